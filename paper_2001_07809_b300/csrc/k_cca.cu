// Connected components analysis and small-component removal (Section III).
//
// Labelling (8-connectivity) is union-find: a warp labels each 32x32 tile by
// sweeping its rows in order with one node per horizontal run (in shared
// memory), then pixels on tile borders unite across tiles in global memory,
// then every tile-local root is chased to its component root while the sizes
// are counted.  Unions always hang the larger root under the smaller
// (atomicMin), so a component's final root is its smallest linear index: the
// same label a raster-order flood fill gives.
//
// Removal: the components are ordered by (size, label) and the longest
// prefix holding at most floor(frac * N_b) pixels is removed.  On the device
// that prefix is "every component smaller than s*, plus the m size-s*
// components with the smallest labels", with s* and m found from a histogram
// of component sizes, and the cut label T found from per-row counts; both
// counts run over the list of roots rather than over every pixel.  No host
// round-trip, so the whole sequence can be captured in a CUDA graph.
#include <algorithm>
#include "sb_common.cuh"

namespace sb {

namespace {
constexpr int CT = 32;                 // CCA tile side

// Root of x: follows at most `limit` parent links (CcaJob::union_limit); a
// chain that is longer clears ok (the run is reported as SB_ERR_TIMEOUT) and
// returns the node reached.  Every link points to a smaller index, so the walk
// always stays inside the image and ends.
__device__ __forceinline__ int find_root(const int* P, int x, int limit, bool& ok) {
  for (int guard = 0;; ++guard) {
    const int p = P[x];
    if (p == x) return x;
    if (guard >= limit) {
      ok = false;
      return x;
    }
    x = p;
  }
}

// Lock-free union (both roots hang the larger index under the smaller), at
// most `limit` attempts.
__device__ __forceinline__ bool unite(int* P, int a, int b, int limit, bool& ok) {
  for (int it = 0; it < limit; ++it) {
    a = find_root(P, a, limit, ok);
    b = find_root(P, b, limit, ok);
    if (a == b) return true;
    if (a < b) {
      int old = atomicMin(&P[b], a);
      if (old == b) return true;
      b = old;
    } else {
      int old = atomicMin(&P[a], b);
      if (old == a) return true;
      a = old;
    }
  }
  return false;
}
}  // namespace

// Tile-local labelling, one warp per 32x32 tile, rows in order (the classic
// raster two-pass scheme with a warp holding one row): lane x of the warp is
// tile column x.  The 32 row masks are ballots of the map (all rows loaded up
// front); each horizontal run of a row is one union-find node, named by its
// first pixel (tile-local index y * 32 + start), which is the smallest index
// of the run.  A run of row y touches the runs of row y - 1 that cross its
// columns widened by one on each side (8-connectivity); the lane at its start
// hangs the new node under the root of the first of them and unites that
// tree with the trees of the others (rare: where two branches meet).  Every
// link goes from a larger index to a smaller one, so a component's root is
// its smallest index, the label the raster flood fill gives.  A last pass
// finds every pixel's root from the row masks and writes the labels.
constexpr int kCcaWarps = 8;   // tiles per CTA (along x)

__device__ __forceinline__ int run_start(unsigned mask, int c) {
  const unsigned z = ~mask & ((1u << c) - 1u);   // clear columns left of c (c = 0: none)
  return z ? 32 - __clz(z) : 0;
}

__global__ void __launch_bounds__(kCcaWarps * 32) k_cca_local(const CcaJob* __restrict__ jobs, uint32_t* dev_err) {
  __shared__ int s_par[kCcaWarps][CT * CT];
  const CcaJob J = jobs[blockIdx.z];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tx0 = (blockIdx.x * kCcaWarps + warp) * CT, ty0 = blockIdx.y * CT;
  if (tx0 >= J.w || ty0 >= J.h) return;   // whole warps leave together
  const int w = J.w, h = J.h;
  int* P = s_par[warp];
  const int x = tx0 + lane;
  // the tile's 32 bytes of column `lane`, then lane y keeps the mask of row y
  unsigned colbits = 0;
  {
    uint8_t v[CT];
#pragma unroll
    for (int y = 0; y < CT; ++y) v[y] = (x < w && ty0 + y < h) ? J.b[(int64_t)(ty0 + y) * w + x] : (uint8_t)0;
#pragma unroll
    for (int y = 0; y < CT; ++y) colbits |= (v[y] ? 1u : 0u) << y;
  }
  unsigned rowmask = 0;
#pragma unroll
  for (int y = 0; y < CT; ++y) {
    const unsigned m = __ballot_sync(0xffffffffu, (colbits >> y) & 1u);
    if (lane == y) rowmask = m;
  }
  bool ok = true;
  unsigned prev = 0;
  for (int y = 0; y < CT; ++y) {
    const unsigned cur = __shfl_sync(0xffffffffu, rowmask, y);
    if (cur) {
      // the lane at the start of each run links the run (a fresh node) to the
      // root of the first run above it touches, and unites that tree with the
      // tree of every further run above it touches
      const unsigned starts = cur & ~(cur << 1);
      if ((starts >> lane) & 1u) {
        const int C = y * CT + lane;
        const unsigned inv = ~(cur >> lane);
        const int len = inv ? __ffs(inv) - 1 : CT - lane;
        const unsigned run = (len == 32 ? 0xffffffffu : ((1u << len) - 1u)) << lane;
        const unsigned T = prev & (run | (run << 1) | (run >> 1));   // columns above it touches
        if (!T) {
          P[C] = C;
        } else {
          const int s1 = run_start(prev, __ffs(T) - 1);
          const int r1 = find_root(P, (y - 1) * CT + s1, J.union_limit, ok);
          P[C] = r1;   // r1 < C: the smaller index stays the root
          unsigned others = T & (prev & ~(prev << 1)) & ~(1u << s1);   // starts of the other runs above
          while (others) {
            const int b = __ffs(others) - 1;
            others &= others - 1u;
            ok &= unite(P, r1, (y - 1) * CT + b, J.union_limit, ok);
          }
        }
      }
      __syncwarp();
    }
    prev = cur;
  }
  // labels: every pixel's root, as a linear index of the image
  for (int y = 0; y < CT && ty0 + y < h; ++y) {
    const unsigned cur = __shfl_sync(0xffffffffu, rowmask, y);
    if (x >= w) continue;
    int v = -1;
    if ((cur >> lane) & 1u) {
      const int root = find_root(P, y * CT + run_start(cur, lane), J.union_limit, ok);
      v = (ty0 + (root >> 5)) * w + tx0 + (root & (CT - 1));
    }
    J.lab[(int64_t)(ty0 + y) * w + x] = v;
  }
  if (!ok) atomicOr(dev_err, DEV_ERR_CCA_ITER);
}

constexpr int kMergeTiles = 4;   // tiles per CTA of k_cca_merge (along x)
__global__ void __launch_bounds__(128) k_cca_merge(const CcaJob* __restrict__ jobs, uint32_t* dev_err) {
  const CcaJob J = jobs[blockIdx.z];
  const int ty0 = blockIdx.y * CT;
  if (blockIdx.x * kMergeTiles * CT >= J.w || ty0 >= J.h) return;
  const int w = J.w, h = J.h;
  bool ok = true;
  // tile border pixels: top row (32), left column (31 more), right column (31 more)
  for (int tt = threadIdx.x; tt < kMergeTiles * 3 * CT; tt += blockDim.x) {
    const int tx0 = (blockIdx.x * kMergeTiles + tt / (3 * CT)) * CT, t = tt % (3 * CT);
    if (tx0 >= w) continue;
    int lx, ly;
    if (t < CT) { lx = t; ly = 0; }
    else if (t < 2 * CT - 1) { lx = 0; ly = t - CT + 1; }
    else if (t < 3 * CT - 2) { lx = CT - 1; ly = t - 2 * CT + 2; }
    else continue;
    const int x = tx0 + lx, y = ty0 + ly;
    if (x >= w || y >= h) continue;
    const int p = y * w + x;
    if (!J.b[p]) continue;
    const int nx[4] = {x - 1, x - 1, x, x + 1}, ny[4] = {y, y - 1, y - 1, y - 1};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int qx = nx[k], qy = ny[k];
      if (qx < 0 || qy < 0 || qx >= w) continue;
      if (qx >= tx0 && qx < tx0 + CT && qy >= ty0) continue;  // same tile: done locally
      const int q = qy * w + qx;
      if (J.b[q]) ok &= unite(J.lab, p, q, J.union_limit, ok);
    }
  }
  if (!ok) atomicOr(dev_err, DEV_ERR_CCA_ITER);
}

// Final labels and component sizes.  After the tile labelling every pixel's
// label is its tile-local root; the border merge then re-points some of those
// roots (to a root in this tile or another).  So a pixel p's local root u is
// its label when that lies in the tile, else p itself (a local root whose
// label the merge changed to another tile).  A 32x32 tile counts its pixels
// per local root in shared memory, then only the referenced local roots
// follow their parent chains in global memory (one to a few hops) to the
// component root R, add their counts to size[R] and, when a local root is R
// itself, append it to the job's root list; a last pass writes R as every
// pixel's label.  The tile's boundary pixels are added to N_b.
__device__ __forceinline__ int tile_local(int v, int base, int w, float inv_w) {
  const int d = v - base;   // v = base + dy * w + dx for a pixel of the tile
  if (d < 0) return -1;
  int dy = (int)((float)d * inv_w);
  if (dy * w > d) --dy;
  else if ((dy + 1) * w <= d) ++dy;   // exact for dy < 32, where it matters
  if (dy >= CT) return -1;
  const int dx = d - dy * w;
  return dx < CT && dx < w ? dy * CT + dx : -1;
}

constexpr int kCountTiles = 2;   // tiles per CTA of k_cc_count (along x)
__global__ void __launch_bounds__(256) k_cc_count(const CcaJob* __restrict__ jobs, uint32_t* dev_err) {
  constexpr int kPer = CT * CT / 256;   // pixels per thread and tile
  __shared__ unsigned s_cnt[kCountTiles][CT * CT];   // pixels per local root
  __shared__ int s_root[kCountTiles][CT * CT];       // component root of each referenced local root
  __shared__ unsigned s_total;
  const CcaJob J = jobs[blockIdx.z];
  const int w = J.w, h = J.h;
  const int ty0 = blockIdx.y * CT;
  if (blockIdx.x * kCountTiles * CT >= w || ty0 >= h) return;
  const float inv_w = 1.0f / (float)w;
  for (int i = threadIdx.x; i < kCountTiles * CT * CT; i += blockDim.x) (&s_cnt[0][0])[i] = 0u;
  if (threadIdx.x == 0) s_total = 0;
  __syncthreads();
  int u[kCountTiles][kPer], v[kCountTiles][kPer];
  unsigned mine = 0;
  bool ok = true;
#pragma unroll
  for (int tt = 0; tt < kCountTiles; ++tt)
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int i = threadIdx.x + 256 * k;
      const int x = (blockIdx.x * kCountTiles + tt) * CT + (i & (CT - 1)), y = ty0 + (i >> 5);
      v[tt][k] = (x < w && y < h) ? J.lab[(int64_t)y * w + x] : -1;
    }
#pragma unroll
  for (int tt = 0; tt < kCountTiles; ++tt) {
    const int tx0 = (blockIdx.x * kCountTiles + tt) * CT;
    const int base = ty0 * w + tx0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      u[tt][k] = -1;
      if (v[tt][k] >= 0) {
        const int i = threadIdx.x + 256 * k;
        const int t = tile_local(v[tt][k], base, w, inv_w);
        u[tt][k] = t >= 0 ? t : i;
        atomicAdd(&s_cnt[tt][u[tt][k]], 1u);
        ++mine;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int tt = 0; tt < kCountTiles; ++tt) {
    const int tx0 = (blockIdx.x * kCountTiles + tt) * CT;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int i = threadIdx.x + 256 * k;
      const unsigned c = s_cnt[tt][i];
      if (c) {   // pixel i is a local root some pixel of the tile refers to
        const int g = (ty0 + (i >> 5)) * w + tx0 + (i & (CT - 1));
        const int R = find_root(J.lab, g, J.union_limit, ok);
        s_root[tt][i] = R;
        atomicAdd(&J.size[R], c);
        if (R == g) J.roots[atomicAdd(reinterpret_cast<unsigned long long*>(&J.cut[5]), 1ull)] = R;
      }
    }
  }
  for (int o = 16; o; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(&s_total, mine);
  __syncthreads();
#pragma unroll
  for (int tt = 0; tt < kCountTiles; ++tt) {
    const int tx0 = (blockIdx.x * kCountTiles + tt) * CT;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      if (u[tt][k] < 0) continue;
      const int R = s_root[tt][u[tt][k]];
      if (R != v[tt][k]) {
        const int i = threadIdx.x + 256 * k;
        J.lab[(int64_t)(ty0 + (i >> 5)) * w + tx0 + (i & (CT - 1))] = R;   // other tiles may follow it: R is an ancestor
      }
    }
  }
  if (threadIdx.x == 0 && s_total) atomicAdd(reinterpret_cast<unsigned long long*>(&J.cut[0]), (unsigned long long)s_total);
  if (!ok) atomicOr(dev_err, DEV_ERR_CCA_ITER);
}

__device__ __forceinline__ int64_t removal_limit(const CcaJob& J) {
  return (int64_t)floor(__dmul_rn(J.frac, (double)J.cut[0]));
}

__global__ void __launch_bounds__(256) k_cc_hist(const CcaJob* __restrict__ jobs) {
  const CcaJob J = jobs[blockIdx.y];
  const int64_t nroots = J.cut[5];
  const int64_t limit = removal_limit(J);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nroots; i += stride) {
    const uint32_t s = J.size[J.roots[i]];
    if ((int64_t)s <= limit && (int64_t)s < J.shist_len) atomicAdd(&J.shist[s], 1u);
  }
}

// One CTA per job: s* = smallest size whose cumulative pixel count exceeds the
// limit, m = how many size-s* components still fit.
__global__ void __launch_bounds__(1024) k_cc_cut(const CcaJob* __restrict__ jobs) {
  __shared__ long long s_part[1024];
  __shared__ long long s_first;
  const CcaJob J = jobs[blockIdx.x];
  const int64_t limit = removal_limit(J);
  const int64_t len = limit < (int64_t)J.shist_len - 1 ? limit : (int64_t)J.shist_len - 1;  // sizes 1..len
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t per = (len + nt - 1) / nt;
  const int64_t a = 1 + tid * per, b = a + per < len + 1 ? a + per : len + 1;
  long long loc = 0;
  for (int64_t s = a; s < b; ++s) loc += (long long)s * J.shist[s];
  s_part[tid] = loc;
  if (tid == 0) s_first = LLONG_MAX;
  __syncthreads();
  // inclusive scan over threads (Hillis-Steele, 1024 entries)
  for (int o = 1; o < nt; o <<= 1) {
    long long v = tid >= o ? s_part[tid - o] : 0;
    __syncthreads();
    s_part[tid] += v;
    __syncthreads();
  }
  long long run = tid ? s_part[tid - 1] : 0;
  long long found = LLONG_MAX, found_before = 0;
  for (int64_t s = a; s < b; ++s) {
    long long nxt = run + (long long)s * J.shist[s];
    if (nxt > limit) { found = s; found_before = run; atomicMin(&s_first, found); break; }
    run = nxt;
  }
  __syncthreads();
  if (found != LLONG_MAX && found == s_first) {
    // the unique thread holding the first crossing: m size-s* components still fit
    J.cut[2] = found;
    J.cut[3] = (limit - found_before) / found;
  }
  if (tid == 0) {
    if (s_first == LLONG_MAX) {  // every component of size <= limit goes
      J.cut[2] = limit + 1;
      J.cut[3] = 0;
    }
    J.cut[1] = limit;
    J.cut[4] = -1;
  }
}

// Per row: how many roots have size s* (only when m > 0); rowcnt is zero on entry.
__global__ void __launch_bounds__(256) k_cc_rowcount(const CcaJob* __restrict__ jobs) {
  const CcaJob J = jobs[blockIdx.y];
  if (J.cut[3] <= 0) return;
  const uint32_t sstar = (uint32_t)J.cut[2];
  const int64_t nroots = J.cut[5];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nroots; i += stride) {
    const int v = J.roots[i];
    if (J.size[v] == sstar) atomicAdd(&J.rowcnt[v / J.w], 1u);
  }
}

// One CTA per job: T = label of the m-th (0-based) size-s* root in raster order.
__global__ void __launch_bounds__(1024) k_cc_select(const CcaJob* __restrict__ jobs) {
  __shared__ long long s_part[1024];
  __shared__ int s_row;
  __shared__ long long s_before;
  const CcaJob J = jobs[blockIdx.x];
  const long long m = J.cut[3];
  if (m <= 0) return;
  const uint32_t sstar = (uint32_t)J.cut[2];
  const int tid = threadIdx.x, nt = blockDim.x, h = J.h;
  const int per = (h + nt - 1) / nt;
  const int a = tid * per, b = a + per < h ? a + per : h;
  long long loc = 0;
  for (int y = a; y < b; ++y) loc += J.rowcnt[y];
  s_part[tid] = loc;
  if (tid == 0) s_row = INT_MAX;
  __syncthreads();
  for (int o = 1; o < nt; o <<= 1) {
    long long v = tid >= o ? s_part[tid - o] : 0;
    __syncthreads();
    s_part[tid] += v;
    __syncthreads();
  }
  long long run = tid ? s_part[tid - 1] : 0;
  int cand = INT_MAX;
  long long cand_before = 0;
  for (int y = a; y < b; ++y) {
    long long nxt = run + J.rowcnt[y];
    if (m < nxt) { cand = y; cand_before = run; break; }
    run = nxt;
  }
  if (cand != INT_MAX) atomicMin(&s_row, cand);  // every later thread also crosses: keep the first row
  __syncthreads();
  if (cand != INT_MAX && cand == s_row) s_before = cand_before;
  __syncthreads();
  if (tid < 32 && s_row != INT_MAX) {  // warp 0 walks the row 32 pixels at a time
    long long k = m - s_before;
    const int64_t base = (int64_t)s_row * J.w;
    for (int x0 = 0; x0 < J.w; x0 += 32) {
      const int x = x0 + tid;
      const int64_t p = base + x;
      const bool hit = x < J.w && J.lab[p] == (int)p && J.size[p] == sstar;
      const unsigned mask = __ballot_sync(0xffffffffu, hit);
      const int c = __popc(mask);
      if (k < c) {
        // position of the k-th set bit
        unsigned mm = mask;
        for (long long i = 0; i < k; ++i) mm &= mm - 1;
        if (tid == __ffs(mm) - 1) J.cut[4] = p;
        break;
      }
      k -= c;
    }
  }
}

__global__ void __launch_bounds__(256) k_cc_filter(const CcaJob* __restrict__ jobs) {
  const CcaJob J = jobs[blockIdx.y];
  const int64_t n = (int64_t)J.w * J.h;
  const uint32_t sstar = (uint32_t)J.cut[2];
  const long long T = J.cut[4];
  auto keep = [&](int v) -> uint32_t {
    if (v < 0) return 0u;
    const uint32_t sz = J.size[v];
    return sz < sstar || (sz == sstar && (long long)v < T) ? 0u : 1u;
  };
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // four pixels per step (16-byte label loads, one size lookup per distinct
  // label: neighbours mostly share their root), then the last n % 4 pixels
  const int64_t n4 = n / 4;
  const bool vec = ((reinterpret_cast<uintptr_t>(J.lab) | reinterpret_cast<uintptr_t>(J.out)) & 15) == 0;
  if (vec) {
    for (int64_t q = t0; q < n4; q += stride) {
      const int4 v = reinterpret_cast<const int4*>(J.lab)[q];
      const uint32_t k0 = keep(v.x);
      const uint32_t k1 = v.y == v.x ? k0 : keep(v.y);
      const uint32_t k2 = v.z == v.y ? k1 : keep(v.z);
      const uint32_t k3 = v.w == v.z ? k2 : keep(v.w);
      reinterpret_cast<uint32_t*>(J.out)[q] = k0 | (k1 << 8) | (k2 << 16) | (k3 << 24);
    }
  }
  for (int64_t p = (vec ? 4 * n4 : 0) + t0; p < n; p += stride) J.out[p] = (uint8_t)keep(J.lab[p]);
}

void launch_cca(const CcaJob* jobs, int n_jobs, int max_w, int max_h, uint32_t* dev_err, cudaStream_t s) {
  if (n_jobs <= 0) return;
  dim3 tiles((max_w + CT - 1) / CT, (max_h + CT - 1) / CT, n_jobs);
  const int tiles_x = (max_w + CT - 1) / CT;
  k_cca_local<<<dim3((tiles_x + kCcaWarps - 1) / kCcaWarps, tiles.y, n_jobs), kCcaWarps * 32, 0, s>>>(jobs, dev_err);
  k_cca_merge<<<dim3((tiles_x + kMergeTiles - 1) / kMergeTiles, tiles.y, n_jobs), 128, 0, s>>>(jobs, dev_err);
}

void launch_cc_filter(const CcaJob* jobs, int n_jobs, int max_w, int max_h, uint32_t* dev_err, cudaStream_t s) {
  if (n_jobs <= 0) return;
  const int64_t n = (int64_t)max_w * max_h;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // filter CTAs per job: one per 2048 pixels, at most 8 waves per SM, and no more
  // than 16 waves of the whole batch in all (a large batch needs few per job)
  int64_t bpj64 = std::min<int64_t>((n + 256 * 8 - 1) / (256 * 8), 8 * (int64_t)sms);
  bpj64 = std::min<int64_t>(bpj64, (16 * 8 * (int64_t)sms + n_jobs - 1) / n_jobs);
  const int bpj = (int)std::max<int64_t>(1, bpj64);
  const int tiles_x = (max_w + CT - 1) / CT;
  k_cc_count<<<dim3((tiles_x + kCountTiles - 1) / kCountTiles, (max_h + CT - 1) / CT, n_jobs), 256, 0, s>>>(jobs, dev_err);
  // root-list passes: roots are few; four waves of the batch in all
  const int rpj = (int)std::max<int64_t>(1, std::min<int64_t>(std::min(bpj, sms), (4 * 8 * (int64_t)sms + n_jobs - 1) / n_jobs));
  k_cc_hist<<<dim3(rpj, n_jobs), 256, 0, s>>>(jobs);
  k_cc_cut<<<n_jobs, 1024, 0, s>>>(jobs);
  k_cc_rowcount<<<dim3(rpj, n_jobs), 256, 0, s>>>(jobs);
  k_cc_select<<<n_jobs, 1024, 0, s>>>(jobs);
  k_cc_filter<<<dim3(bpj, n_jobs), 256, 0, s>>>(jobs);
}

}  // namespace sb
