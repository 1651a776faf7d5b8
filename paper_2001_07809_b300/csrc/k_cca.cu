// Connected components analysis and small-component removal (Section III).
//
// Labelling (8-connectivity) is union-find: each 32x32 tile first unites its
// pixels in shared memory (at most two unions per pixel, by the decision tree
// of two-pass labelling), then pixels on tile borders unite across tiles in
// global memory, then every pixel jumps to its root while the sizes are
// counted.  Unions always hang the larger root under the smaller (atomicMin),
// so a component's final root is its smallest linear index: the same label a
// raster-order flood fill gives.
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
constexpr int kUnionLimit = 1 << 22;   // retries of one union before flagging an error

__device__ __forceinline__ int find_root(const int* P, int x) {
  int guard = 0;
  while (true) {
    int p = P[x];
    if (p == x || ++guard > kUnionLimit) return x;
    x = p;
  }
}

// Lock-free union (both roots hang the larger index under the smaller).
__device__ __forceinline__ bool unite(int* P, int a, int b) {
  for (int it = 0; it < kUnionLimit; ++it) {
    a = find_root(P, a);
    b = find_root(P, b);
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
// of the run.  Row y's runs are united with the runs of row y - 1 they touch
// (8-connectivity: columns x - 1 .. x + 1), one union per (run above, run
// below) pair: lane q takes the pairs that first touch at column q of the row
// above.  Unions hang the larger root under the smaller, so a component's
// root is its smallest index, the label the raster flood fill gives.  A last
// pass finds every pixel's root from the row masks and writes the labels.
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
      const bool set = (cur >> lane) & 1u;
      if (set && run_start(cur, lane) == lane) P[y * CT + lane] = y * CT + lane;   // a new node per run
      __syncwarp();
      if (prev && ((prev >> lane) & 1u)) {
        const int q = lane;
        const int A = (y - 1) * CT + run_start(prev, q);                 // the run above through column q
        const bool left_above = q > 0 && ((prev >> (q - 1)) & 1u);       // column q - 1 above: same run, its lane
        auto cb = [&](int c) { return c >= 0 && c < CT && ((cur >> c) & 1u); };
        if (left_above) {
          // lane q - 1 took the runs through columns q - 2 .. q; a run starting at q + 1 is new
          if (cb(q + 1) && !cb(q)) ok &= unite(P, A, y * CT + q + 1);
        } else {
          if (cb(q - 1)) ok &= unite(P, A, y * CT + run_start(cur, q - 1));
          if (cb(q) && !cb(q - 1)) ok &= unite(P, A, y * CT + q);
          if (cb(q + 1) && !cb(q)) ok &= unite(P, A, y * CT + q + 1);
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
      const int root = find_root(P, y * CT + run_start(cur, lane));
      v = (ty0 + (root >> 5)) * w + tx0 + (root & (CT - 1));
    }
    J.lab[(int64_t)(ty0 + y) * w + x] = v;
  }
  if (!ok) atomicOr(dev_err, DEV_ERR_CCA_ITER);
}

__global__ void __launch_bounds__(256) k_cca_merge(const CcaJob* __restrict__ jobs, uint32_t* dev_err) {
  const CcaJob J = jobs[blockIdx.z];
  const int tx0 = blockIdx.x * CT, ty0 = blockIdx.y * CT;
  if (tx0 >= J.w || ty0 >= J.h) return;
  const int w = J.w, h = J.h;
  bool ok = true;
  // tile border pixels: top row (32), left column (31 more), right column (31 more)
  for (int t = threadIdx.x; t < 3 * CT; t += blockDim.x) {
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
      if (J.b[q]) ok &= unite(J.lab, p, q);
    }
  }
  if (!ok) atomicOr(dev_err, DEV_ERR_CCA_ITER);
}

// Final labels and component sizes: every pixel of a 32x32 tile follows its
// parent chain to the root (and stores it: the label is then the root), the
// tile counts its pixels per root in a small shared-memory hash table and
// adds one total per (tile, root) to the global size array, so a large
// component costs one atomic per tile it touches instead of one per pixel.
// Roots append themselves to the job's root list, and the tile's boundary
// pixels are added to N_b.
__global__ void __launch_bounds__(256) k_cc_count(const CcaJob* __restrict__ jobs) {
  constexpr int HS = 256;  // hash slots (a tile rarely holds more than a few dozen roots)
  __shared__ int s_key[HS];
  __shared__ unsigned s_cnt[HS];
  __shared__ unsigned s_total;
  const CcaJob J = jobs[blockIdx.z];
  const int tx0 = blockIdx.x * CT, ty0 = blockIdx.y * CT;
  if (tx0 >= J.w || ty0 >= J.h) return;
  for (int i = threadIdx.x; i < HS; i += blockDim.x) { s_key[i] = -1; s_cnt[i] = 0; }
  if (threadIdx.x == 0) s_total = 0;
  __syncthreads();
  unsigned mine = 0;
  for (int i = threadIdx.x; i < CT * CT; i += blockDim.x) {
    const int x = tx0 + (i & (CT - 1)), y = ty0 + (i >> 5);
    if (x >= J.w || y >= J.h) continue;
    const int64_t p = (int64_t)y * J.w + x;
    int v = J.lab[p];
    if (v < 0) continue;
    ++mine;
    const int f = find_root(J.lab, v);
    if (f != v) J.lab[p] = f;   // only shortens paths other tiles may be following
    if (f == (int)p) J.roots[atomicAdd(reinterpret_cast<unsigned long long*>(&J.cut[5]), 1ull)] = f;
    v = f;
    unsigned hsh = ((unsigned)v * 2654435761u) >> 24;  // 8 bits
    bool placed = false;
    volatile int* vkey = s_key;
    for (int probe = 0; probe < HS; ++probe) {
      const int slot = (hsh + probe) & (HS - 1);
      const int k = vkey[slot];
      if (k == v || (k == -1 && (atomicCAS(&s_key[slot], -1, v) == -1 || vkey[slot] == v))) {
        atomicAdd(&s_cnt[slot], 1u);
        placed = true;
        break;
      }
    }
    if (!placed) atomicAdd(&J.size[v], 1u);  // table full: count directly
  }
  for (int o = 16; o; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(&s_total, mine);
  __syncthreads();
  for (int i = threadIdx.x; i < HS; i += blockDim.x)
    if (s_key[i] >= 0 && s_cnt[i]) atomicAdd(&J.size[s_key[i]], s_cnt[i]);
  if (threadIdx.x == 0 && s_total) atomicAdd(reinterpret_cast<unsigned long long*>(&J.cut[0]), (unsigned long long)s_total);
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
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
    const int v = J.lab[p];
    uint8_t keep = 0;
    if (v >= 0) {
      const uint32_t sz = J.size[v];
      const bool gone = sz < sstar || (sz == sstar && (long long)v < T);
      keep = gone ? 0 : 1;
    }
    J.out[p] = keep;
  }
}

void launch_cca(const CcaJob* jobs, int n_jobs, int max_w, int max_h, uint32_t* dev_err, cudaStream_t s) {
  if (n_jobs <= 0) return;
  dim3 tiles((max_w + CT - 1) / CT, (max_h + CT - 1) / CT, n_jobs);
  const int tiles_x = (max_w + CT - 1) / CT;
  k_cca_local<<<dim3((tiles_x + kCcaWarps - 1) / kCcaWarps, tiles.y, n_jobs), kCcaWarps * 32, 0, s>>>(jobs, dev_err);
  k_cca_merge<<<tiles, 128, 0, s>>>(jobs, dev_err);
}

void launch_cc_filter(const CcaJob* jobs, int n_jobs, int max_w, int max_h, cudaStream_t s) {
  if (n_jobs <= 0) return;
  const int64_t n = (int64_t)max_w * max_h;
  int bpj = (int)((n + 256 * 8 - 1) / (256 * 8));
  if (bpj > 1184) bpj = 1184;
  if (bpj < 1) bpj = 1;
  k_cc_count<<<dim3((max_w + CT - 1) / CT, (max_h + CT - 1) / CT, n_jobs), 256, 0, s>>>(jobs);
  const int rpj = std::max(1, std::min(bpj, 148));   // root-list passes: roots are few
  k_cc_hist<<<dim3(rpj, n_jobs), 256, 0, s>>>(jobs);
  k_cc_cut<<<n_jobs, 1024, 0, s>>>(jobs);
  k_cc_rowcount<<<dim3(rpj, n_jobs), 256, 0, s>>>(jobs);
  k_cc_select<<<n_jobs, 1024, 0, s>>>(jobs);
  k_cc_filter<<<dim3(bpj, n_jobs), 256, 0, s>>>(jobs);
}

}  // namespace sb
