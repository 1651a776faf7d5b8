// Connected components analysis and small-component removal (Section III).
//
// Labelling (8-connectivity) is union-find at two levels.  A warp labels each
// 32x32 tile in shared memory, sweeping its rows in order with one node per
// horizontal run, and writes every pixel's tile-local root as a 16-bit index
// (y * 32 + x within the tile, 0xFFFF off the map).  Only the tile-local roots
// have a node in the image-level forest: at the linear index g of a local
// root, J.node[2g] is its parent and J.node[2g + 1] the component's size once g
// is a component root; no other slot is read or written, so nothing has to
// clear the table.  Pixels on tile borders then unite the nodes of their local
// roots across tiles, and every local root is chased to its component root
// while the sizes are counted.  Unions always hang the larger root under the
// smaller (atomicMin), and a local root is the smallest index of its piece of
// the tile, so a component's final root is its smallest linear index: the same
// label a raster-order flood fill gives.
//
// Removal: the components are ordered by (size, label) and the longest
// prefix holding at most floor(frac * N_b) pixels is removed.  On the device
// that prefix is "every component smaller than s*, plus the m size-s*
// components with the smallest labels", with s* and m found from a histogram
// of component sizes, and the cut label T found from per-row counts; both
// counts run over the list of roots rather than over every pixel.  No host
// round-trip, so the whole sequence can be captured in a CUDA graph.
//
// Traffic per pixel: the map is read once (1 byte), the 16-bit labels are
// written once and read twice (counting, filtering), the filtered map is
// written once (1 byte); the node table is touched at local roots only.
#include <algorithm>
#include "sb_common.cuh"

namespace sb {

namespace {
constexpr int CT = 32;                  // CCA tile side
constexpr uint16_t kOffMap = 0xFFFF;    // tile-local label of a pixel off the map

// Parent of node x: P[x] in a tile's shared-memory forest (S = 1), P[2x] in
// the image-level node table (S = 2).
template <int S>
__device__ __forceinline__ int* parent_of(int* P, int x) {
  if constexpr (S == 1) return P + x;
  else return P + 2 * (int64_t)x;
}

// Root of x: follows at most `limit` parent links (CcaJob::union_limit); a
// chain that is longer clears ok (the run is reported as SB_ERR_TIMEOUT) and
// returns the node reached.  Every link points to a smaller index, so the walk
// always stays inside the image and ends.
template <int S>
__device__ __forceinline__ int find_root(int* P, int x, int limit, bool& ok) {
  for (int guard = 0;; ++guard) {
    const int p = *parent_of<S>(P, x);
    if (p == x || !SB_CHECK(p >= 0 && p < x, 301u)) return x;
    if (guard >= limit) {
      ok = false;
      return x;
    }
    x = p;
  }
}

// Lock-free union (both roots hang the larger index under the smaller), at
// most `limit` attempts.
template <int S>
__device__ __forceinline__ bool unite(int* P, int a, int b, int limit, bool& ok) {
  for (int it = 0; it < limit; ++it) {
    a = find_root<S>(P, a, limit, ok);
    b = find_root<S>(P, b, limit, ok);
    if (a == b) return true;
    if (a < b) {
      int old = atomicMin(parent_of<S>(P, b), a);
      if (old == b) return true;
      b = old;
    } else {
      int old = atomicMin(parent_of<S>(P, a), b);
      if (old == a) return true;
      a = old;
    }
  }
  return false;
}

// Bit i set when byte i of v is nonzero (i = 0..3): the high bit of each
// nonzero byte is gathered by a carry-free multiply.
__device__ __forceinline__ unsigned nz_bits(unsigned v) {
  const unsigned t = (((v & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | v) & 0x80808080u;
  return ((t >> 7) * 0x01020408u) >> 24;
}

// Linear index of the local root named by label li of pixel (x, y).
__device__ __forceinline__ int64_t local_root_at(int x, int y, int li, int w) {
  return (int64_t)((y & ~(CT - 1)) + (li >> 5)) * w + (x & ~(CT - 1)) + (li & (CT - 1));
}

__device__ __forceinline__ uint32_t comp_size(const CcaJob& J, int64_t r) {
  return (uint32_t)J.node[2 * r + 1];
}
}  // namespace

// Tile-local labelling, one warp per 32x32 tile.  Lane y holds the mask of
// tile row y; each horizontal run of a row is one union-find node, named by its
// first pixel (tile-local index y * 32 + start), which is the smallest index of
// the run.  A run of row y touches the runs of row y - 1 that cross its
// columns widened by one on each side (8-connectivity); every lane unites each
// run of its row with each run above it touches, all rows at once, with the
// lock-free union of the image-level merge (shared-memory atomics).  Every
// link goes from a larger index to a smaller one, so a piece's root is its
// smallest index.  A last sweep, lane x of the warp on tile column x,
// rows in order, finds every pixel's root, writes it as the pixel's
// label and points each run's node straight at it (so the searches of later
// rows take one or two links), and gives every local root its node in the
// image-level table (parent itself, size 0).
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
  unsigned rowmask = 0;   // lane y: bit c set when pixel (tx0 + c, ty0 + y) is on the map
  if (tx0 + CT <= w && (w & 15) == 0 && (reinterpret_cast<uintptr_t>(J.b) & 15) == 0) {
    // whole tile rows: lane y reads its row's 32 bytes as two 16-byte loads
    if (ty0 + lane < h) {
      const uint4* row = reinterpret_cast<const uint4*>(J.b + (int64_t)(ty0 + lane) * w + tx0);
      const uint4 a = row[0], c = row[1];
      rowmask = nz_bits(a.x) | nz_bits(a.y) << 4 | nz_bits(a.z) << 8 | nz_bits(a.w) << 12 |
                nz_bits(c.x) << 16 | nz_bits(c.y) << 20 | nz_bits(c.z) << 24 | nz_bits(c.w) << 28;
    }
  } else {
    // ragged tile: the 32 bytes of column `lane`, then one ballot per row
    unsigned colbits = 0;
    uint8_t v[CT];
#pragma unroll
    for (int y = 0; y < CT; ++y) v[y] = (x < w && ty0 + y < h) ? J.b[(int64_t)(ty0 + y) * w + x] : (uint8_t)0;
#pragma unroll
    for (int y = 0; y < CT; ++y) colbits |= (v[y] ? 1u : 0u) << y;
#pragma unroll
    for (int y = 0; y < CT; ++y) {
      const unsigned m = __ballot_sync(0xffffffffu, (colbits >> y) & 1u);
      if (lane == y) rowmask = m;
    }
  }
  bool ok = true;
  {
    // every row at once: lane y makes a node of each run of its row, then links
    // each run to every run of row y - 1 it touches
    const unsigned cur = rowmask;
    const unsigned above = __shfl_up_sync(0xffffffffu, rowmask, 1);
    const unsigned prev = lane > 0 ? above : 0u;
    const unsigned starts = cur & ~(cur << 1), pstarts = prev & ~(prev << 1);
    for (unsigned m = starts; m; m &= m - 1u) {
      const int c = __ffs(m) - 1;
      P[lane * CT + c] = lane * CT + c;
    }
    __syncwarp();
    for (unsigned m = starts; m; m &= m - 1u) {
      const int c = __ffs(m) - 1;
      const unsigned inv = ~(cur >> c);
      const int len = inv ? __ffs(inv) - 1 : CT - c;
      const unsigned run = (len == 32 ? 0xffffffffu : ((1u << len) - 1u)) << c;
      const unsigned T = prev & (run | (run << 1) | (run >> 1));   // columns above it touches
      if (!T) continue;
      const int C = lane * CT + c;
      const int s1 = run_start(prev, __ffs(T) - 1);   // the first run above, which may start left of T
      ok &= unite<1>(P, C, (lane - 1) * CT + s1, J.union_limit, ok);
      for (unsigned o = T & pstarts & ~(1u << s1); o; o &= o - 1u)   // the other runs above
        ok &= unite<1>(P, C, (lane - 1) * CT + __ffs(o) - 1, J.union_limit, ok);
    }
    __syncwarp();
  }
  // labels, rows in order (a node another lane is re-pointing still leads to
  // the same root, whichever value a search reads)
  for (int y = 0; y < CT && ty0 + y < h; ++y) {
    const unsigned cur = __shfl_sync(0xffffffffu, rowmask, y);
    uint16_t v = kOffMap;
    if ((cur >> lane) & 1u) {
      const int C = y * CT + run_start(cur, lane);
      const int root = find_root<1>(P, C, J.union_limit, ok);
      v = (uint16_t)root;
      if (C == y * CT + lane) {   // the run's first lane
        if (root != C) {
          P[C] = root;
        } else {
          const int64_t g = (int64_t)(ty0 + y) * w + x;
          if (SB_CHECK(x < w, 302u)) reinterpret_cast<int2*>(J.node)[g] = make_int2((int)g, 0);
        }
      }
    }
    if (x < w) J.lab[(int64_t)(ty0 + y) * w + x] = v;
  }
  if (!ok) atomicOr(dev_err, DEV_ERR_CCA_ITER);
}

// Border merge: every map pixel on a tile's top row or left or right column
// unites the node of its local root with the node of each 8-neighbour's local
// root in another tile (neighbours above and to the left; the pixels below and
// to the right of a border are the next tiles' border pixels).
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
    const int lp = J.lab[(int64_t)y * w + x];
    if (lp == kOffMap || !SB_CHECK(lp < CT * CT, 303u)) continue;
    const int a = (int)local_root_at(x, y, lp, w);
    const int nx[4] = {x - 1, x - 1, x, x + 1}, ny[4] = {y, y - 1, y - 1, y - 1};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int qx = nx[k], qy = ny[k];
      if (qx < 0 || qy < 0 || qx >= w) continue;
      if (qx >= tx0 && qx < tx0 + CT && qy >= ty0) continue;  // same tile: done locally
      const int lq = J.lab[(int64_t)qy * w + qx];
      if (lq != kOffMap && SB_CHECK(lq < CT * CT, 303u)) ok &= unite<2>(J.node, a, (int)local_root_at(qx, qy, lq, w), J.union_limit, ok);
    }
  }
  if (!ok) atomicOr(dev_err, DEV_ERR_CCA_ITER);
}

// Component sizes.  A 32x32 tile counts its pixels per local root in shared
// memory; then each local root some pixel refers to follows its parent chain
// in the node table (one to a few links) to the component root R, adds its
// count to R's size, points its own node straight at R (so the filter needs
// one link) and, when it is R itself, appends R to the job's root list.  The
// tile's map pixels are added to N_b.
constexpr int kCountTiles = 2;   // tiles per CTA of k_cc_count (along x)
__global__ void __launch_bounds__(256) k_cc_count(const CcaJob* __restrict__ jobs, uint32_t* dev_err) {
  constexpr int kPer = CT * CT / 256;   // pixels per thread and tile
  __shared__ unsigned s_cnt[kCountTiles][CT * CT];   // pixels per local root
  __shared__ unsigned s_total;
  const CcaJob J = jobs[blockIdx.z];
  const int w = J.w, h = J.h;
  const int ty0 = blockIdx.y * CT;
  if (blockIdx.x * kCountTiles * CT >= w || ty0 >= h) return;
  for (int i = threadIdx.x; i < kCountTiles * CT * CT; i += blockDim.x) (&s_cnt[0][0])[i] = 0u;
  if (threadIdx.x == 0) s_total = 0;
  int li[kCountTiles][kPer];
#pragma unroll
  for (int tt = 0; tt < kCountTiles; ++tt)
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int i = threadIdx.x + 256 * k;
      const int x = (blockIdx.x * kCountTiles + tt) * CT + (i & (CT - 1)), y = ty0 + (i >> 5);
      li[tt][k] = (x < w && y < h) ? J.lab[(int64_t)y * w + x] : kOffMap;
    }
  __syncthreads();
  unsigned mine = 0;
  bool ok = true;
#pragma unroll
  for (int tt = 0; tt < kCountTiles; ++tt)
#pragma unroll
    for (int k = 0; k < kPer; ++k)
      if (li[tt][k] != kOffMap && SB_CHECK(li[tt][k] < CT * CT, 304u)) {
        atomicAdd(&s_cnt[tt][li[tt][k]], 1u);
        ++mine;
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
        const int R = find_root<2>(J.node, g, J.union_limit, ok);
        atomicAdd(reinterpret_cast<unsigned*>(&J.node[2 * (int64_t)R + 1]), c);
        if (R == g) {
          const unsigned long long at = atomicAdd(reinterpret_cast<unsigned long long*>(&J.cut[5]), 1ull);
          if (SB_CHECK(at < (unsigned long long)((w + 1) / 2) * ((h + 1) / 2), 305u)) J.roots[at] = R;
        } else {
          J.node[2 * (int64_t)g] = R;   // another tile's search through g still reaches R
        }
      }
    }
  }
  for (int o = 16; o; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(&s_total, mine);
  __syncthreads();
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
    const int v = J.roots[i];
    if (!SB_CHECK(v >= 0 && v < J.w * J.h, 306u)) continue;
    const uint32_t s = comp_size(J, v);
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
    if (!SB_CHECK(v >= 0 && v < J.w * J.h, 306u)) continue;
    if (comp_size(J, v) == sstar) atomicAdd(&J.rowcnt[v / J.w], 1u);
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
    const int y = s_row;
    const int64_t base = (int64_t)y * J.w;
    for (int x0 = 0; x0 < J.w; x0 += 32) {
      const int x = x0 + tid;
      const int64_t p = base + x;
      // p is a component root of size s*: a local root (its label names
      // itself) whose node is its own parent
      bool hit = false;
      if (x < J.w && J.lab[p] == (((y & (CT - 1)) << 5) | (x & (CT - 1))))
        hit = J.node[2 * p] == (int)p && comp_size(J, p) == sstar;
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

// The filtered map (and, when asked for, every pixel's component label),
// kFilterTiles 32x32 tiles per CTA.  Thread t holds eight pixels of one tile
// row; the tile's pixels first mark the local roots they refer to, then each
// marked local root is resolved once (its node points straight at its
// component root R after counting; R's component stays unless it is smaller
// than s*, or of size s* with a label below T), all of them in parallel, and
// the pixels take their local root's result from shared memory.
constexpr int kFilterTiles = 2;
__global__ void __launch_bounds__(256) k_cc_filter(const CcaJob* __restrict__ jobs) {
  constexpr int kMark = -2;
  __shared__ int s_R[kFilterTiles][CT * CT];          // component root per local root (-1: unused)
  __shared__ uint8_t s_keep[kFilterTiles][CT * CT];
  const CcaJob J = jobs[blockIdx.z];
  const int w = J.w, h = J.h;
  const int ty0 = blockIdx.y * CT;
  if (blockIdx.x * kFilterTiles * CT >= w || ty0 >= h) return;
  const uint32_t sstar = (uint32_t)J.cut[2];
  const long long T = J.cut[4];
  const int tid = threadIdx.x, tt = tid >> 7, ly = (tid >> 2) & (CT - 1), c8 = (tid & 3) * 8;
  const int tx0 = (blockIdx.x * kFilterTiles + tt) * CT, x0 = tx0 + c8, y = ty0 + ly;
  for (int i = tid; i < kFilterTiles * CT * CT; i += blockDim.x) (&s_R[0][0])[i] = -1;
  // this thread's eight labels (one 16-byte load where the row allows it)
  uint16_t li[8];
  const int64_t p0 = (int64_t)y * w + x0;
  const bool inside = y < h && x0 + 8 <= w;
  const bool vec = inside && (w & 7) == 0 && (reinterpret_cast<uintptr_t>(J.lab) & 15) == 0;
  if (vec) {
    const uint4 v = *reinterpret_cast<const uint4*>(J.lab + p0);
    const uint32_t wd[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < 8; ++j) li[j] = (uint16_t)(wd[j >> 1] >> (16 * (j & 1)));
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j) li[j] = (y < h && x0 + j < w) ? J.lab[p0 + j] : kOffMap;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < 8; ++j)
    if (li[j] != kOffMap && SB_CHECK(li[j] < CT * CT, 307u)) s_R[tt][li[j]] = kMark;
  __syncthreads();
  for (int i = tid; i < kFilterTiles * CT * CT; i += blockDim.x) {
    if ((&s_R[0][0])[i] != kMark) continue;
    const int ti = i >> 10, l = i & (CT * CT - 1);
    const int64_t g = (int64_t)(ty0 + (l >> 5)) * w + (blockIdx.x * kFilterTiles + ti) * CT + (l & (CT - 1));
    int R = J.node[2 * g];
    if (!SB_CHECK(R >= 0 && R < w * h, 308u)) R = -1;
    uint8_t k = 0;
    if (R >= 0) {
      const uint32_t sz = comp_size(J, R);
      k = sz < sstar || (sz == sstar && (long long)R < T) ? 0 : 1;
    }
    (&s_R[0][0])[i] = R;
    (&s_keep[0][0])[i] = k;
  }
  __syncthreads();
  if (y >= h || x0 >= w) return;
  uint32_t o[2] = {0u, 0u};
  int R[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const bool on = li[j] != kOffMap && li[j] < CT * CT;
    R[j] = on ? s_R[tt][li[j]] : -1;
    o[j >> 2] |= (uint32_t)(on ? s_keep[tt][li[j]] : 0) << (8 * (j & 3));
  }
  if (vec && (reinterpret_cast<uintptr_t>(J.out) & 7) == 0) {
    *reinterpret_cast<uint2*>(J.out + p0) = make_uint2(o[0], o[1]);
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (x0 + j < w) J.out[p0 + j] = (uint8_t)(o[j >> 2] >> (8 * (j & 3)));
  }
  if (J.labels_out) {
    if (vec && (reinterpret_cast<uintptr_t>(J.labels_out) & 15) == 0) {
      int4* lo = reinterpret_cast<int4*>(J.labels_out + p0);
      lo[0] = make_int4(R[0], R[1], R[2], R[3]);
      lo[1] = make_int4(R[4], R[5], R[6], R[7]);
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (x0 + j < w) J.labels_out[p0 + j] = R[j];
    }
  }
}

void launch_cca(const CcaJob* jobs, int n_jobs, int max_w, int max_h, uint32_t* dev_err, cudaStream_t s) {
  if (n_jobs <= 0) return;
  const int tiles_x = (max_w + CT - 1) / CT, tiles_y = (max_h + CT - 1) / CT;
  k_cca_local<<<dim3((tiles_x + kCcaWarps - 1) / kCcaWarps, tiles_y, n_jobs), kCcaWarps * 32, 0, s>>>(jobs, dev_err);
  k_cca_merge<<<dim3((tiles_x + kMergeTiles - 1) / kMergeTiles, tiles_y, n_jobs), 128, 0, s>>>(jobs, dev_err);
}

void launch_cc_filter(const CcaJob* jobs, int n_jobs, int max_w, int max_h, uint32_t* dev_err, cudaStream_t s) {
  if (n_jobs <= 0) return;
  const int64_t n = (int64_t)max_w * max_h;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int tiles_x = (max_w + CT - 1) / CT;
  k_cc_count<<<dim3((tiles_x + kCountTiles - 1) / kCountTiles, (max_h + CT - 1) / CT, n_jobs), 256, 0, s>>>(jobs, dev_err);
  // root-list passes: roots are few; one CTA per 2048 pixels of a job, at most one
  // per SM, and four waves of the batch in all
  const int64_t per_job = std::min<int64_t>((n + 2047) / 2048, sms);
  const int rpj = (int)std::max<int64_t>(1, std::min<int64_t>(per_job, (4 * 8 * (int64_t)sms + n_jobs - 1) / n_jobs));
  k_cc_hist<<<dim3(rpj, n_jobs), 256, 0, s>>>(jobs);
  k_cc_cut<<<n_jobs, 1024, 0, s>>>(jobs);
  k_cc_rowcount<<<dim3(rpj, n_jobs), 256, 0, s>>>(jobs);
  k_cc_select<<<n_jobs, 1024, 0, s>>>(jobs);
  k_cc_filter<<<dim3((tiles_x + kFilterTiles - 1) / kFilterTiles, (max_h + CT - 1) / CT, n_jobs), 256, 0, s>>>(jobs);
}

SB_CHECKS_UNIT(cca)

}  // namespace sb
