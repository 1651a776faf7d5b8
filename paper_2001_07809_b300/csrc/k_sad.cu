// Disparity of boundary pixels (Section III): winner-takes-all SAD over
// d = 0..D of block x block windows of L, cost O(N_b w^2 d).  Two exact
// implementations share the key encoding key = (cost << 10) | d, so the
// smallest key is the smallest cost with ties to the smallest d.
//
// Box-sum variant (dense over the domain, O(|Omega| d) with a few integer
// operations per pixel and disparity): a CTA owns a strip of TX output
// columns, a band of rows and a chunk of 32 disparities.
//   Stage A: thread t owns column c = x0 - r + t and keeps the 32 vertical
//     window sums V_d(y, c) = sum_{|i|<=r} |L(y+i, c) - R(y+i, c-d)| in
//     registers, sliding down one row per step.  Four disparities at a time:
//     one packed |L - R| of four bytes for the entering row and one for the
//     leaving row (vabsdiff4), interleaved with prmt, and two mixed-sign dp4a
//     add (entering - leaving) per disparity.  Rows are staged in a shared
//     memory ring so that every byte is read from HBM once per CTA.
//   Stage B: lanes = disparities; a warp slides the horizontal sum
//     S = sum_{|j|<=r} V(c+j) along its row segment and, at anchor pixels
//     (warp-uniform test), reduces (S << 10 | d) over the 32 lanes with
//     redux.sync and atomically keeps the minimum in the per-pixel key.
// Direct variant (for low boundary density and small blocks): a warp per
// anchor, lanes = disparities, vabsdiff4.add over the re-aligned 4-byte
// words of each window row.
#include "sb_common.cuh"

namespace sb {

namespace {
constexpr int kThreads = 256;
constexpr int kGroup = 4;        // rows per Stage A -> Stage B hand-off
constexpr int kVsColBytes = 64;  // 32 disparities x uint16
constexpr int kRowBytes = 576;   // staged bytes per row: 256 L + up to 320 R

__device__ __forceinline__ uint32_t dp4a_us(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("dp4a.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

__device__ __forceinline__ int vs_off(int g, int col, int lane) {
  return g * (kThreads * kVsColBytes) + col * kVsColBytes + 16 * ((lane >> 3) ^ ((col >> 1) & 3)) + 2 * (lane & 7);
}

__device__ __forceinline__ int floor4(int v) { return v >= 0 ? (v & ~3) : -(((-v) + 3) & ~3); }
}  // namespace

__host__ __device__ int sad_boxsum_strip(int r) { return (kThreads - 2 * r) & ~7; }

__global__ void __launch_bounds__(kThreads, 2) k_sad_boxsum(const SadJob* __restrict__ jobs,
                                                            const SadItem* __restrict__ items) {
  extern __shared__ __align__(16) uint8_t smem[];
  const SadItem it = items[blockIdx.x];
  const SadJob J = jobs[it.job];
  const int r = J.r, D = J.D, w = J.w;
  const int ring = 2 * r + 1 + kGroup;
  uint8_t* s_ring = smem;                                 // ring rows of kRowBytes
  uint8_t* s_zero = smem + ring * kRowBytes;              // one zero row
  uint8_t* s_vs = s_zero + kRowBytes;                     // kGroup x 256 columns x 64 B
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int TX = sad_boxsum_strip(r);
  const int NC = TX + 2 * r;
  const int x0 = it.x0, d0 = it.d0;
  const int xo0 = D + r, xo1 = w - 1 - r;                 // Omega columns
  const int cstart = x0 - r;                              // strip column 0
  const int rbase = floor4(cstart - d0 - 31);             // first staged R byte (4-aligned)
  const int y_first = it.y0;                              // first output row of the band (>= r)
  const int y_last = it.y1;                               // last output row (inclusive)

  for (int i = tid; i < kRowBytes / 4; i += kThreads) reinterpret_cast<uint32_t*>(s_zero)[i] = 0u;

  // Stage A state
  uint32_t V[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) V[k] = 0u;
  const int c = cstart + tid;
  const int rel = (c - d0 - 31) - rbase;                  // >= 0 by construction
  const int q = rel >> 2, sh = (rel & 3) * 8;

  // virtual output rows run from y_first - 2r (warm-up) to y_last
  for (int yg = y_first - 2 * r; yg <= y_last; yg += kGroup) {
    const int ng = min(kGroup, y_last - yg + 1);
    __syncthreads();  // previous readers of the ring slots being refilled are done
    // stage entering rows yin = yg + k + r for k < ng
    for (int k = 0; k < ng; ++k) {
      const int yin = yg + k + r;
      uint8_t* row = s_ring + ((yin % ring + ring) % ring) * kRowBytes;
      const uint8_t* gl = J.Ll + (int64_t)yin * w;
      const uint8_t* gr = J.Lr + (int64_t)yin * w;
      for (int i = tid; i < kRowBytes; i += kThreads) {
        uint8_t v = 0;
        if (i < 256) {
          const int x = cstart + i;
          if (x >= 0 && x < w) v = gl[x];
        } else {
          const int x = rbase + (i - 256);
          if (x >= 0 && x < w) v = gr[x];
        }
        row[i] = v;
      }
    }
    __syncthreads();
    // Stage A: ng row steps
    for (int k = 0; k < ng; ++k) {
      const int y = yg + k;  // output row of this step (virtual when < y_first)
      const int yin = y + r, yout = y - r - 1;
      const uint8_t* rin = s_ring + ((yin % ring + ring) % ring) * kRowBytes;
      const uint8_t* rout = (yout < y_first - r) ? s_zero : s_ring + ((yout % ring + ring) % ring) * kRowBytes;
      if (tid < NC) {
        const uint32_t Lin = (uint32_t)rin[tid] * 0x01010101u;
        const uint32_t Lout = (uint32_t)rout[tid] * 0x01010101u;
        const uint32_t* Rin = reinterpret_cast<const uint32_t*>(rin + 256) + q;
        const uint32_t* Rout = reinterpret_cast<const uint32_t*>(rout + 256) + q;
        uint32_t wi = Rin[0], wo = Rout[0];
#pragma unroll
        for (int g = 0; g < 8; ++g) {
          const uint32_t wi2 = Rin[g + 1], wo2 = Rout[g + 1];
          const uint32_t ri = __funnelshift_r(wi, wi2, sh), ro = __funnelshift_r(wo, wo2, sh);
          wi = wi2;
          wo = wo2;
          const uint32_t ai = __vabsdiffu4(Lin, ri), ao = __vabsdiffu4(Lout, ro);
          const uint32_t lo = __byte_perm(ai, ao, 0x5140), hi = __byte_perm(ai, ao, 0x7362);
          // byte b of word g holds disparity d0 + 31 - 4g - b
          V[31 - 4 * g] = dp4a_us(lo, 0x0000FF01u, V[31 - 4 * g]);
          V[30 - 4 * g] = dp4a_us(lo, 0xFF010000u, V[30 - 4 * g]);
          V[29 - 4 * g] = dp4a_us(hi, 0x0000FF01u, V[29 - 4 * g]);
          V[28 - 4 * g] = dp4a_us(hi, 0xFF010000u, V[28 - 4 * g]);
        }
        if (y >= y_first) {
          uint4* dst = reinterpret_cast<uint4*>(s_vs + k * (kThreads * kVsColBytes) + tid * kVsColBytes);
#pragma unroll
          for (int qd = 0; qd < 4; ++qd) {
            uint4 v;
            v.x = __byte_perm(V[8 * qd + 0], V[8 * qd + 1], 0x5410);
            v.y = __byte_perm(V[8 * qd + 2], V[8 * qd + 3], 0x5410);
            v.z = __byte_perm(V[8 * qd + 4], V[8 * qd + 5], 0x5410);
            v.w = __byte_perm(V[8 * qd + 6], V[8 * qd + 7], 0x5410);
            dst[qd ^ ((tid >> 1) & 3)] = v;
          }
        }
      }
    }
    if (yg + ng - 1 < y_first) continue;  // still warming up
    __syncthreads();
    // Stage B: warp -> (row slot, half strip); lane -> disparity
    {
      const int g = warp >> 1, half = warp & 1;
      const int y = yg + g;
      if (g < ng && y >= y_first) {
        const int HW = TX / 2;
        const int xa = half * HW, xb = min(half * HW + HW, TX);
        const int d = d0 + lane;
        const bool dvalid = d <= D;
        const uint16_t* vs = reinterpret_cast<const uint16_t*>(s_vs);
        auto V16 = [&](int col) -> uint32_t { return vs[vs_off(g, col, lane) >> 1]; };
        uint32_t S = 0;
        for (int j = 0; j <= 2 * r; ++j) S += V16(xa + j);
        const uint8_t* brow = J.bmap + (int64_t)y * w;
        uint32_t* krow = J.key + (int64_t)y * w;
        for (int xbase = xa; xbase < xb; xbase += 32) {
          const int xl = x0 + xbase + lane;
          bool anc = false;
          if (xbase + lane < xb && xl >= xo0 && xl <= xo1) anc = (xl == xo0) || (xl == xo1) || brow[xl];
          uint32_t mask = __ballot_sync(0xffffffffu, anc);
          const int n = min(32, xb - xbase);
          for (int i = 0; i < n; ++i) {
            const int xi = xbase + i;
            if (xi > xa) S += V16(xi + 2 * r) - V16(xi - 1);
            if (mask & (1u << i)) {
              const uint32_t key = dvalid ? ((S << SB_KEY_DBITS) | (uint32_t)d) : 0xFFFFFFFFu;
              const uint32_t kmin = __reduce_min_sync(0xffffffffu, key);
              if (lane == 0) atomicMin(&krow[x0 + xi], kmin);
            }
          }
        }
      }
    }
  }
}

int sad_boxsum_smem_bytes(int r) {
  const int ring = 2 * r + 1 + kGroup;
  return (ring + 1) * kRowBytes + kGroup * kThreads * kVsColBytes;
}

void launch_sad_boxsum(const SadJob* jobs, const SadItem* items, int n_items, cudaStream_t s) {
  if (n_items <= 0) return;
  static int configured = 0;
  const int smem = sad_boxsum_smem_bytes(31);
  if (!configured) {
    cudaFuncSetAttribute(k_sad_boxsum, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    configured = 1;
  }
  k_sad_boxsum<<<n_items, kThreads, smem, s>>>(jobs, items);
}

// ----------------------------------------------------------------- direct
namespace {
// 4 bytes at byte offset off (a multiple of 4) of an image of n bytes; bytes
// past the end read as 0, a base that is not 4-byte aligned uses byte loads.
__device__ __forceinline__ uint32_t load_word(const uint8_t* base, int64_t off, int64_t n) {
  if (off + 3 < n && ((reinterpret_cast<uintptr_t>(base) & 3) == 0))
    return __ldg(reinterpret_cast<const uint32_t*>(base + off));
  uint32_t v = 0;
  for (int b = 0; b < 4; ++b) v |= (off + b < n ? (uint32_t)__ldg(base + off + b) : 0u) << (8 * b);
  return v;
}
}  // namespace
// One warp per (row, 32-column chunk); every anchor of the chunk is matched
// by the whole warp, lanes = disparities d0 + lane for d0 = 0, 32, ...
__global__ void __launch_bounds__(256) k_sad_direct(const SadJob* __restrict__ jobs) {
  const SadJob J = jobs[blockIdx.z];
  const int r = J.r, D = J.D, w = J.w, B = 2 * r + 1;
  const int y = r + blockIdx.y;
  if (y > J.h - 1 - r) return;
  const int lane = threadIdx.x & 31;
  const int xo0 = D + r, xo1 = w - 1 - r;
  const int x = xo0 + (blockIdx.x * 8 + (threadIdx.x >> 5)) * 32 + lane;
  bool anc = false;
  if (x <= xo1) anc = (x == xo0) || (x == xo1) || J.bmap[(int64_t)y * w + x];
  uint32_t mask = __ballot_sync(0xffffffffu, anc);
  const int nw = (B + 3) >> 2;                         // words per window row
  const int64_t nimg = (int64_t)w * J.h;
  const uint32_t lastmask = (B & 3) ? (0xFFFFFFFFu >> (8 * (4 - (B & 3)))) : 0xFFFFFFFFu;
  while (mask) {
    const int i = __ffs(mask) - 1;
    mask &= mask - 1;
    const int xa = x - lane + i;                        // the anchor
    uint32_t best = 0xFFFFFFFFu;
    for (int d0 = 0; d0 <= D; d0 += 32) {
      const int d = d0 + lane;
      const bool dv = d <= D;
      const int dd = dv ? d : D;                        // keep addresses inside the image
      uint32_t acc = 0;
      const int lstart = xa - r, rstart = xa - r - dd;
      for (int iy = -r; iy <= r; ++iy) {
        // word-aligned absolute offsets of the window starts in this row
        const int64_t row = (int64_t)(y + iy) * w;
        const int64_t labs = row + lstart, rabs = row + rstart;
        const int64_t la = labs & ~(int64_t)3, ra = rabs & ~(int64_t)3;
        const int lsh = (int)(labs & 3) * 8, rsh = (int)(rabs & 3) * 8;
        uint32_t lp = load_word(J.Ll, la, nimg), rp = load_word(J.Lr, ra, nimg);
        for (int k = 0; k < nw; ++k) {
          const uint32_t ln = load_word(J.Ll, la + 4 * k + 4, nimg);
          const uint32_t rn = load_word(J.Lr, ra + 4 * k + 4, nimg);
          uint32_t lw = __funnelshift_r(lp, ln, lsh), rw = __funnelshift_r(rp, rn, rsh);
          lp = ln;
          rp = rn;
          if (k == nw - 1) { lw &= lastmask; rw &= lastmask; }
          asm("vabsdiff4.u32.u32.u32.add %0, %1, %2, %0;" : "+r"(acc) : "r"(lw), "r"(rw));
        }
      }
      const uint32_t key = dv ? ((acc << SB_KEY_DBITS) | (uint32_t)d) : 0xFFFFFFFFu;
      best = min(best, __reduce_min_sync(0xffffffffu, key));
    }
    if (lane == 0) J.key[(int64_t)y * w + xa] = best;
  }
}

void launch_sad_direct(const SadJob* jobs, int n_jobs, int max_w, int max_h, cudaStream_t s) {
  if (n_jobs <= 0) return;
  dim3 grid((max_w + 255) / 256, max_h, n_jobs);
  k_sad_direct<<<grid, 256, 0, s>>>(jobs);
}

// keys -> disparity (uint16, UNDET off the anchors) and cost
__global__ void __launch_bounds__(256) k_sad_finalize(const SadJob* __restrict__ jobs) {
  const SadJob J = jobs[blockIdx.y];
  const int w = J.w, h = J.h, r = J.r;
  const int xo0 = J.D + r, xo1 = w - 1 - r;
  const int64_t n = (int64_t)w * h;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
    const int y = (int)(p / w), x = (int)(p - (int64_t)y * w);
    const bool in = y >= r && y <= h - 1 - r && x >= xo0 && x <= xo1;
    const bool anc = in && (x == xo0 || x == xo1 || J.bmap[p]);
    uint16_t dv = SB_UNDET16;
    uint32_t cv = 0;
    if (anc) {
      const uint32_t k = J.key[p];
      dv = (uint16_t)(k & ((1u << SB_KEY_DBITS) - 1));
      cv = k >> SB_KEY_DBITS;
    }
    J.disp[p] = dv;
    if (J.cost) J.cost[p] = cv;
  }
}

void launch_sad_finalize(const SadJob* jobs, int n_jobs, int max_w, int max_h, cudaStream_t s) {
  if (n_jobs <= 0) return;
  const int64_t n = (int64_t)max_w * max_h;
  int bpj = (int)((n + 256 * 8 - 1) / (256 * 8));
  if (bpj > 1184) bpj = 1184;
  if (bpj < 1) bpj = 1;
  k_sad_finalize<<<dim3(bpj, n_jobs), 256, 0, s>>>(jobs);
}

}  // namespace sb
