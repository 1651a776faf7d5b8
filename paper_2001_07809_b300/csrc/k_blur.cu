// Depth-based selective blurring (Section III, Eq. 1 and 2).
//
// The normalised 2-D Gaussian h(n1, n2) = g(n1) g(n2) with g the normalised
// 1-D Gaussian, so the blur is two FP32 passes over a shared-memory tile:
// a horizontal pass over the input rows the tile needs (replicated edges),
// then a vertical pass.  Each thread produces 16 consecutive outputs per
// pass, sliding a 16-value register window over the input so that every
// shared-memory load feeds 16 FMAs (the tap is a warp-uniform broadcast);
// taps are padded with zeros only to a multiple of 8.  The three channels
// are staged together when the tile fits in shared memory.
// Only pixels whose disparity lies in no range of interest take the blurred
// value; the rest are copied, and a tile with no such pixel is copied as is.
#include "sb_common.cuh"

namespace sb {

namespace {
constexpr int BX = 64;    // output columns per tile
constexpr int BY = 112;   // output rows per tile (a multiple of OB)
constexpr int OB = 16;    // outputs per thread per pass (register window)
constexpr int kBlurThreads = 256;
constexpr int kAll3Limit = 110 * 1024;  // stage the three channels together up to this size (2 CTAs/SM)

__host__ __device__ inline int rup8(int v) { return (v + 7) & ~7; }

__device__ __forceinline__ bool in_focus(uint16_t d, const int* lo, const int* hi, int n) {
  for (int i = 0; i < n; ++i)
    if ((int)d >= lo[i] && (int)d <= hi[i]) return true;
  return false;
}

// exact u8 -> float: 2^23 + b as a float, minus 2^23
__device__ __forceinline__ float u8f(uint8_t b) { return __int_as_float(0x4B000000 | b) - 8388608.0f; }

// acc[o] += sum_t tap[t] * x[o + t] for o < OB, t < nt (nt a multiple of 8),
// where x(j) loads input j.  The window win holds x[t + (o..o+15)] rotated so
// that every index is static: full blocks of 16 taps, then at most one half block.
template <class LOAD>
__device__ __forceinline__ void conv16(float (&acc)[OB], const float* tap, int nt, LOAD x) {
  float win[OB];
#pragma unroll
  for (int o = 0; o < OB; ++o) { acc[o] = 0.f; win[o] = x(o); }
  int t = 0;
  for (; t + OB <= nt; t += OB) {
#pragma unroll
    for (int u = 0; u < OB; ++u) {
      const float tp = tap[t + u];
#pragma unroll
      for (int o = 0; o < OB; ++o) acc[o] = fmaf(tp, win[(u + o) % OB], acc[o]);
      win[u] = x(t + u + OB);
    }
  }
  if (t < nt) {  // half block of 8 taps
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float tp = tap[t + u];
#pragma unroll
      for (int o = 0; o < OB; ++o) acc[o] = fmaf(tp, win[(u + o) % OB], acc[o]);
      win[u] = x(t + u + OB);
    }
  }
}
}  // namespace

// shared memory: taps (2R+1 padded with zeros to nt = a multiple of 8), the
// horizontal results as float [(BY + nt)][BX], the tile's blur mask
// [BY][BX], then the input tile as bytes [(BY + nt)][(BX + nt)] x (3 channels
// interleaved, or 1 channel when three do not fit).
__host__ __device__ int blur_smem_bytes(int R, int* all3) {
  const int nt = rup8(2 * R + 1);
  const int iw = BX + nt, ih = BY + nt;  // the windows read input indices up to nt + 15
  const int base = (nt + ih * BX) * 4 + BY * BX + 16;
  const int three = base + iw * ih * 3;
  if (three <= kAll3Limit) { if (all3) *all3 = 1; return three; }
  if (all3) *all3 = 0;
  return base + iw * ih;
}
__host__ __device__ int blur_smem_bytes(int R) { return blur_smem_bytes(R, nullptr); }

__global__ void __launch_bounds__(kBlurThreads) k_blur(const BlurJob* __restrict__ jobs) {
  extern __shared__ __align__(16) float fsm[];
  __shared__ int s_any;
  __shared__ int s_lo[8], s_hi[8];
  const BlurJob J = jobs[blockIdx.z];
  const int w = J.w, h = J.h, R = J.R;
  const int tx0 = blockIdx.x * BX, ty0 = blockIdx.y * BY;
  if (tx0 >= w || ty0 >= h) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ox = min(BX, w - tx0), oy = min(BY, h - ty0);
  const int nr = J.n_ranges;
  int all3;
  blur_smem_bytes(R, &all3);
  const int nt = rup8(2 * R + 1);
  const int iw = BX + nt, ih = BY + nt;
  const int nch = all3 ? 3 : 1;
  float* s_tap = fsm;
  float* s_h = s_tap + nt;
  uint8_t* s_mask = reinterpret_cast<uint8_t*>(s_h + ih * BX);
  uint8_t* s_in = s_mask + BY * BX;
  if (tid < 8) { s_lo[tid] = J.lo[tid]; s_hi[tid] = J.hi[tid]; }
  if (tid == 0) s_any = 0;
  __syncthreads();
  // blur mask of the tile (1 = blurred: the disparity is in no range of interest)
  int any = 0;
  for (int t = tid; t < BY * BX; t += kBlurThreads) {
    const int i = t / BX, j = t % BX;  // BX is a power of two
    uint8_t m = 0;
    if (i < oy && j < ox) m = !in_focus(J.disp[(int64_t)(ty0 + i) * w + tx0 + j], s_lo, s_hi, nr);
    s_mask[t] = m;
    any |= m;
  }
  if (any) s_any = 1;
  __syncthreads();
  if (!s_any) {
    for (int i = warp; i < oy; i += kBlurThreads / 32) {
      const int64_t row = ((int64_t)(ty0 + i) * w + tx0) * 3;
      for (int b = lane; b < ox * 3; b += 32) J.out[row + b] = J.rgb[row + b];
    }
    return;
  }
  for (int t = tid; t < nt; t += kBlurThreads) s_tap[t] = t <= 2 * R ? J.taps[t] : 0.0f;
  // stage channels c0 .. c0+nch-1 of the input tile (edges replicated): rows that
  // lie inside the image columns are one contiguous run of bytes
  auto stage = [&](int c0) {
    for (int i = warp; i < ih; i += kBlurThreads / 32) {
      const int y = min(max(ty0 - R + i, 0), h - 1);
      const int xs = tx0 - R;
      uint8_t* dst = s_in + i * iw * nch;
      const uint8_t* src_row = J.rgb + (int64_t)y * w * 3;
      if (nch == 3 && xs >= 0 && xs + iw <= w) {
        const uint8_t* src = src_row + (int64_t)xs * 3;
        for (int b = lane; b < iw * 3; b += 32) dst[b] = src[b];
      } else {
        for (int b = lane; b < iw * nch; b += 32) {
          const int j = nch == 3 ? b / 3 : b, c = nch == 3 ? b - 3 * j : 0;
          const int x = min(max(xs + j, 0), w - 1);
          dst[b] = src_row[x * 3 + c0 + c];
        }
      }
    }
  };
  if (all3) stage(0);
  for (int ch = 0; ch < 3; ++ch) {
    const int c = all3 ? ch : 0;
    if (!all3) {
      __syncthreads();
      stage(ch);
    }
    __syncthreads();
    // horizontal pass: rows 0 .. BY+nt-1, 16 outputs per task
    {
      const int tasks_per_row = BX / OB;
      const int rows = BY + nt;
      for (int task = tid; task < rows * tasks_per_row; task += kBlurThreads) {
        const int i = task / tasks_per_row, j0 = (task % tasks_per_row) * OB;
        const uint8_t* in = s_in + ((i * iw) + j0) * nch + c;  // output j0+o uses in[o .. o+2R]
        float acc[OB];
        conv16(acc, s_tap, nt, [&](int j) { return u8f(in[j * nch]); });
#pragma unroll
        for (int o = 0; o < OB; ++o) s_h[i * BX + j0 + o] = acc[o];
      }
    }
    __syncthreads();
    // vertical pass: 16 output rows per task, one column
    {
      const int tasks = BX * (BY / OB);
      for (int task = tid; task < tasks; task += kBlurThreads) {
        const int col = task % BX, i0 = (task / BX) * OB;
        const float* hc = s_h + i0 * BX + col;  // output row i0+o uses hc rows o .. o+2R
        float acc[OB];
        conv16(acc, s_tap, nt, [&](int j) { return hc[j * BX]; });
        if (col < ox) {
#pragma unroll
          for (int o = 0; o < OB; ++o) {
            const int i = i0 + o;
            if (i < oy) {
              uint8_t v;
              if (s_mask[i * BX + col]) {
                const int q = __float2int_rd(acc[o] + 0.5f);
                v = (uint8_t)min(max(q, 0), 255);
              } else {
                v = s_in[((i + R) * iw + col + R) * nch + c];  // the original pixel
              }
              J.out[((int64_t)(ty0 + i) * w + tx0 + col) * 3 + ch] = v;
            }
          }
        }
      }
    }
  }
}

void launch_blur(const BlurJob* jobs, int n_jobs, int max_w, int max_h, int max_R, cudaStream_t s) {
  if (n_jobs <= 0) return;
  // every job's own layout (three channels or one) fits in the largest job's size
  int smem = 0;
  for (int R = 0; R <= max_R; ++R) smem = smem > blur_smem_bytes(R) ? smem : blur_smem_bytes(R);
  cudaFuncSetAttribute(k_blur, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  dim3 grid((max_w + BX - 1) / BX, (max_h + BY - 1) / BY, n_jobs);
  k_blur<<<grid, kBlurThreads, smem, s>>>(jobs);
}

}  // namespace sb
