// Depth-based selective blurring (Section III, Eq. 1 and 2).
//
// The normalised 2-D Gaussian h(n1, n2) = g(n1) g(n2) with g the normalised
// 1-D Gaussian, so the blur is two FP32 passes over a shared-memory tile:
// a horizontal pass over the input rows the tile needs (replicated edges),
// then a vertical pass.  Each thread produces 16 consecutive outputs per
// pass, sliding a 16-value register window over the input so that every
// shared-memory load feeds 16 FMAs (the tap is a warp-uniform broadcast).
// Only pixels whose disparity lies in no range of interest take the blurred
// value; the rest are copied, and a tile with no such pixel is copied as is.
#include "sb_common.cuh"

namespace sb {

namespace {
constexpr int BX = 64;    // output columns per tile
constexpr int BY = 128;   // output rows per tile
constexpr int OB = 16;    // outputs per thread per pass (register window)
constexpr int kBlurThreads = 256;

__host__ __device__ inline int rup16(int v) { return (v + 15) & ~15; }

__device__ __forceinline__ bool in_focus(uint16_t d, const BlurJob& J) {
  for (int i = 0; i < J.n_ranges; ++i)
    if ((int)d >= J.lo[i] && (int)d <= J.hi[i]) return true;
  return false;
}
}  // namespace

// shared memory: taps (padded to a multiple of 16, zeros after 2R+1) and
// the horizontal results as float [(BY + nt)][BX], then the input tile of
// one channel as bytes [(BY + nt)][(BX + nt)] (2R halo plus padding).
int blur_smem_bytes(int R) {
  const int nt = rup16(2 * R + 1);
  const int iw = BX + nt, ih = BY + nt;
  return (nt + ih * BX) * 4 + iw * ih + 16;
}

namespace {
// exact u8 -> float: 2^23 + b as a float, minus 2^23
__device__ __forceinline__ float u8f(uint8_t b) { return __int_as_float(0x4B000000 | b) - 8388608.0f; }
}  // namespace

__global__ void __launch_bounds__(kBlurThreads) k_blur(const BlurJob* __restrict__ jobs) {
  extern __shared__ __align__(16) float fsm[];
  __shared__ int s_any;
  const BlurJob J = jobs[blockIdx.z];
  const int w = J.w, h = J.h, R = J.R;
  const int tx0 = blockIdx.x * BX, ty0 = blockIdx.y * BY;
  if (tx0 >= w || ty0 >= h) return;
  const int tid = threadIdx.x;
  const int ox = min(BX, w - tx0), oy = min(BY, h - ty0);

  // is any pixel of the tile blurred?
  if (tid == 0) s_any = 0;
  __syncthreads();
  int any = 0;
  for (int t = tid; t < ox * oy; t += kBlurThreads) {
    const int y = ty0 + t / ox, x = tx0 + t % ox;
    if (!in_focus(J.disp[(int64_t)y * w + x], J)) { any = 1; break; }
  }
  if (any) s_any = 1;
  __syncthreads();
  if (!s_any) {
    for (int t = tid; t < ox * oy * 3; t += kBlurThreads) {
      const int px = t / 3, ch = t % 3;
      const int64_t p = (int64_t)(ty0 + px / ox) * w + tx0 + px % ox;
      J.out[3 * p + ch] = J.rgb[3 * p + ch];
    }
    return;
  }

  const int nt = rup16(2 * R + 1);            // padded tap count
  const int iw = BX + nt, ih = BY + nt;       // input tile (covers 2R halo + padding)
  float* s_tap = fsm;
  float* s_h = s_tap + nt;
  uint8_t* s_in = reinterpret_cast<uint8_t*>(s_h + ih * BX);
  for (int t = tid; t < nt; t += kBlurThreads) s_tap[t] = t <= 2 * R ? J.taps[t] : 0.0f;

  for (int ch = 0; ch < 3; ++ch) {
    __syncthreads();
    // stage the input channel: tile rows ty0 - R .. and columns tx0 - R .., edges replicated
    for (int t = tid; t < iw * ih; t += kBlurThreads) {
      const int i = t / iw, j = t % iw;
      const int y = min(max(ty0 - R + i, 0), h - 1), x = min(max(tx0 - R + j, 0), w - 1);
      s_in[t] = J.rgb[((int64_t)y * w + x) * 3 + ch];
    }
    __syncthreads();
    // horizontal pass: rows 0..BY+2R-1 (+ padding rows), 16 outputs per task
    {
      const int tasks_per_row = BX / OB;
      const int rows = BY + nt;
      for (int task = tid; task < rows * tasks_per_row; task += kBlurThreads) {
        const int i = task / tasks_per_row, j0 = (task % tasks_per_row) * OB;
        const uint8_t* in = s_in + i * iw + j0;  // output j0+o uses in[o .. o+2R]
        float acc[OB], win[OB];
#pragma unroll
        for (int o = 0; o < OB; ++o) { acc[o] = 0.f; win[o] = u8f(in[o]); }
        for (int t = 0; t < nt; t += OB) {
#pragma unroll
          for (int u = 0; u < OB; ++u) {
            const float tp = s_tap[t + u];
#pragma unroll
            for (int o = 0; o < OB; ++o) acc[o] = fmaf(tp, win[(u + o) % OB], acc[o]);
            win[u] = u8f(in[t + u + OB]);
          }
        }
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
        float acc[OB], win[OB];
#pragma unroll
        for (int o = 0; o < OB; ++o) { acc[o] = 0.f; win[o] = hc[o * BX]; }
        for (int t = 0; t < nt; t += OB) {
#pragma unroll
          for (int u = 0; u < OB; ++u) {
            const float tp = s_tap[t + u];
#pragma unroll
            for (int o = 0; o < OB; ++o) acc[o] = fmaf(tp, win[(u + o) % OB], acc[o]);
            win[u] = hc[(t + u + OB) * BX];
          }
        }
        const int x = tx0 + col;
        if (x < w) {
#pragma unroll
          for (int o = 0; o < OB; ++o) {
            const int y = ty0 + i0 + o;
            if (y < h) {
              const int64_t p = (int64_t)y * w + x;
              uint8_t v;
              if (in_focus(J.disp[p], J)) {
                v = J.rgb[3 * p + ch];
              } else {
                const int q = __float2int_rd(acc[o] + 0.5f);
                v = (uint8_t)min(max(q, 0), 255);
              }
              J.out[3 * p + ch] = v;
            }
          }
        }
      }
    }
  }
}

void launch_blur(const BlurJob* jobs, int n_jobs, int max_w, int max_h, int max_R, cudaStream_t s) {
  if (n_jobs <= 0) return;
  const int smem = blur_smem_bytes(max_R);
  cudaFuncSetAttribute(k_blur, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  dim3 grid((max_w + BX - 1) / BX, (max_h + BY - 1) / BY, n_jobs);
  k_blur<<<grid, kBlurThreads, smem, s>>>(jobs);
}

}  // namespace sb
