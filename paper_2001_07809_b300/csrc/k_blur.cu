// Depth-based selective blurring (Section III, Eq. 1 and 2).
//
// The normalised 2-D Gaussian h(n1, n2) = g(n1) g(n2) with g the normalised
// 1-D Gaussian, so the blur is two FP32 passes over a shared-memory tile:
// a horizontal pass over the input rows the tile needs (replicated edges),
// then a vertical pass.  Each thread produces 16 consecutive outputs per
// pass, sliding a 16-value register window over the input so that every
// shared-memory load feeds 16 FMAs (the tap is a warp-uniform broadcast);
// exactly 2R+1 taps are applied (whole blocks of 16, then a predicated
// tail).  The three channels are staged together, by 16-byte cp.async copies
// of each input row's byte run, when the tile fits in shared memory.
// Only pixels whose disparity lies in no range of interest take the blurred
// value; the rest are copied, and a tile with no such pixel is copied as is.
#include <algorithm>
#include "sb_common.cuh"

namespace sb {

namespace {
constexpr int BX = 64;    // output columns per tile
// Output rows per tile (a multiple of OB), a template parameter: 112 (two
// CTAs per SM at sigma 8) or 64 (more halo rows per output row, but three
// CTAs per SM); the autotuner picks per batch shape.
constexpr int OB = 16;    // outputs per thread per pass (register window)
constexpr int kBlurThreads = 256;
constexpr int kAll3Limit = 110 * 1024;  // stage the three channels together up to this size (2 CTAs/SM)
constexpr int HS = BX + 1;               // row stride of the horizontal results: conflict-light stores


__device__ __forceinline__ bool in_focus(uint16_t d, const int* lo, const int* hi, int n) {
  for (int i = 0; i < n; ++i)
    if ((int)d >= lo[i] && (int)d <= hi[i]) return true;
  return false;
}

// exact u8 -> float: 2^23 + b as a float, minus 2^23
__device__ __forceinline__ float u8f(uint8_t b) { return __int_as_float(0x4B000000 | b) - 8388608.0f; }

// One tap of the register-window convolution at rotation offset OFF + u:
// win[(OFF + u + o) % OB] holds x[t + u + o]; afterwards the freed slot takes
// x[t + u + OB].
template <int OFF, int U, class LOAD>
__device__ __forceinline__ void conv_tap(float (&acc)[OB], float (&win)[OB], float tp, int t, LOAD x) {
#pragma unroll
  for (int o = 0; o < OB; ++o) acc[o] = fmaf(tp, win[(OFF + U + o) % OB], acc[o]);
  win[(OFF + U) % OB] = x(t + U + OB);
}

// at most 7 single taps t .. t+rem-1 at rotation offset OFF
template <int OFF, class LOAD>
__device__ __forceinline__ void conv_tail(float (&acc)[OB], float (&win)[OB], const float* tap, int t, int rem,
                                          LOAD x) {
  if (rem > 0) conv_tap<OFF, 0>(acc, win, tap[t], t, x);
  if (rem > 1) conv_tap<OFF, 1>(acc, win, tap[t + 1], t, x);
  if (rem > 2) conv_tap<OFF, 2>(acc, win, tap[t + 2], t, x);
  if (rem > 3) conv_tap<OFF, 3>(acc, win, tap[t + 3], t, x);
  if (rem > 4) conv_tap<OFF, 4>(acc, win, tap[t + 4], t, x);
  if (rem > 5) conv_tap<OFF, 5>(acc, win, tap[t + 5], t, x);
  if (rem > 6) conv_tap<OFF, 6>(acc, win, tap[t + 6], t, x);
}

// acc[o] = sum_{t < nt} tap[t] * x[o + t] for o < OB, where x(j) loads input
// j (inputs up to index nt - 1 + OB are loaded; the last OB - 1 of them only
// refill the window).  Whole blocks of 16 taps keep every window index static
// by rotating the slots; the remainder is at most one half block and 7 taps.
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
  const int rem = nt - t;
  if (rem >= 8) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float tp = tap[t + u];
#pragma unroll
      for (int o = 0; o < OB; ++o) acc[o] = fmaf(tp, win[(u + o) % OB], acc[o]);
      win[u] = x(t + u + OB);
    }
    conv_tail<8>(acc, win, tap, t + 8, rem - 8, x);
  } else {
    conv_tail<0>(acc, win, tap, t, rem, x);
  }
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(src));
}

struct BlurGeo {
  int nt, ih, hrows, iw, sr, base, all3, bytes;
};

// Shared-memory layout for radius R: taps [nt] (16-byte padded), horizontal
// results float [hrows = BY + 2R + 1][HS] (the last row is only read as a
// window refill), the blur mask [BY][BX], then the input tile: three
// interleaved channels, rows of sr bytes that start at a per-row offset of
// 0..15 bytes (the cp.async source alignment), or one channel [ih][iw].
template <int BY>
__host__ __device__ inline BlurGeo blur_geo(int R) {
  BlurGeo g;
  g.nt = 2 * R + 1;
  g.ih = BY + 2 * R;
  g.hrows = g.ih + 1;
  g.iw = BX + 2 * R + 1;
  g.sr = ((g.iw * 3 + 15 + 15) / 16) * 16;
  g.base = ((((g.nt + 3) & ~3) * 4 + g.hrows * HS * 4 + BY * BX) + 15) & ~15;
  const int three = g.base + g.ih * g.sr;
  g.all3 = three <= kAll3Limit;
  g.bytes = g.all3 ? three : g.base + g.ih * g.iw;
  return g;
}
}  // namespace

__host__ __device__ int blur_smem_bytes(int R, int by) { return by == 64 ? blur_geo<64>(R).bytes : blur_geo<112>(R).bytes; }

template <int BY>
__global__ void __launch_bounds__(kBlurThreads) k_blur(const BlurJob* __restrict__ jobs) {
  extern __shared__ __align__(16) float fsm[];
  __shared__ int s_any;
  __shared__ int s_lo[8], s_hi[8];
  __shared__ uint8_t s_off[BY + 2 * 96];   // per input row: byte offset of its run (R <= 96)
  const BlurJob J = jobs[blockIdx.z];
  const int w = J.w, h = J.h, R = J.R;
  const int tx0 = blockIdx.x * BX, ty0 = blockIdx.y * BY;
  if (tx0 >= w || ty0 >= h) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ox = min(BX, w - tx0), oy = min(BY, h - ty0);
  const int nr = J.n_ranges;
  const BlurGeo G = blur_geo<BY>(R);
  const int nt = G.nt, iw = G.iw, ih = G.ih, sr = G.sr;
  const int nch = G.all3 ? 3 : 1;
  float* s_tap = fsm;
  float* s_h = fsm + ((nt + 3) & ~3);
  uint8_t* s_mask = reinterpret_cast<uint8_t*>(s_h + G.hrows * HS);
  uint8_t* s_in = reinterpret_cast<uint8_t*>(fsm) + G.base;
  const int xs = tx0 - R;
  const bool interior = xs >= 0 && xs + iw <= w;
  const int64_t nbytes = (int64_t)w * h * 3;
  const bool fast = interior && G.all3 && ((reinterpret_cast<uintptr_t>(J.rgb) & 15) == 0);
  if (tid < 8) { s_lo[tid] = jobs[blockIdx.z].lo[tid]; s_hi[tid] = jobs[blockIdx.z].hi[tid]; }
  if (tid == 0) s_any = 0;
  // three channels, interior tile: each input row is one run of iw*3 bytes,
  // copied as the 16-byte chunks that cover it (issued before the mask so the
  // copies overlap the mask loads)
  if (fast) {
    const int nchunk = (iw * 3 + 15 + 15) / 16;
    for (int i = warp; i < ih; i += kBlurThreads / 32) {
      const int y = min(max(ty0 - R + i, 0), h - 1);
      const int64_t s0 = ((int64_t)y * w + xs) * 3, a16 = s0 & ~(int64_t)15;
      if (lane == 0) s_off[i] = (uint8_t)(s0 - a16);
      uint8_t* dst = s_in + i * sr;
      for (int c = lane; c < nchunk; c += 32) {
        const int64_t src = a16 + 16 * c;
        if (src + 16 <= nbytes) {
          cp_async16(dst + 16 * c, J.rgb + src);
        } else {
          for (int k = 0; k < 16; ++k) dst[16 * c + k] = J.rgb[min(src + k, nbytes - 1)];
        }
      }
    }
    asm volatile("cp.async.commit_group;\n" ::);
  }
  __syncthreads();
  // blur mask of the tile (1 = blurred: the disparity is in no range of interest)
  int any = 0;
#pragma unroll 7
  for (int t = tid; t < BY * BX; t += kBlurThreads) {
    const int i = t / BX, j = t % BX;  // BX is a power of two
    uint8_t m = 0;
    if (i < oy && j < ox) m = !in_focus(J.disp[(int64_t)(ty0 + i) * w + tx0 + j], s_lo, s_hi, nr);
    s_mask[t] = m;
    any |= m;
  }
  if (any) s_any = 1;
  if (fast) asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  if (!s_any) {  // nothing to blur: copy the tile (from the staged rows when there are any)
    for (int i = warp; i < oy; i += kBlurThreads / 32) {
      const int64_t row = ((int64_t)(ty0 + i) * w + tx0) * 3;
      if (fast) {
        const uint8_t* src = s_in + (i + R) * sr + s_off[i + R] + R * 3;
        for (int b = lane; b < ox * 3; b += 32) J.out[row + b] = src[b];
      } else {
        for (int b = lane; b < ox * 3; b += 32) J.out[row + b] = J.rgb[row + b];
      }
    }
    return;
  }
  for (int t = tid; t < nt; t += kBlurThreads) s_tap[t] = J.taps[t];
  // byte-wise staging (edge tiles, unaligned images, or one channel at a
  // time): channels c0 .. c0+nch-1, edges replicated, row offset 0
  auto stage = [&](int c0) {
    const int stride = nch == 3 ? sr : iw;
    for (int i = warp; i < ih; i += kBlurThreads / 32) {
      const int y = min(max(ty0 - R + i, 0), h - 1);
      uint8_t* dst = s_in + i * stride;
      const uint8_t* src_row = J.rgb + (int64_t)y * w * 3;
      if (lane == 0) s_off[i] = 0;
      for (int b = lane; b < iw * nch; b += 32) {
        const int j = nch == 3 ? b / 3 : b, c = nch == 3 ? b - 3 * j : 0;
        const int x = min(max(xs + j, 0), w - 1);
        dst[b] = src_row[x * 3 + c0 + c];
      }
    }
  };
  if (G.all3 && !fast) stage(0);
  const int stride = nch == 3 ? sr : iw;
  for (int ch = 0; ch < 3; ++ch) {
    const int c = G.all3 ? ch : 0;
    if (!G.all3) {
      __syncthreads();
      stage(ch);
    }
    __syncthreads();
    // horizontal pass: input rows 0 .. BY+2R-1, 16 outputs per task
    {
      const int tasks_per_row = BX / OB;
      for (int task = tid; task < ih * tasks_per_row; task += kBlurThreads) {
        const int i = task / tasks_per_row, j0 = (task % tasks_per_row) * OB;
        const uint8_t* in = s_in + i * stride + s_off[i] + j0 * nch + c;  // output j0+o uses in[o .. o+2R]
        float acc[OB];
        conv16(acc, s_tap, nt, [in, nch](int j) { return u8f(in[j * nch]); });
#pragma unroll
        for (int o = 0; o < OB; ++o) s_h[i * HS + j0 + o] = acc[o];
      }
    }
    __syncthreads();
    // vertical pass: 16 output rows per task, one column
    {
      const int tasks = BX * (BY / OB);
      for (int task = tid; task < tasks; task += kBlurThreads) {
        const int col = task % BX, i0 = (task / BX) * OB;
        const float* hc = s_h + i0 * HS + col;  // output row i0+o uses hc rows o .. o+2R
        float acc[OB];
        conv16(acc, s_tap, nt, [hc](int j) { return hc[j * HS]; });
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
                v = s_in[(i + R) * stride + s_off[i + R] + (col + R) * nch + c];  // the original pixel
              }
              J.out[((int64_t)(ty0 + i) * w + tx0 + col) * 3 + ch] = v;
            }
          }
        }
      }
    }
  }
}

template <int BY>
void launch_blur_by(const BlurJob* jobs, int n_jobs, int max_w, int max_h, int max_R, cudaStream_t s) {
  // every job's own layout (three channels or one) fits in the largest job's size
  int smem = 0;
  for (int R = 0; R <= max_R; ++R) smem = std::max(smem, blur_geo<BY>(R).bytes);
  cudaFuncSetAttribute(k_blur<BY>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  dim3 grid((max_w + BX - 1) / BX, (max_h + BY - 1) / BY, n_jobs);
  k_blur<BY><<<grid, kBlurThreads, smem, s>>>(jobs);
}

void launch_blur(const BlurJob* jobs, int n_jobs, int max_w, int max_h, int max_R, int by, cudaStream_t s) {
  if (n_jobs <= 0) return;
  if (by == 64)
    launch_blur_by<64>(jobs, n_jobs, max_w, max_h, max_R, s);
  else
    launch_blur_by<112>(jobs, n_jobs, max_w, max_h, max_R, s);
}

}  // namespace sb
