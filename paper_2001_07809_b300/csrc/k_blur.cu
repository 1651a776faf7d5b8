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
// A second form (k_blur_strip, below) walks 64-column strips down the image
// and keeps the horizontally filtered rows in a ring, so no halo row is
// filtered twice; both forms apply the same taps in the same order.
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

// tap x value + accumulator, one channel (float) or two (float2: a packed
// FP32 FMA, two channels per instruction)
__device__ __forceinline__ float fma_t(float tp, float w, float a) { return fmaf(tp, w, a); }
__device__ __forceinline__ float2 fma_t(float tp, float2 w, float2 a) { return __ffma2_rn(make_float2(tp, tp), w, a); }
template <class T> __device__ __forceinline__ T zero_t();
template <> __device__ __forceinline__ float zero_t<float>() { return 0.f; }
template <> __device__ __forceinline__ float2 zero_t<float2>() { return make_float2(0.f, 0.f); }

// One tap of the register-window convolution at rotation offset OFF + u:
// win[(OFF + u + o) % OB] holds x[t + u + o]; afterwards the freed slot takes
// x[t + u + OB].
template <int OFF, int U, int N, class T, class LOAD>
__device__ __forceinline__ void conv_tap(T (&acc)[N], T (&win)[N], float tp, int t, LOAD x) {
#pragma unroll
  for (int o = 0; o < N; ++o) acc[o] = fma_t(tp, win[(OFF + U + o) % N], acc[o]);
  win[(OFF + U) % N] = x(t + U + N);
}

// at most 7 single taps t .. t+rem-1 at rotation offset OFF
template <int OFF, int N, class T, class LOAD>
__device__ __forceinline__ void conv_tail(T (&acc)[N], T (&win)[N], const float* tap, int t, int rem,
                                          LOAD x) {
  if (rem > 0) conv_tap<OFF, 0, N>(acc, win, tap[t], t, x);
  if (rem > 1) conv_tap<OFF, 1, N>(acc, win, tap[t + 1], t, x);
  if (rem > 2) conv_tap<OFF, 2, N>(acc, win, tap[t + 2], t, x);
  if (rem > 3) conv_tap<OFF, 3, N>(acc, win, tap[t + 3], t, x);
  if (rem > 4) conv_tap<OFF, 4, N>(acc, win, tap[t + 4], t, x);
  if (rem > 5) conv_tap<OFF, 5, N>(acc, win, tap[t + 5], t, x);
  if (rem > 6) conv_tap<OFF, 6, N>(acc, win, tap[t + 6], t, x);
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
    conv_tail<8, OB>(acc, win, tap, t + 8, rem - 8, x);
  } else {
    conv_tail<0, OB>(acc, win, tap, t, rem, x);
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
  if (ox == BX && ((reinterpret_cast<uintptr_t>(J.disp) | ((int64_t)w * 2) | (tx0 * 2)) & 15) == 0) {
    // eight disparities per 16-byte load, all of a thread's loads issued first
    constexpr int kG = (BY * BX / 8 + kBlurThreads - 1) / kBlurThreads;
    uint4 dv[kG];
#pragma unroll
    for (int k = 0; k < kG; ++k) {
      const int g = tid + k * kBlurThreads, i = g / (BX / 8), c = (g % (BX / 8)) * 8;
      dv[k] = g < BY * BX / 8 && i < oy ? *reinterpret_cast<const uint4*>(J.disp + (int64_t)(ty0 + i) * w + tx0 + c)
                                        : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int k = 0; k < kG; ++k) {
      const int g = tid + k * kBlurThreads, i = g / (BX / 8);
      if (g >= BY * BX / 8) continue;
      const uint32_t wv[4] = {dv[k].x, dv[k].y, dv[k].z, dv[k].w};
      uint32_t lo = 0, hi = 0;   // mask bytes of pixels 0..3 and 4..7
      if (i < oy)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const uint32_t m = !in_focus((uint16_t)(wv[j >> 1] >> (16 * (j & 1))), s_lo, s_hi, nr);
          if (j < 4) lo |= m << (8 * j);
          else hi |= m << (8 * (j - 4));
        }
      reinterpret_cast<uint32_t*>(s_mask)[2 * g] = lo;       // s_mask is 4-byte aligned (not 8)
      reinterpret_cast<uint32_t*>(s_mask)[2 * g + 1] = hi;
      any |= (lo | hi) != 0;
    }
  } else {
#pragma unroll 7
    for (int t = tid; t < BY * BX; t += kBlurThreads) {
      const int i = t / BX, j = t % BX;  // BX is a power of two
      uint8_t m = 0;
      if (i < oy && j < ox) m = !in_focus(J.disp[(int64_t)(ty0 + i) * w + tx0 + j], s_lo, s_hi, nr);
      s_mask[t] = m;
      any |= m;
    }
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

// ----------------------------------------------------------------- strip form
// A CTA walks down a strip of BX output columns over a band of kBandRows output
// rows, kSB output rows per step.  The horizontal results live in a ring of
// M = 2R + kSB + 1 rows per channel (the rows the vertical pass of one step
// reads), so no input row is filtered twice; the ring advances kSB rows per
// step.  Input rows for the next batch of horizontal rows are copied with
// cp.async while the current batch or the vertical pass runs.  The blur mask
// of the whole band is taken once, as bits, at the start; a step with no
// blurred pixel is copied, and a batch of horizontal rows that no remaining
// blurred step reads is skipped.
namespace {
constexpr int kSB = 32;              // output rows per step
constexpr int kStripThreads = 384;   // = kSB x 3 channels x BX/OB (horizontal) = BX x 3 x kSB/OB (vertical)
constexpr int kBandRows = 512;       // output rows per CTA
constexpr int kMaxSteps = kBandRows / kSB;
// channel c's ring starts at c * (M * HS + kChPad) floats: with the 4-float
// pad, the horizontal pass's stores of the three channels and four column
// segments a warp holds fall in different banks (2-way at most, 6-way without)
constexpr int kChPad = 4;

struct StripGeo {
  int nt, F, M, iw, sr, h_off, in_off, out_off, bytes;
};
// F: filtered rows one step reads (2R + kSB + 1); M: ring rows, F rounded up
// to a multiple of OB so that a block of OB consecutive ring rows starting at
// a multiple of OB never wraps
__host__ __device__ inline StripGeo strip_geo(int R) {
  StripGeo g;
  g.nt = 2 * R + 1;
  g.F = 2 * R + kSB + 1;
  g.M = (g.F + OB - 1) / OB * OB;
  g.iw = BX + 2 * R + 1;
  g.sr = ((g.iw * 3 + 15 + 15) / 16) * 16;
  g.h_off = ((g.nt + 3) & ~3) * 4;                                   // taps first
  g.in_off = (g.h_off + (3 * g.M * HS + 2 * kChPad) * 4 + 15) & ~15;  // then the ring, 3 channels (cp.async
                                                                     // destinations need 16-byte alignment)
  g.out_off = g.in_off + 2 * kSB * g.sr;                             // then two input buffers
  g.bytes = g.out_off + kSB * BX * 3;                                // then one step's output rows
  return g;
}
}  // namespace

// conv16 over ring rows b0 + j (mod M) of one column (hc: the column's row-0
// entry, row stride HS); b0 and M are multiples of OB, so the wrap is taken
// once per block of OB rows
// rd(k): the value (one channel, or two channels as a float2) at float
// offset k of the channel plane(s) of the ring
template <int N, class T, class RD>
__device__ __forceinline__ void conv16_ring(T (&acc)[N], const float* tap, int nt, RD rd, int b0, int M) {
  auto block = [&](int j) {   // j: a multiple of N
    int q = b0 + j;
    if (q >= M) q -= M;
    return q * HS;
  };
  T win[N];
  const int p = block(0);
#pragma unroll
  for (int o = 0; o < N; ++o) { acc[o] = zero_t<T>(); win[o] = rd(p + o * HS); }
  int t = 0;
  for (; t + N <= nt; t += N) {
    const int pn = block(t + N);
#pragma unroll
    for (int u = 0; u < N; ++u) {
      const float tp = tap[t + u];
#pragma unroll
      for (int o = 0; o < N; ++o) acc[o] = fma_t(tp, win[(u + o) % N], acc[o]);
      win[u] = rd(pn + u * HS);
    }
  }
  const int rem = nt - t;
  const int pn = block(t + N);   // the refills of the remaining taps: rows t + N .. t + N + rem - 1
  auto x = [pn, t, rd](int j) { return rd(pn + (j - t - N) * HS); };
  if (N == 16 && rem >= 8) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float tp = tap[t + u];
#pragma unroll
      for (int o = 0; o < N; ++o) acc[o] = fma_t(tp, win[(u + o) % N], acc[o]);
      win[u] = rd(pn + u * HS);
    }
    conv_tail<8 % N, N>(acc, win, tap, t + 8, rem - 8, x);
  } else {
    conv_tail<0, N>(acc, win, tap, t, rem, x);
  }
}

__host__ __device__ bool blur_strip_fits(int R) { return strip_geo(R).bytes <= 200 * 1024; }

__global__ void __launch_bounds__(kStripThreads, 2) k_blur_strip(const BlurJob* __restrict__ jobs) {
  extern __shared__ __align__(16) float fsm[];
  __shared__ uint32_t s_mbits[kBandRows * BX / 32];   // 1 = blurred
  __shared__ int s_flag[kMaxSteps];
  // bit q of s_vq[h]: output rows 16q .. 16q + 15 of the band hold a blurred pixel in
  // columns 32h .. 32h + 31 (one vertical task block of a warp: OB rows x 32 columns)
  __shared__ uint32_t s_vq[2];
  static_assert(2 * kMaxSteps <= 32 && kSB == 2 * OB, "two task blocks per step, one bit each");
  __shared__ int s_lo[8], s_hi[8];
  __shared__ uint8_t s_off[2][kSB];
  const BlurJob J = jobs[blockIdx.z];
  const int w = J.w, h = J.h, R = J.R;
  const int tx0 = blockIdx.x * BX, yb0 = blockIdx.y * kBandRows;
  if (tx0 >= w || yb0 >= h) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kWarps = kStripThreads / 32;
  const int ox = min(BX, w - tx0), rows = min(kBandRows, h - yb0);
  const int nsteps = (rows + kSB - 1) / kSB;
  const StripGeo G = strip_geo(R);
  const int nt = G.nt, M = G.M, iw = G.iw, sr = G.sr;
  float* s_tap = fsm;
  float* s_h = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(fsm) + G.h_off);
  uint8_t* s_in = reinterpret_cast<uint8_t*>(fsm) + G.in_off;
  uint8_t* s_out = reinterpret_cast<uint8_t*>(fsm) + G.out_off;   // one step's output rows (BX * 3 bytes each)
  const int xs = tx0 - R;
  const bool interior = xs >= 0 && xs + iw <= w;
  const int64_t nbytes = (int64_t)w * h * 3;
  const bool fast = interior && ((reinterpret_cast<uintptr_t>(J.rgb) & 15) == 0);
  // whole strips of a 16-byte aligned image whose rows are multiples of 16 bytes: a step's
  // output rows are assembled in shared memory (original rows copied in, blurred bytes
  // written over them) and stored 16 bytes at a time
  const bool vout = ox == BX && ((w * 3) & 15) == 0 &&
                    ((reinterpret_cast<uintptr_t>(J.rgb) | reinterpret_cast<uintptr_t>(J.out)) & 15) == 0;
  constexpr int kRowChunks = BX * 3 / 16;   // 16-byte chunks of an output row
  static_assert(kSB * kRowChunks == kStripThreads, "one output chunk per thread and step");
  if (tid < 8) { s_lo[tid] = jobs[blockIdx.z].lo[tid]; s_hi[tid] = jobs[blockIdx.z].hi[tid]; }
  for (int t = tid; t < nt; t += kStripThreads) s_tap[t] = J.taps[t];
  __syncthreads();
  // mask bits of the band (little-endian: bit j of word q is pixel 32q + j) and per-step flags
  const int nr = J.n_ranges;
  const int npix = kSB * nsteps * BX;
  uint8_t* mbytes = reinterpret_cast<uint8_t*>(s_mbits);   // byte g: pixels 8g .. 8g+7 of the band, bit j = pixel 8g+j
  const bool vec8 = ox == BX && ((reinterpret_cast<uintptr_t>(J.disp) | ((int64_t)w * 2) | (tx0 * 2)) & 15) == 0;
  if (vec8) {
    // eight disparities per 16-byte load, all of a thread's loads in flight
    constexpr int kG = (kBandRows * BX / 8 + kStripThreads - 1) / kStripThreads;   // groups per thread
    uint4 dv[kG];
#pragma unroll
    for (int k = 0; k < kG; ++k) {
      const int g = tid + k * kStripThreads, i = g / (BX / 8), c = (g % (BX / 8)) * 8;
      dv[k] = g * 8 < npix && i < rows
                  ? *reinterpret_cast<const uint4*>(J.disp + (int64_t)(yb0 + i) * w + tx0 + c)
                  : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int k = 0; k < kG; ++k) {
      const int g = tid + k * kStripThreads, i = g / (BX / 8);
      if (g * 8 >= npix) continue;
      const uint32_t wv[4] = {dv[k].x, dv[k].y, dv[k].z, dv[k].w};
      uint32_t m = 0;
      if (i < rows)
#pragma unroll
        for (int j = 0; j < 8; ++j)
          m |= (uint32_t)!in_focus((uint16_t)(wv[j >> 1] >> (16 * (j & 1))), s_lo, s_hi, nr) << j;
      mbytes[g] = (uint8_t)m;
    }
  } else {
    for (int g = tid; g * 8 < npix; g += kStripThreads) {
      const int i = g / (BX / 8), c0 = (g % (BX / 8)) * 8;
      uint32_t m = 0;
      if (i < rows)
        for (int j = 0; j < 8; ++j)
          if (c0 + j < ox) m |= (uint32_t)!in_focus(J.disp[(int64_t)(yb0 + i) * w + tx0 + c0 + j], s_lo, s_hi, nr) << j;
      mbytes[g] = (uint8_t)m;
    }
  }
  __syncthreads();
  if (tid < 2) s_vq[tid] = 0u;
  __syncthreads();
  for (int st = tid; st < nsteps; st += kStripThreads) {
    int any = 0;
    for (int q = st * kSB * (BX / 32); q < (st + 1) * kSB * (BX / 32); ++q) any |= s_mbits[q] != 0u;
    s_flag[st] = any;
  }
  if (tid < 2 * 2 * nsteps) {   // thread (q, half): task block q, columns 32 half ..
    const int q = tid >> 1, hf = tid & 1;
    uint32_t any = 0;
    for (int i = 0; i < OB; ++i) any |= s_mbits[(OB * q + i) * (BX / 32) + hf];
    if (any) atomicOr(&s_vq[hf], 1u << q);
  }
  __syncthreads();
  int any_step = 0;
  for (int st = 0; st < nsteps; ++st) any_step |= s_flag[st];
  if (!any_step) {   // nothing to blur in the band: copy it
    if (vout) {
      for (int c = tid; c < rows * kRowChunks; c += kStripThreads) {
        const int i = c / kRowChunks, q = c - i * kRowChunks;
        const int64_t at = ((int64_t)(yb0 + i) * w + tx0) * 3 + 16 * q;
        *reinterpret_cast<uint4*>(J.out + at) = *reinterpret_cast<const uint4*>(J.rgb + at);
      }
      return;
    }
    for (int i = warp; i < rows; i += kWarps) {
      const int64_t row = ((int64_t)(yb0 + i) * w + tx0) * 3;
      for (int b = lane; b < ox * 3; b += 32) J.out[row + b] = J.rgb[row + b];
    }
    return;
  }
  // horizontal batches: first the ring fill (rows yb0 - R .. yb0 + kSB + R,
  // kSB at a time), then one batch per step s >= 1 (rows y_s + R + 1 ..
  // y_s + kSB + R, read first by step s)
  const int F = G.F;
  const int nfill = (F + kSB - 1) / kSB;
  const int nbatch = nfill + nsteps - 1;
  auto batch_row0 = [&](int k) { return k < nfill ? yb0 - R + kSB * k : yb0 + kSB * (k - nfill + 1) + R + 1; };
  auto batch_rows = [&](int k) { return k < nfill ? min(kSB, F - kSB * k) : kSB; };
  // the column halves of batch k some running vertical task block reads: block q
  // (output rows yb0 + 16q .. + 15) reads rows yb0 + 16q - R .. yb0 + 16q + 15 + R
  auto batch_halves = [&](int k) -> unsigned {
    const int a = batch_row0(k) - yb0, b = a + batch_rows(k) - 1;
    // q0 = ceil((a - (OB - 1) - R) / OB), q1 = floor((b + R) / OB); a >= -R and R <= 96 keep the shifted
    // numerators positive, so the divisions round down
    const int q0 = max(0, (a - R + 16 * OB) / OB - 16), q1 = min(2 * nsteps - 1, (b + R + 16 * OB) / OB - 16);
    if (q0 > q1) return 0u;
    const uint32_t range = (q1 - q0 == 31 ? 0xffffffffu : ((2u << (q1 - q0)) - 1u)) << q0;
    return ((s_vq[0] & range) ? 1u : 0u) | ((s_vq[1] & range) ? 2u : 0u);
  };
  auto stage = [&](int k, int buf) {
    const int a = batch_row0(k), n = batch_rows(k);
    uint8_t* base = s_in + buf * kSB * sr;
    for (int i = warp; i < n; i += kWarps) {
      const int y = min(max(a + i, 0), h - 1);
      uint8_t* dst = base + i * sr;
      if (fast) {
        const int64_t s0 = ((int64_t)y * w + xs) * 3, a16 = s0 & ~(int64_t)15;
        if (lane == 0) s_off[buf][i] = (uint8_t)(s0 - a16);
        const int nchunk = (iw * 3 + 15 + 15) / 16;
        for (int c = lane; c < nchunk; c += 32) {
          const int64_t src = a16 + 16 * c;
          if (src + 16 <= nbytes) {
            cp_async16(dst + 16 * c, J.rgb + src);
          } else {
            for (int q = 0; q < 16; ++q) dst[16 * c + q] = J.rgb[min(src + q, nbytes - 1)];
          }
        }
      } else {
        if (lane == 0) s_off[buf][i] = 0;
        const uint8_t* src_row = J.rgb + (int64_t)y * w * 3;
        for (int b = lane; b < iw * 3; b += 32) {
          const int j = b / 3, c = b - 3 * j;
          dst[b] = src_row[min(max(xs + j, 0), w - 1) * 3 + c];
        }
      }
    }
    asm volatile("cp.async.commit_group;\n" ::);
  };
  auto slot = [&](int y) { return (y - (yb0 - R)) % M; };   // ring row of image row y >= yb0 - R
  // vout: the original rows of step st into s_out, as a cp.async group of its own
  // (committed before the next horizontal batch's group, so that waiting for all
  // groups but the newest completes it while that batch is still in flight)
  auto prefetch = [&](int st) {
    const int ys = yb0 + kSB * st, nrow = min(kSB, rows - kSB * st);
    const int i = tid / kRowChunks, q = tid - i * kRowChunks;
    if (i < nrow) cp_async16(s_out + i * (BX * 3) + 16 * q, J.rgb + ((int64_t)(ys + i) * w + tx0) * 3 + 16 * q);
    asm volatile("cp.async.commit_group;\n" ::);
  };
  // task = (column half, row, channel, block of OB outputs), half outermost so that
  // a warp's tasks share a half; a half no running vertical block reads is skipped
  auto hpass = [&](int k, int buf) {
    const int a = batch_row0(k), n = batch_rows(k);
    const unsigned halves = batch_halves(k);
    const uint8_t* base = s_in + buf * kSB * sr;
    constexpr int kPerRow = 3 * (BX / 2 / OB);   // tasks of one row and half
    for (int task = tid; task < n * 3 * (BX / OB); task += kStripThreads) {
      const int hf = task / (n * kPerRow), r2 = task - hf * (n * kPerRow);
      if (!((halves >> hf) & 1u)) continue;
      const int i = r2 / kPerRow, rest = r2 - i * kPerRow;
      const int ch = rest / (BX / 2 / OB), j0 = hf * (BX / 2) + (rest - ch * (BX / 2 / OB)) * OB;
      const uint8_t* in = base + i * sr + s_off[buf][i] + j0 * 3 + ch;   // output j0+o uses in[3(o .. o+2R)]
      float acc[OB];
      conv16(acc, s_tap, nt, [in](int j) { return u8f(in[j * 3]); });
      float* dst = s_h + ch * (M * HS + kChPad) + slot(a + i) * HS + j0;
#pragma unroll
      for (int o = 0; o < OB; ++o) dst[o] = acc[o];
    }
  };
  stage(0, 0);
  for (int k = 0; k < nfill; ++k) {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    if (vout && k == nfill - 1) prefetch(0);
    if (k + 1 < nbatch) stage(k + 1, (k + 1) & 1);
    else if (vout && k == nfill - 1) asm volatile("cp.async.commit_group;\n" ::);   // (an empty group)
    hpass(k, k & 1);
  }
  for (int st = 0; st < nsteps; ++st) {
    if (vout) asm volatile("cp.async.wait_group 1;\n" ::: "memory");   // this step's original rows
    __syncthreads();   // the ring holds every row step st reads
    const int ys = yb0 + kSB * st, nrow = min(kSB, rows - kSB * st);
    if (s_flag[st] && vout) {
      // vertical pass, staged-output form: thread groups 0-3 take the R and G
      // planes together (packed FP32 FMAs, float2) over blocks of 8 output
      // rows, groups 4-5 the B plane over blocks of 16 (the same registers per
      // thread), so every thread has a task
      constexpr int kPair = OB / 2;   // output rows of an R+G task
      const int col = tid % BX, rest = tid / BX;
      if (rest < 4) {
        const int i0 = rest * kPair;
        const bool need = (s_vq[col >> 5] >> (2 * st + (i0 >= OB))) & 1u;
        if (need) {
          const float* hr = s_h + col;
          const float* hg = s_h + (M * HS + kChPad) + col;
          float2 acc[kPair];
          conv16_ring(acc, s_tap, nt, [hr, hg](int k) { return make_float2(hr[k], hg[k]); }, slot(ys + i0 - R), M);
#pragma unroll
          for (int o = 0; o < kPair; ++o) {
            const int i = i0 + o;
            if (i < nrow && ((s_mbits[((kSB * st + i) * BX + col) >> 5] >> (col & 31)) & 1u)) {
              const int q0 = __float2int_rd(acc[o].x + 0.5f), q1 = __float2int_rd(acc[o].y + 0.5f);
              s_out[i * (BX * 3) + col * 3] = (uint8_t)min(max(q0, 0), 255);
              s_out[i * (BX * 3) + col * 3 + 1] = (uint8_t)min(max(q1, 0), 255);
            }
          }
        }
      } else {
        const int blk = rest - 4, i0 = blk * OB;
        const bool need = (s_vq[col >> 5] >> (2 * st + blk)) & 1u;
        if (need) {
          const float* hb = s_h + 2 * (M * HS + kChPad) + col;
          float acc[OB];
          conv16_ring(acc, s_tap, nt, [hb](int k) { return hb[k]; }, slot(ys + i0 - R), M);
#pragma unroll
          for (int o = 0; o < OB; ++o) {
            const int i = i0 + o;
            if (i < nrow && ((s_mbits[((kSB * st + i) * BX + col) >> 5] >> (col & 31)) & 1u)) {
              const int q = __float2int_rd(acc[o] + 0.5f);
              s_out[i * (BX * 3) + col * 3 + 2] = (uint8_t)min(max(q, 0), 255);
            }
          }
        }
      }
    } else if (s_flag[st]) {
      // vertical pass: task = (column, channel, block of OB output rows)
      const int col = tid % BX, rest = tid / BX, ch = rest % 3, blk = rest / 3;
      const int i0 = blk * OB;
      const int b0 = slot(ys + i0 - R);
      // a warp's tasks are 32 columns (one word of a mask row) x OB rows of one
      // channel; in the staged-output form a warp none of whose pixels is
      // blurred has nothing to write and skips its convolution
      const bool need = (s_vq[col >> 5] >> (2 * st + blk)) & 1u;
      float acc[OB];
      const float* hc = s_h + ch * (M * HS + kChPad) + col;
      if (need) conv16_ring(acc, s_tap, nt, [hc](int k) { return hc[k]; }, b0, M);
      if (vout && need) {
#pragma unroll
        for (int o = 0; o < OB; ++o) {
          const int i = i0 + o;
          if (i < nrow && ((s_mbits[((kSB * st + i) * BX + col) >> 5] >> (col & 31)) & 1u)) {
            const int q = __float2int_rd(acc[o] + 0.5f);
            s_out[i * (BX * 3) + col * 3 + ch] = (uint8_t)min(max(q, 0), 255);
          }
        }
      } else if (col < ox) {
#pragma unroll
        for (int o = 0; o < OB; ++o) {
          const int i = i0 + o;
          if (i < nrow) {
            const int bi = kSB * st + i;   // band row
            const int64_t at = ((int64_t)(ys + i) * w + tx0 + col) * 3 + ch;
            uint8_t v;
            if ((s_mbits[(bi * BX + col) >> 5] >> (col & 31)) & 1u) {
              const int q = __float2int_rd(acc[o] + 0.5f);
              v = (uint8_t)min(max(q, 0), 255);
            } else {
              v = J.rgb[at];
            }
            J.out[at] = v;
          }
        }
      }
    } else if (!vout) {
      for (int i = warp; i < nrow; i += kWarps) {
        const int64_t row = ((int64_t)(ys + i) * w + tx0) * 3;
        for (int b = lane; b < ox * 3; b += 32) J.out[row + b] = J.rgb[row + b];
      }
    }
    if (vout) {
      __syncthreads();   // the step's blurred bytes are in s_out
      const int i = tid / kRowChunks, q = tid - i * kRowChunks;
      if (i < nrow)
        *reinterpret_cast<uint4*>(J.out + ((int64_t)(ys + i) * w + tx0) * 3 + 16 * q) =
            *reinterpret_cast<const uint4*>(s_out + i * (BX * 3) + 16 * q);
    }
    const int k = nfill + st;   // the batch step st + 1 reads first
    if (k < nbatch) {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
      __syncthreads();   // batch k staged; every vertical read of the ring slots it replaces is done
      if (vout) prefetch(st + 1);   // s_out was stored before the barrier
      if (k + 1 < nbatch) stage(k + 1, (k + 1) & 1);
      else if (vout) asm volatile("cp.async.commit_group;\n" ::);   // (an empty group)
      if (batch_halves(k)) hpass(k, k & 1);
    }
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
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
  if (by == kBlurStrip && blur_strip_fits(max_R)) {
    const int smem = strip_geo(max_R).bytes;
    cudaFuncSetAttribute(k_blur_strip, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    dim3 grid((max_w + BX - 1) / BX, (max_h + kBandRows - 1) / kBandRows, n_jobs);
    k_blur_strip<<<grid, kStripThreads, smem, s>>>(jobs);
    return;
  }
  if (by == 64)
    launch_blur_by<64>(jobs, n_jobs, max_w, max_h, max_R, s);
  else
    launch_blur_by<112>(jobs, n_jobs, max_w, max_h, max_R, s);
}

SB_CHECKS_UNIT(blur)

}  // namespace sb
