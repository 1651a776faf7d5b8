// Colour space conversion with the fused 256-bin histogram, and histogram
// K-means (Section III, "Colour Space Conversion" and "Segmentation").
//
// Lightness: per pixel Y16 = (13933 lin[R] + 46871 lin[G] + 4732 lin[B] + 32768) >> 16
// with lin[c] = round(65535 * sRGB^-1(c/255)), then L = round(2.55 L*(Y16/65535)).
// The 65536-entry L table is held compressed in shared memory: one 32-bit
// entry per 16 consecutive Y16 values, the L of the first of them and the
// Y16 at which L steps up by one (L* rises by less than one level over 16
// consecutive Y16 values, which the host checks when it builds the table),
// so a pixel takes one table read and one compare.
// HBM-bound: 3 bytes in, 1 byte out per pixel, 16 pixels per thread step
// with 16-byte loads and stores.
#include "sb_common.cuh"

namespace sb {

__device__ __forceinline__ uint32_t lightness_px(uint32_t r, uint32_t g, uint32_t b, const uint16_t* s_lin,
                                                 const uint32_t* s_ct) {
  const uint32_t y = (13933u * s_lin[r] + 46871u * s_lin[g] + 4732u * s_lin[b] + 32768u) >> 16;
  const uint32_t e = s_ct[y >> 4];
  return (e & 255u) + (y >= (e >> 8) ? 1u : 0u);
}

__global__ void __launch_bounds__(256) k_lightness(const LightJob* __restrict__ jobs, const uint16_t* __restrict__ lin,
                                                   const uint32_t* __restrict__ ct) {
  __shared__ uint16_t s_lin[256];
  __shared__ __align__(16) uint32_t s_ct[4096];
  __shared__ uint32_t s_hist[8][256];
  const LightJob J = jobs[blockIdx.y];
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int i = tid; i < 256; i += 256) s_lin[i] = lin[i];
  for (int i = tid; i < 4096 / 4; i += 256) reinterpret_cast<uint4*>(s_ct)[i] = reinterpret_cast<const uint4*>(ct)[i];
  for (int i = tid; i < 8 * 256; i += 256) (&s_hist[0][0])[i] = 0;
  __syncthreads();

  const bool want_hist = J.hist != nullptr;
  const bool vec = !J.mirror && ((reinterpret_cast<uintptr_t>(J.rgb) | reinterpret_cast<uintptr_t>(J.L)) & 15) == 0;
  const int64_t n = J.n_px;
  const int64_t n16 = vec ? n / 16 : 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + tid; c < n16; c += stride) {
    const uint4* src = reinterpret_cast<const uint4*>(J.rgb + c * 48);
    uint4 a = __ldcs(src), b = __ldcs(src + 1), d = __ldcs(src + 2);
    uint32_t w[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, d.x, d.y, d.z, d.w};
    uint32_t o[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t packed = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int p = q * 4 + k;          // pixel within the 16
        const int byte0 = 3 * p;          // first byte of the pixel in the 48
        uint32_t rr = (w[byte0 >> 2] >> (8 * (byte0 & 3))) & 255u;
        uint32_t gg = (w[(byte0 + 1) >> 2] >> (8 * ((byte0 + 1) & 3))) & 255u;
        uint32_t bb = (w[(byte0 + 2) >> 2] >> (8 * ((byte0 + 2) & 3))) & 255u;
        uint32_t l = lightness_px(rr, gg, bb, s_lin, s_ct);
        if (want_hist) atomicAdd(&s_hist[warp][l], 1u);
        packed |= l << (8 * k);
      }
      o[q] = packed;
    }
    __stcs(reinterpret_cast<uint4*>(J.L) + c, make_uint4(o[0], o[1], o[2], o[3]));
  }
  // scalar tail (and the whole image when the pointers are not 16-byte aligned,
  // or when the rows are written mirrored)
  for (int64_t p = n16 * 16 + (int64_t)blockIdx.x * blockDim.x + tid; p < n; p += stride) {
    uint32_t l = lightness_px(J.rgb[3 * p], J.rgb[3 * p + 1], J.rgb[3 * p + 2], s_lin, s_ct);
    if (want_hist) atomicAdd(&s_hist[warp][l], 1u);
    int64_t q = p;
    if (J.mirror) {   // pixel x of row y goes to w-1-x
      const int64_t y = p / J.w;
      q = y * J.w + (J.w - 1 - (p - y * J.w));
    }
    J.L[q] = (uint8_t)l;
  }
  if (want_hist) {
    __syncthreads();
    for (int i = tid; i < 256; i += 256) {
      uint32_t t = 0;
#pragma unroll
      for (int w8 = 0; w8 < 8; ++w8) t += s_hist[w8][i];
      if (t) atomicAdd(&J.hist[i], t);
    }
  }
}

void launch_lightness(const LightJob* jobs, int n_jobs, int blocks_per_job, const uint16_t* lin,
                      const uint32_t* ct, cudaStream_t s) {
  if (n_jobs <= 0) return;
  dim3 grid(blocks_per_job, n_jobs);
  k_lightness<<<grid, 256, 0, s>>>(jobs, lin, ct);
}

__global__ void __launch_bounds__(256) k_labels(const LabelJob* __restrict__ jobs) {
  __shared__ uint8_t s_lut[256];
  const LabelJob J = jobs[blockIdx.y];
  s_lut[threadIdx.x] = J.lut[threadIdx.x];
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < J.n_px; p += stride) J.labels[p] = s_lut[J.L[p]];
}

// 256-bin histogram of an 8-bit image (hist must be zeroed).
__global__ void __launch_bounds__(256) k_histogram_u8(const uint8_t* __restrict__ L, int64_t n, uint32_t* hist) {
  __shared__ uint32_t s_hist[8][256];
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int i = tid; i < 8 * 256; i += 256) (&s_hist[0][0])[i] = 0;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + tid; p < n; p += stride) atomicAdd(&s_hist[warp][L[p]], 1u);
  __syncthreads();
  uint32_t t = 0;
#pragma unroll
  for (int w8 = 0; w8 < 8; ++w8) t += s_hist[w8][tid];
  if (t) atomicAdd(&hist[tid], t);
}

void launch_histogram_u8(const uint8_t* L, int64_t n, uint32_t* hist, cudaStream_t s) {
  int blocks = (int)((n + 256 * 16 - 1) / (256 * 16));
  blocks = blocks < 1 ? 1 : (blocks > 592 ? 592 : blocks);
  k_histogram_u8<<<blocks, 256, 0, s>>>(L, n, hist);
}

void launch_labels(const LabelJob* jobs, int n_jobs, int blocks_per_job, cudaStream_t s) {
  if (n_jobs <= 0) return;
  k_labels<<<dim3(blocks_per_job, n_jobs), 256, 0, s>>>(jobs);
}

// Histogram K-means: one CTA of 256 threads per image, thread b owns bin b.
// FP64 with explicit round-to-nearest intrinsics so no multiply-add is fused
// (the CPU computes the same expressions in the same order).  A cluster's
// pixel count and sum of lightness are integers, so the order in which they
// are added does not change them: each warp sums the bins of every cluster it
// holds with redux.sync, and one lane per (warp, cluster) adds the result in
// shared memory (at most eight adds to one address, instead of one per bin).
__global__ void __launch_bounds__(256) k_kmeans(const KmeansJob* __restrict__ jobs) {
  __shared__ double s_c[256];
  __shared__ unsigned long long s_num[256], s_den[256];
  __shared__ int s_lmin, s_lmax;
  const KmeansJob J = jobs[blockIdx.x];
  const int b = threadIdx.x, K = J.k, lane = b & 31;
  const uint32_t hb = J.hist[b];
  if (b == 0) { s_lmin = 256; s_lmax = -1; }
  __syncthreads();
  {
    const int wmin = (int)__reduce_min_sync(0xffffffffu, hb ? (unsigned)b : 256u);
    const int wmax = (int)__reduce_max_sync(0xffffffffu, hb ? (unsigned)b + 1u : 0u) - 1;
    if (lane == 0 && wmax >= 0) { atomicMin(&s_lmin, wmin); atomicMax(&s_lmax, wmax); }
  }
  __syncthreads();
  const int lmin = s_lmin, lmax = s_lmax;
  if (lmax < 0) {  // empty image
    if (b < K) J.centroids[b] = 0.0;
    J.lut[b] = 0;
    if (b == 0 && J.iters) *J.iters = 0;
    return;
  }
  if (b < K) {
    double t = __dmul_rn((double)b + 0.5, (double)(lmax - lmin));
    s_c[b] = __dadd_rn((double)lmin, __ddiv_rn(t, (double)K));
  }
  __syncthreads();
  auto assign = [&]() -> int {
    int best = 0;
    double bd = fabs(__dsub_rn((double)b, s_c[0]));
    for (int k = 1; k < K; ++k) {
      double dk = fabs(__dsub_rn((double)b, s_c[k]));
      if (dk < bd) { bd = dk; best = k; }
    }
    return best;
  };
  // exact sum of v over the lanes where `in` (v < 2^39: 24-bit pieces, so no
  // 32-bit partial sum of 32 lanes overflows)
  auto warp_sum = [&](uint64_t v, bool in) -> unsigned long long {
    const unsigned lo = in ? (unsigned)(v & 0xFFFFFFu) : 0u, hi = in ? (unsigned)(v >> 24) : 0u;
    return ((unsigned long long)__reduce_add_sync(0xffffffffu, hi) << 24) + __reduce_add_sync(0xffffffffu, lo);
  };
  int a = assign();
  int it = 0;
  while (it < J.max_iter) {
    ++it;
    if (b < K) { s_num[b] = 0ull; s_den[b] = 0ull; }
    __syncthreads();
    for (unsigned todo = __ballot_sync(0xffffffffu, hb != 0); todo;) {   // clusters this warp holds
      const int k = __shfl_sync(0xffffffffu, a, __ffs(todo) - 1);
      const bool in = hb != 0 && a == k;
      const unsigned grp = __ballot_sync(0xffffffffu, in);
      const unsigned long long num = warp_sum((uint64_t)hb * (uint64_t)b, in), den = warp_sum(hb, in);
      if (lane == __ffs(grp) - 1) {
        atomicAdd(&s_num[k], num);
        atomicAdd(&s_den[k], den);
      }
      todo &= ~grp;
    }
    __syncthreads();
    if (b < K && s_den[b] > 0ull) s_c[b] = __ddiv_rn(__ull2double_rn(s_num[b]), __ull2double_rn(s_den[b]));
    __syncthreads();
    int a2 = assign();
    int changed = __syncthreads_or(a2 != a);
    a = a2;
    if (!changed) break;
  }
  if (b < K) J.centroids[b] = s_c[b];
  J.lut[b] = (uint8_t)a;
  if (b == 0 && J.iters) *J.iters = it;
}

void launch_kmeans(const KmeansJob* jobs, int n_jobs, cudaStream_t s) {
  if (n_jobs <= 0) return;
  k_kmeans<<<n_jobs, 256, 0, s>>>(jobs);
}

SB_CHECKS_UNIT(segment)

}  // namespace sb
