// Instruction-throughput microbenchmark: the issue rate of this GPU for the
// instructions the box-sum and direct SAD kernels are built from, measured
// rather than taken from a data sheet (the roofline of an integer-bound
// kernel needs the integer rate, which no copy or GEMM benchmark gives).
//
// Each thread runs 8 independent dependency chains of one instruction for
// a fixed number of iterations over a grid of 8 CTAs of 256 threads per SM;
// throughput = instructions x lanes / kernel time (CUDA events).
#include <cuda_runtime.h>
#include <stdint.h>

namespace {
constexpr int kChains = 8;
constexpr int kIters = 4096;

template <int OP>
__global__ void __launch_bounds__(256) k_peak(uint32_t* out, uint32_t seed) {
  uint32_t a[kChains], b[kChains];
  float f[kChains];
  uint64_t f2[kChains];   // packed float pairs (fma.rn.f32x2)
#pragma unroll
  for (int i = 0; i < kChains; ++i) {
    a[i] = seed * (threadIdx.x + 1 + i);
    b[i] = seed ^ (i * 0x9e3779b9u + threadIdx.x);
    f[i] = (float)(a[i] & 255);
    asm("mov.b64 %0, {%1, %2};" : "=l"(f2[i]) : "f"(f[i]), "f"(f[i] + 1.f));
  }
  const uint32_t c = seed + 7;
  const float fb = 1.0001f;
  uint64_t fb2;
  asm("mov.b64 %0, {%1, %1};" : "=l"(fb2) : "f"(fb));
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
      if (OP == 0) asm volatile("add.u32 %0, %0, %1;" : "+r"(a[i]) : "r"(b[i]));
      if (OP == 1) asm volatile("vabsdiff4.u32.u32.u32.add %0, %1, %2, %0;" : "+r"(a[i]) : "r"(b[i]), "r"(c));
      if (OP == 2) asm volatile("fma.rn.f32 %0, %0, %1, %1;" : "+f"(f[i]) : "f"(fb));
      if (OP == 3) asm volatile("prmt.b32 %0, %0, %1, 0x5140;" : "+r"(a[i]) : "r"(b[i]));
      if (OP == 4) asm volatile("fma.rn.f32x2 %0, %0, %1, %1;" : "+l"(f2[i]) : "l"(fb2));
      if (OP == 5) asm volatile("shf.r.wrap.b32 %0, %0, %1, %2;" : "+r"(a[i]) : "r"(b[i]), "r"(c & 24u));
      if (OP == 6) asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[i]) : "r"(b[i]), "r"(c));
      if (OP == 7) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[i]) : "r"(b[i]), "r"(c));
      if (OP == 8) asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(a[i]) : "r"(b[i]), "r"(c));
      if (OP == 9) asm volatile("redux.sync.min.u32 %0, %1, 0xffffffff;" : "=r"(a[i]) : "r"(a[i] ^ b[i]));
      if (OP == 10) asm volatile("vabsdiff4.u32.u32.u32 %0.b20, %0, %1, %0;" : "+r"(a[i]) : "r"(b[i]));
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i] + (uint32_t)f[i] + (uint32_t)f2[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int OP>
int time_op(int blocks, uint32_t* out, double* per_s) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return 1;
  k_peak<OP><<<blocks, 256>>>(out, 3);   // warm-up
  cudaEventRecord(e0);
  k_peak<OP><<<blocks, 256>>>(out, 5);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cudaGetLastError() != cudaSuccess || ms <= 0.f) return 1;
  *per_s = (double)blocks * 256 * kIters * kChains / (ms * 1e-3);
  return 0;
}
}  // namespace

// rates[0..10]: thread-instructions per second of add.u32, vabsdiff4 (4 byte
// cells each), fma.f32, prmt, fma.f32x2 (two FMAs each), shf.r.wrap, lop3,
// mad.lo.u32, mad.hi.u32, redux.sync.min.u32 (per participating thread) and
// vabsdiff4 with a destination byte mask, on the current device.  Returns 0
// on success.
extern "C" int sb_peak_measure(double* rates) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  uint32_t* out = nullptr;
  const int blocks = sms * 8;
  if (cudaMalloc(&out, (size_t)blocks * 256 * 4) != cudaSuccess) return 1;
  int rc = time_op<0>(blocks, out, &rates[0]);
  rc |= time_op<1>(blocks, out, &rates[1]);
  rc |= time_op<2>(blocks, out, &rates[2]);
  rc |= time_op<3>(blocks, out, &rates[3]);
  rc |= time_op<4>(blocks, out, &rates[4]);
  rc |= time_op<5>(blocks, out, &rates[5]);
  rc |= time_op<6>(blocks, out, &rates[6]);
  rc |= time_op<7>(blocks, out, &rates[7]);
  rc |= time_op<8>(blocks, out, &rates[8]);
  rc |= time_op<9>(blocks, out, &rates[9]);
  rc |= time_op<10>(blocks, out, &rates[10]);
  cudaFree(out);
  return rc;
}
