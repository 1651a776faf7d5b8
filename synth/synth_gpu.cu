// CUDA build of the synthetic stereo generator: the same per-pixel integer
// core as synth.c (synth_core.h), one thread per pixel, so the device makes
// the same bytes as the host.  Used to create large batches of 4096x2304
// pairs directly in device memory.
#include <cuda_runtime.h>
#include <stdint.h>

#define SYNTH_FN __host__ __device__ static inline
#include "synth_core.h"

__global__ void __launch_bounds__(256) k_synth_render(synth_scene sc, const synth_layer* __restrict__ layers,
                                                      const layer_pose* __restrict__ poses, uint8_t* left,
                                                      uint8_t* right, float* gt) {
  __shared__ synth_layer s_layers[64];
  __shared__ layer_pose s_pose[64];
  for (int i = threadIdx.x; i < sc.n_layers; i += blockDim.x) {
    s_layers[i] = layers[i];
    s_pose[i] = poses[i];
  }
  __syncthreads();
  const int64_t n = (int64_t)sc.w * sc.h;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t y = p / sc.w, x = p - y * sc.w;
    synth_pixel(&sc, s_layers, s_pose, x, y, left, right, gt);
  }
}

// Render one pair into device buffers on `stream` (left/right: h*w*3 bytes,
// gt: h*w floats or NULL).  Returns 0, or a CUDA error code.
extern "C" int synth_render_device(const synth_scene* sc, uint8_t* left, uint8_t* right, float* gt, void* stream) {
  if (!sc || sc->n_layers < 1 || sc->n_layers > 64) return -1;
  cudaStream_t s = (cudaStream_t)stream;
  layer_pose pose[64];
  for (int k = 0; k < sc->n_layers; ++k) pose[k] = pose_of(&sc->layers[k], sc->frame);
  void* buf = nullptr;
  const size_t lb = sizeof(synth_layer) * sc->n_layers, pb = sizeof(layer_pose) * sc->n_layers;
  cudaError_t e = cudaMallocAsync(&buf, lb + pb + 16, s);
  if (e != cudaSuccess) return (int)e;
  uint8_t* d = (uint8_t*)buf;
  layer_pose* dp = (layer_pose*)(d + ((lb + 15) & ~(size_t)15));
  cudaMemcpyAsync(d, sc->layers, lb, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(dp, pose, pb, cudaMemcpyHostToDevice, s);
  const int64_t n = (int64_t)sc->w * sc->h;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 148 * 16) blocks = 148 * 16;
  k_synth_render<<<blocks, 256, 0, s>>>(*sc, (const synth_layer*)d, dp, left, right, gt);
  e = cudaGetLastError();
  cudaStreamSynchronize(s);   // the pose array lives on this host stack
  cudaFreeAsync(buf, s);
  return (int)e;
}
