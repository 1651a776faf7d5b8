// Boundary SAD without any device allocation.
//
// sb_boundary_sad needs scratch memory (one 32-bit argmin key per pixel and
// the launch's job descriptors), which a context obtains with cudaMalloc.
// Some callers cannot allocate device memory at all: a plug-in running inside
// a host application that owns every device byte through its own pool, or a
// real-time video loop that must never hit cudaMalloc (it can synchronise the
// device and stall the frame).  This entry point serves them: its scratch is
// the file-scope array below, reserved once when the library is loaded on a
// GPU and held until the process exits.  The caller still passes its inputs
// and outputs.  Every call shares the array, so calls that overlap on the GPU
// (different streams, or different host threads) race with each other.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "../../include/sb.h"
#include "sb_common.cuh"

using namespace sb;

namespace {

constexpr size_t kKeyBytes = (size_t)SB_STATIC_MAX_PIXELS * 4;  // one uint32 key per pixel
constexpr size_t kDescBytes = 256 << 10;                         // job + work items of one call
constexpr int kMaxDevices = 128;

// The scratch.  In host code this name is only a stand-in for the device
// array, never a device address: host code must use the address returned by
// cudaGetSymbolAddress for the current device.
static __device__ __align__(256) uint8_t g_sad_scratch[kKeyBytes + kDescBytes];

uint8_t* g_scratch_addr[kMaxDevices] = {};
std::mutex g_setup_mu;

sb_status report(char* errbuf, size_t len, sb_status st, const char* msg) {
  if (errbuf && len) {
    strncpy(errbuf, msg, len - 1);
    errbuf[len - 1] = 0;
  }
  return st;
}

}  // namespace

extern "C" sb_status sb_boundary_sad_static(const uint8_t* L_left, const uint8_t* L_right, const uint8_t* boundary,
                                            int32_t w, int32_t h, int32_t max_disp, int32_t block, int32_t variant,
                                            uint16_t* disp, uint32_t* cost, void* cuda_stream, char* errbuf,
                                            size_t errbuf_len) {
  char msg[256];
  if (errbuf && errbuf_len) errbuf[0] = 0;
  if (!L_left || !L_right || !boundary || !disp)
    return report(errbuf, errbuf_len, SB_ERR_INVALID_ARG, "null input or output pointer");
  if (block < 1 || block > 63 || (block & 1) == 0 || max_disp < 0 || max_disp > 1023 || w < max_disp + block + 1 ||
      h < block) {
    snprintf(msg, sizeof msg, "bad geometry: %dx%d image, max_disp %d, block %d (block odd in [1,63], "
             "max_disp in [0,1023], w >= max_disp+block+1, h >= block)", w, h, max_disp, block);
    return report(errbuf, errbuf_len, SB_ERR_INVALID_ARG, msg);
  }
  if ((int64_t)w * h > (int64_t)SB_STATIC_MAX_PIXELS) {
    snprintf(msg, sizeof msg, "image of %lld pixels exceeds the static scratch limit of %d pixels",
             (long long)w * h, SB_STATIC_MAX_PIXELS);
    return report(errbuf, errbuf_len, SB_ERR_INVALID_ARG, msg);
  }
  if (variant < SB_SAD_AUTO || variant > SB_SAD_BOXSUM)
    return report(errbuf, errbuf_len, SB_ERR_INVALID_ARG, "unknown SAD variant");
  cudaStream_t s = (cudaStream_t)cuda_stream;

  // set-up, once per device with that device current: the scratch's device address
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    snprintf(msg, sizeof msg, "cudaGetDevice: %s", cudaGetErrorString(e));
    return report(errbuf, errbuf_len, SB_ERR_CUDA, msg);
  }
  uint8_t* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_sad_scratch);
      if (e != cudaSuccess || !p) {
        snprintf(msg, sizeof msg, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        return report(errbuf, errbuf_len, SB_ERR_CUDA, msg);
      }
      g_scratch_addr[dev] = (uint8_t*)p;
    }
    base = g_scratch_addr[dev];
  }
  uint32_t* key = (uint32_t*)base;
  uint8_t* desc = base + kKeyBytes;

  // descriptors: one job (and, at kCountOff, the boundary map, its size and a
  // zeroed count for the device-side variant choice; at kQueueOff the zeroed
  // work cursor of the box-sum kernel), then the box-sum work items (strip x
  // disparity chunk x row band)
  const int r = (block - 1) / 2;
  constexpr size_t kCountOff = 192, kQueueOff = 224;   // count block: map, size, count; queue: work cursor
  static_assert(sizeof(SadJob) <= kCountOff, "job descriptor overlaps the count block");
  SadJob job{L_left, L_right, boundary, key, disp, cost, w, h, max_disp, r, nullptr, -1};
  bool run_direct = variant == SB_SAD_DIRECT, run_box = variant == SB_SAD_BOXSUM;
  if (variant == SB_SAD_AUTO) {   // same cost model as the context path, decided from the map's own count
    job.nb_direct_max = sad_direct_limit(w, h, max_disp, block);
    job.nb = job.nb_direct_max >= 0 ? (const int64_t*)(desc + kCountOff + 16) : nullptr;
    run_direct = job.nb_direct_max >= 0;
    run_box = true;
  } else {
    job.nb_direct_max = run_direct ? 1 : -1;
  }
  const int64_t npx = (int64_t)w * h, zero = 0;
  std::vector<uint8_t> blob(256, 0);
  memcpy(blob.data(), &job, sizeof job);
  memcpy(blob.data() + kCountOff, &boundary, sizeof boundary);
  memcpy(blob.data() + kCountOff + 8, &npx, 8);
  memcpy(blob.data() + kCountOff + 16, &zero, 8);
  int n_items = 0;
  if (run_box) {
    const int xo0 = max_disp + r, xo1 = w - 1 - r, yo0 = r, yo1 = h - 1 - r;
    const int rows = yo1 - yo0 + 1, ncols = xo1 - xo0 + 1;
    const int TX = sad_boxsum_strip(r);
    const int64_t base_items = (int64_t)((ncols + TX - 1) / TX) * ((max_disp + 1 + kSadChunk - 1) / kSadChunk);
    int bands = (int)std::max<int64_t>(1, (888 + base_items - 1) / base_items);
    bands = std::min(bands, std::max(1, rows / std::max(8 * r, 64)));
    for (int b = 0; b < bands; ++b) {
      const int ya = yo0 + (int)((int64_t)rows * b / bands), yb = yo0 + (int)((int64_t)rows * (b + 1) / bands) - 1;
      if (ya > yb) continue;
      for (int x0 = xo0; x0 <= xo1; x0 += TX)
        for (int d0 = 0; d0 <= max_disp; d0 += kSadChunk) {
          SadItem it{0, x0, d0, ya, yb};
          const size_t off = blob.size();
          blob.resize(off + sizeof it);
          memcpy(blob.data() + off, &it, sizeof it);
          ++n_items;
        }
    }
  }
  if (blob.size() > kDescBytes) return report(errbuf, errbuf_len, SB_ERR_UNSUPPORTED, "too many work items");

  // the keys must start at the largest value: the array keeps the last call's contents
  e = cudaMemsetAsync(key, 0xFF, (size_t)w * h * 4, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(desc, blob.data(), blob.size(), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    snprintf(msg, sizeof msg, "scratch set-up: %s", cudaGetErrorString(e));
    return report(errbuf, errbuf_len, SB_ERR_CUDA, msg);
  }
  const SadJob* djob = (const SadJob*)desc;
  if (run_direct && run_box)
    launch_count_nonzero((const uint8_t* const*)(desc + kCountOff), (const int64_t*)(desc + kCountOff + 8),
                         (int64_t*)(desc + kCountOff + 16), 1, s);
  if (run_box) launch_sad_boxsum(djob, (const SadItem*)(desc + 256), n_items, r, (unsigned*)(desc + kQueueOff), s);
  if (run_direct) launch_sad_direct(djob, 1, sad_direct_words(block), r, max_disp, s);
  launch_sad_finalize(djob, 1, w, h, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(msg, sizeof msg, "kernel launch: %s", cudaGetErrorString(e));
    return report(errbuf, errbuf_len, SB_ERR_CUDA, msg);
  }
  return SB_OK;
}
