// Boundary SAD without any device allocation.
//
// sb_boundary_sad needs scratch memory (one 32-bit argmin key per pixel and
// the launch's job and work-item descriptors), which a context obtains with
// cudaMalloc.  Some callers cannot allocate device memory at all: a plug-in
// running inside a host application that owns every device byte through its
// own pool, or a real-time video loop that must never hit cudaMalloc (it can
// synchronise the device and stall the frame).  This entry point serves them:
// its scratch is the file-scope array below, which every GPU that loads the
// library's device code holds until the process exits.  The device code is
// loaded, and the array reserved, on the first call on a device (CUDA loads
// modules lazily), so such callers make one warm-up call before their
// real-time loop.  The caller still passes its inputs and outputs.  Every call
// shares the array, so calls that overlap on the GPU (different streams, or
// different host threads) race with each other.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "../../include/sb.h"
#include "sb_common.cuh"

using namespace sb;

namespace {

constexpr size_t kKeyBytes = (size_t)SB_STATIC_MAX_PIXELS * 4;  // one uint32 key per pixel
constexpr size_t kDescBytes = 256 << 10;                         // job, counters and work items of one call
constexpr size_t kItemsOff = 256;                                // work items start here in the descriptor area
constexpr int kMaxItems = (int)((kDescBytes - kItemsOff) / sizeof(SadItem));
static_assert(kMaxItems == SB_STATIC_MAX_ITEMS, "the header's work-item limit matches the descriptor area");
constexpr size_t kCountOff = 192;   // boundary map pointer, its size, the zeroed count (device-side variant choice)
constexpr size_t kQueueOff = 224;   // zeroed work cursors of the box-sum and tail kernels
constexpr int kMaxDevices = 128;

// The scratch.  In host code this name is only a stand-in for the device
// array, never a device address: host code uses the address that
// cudaGetSymbolAddress returns in the current context.
static __device__ __align__(256) uint8_t g_sad_scratch[kKeyBytes + kDescBytes];

// Per device: the context the address was looked up in (its unique id), the
// address and the SM count.  A symbol's address belongs to a context, so a new
// context on the device (a host application's own driver context, or the
// primary context re-created after cudaDeviceReset) repeats the look-up.
struct Setup {
  unsigned long long ctx_id = 0;
  uint8_t* addr = nullptr;
  int sms = 0;
};
Setup g_setup[kMaxDevices];
std::mutex g_setup_mu;

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

sb_status report(char* errbuf, size_t len, sb_status st, const char* msg) {
  if (errbuf && len) {
    strncpy(errbuf, msg, len - 1);
    errbuf[len - 1] = 0;
  }
  return st;
}

// The id of the current context (0 when the driver entry points are missing).
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = (CtxGetCurrentFn)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (CtxGetIdFn)f;
    looked_up = true;
  }
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (get_current && get_id && get_current(&c) == CUDA_SUCCESS && c && get_id(c, &id) == CUDA_SUCCESS) return id;
  return 0;
}

// Work of one call, passed by value to the set-up kernel: the job, and the
// box-sum and tail work lists in the layout the context path builds for one
// pair (bands x strips x disparity chunks; tail: bands x strips).
struct StaticPlan {
  SadJob job;
  const uint8_t* bmap;
  int64_t npx;
  int32_t n_box, n_tail;
  int32_t xo0, yo0, rows;
  int32_t TX, strips, chunks, bands;        // box-sum items
  int32_t TT, tstrips, tbands, dt0;         // tail items
};

// Writes the descriptors into the scratch: the job at offset 0, the count
// block, zeroed work cursors, then the box-sum items and the tail items.
__global__ void k_static_setup(StaticPlan P, uint8_t* desc) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid == 0) {
    *reinterpret_cast<SadJob*>(desc) = P.job;
    *reinterpret_cast<const uint8_t**>(desc + kCountOff) = P.bmap;
    *reinterpret_cast<int64_t*>(desc + kCountOff + 8) = P.npx;
    *reinterpret_cast<int64_t*>(desc + kCountOff + 16) = 0;
    reinterpret_cast<unsigned*>(desc + kQueueOff)[0] = 0u;
    reinterpret_cast<unsigned*>(desc + kQueueOff)[1] = 0u;
  }
  SadItem* items = reinterpret_cast<SadItem*>(desc + kItemsOff);
  for (int i = tid; i < P.n_box + P.n_tail; i += gridDim.x * blockDim.x) {
    if (!SB_CHECK(i < kMaxItems, 701u)) break;   // the host rejects larger plans
    SadItem it;
    it.job = 0;
    if (i < P.n_box) {
      const int c = i % P.chunks, s = (i / P.chunks) % P.strips, b = i / (P.chunks * P.strips);
      it.x0 = P.xo0 + s * P.TX;
      it.d0 = c * kSadChunk;
      it.y0 = P.yo0 + (int)((int64_t)P.rows * b / P.bands);
      it.y1 = P.yo0 + (int)((int64_t)P.rows * (b + 1) / P.bands) - 1;
    } else {
      const int k = i - P.n_box, s = k % P.tstrips, b = k / P.tstrips;
      it.x0 = P.xo0 + s * P.TT;
      it.d0 = P.dt0;
      it.y0 = P.yo0 + (int)((int64_t)P.rows * b / P.tbands);
      it.y1 = P.yo0 + (int)((int64_t)P.rows * (b + 1) / P.tbands) - 1;
    }
    items[i] = it;
  }
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

  // the work lists, as the context path builds them for one pair
  const int r = (block - 1) / 2;
  bool run_direct = variant == SB_SAD_DIRECT, run_box = variant == SB_SAD_BOXSUM;
  int64_t nb_direct_max = run_direct ? 1 : -1;
  if (variant == SB_SAD_AUTO) {   // same cost model as the context path, decided from the map's own count
    nb_direct_max = sad_direct_limit(w, h, max_disp, block);
    run_direct = nb_direct_max >= 0;
    run_box = true;
  }
  StaticPlan P{};
  P.xo0 = max_disp + r;
  P.yo0 = r;
  P.rows = h - 2 * r;
  const int ncols = w - max_disp - 2 * r;
  const bool tail = sad_has_tail(max_disp);
  if (run_box) {
    const int dend = tail ? sad_tail_first(max_disp) : max_disp + 1;   // box-sum chunks cover d < dend
    P.TX = sad_boxsum_strip(r);
    P.strips = (ncols + P.TX - 1) / P.TX;
    P.chunks = (dend + kSadChunk - 1) / kSadChunk;
    P.bands = 1;
    P.n_box = 0;
    if (P.chunks > 0) {
      // device setup below fixes the SM count; bands are cut so one pair still fills the GPU
      P.n_box = P.strips * P.chunks;
    }
    if (tail) {
      P.TT = sad_tail_strip(r);
      P.tstrips = (ncols + P.TT - 1) / P.TT;
      P.dt0 = sad_tail_first(max_disp);
    }
  }

  // set-up, once per device and context with that device current: the
  // scratch's device address (the first call on a device also loads the
  // library's device code) and the SM count
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    snprintf(msg, sizeof msg, "cudaGetDevice: %s", cudaGetErrorString(e));
    return report(errbuf, errbuf_len, SB_ERR_CUDA, msg);
  }
  uint8_t* base = nullptr;
  int sms = 0;
  {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    Setup& S = g_setup[dev];
    const unsigned long long cid = current_context_id();
    if (!S.addr || cid == 0 || cid != S.ctx_id) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_sad_scratch);
      if (e != cudaSuccess || !p) {
        snprintf(msg, sizeof msg, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        return report(errbuf, errbuf_len, SB_ERR_CUDA, msg);
      }
      int n = 0;
      e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess || n <= 0) {
        snprintf(msg, sizeof msg, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
        return report(errbuf, errbuf_len, SB_ERR_CUDA, msg);
      }
      S.addr = (uint8_t*)p;
      S.sms = n;
      S.ctx_id = cid;
    }
    base = S.addr;
    sms = S.sms;
  }
  uint32_t* key = (uint32_t*)base;
  uint8_t* desc = base + kKeyBytes;

  if (run_box && P.n_box > 0) {
    // row bands as in the context path: enough items for three waves of the persistent
    // grid (bands of at least max(8r, 64) rows); where that leaves CTA slots idle, the
    // count (bands of at least 8 rows) that minimises (rounds) x (band rows + r)
    const int64_t target = (int64_t)sms * 2 * 3, box_slots = (int64_t)sms * 2;
    const int64_t per_target = std::max<int64_t>(1, (target + P.n_box - 1) / P.n_box);
    P.bands = (int)std::min<int64_t>(per_target, std::max(1, P.rows / std::max(8 * r, 64)));
    if ((int64_t)P.n_box * P.bands < box_slots) {
      const int cap = (int)std::min<int64_t>(per_target, std::max(1, P.rows / 8));
      int64_t best_cost = -1;
      for (int t = 1; t <= cap; ++t) {
        const int64_t c = ((int64_t)P.n_box * t + box_slots - 1) / box_slots * ((P.rows + t - 1) / t + r);
        if (best_cost < 0 || c < best_cost) { best_cost = c; P.bands = t; }
      }
    }
    P.n_box *= P.bands;
  }
  if (run_box && tail) {
    // tail bands: the count that minimises (rounds of the persistent grid, six CTAs per SM) x (rows + 2r)
    const int64_t slots = (int64_t)sms * 6;
    int64_t best = -1;
    P.tbands = 1;
    for (int t = 1; t <= 16 && t <= P.rows; ++t) {
      const int64_t rounds = ((int64_t)P.tstrips * t + slots - 1) / slots;
      const int64_t c = rounds * ((P.rows + t - 1) / t + 2 * r);
      if (best < 0 || c < best) { best = c; P.tbands = t; }
    }
    P.n_tail = P.tstrips * P.tbands;
  }
  if ((int64_t)P.n_box + P.n_tail > kMaxItems) {
    snprintf(msg, sizeof msg, "%d work items exceed the static limit of %d (a wide image with a large disparity "
             "range: the items are strips of about 200 columns times chunks of 64 disparities)",
             P.n_box + P.n_tail, kMaxItems);
    return report(errbuf, errbuf_len, SB_ERR_UNSUPPORTED, msg);
  }
  P.job = SadJob{L_left, L_right, boundary, key, disp, cost, w, h, max_disp, r,
                 variant == SB_SAD_AUTO && nb_direct_max >= 0 ? (const int64_t*)(desc + kCountOff + 16) : nullptr,
                 nb_direct_max};
  P.bmap = boundary;
  P.npx = (int64_t)w * h;

  // the keys must start at the largest value: the array keeps the last call's contents
  e = cudaMemsetAsync(key, 0xFF, (size_t)w * h * 4, s);
  if (e != cudaSuccess) {
    snprintf(msg, sizeof msg, "scratch set-up: %s", cudaGetErrorString(e));
    return report(errbuf, errbuf_len, SB_ERR_CUDA, msg);
  }
  // the descriptors are written on the device from the kernel's by-value arguments
  const int n_all = P.n_box + P.n_tail;
  k_static_setup<<<std::max(1, std::min(64, (n_all + 255) / 256)), 256, 0, s>>>(P, desc);
  const SadJob* djob = (const SadJob*)desc;
  const SadItem* items = (const SadItem*)(desc + kItemsOff);
  unsigned* queue = (unsigned*)(desc + kQueueOff);
  if (run_direct && run_box)
    launch_count_nonzero((const uint8_t* const*)(desc + kCountOff), (const int64_t*)(desc + kCountOff + 8),
                         (int64_t*)(desc + kCountOff + 16), 1, s);
  if (run_box) {
    launch_sad_boxsum(djob, items, P.n_box, r, r, w % 16 == 0, queue, s);
    if (P.n_tail > 0) launch_sad_tail(djob, items + P.n_box, P.n_tail, max_disp + 1 - P.dt0, queue + 1, s);
  }
  if (run_direct) launch_sad_direct(djob, 1, sad_direct_words(block), r, max_disp, s);
  launch_sad_finalize(djob, 1, w, h, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(msg, sizeof msg, "kernel launch: %s", cudaGetErrorString(e));
    return report(errbuf, errbuf_len, SB_ERR_CUDA, msg);
  }
  return SB_OK;
}

namespace sb {
SB_CHECKS_UNIT(noalloc)
}  // namespace sb
