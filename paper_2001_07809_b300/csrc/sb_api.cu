// C ABI of the selective-blurring library: context, workspace, argument
// checks, the per-stage entry points and sb_run (per-pair, batched, CUDA
// graph and host-buffer streaming forms).  All arithmetic of the method runs
// in the kernels of the other translation units; this file only sizes,
// places and orders the work.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <functional>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/sb.h"
#include "sb_common.cuh"

using namespace sb;

namespace {

constexpr size_t kAlign = 256;
constexpr int kSegRows = 64;  // Algorithm 2 column segment height
inline size_t al(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

// ------------------------------------------------------------ job uploads
// Small host-to-device transfers (job descriptors, the graph form's blob, the
// error word) are moved by the SMs through the device mapping of pinned host
// memory, not by cudaMemcpyAsync: a copy engine runs its queued copies in
// order, so a few hundred bytes of descriptors would otherwise wait behind
// the bulk image copies other streams (host-buffer streaming, the served
// requests) have queued on the same engine.
__global__ void k_gather16(const uint4* __restrict__ src, uint4* __restrict__ dst, size_t n16) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n16; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}
// bytes (rounded up to 16) from src_mapped, the device address of pinned host
// memory, to dst; both 16-byte aligned
cudaError_t gather_h2d(void* dst, const void* src_mapped, size_t bytes, cudaStream_t s) {
  const size_t n16 = (bytes + 15) / 16;
  if (!n16) return cudaSuccess;
  const unsigned blocks = (unsigned)std::min<size_t>((n16 + 255) / 256, 64);
  k_gather16<<<blocks, 256, 0, s>>>(reinterpret_cast<const uint4*>(src_mapped), reinterpret_cast<uint4*>(dst), n16);
  return cudaGetLastError();
}
__global__ void k_read_word(const uint32_t* __restrict__ src, volatile uint32_t* dst) { *dst = *src; }

// A pinned (mapped) host ring and a device ring of the same size.  Device
// reuse is ordered by the stream; host reuse waits for the copy that read it.
struct Uploader {
  uint8_t* host = nullptr;
  uint8_t* host_dev = nullptr;   // the device address of the host ring
  uint8_t* dev = nullptr;
  size_t cap = 0, head = 0;
  struct Flight { size_t a, b; cudaEvent_t ev; };
  std::vector<Flight> flights;
  std::vector<cudaEvent_t> pool;

  cudaError_t init(size_t bytes) {
    cap = bytes;
    cudaError_t e = cudaHostAlloc(&host, cap, cudaHostAllocMapped);
    if (e != cudaSuccess) return e;
    e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&host_dev), host, 0);
    if (e != cudaSuccess) return e;
    return cudaMalloc(&dev, cap);
  }
  void release() {
    for (auto& f : flights) cudaEventDestroy(f.ev);
    for (auto ev : pool) cudaEventDestroy(ev);
    flights.clear();
    pool.clear();
    if (host) cudaFreeHost(host);
    if (dev) cudaFree(dev);
    host = dev = nullptr;
  }
  // copies n bytes to the device; returns the device address
  void* put(const void* src, size_t bytes, cudaStream_t s, cudaError_t* err) {
    const size_t n = al(bytes ? bytes : 1);
    if (n > cap) { *err = cudaErrorMemoryAllocation; return nullptr; }
    if (head + n > cap) head = 0;
    const size_t a = head, b = head + n;
    // wait for in-flight copies that read [a, b)
    for (size_t i = 0; i < flights.size();) {
      if (flights[i].a < b && a < flights[i].b) {
        cudaEventSynchronize(flights[i].ev);
        pool.push_back(flights[i].ev);
        flights.erase(flights.begin() + i);
      } else {
        ++i;
      }
    }
    if (bytes) memcpy(host + a, src, bytes);
    *err = gather_h2d(dev + a, host_dev + a, n, s);
    cudaEvent_t ev;
    if (!pool.empty()) { ev = pool.back(); pool.pop_back(); }
    else cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    cudaEventRecord(ev, s);
    flights.push_back({a, b, ev});
    head = b;
    return dev + a;
  }
};

// ------------------------------------------------------------ workspace
struct PairWs {
  uint8_t *Ll, *Lr, *refined, *filtered, *lut;
  uint32_t *hist, *size_key, *shist, *rowcnt;
  int32_t* roots;   // component roots of the CCA (at most ceil(w/2) ceil(h/2) with 8-connectivity)
  double* centroids;
  int32_t *node, *iters;   // node: the CCA's node table (2 ints per pixel), later the SAD argmin keys (size_key)
  uint16_t* lab16;         // the CCA's tile-local labels, in the buffer the SAD writes later (sparse)
  int64_t* cut;
  uint16_t *sparse, *filled, *disp, *seg_top, *seg_bot;
  float* taps;
  int32_t shist_len, nseg;
};

struct Geo {
  int w, h;
  sb_params p;
};

size_t pair_ws_bytes(const Geo& g, bool need_disp) {
  const size_t N = (size_t)g.w * g.h;
  const int nseg = (g.h + kSegRows - 1) / kSegRows;
  const size_t shist = (size_t)floor(g.p.cc_remove_fraction * (double)N) + 2;
  size_t b = 0;
  b += al(N) * 4;                        // Ll, Lr, refined, filtered
  b += al(256) + al(256 * 4) + al(256 * 8) + al(8) + al(8 * 8);
  b += al(N * 8);                        // CCA node table, then the SAD argmin keys
  b += al(shist * 4) + al((size_t)g.h * 4) + al(N + g.w + g.h + 1);   // + root list
  b += al(N * 2) * (need_disp ? 3 : 2);  // sparse, filled (+ disp)
  b += al((size_t)nseg * g.w * 2) * 2;
  b += al(200 * 4);
  return b;
}

PairWs carve(uint8_t* base, const Geo& g, bool need_disp) {
  const size_t N = (size_t)g.w * g.h;
  const int nseg = (g.h + kSegRows - 1) / kSegRows;
  const size_t shist = (size_t)floor(g.p.cc_remove_fraction * (double)N) + 2;
  PairWs s{};
  size_t o = 0;
  auto take = [&](size_t n) { uint8_t* p = base + o; o += al(n); return p; };
  s.Ll = take(N);
  s.Lr = take(N);
  s.refined = take(N);
  s.filtered = take(N);
  s.lut = take(256);
  s.hist = (uint32_t*)take(256 * 4);
  s.centroids = (double*)take(256 * 8);
  s.iters = (int32_t*)take(8);
  s.cut = (int64_t*)take(8 * 8);
  s.node = (int32_t*)take(N * 8);
  s.size_key = (uint32_t*)s.node;   // free once the CCA's filter has run
  s.shist = (uint32_t*)take(shist * 4);
  s.rowcnt = (uint32_t*)take((size_t)g.h * 4);
  s.roots = (int32_t*)take(N + g.w + g.h + 1);   // 4 ceil(w/2) ceil(h/2) <= (w+1)(h+1) bytes
  s.sparse = (uint16_t*)take(N * 2);
  s.lab16 = s.sparse;   // the CCA is done with its labels before the SAD writes here
  s.filled = (uint16_t*)take(N * 2);
  s.disp = need_disp ? (uint16_t*)take(N * 2) : nullptr;
  s.seg_top = (uint16_t*)take((size_t)nseg * g.w * 2);
  s.seg_bot = (uint16_t*)take((size_t)nseg * g.w * 2);
  s.taps = (float*)take(200 * 4);
  s.shist_len = (int32_t)shist;
  s.nseg = nseg;
  return s;
}

std::vector<float> gauss_taps(float sigma, int* R_out) {
  const int R = (int)ceil(3.0 * (double)sigma);
  std::vector<double> g(2 * R + 1);
  double tot = 0.0;
  const double s2 = (double)sigma * (double)sigma;
  for (int i = -R; i <= R; ++i) { g[i + R] = exp(-(double)(i * i) / (2.0 * s2)); tot += g[i + R]; }
  std::vector<float> out(2 * R + 1);
  for (int i = 0; i < 2 * R + 1; ++i) out[i] = (float)(g[i] / tot);
  *R_out = R;
  return out;
}

}  // namespace

// ------------------------------------------------------------------ context
// batch shapes whose graphs a context keeps instantiated (each holds only its
// kernel nodes; the job blob and the workspace are the context's)
constexpr size_t kGraphCacheMax = 64;

struct sb_context {
  int device = 0;
  cudaStream_t stream = nullptr;
  size_t budget = 0;
  std::string err;
  uint64_t launches = 0;
  uint8_t* tables = nullptr;  // lin (512 B) | packed L table (4096 x 4 B)
  uint32_t* dev_err = nullptr;
  unsigned* sad_queue = nullptr;  // work-item cursors of the box-sum SAD and tail kernels
  uint8_t* ws = nullptr;
  size_t ws_bytes = 0;
  cudaMemPool_t ws_pool = nullptr;   // the workspace's own stream-ordered pool (keeps freed memory)
  bool ws_pooled = false;            // ws came from ws_pool
  Uploader up;
  cudaStream_t s_in = nullptr, s_out = nullptr;  // host-buffer streaming
  // graph cache (batched form): the instantiated graphs of the most recent
  // batch shapes, least recently used first out
  struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    uint64_t kernels = 0;   // kernel nodes (for sb_launch_count)
    uint64_t used = 0;      // last use (a counter)
  };
  std::map<std::string, GraphEntry> graphs;
  uint64_t graph_clock = 0;
  void drop_graphs() {
    for (auto& g : graphs) cudaGraphExecDestroy(g.second.exec);
    graphs.clear();
  }
  // host-buffer staging
  uint8_t* stage = nullptr;
  size_t stage_bytes = 0;
  // job blob of the graph form: the dry pass records every upload here
  bool dry = false;       // record uploads only: no memsets, no launches
  int sink = 0;           // 0: upload ring, 1: blob
  std::vector<uint8_t> blob;
  uint8_t* blob_dev = nullptr;
  size_t blob_cap = 0;
  uint8_t* blob_host = nullptr;  // pinned (mapped) staging of the blob
  uint8_t* blob_host_dev = nullptr;   // its device address
  uint32_t* err_host = nullptr;       // pinned (mapped) copy of the error word
  uint32_t* err_host_dev = nullptr;
  cudaEvent_t blob_ev = nullptr;
  // stage profiling
  bool prof_on = false;
  cudaEvent_t prof_ev[SB_N_STAGES + 1] = {};
  bool prof_recorded = false;
  bool nvtx_open = false;   // a stage's NVTX range is pushed
  bool capturing = false;
  // autotune cache: launch-group shape (each pair's w, h, D, block) -> the
  // box-sum SAD's work-item target chosen by sb_autotune
  std::map<std::string, int> tuned;
  std::map<std::string, int> tuned_blur;   // same shapes -> blur tile height (112 or 64)
  int sad_target_override = 0;   // set while sb_autotune times a candidate
  int blur_by_override = 0;
  int union_limit = kUnionLimitDefault;   // connected components: parent links / union attempts
  size_t host_first = (size_t)64 << 20;   // host-buffer streaming: first chunk's input bytes (ramp start)
  size_t host_cap = (size_t)1024 << 20;   // and the largest chunk
  int host_chunks = 0;                    // chunks of the last host-buffer run
  int sms = 148;
};

namespace {

sb_status fail(sb_context* ctx, sb_status st, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return st;
}

sb_status cuda_fail(sb_context* ctx, cudaError_t e, const char* where) {
  return fail(ctx, e == cudaErrorMemoryAllocation ? SB_ERR_OOM : SB_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define SB_CUDA(ctx, call)                                    \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);  \
  } while (0)

#define SB_MEMSET(ctx, args)                                                  \
  do {                                                                          \
    if (!(ctx)->dry) {                                                          \
      cudaError_t e_ = cudaMemsetAsync args;                                    \
      if (e_ != cudaSuccess) return cuda_fail(ctx, e_, "cudaMemsetAsync");      \
    }                                                                           \
  } while (0)

#define SB_LAUNCHED(ctx, nk)                                                         \
  do {                                                                               \
    (ctx)->launches += (nk);                                                         \
    cudaError_t e_ = cudaPeekAtLastError();                                          \
    if (e_ != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "kernel launch"); \
  } while (0)

sb_status build_tables(sb_context* ctx) {
  uint16_t lin[256];
  std::vector<uint8_t> lt(65536);
  for (int c = 0; c < 256; ++c) {
    const double v = c / 255.0;
    const double l = v <= 0.04045 ? v / 12.92 : pow((v + 0.055) / 1.055, 2.4);
    lin[c] = (uint16_t)floor(65535.0 * l + 0.5);
  }
  const double e = 216.0 / 24389.0, k = 24389.0 / 27.0;  // (6/29)^3 and (29/3)^3
  for (int y = 0; y < 65536; ++y) {
    const double t = y / 65535.0;
    const double Ls = t > e ? 116.0 * cbrt(t) - 16.0 : k * t;
    double v = floor(2.55 * Ls + 0.5);
    lt[y] = (uint8_t)(v < 0 ? 0 : (v > 255 ? 255 : v));
  }
  uint8_t coarse[4096];
  uint32_t thr[257];
  for (int i = 0; i < 4096; ++i) coarse[i] = lt[i * 16];
  for (int l = 0; l <= 256; ++l) {
    uint32_t t = 65536;
    for (int y = 0; y < 65536; ++y)
      if (lt[y] >= l) { t = (uint32_t)y; break; }
    thr[l] = t;
  }
  // packed: entry i = coarse[i] | thr[coarse[i] + 1] << 8 (thresholds <= 65536 fit in 24 bits),
  // so a pixel needs one lookup: L = (e & 255) + (Y16 >= e >> 8)
  uint32_t ct[4096];
  for (int i = 0; i < 4096; ++i) ct[i] = (uint32_t)coarse[i] | (thr[coarse[i] + 1] << 8);
  for (int y = 0; y < 65536; ++y) {  // the compressed form must reproduce the table
    const uint32_t e = ct[y >> 4];
    const int v = (int)(e & 255u) + ((uint32_t)y >= (e >> 8) ? 1 : 0);
    if (v != lt[y]) return fail(ctx, SB_ERR_UNSUPPORTED, "lightness table compression check failed at %d", y);
  }
  uint8_t host[512 + 4096 * 4];
  memcpy(host, lin, 512);
  memcpy(host + 512, ct, 4096 * 4);
  SB_CUDA(ctx, cudaMalloc(&ctx->tables, sizeof host));
  SB_CUDA(ctx, cudaMemcpy(ctx->tables, host, sizeof host, cudaMemcpyHostToDevice));
  return SB_OK;
}

const uint16_t* t_lin(sb_context* c) { return (const uint16_t*)c->tables; }
const uint32_t* t_ct(sb_context* c) { return (const uint32_t*)(c->tables + 512); }

sb_status ensure_ws(sb_context* ctx, size_t bytes) {
  if (bytes <= ctx->ws_bytes) return SB_OK;
  if (ctx->budget && bytes > ctx->budget)
    return fail(ctx, SB_ERR_OOM, "workspace of %zu bytes exceeds the budget of %zu bytes", bytes, ctx->budget);
  // grow by at least half again, so that a context fed batches of varying
  // size (a serving loop) re-allocates a few times only
  size_t grow = ctx->ws_bytes + ctx->ws_bytes / 2;
  if (ctx->budget && grow > ctx->budget) grow = ctx->budget;
  if (!ctx->capturing) {
    // stream-ordered: the old workspace is released after the work queued on
    // this stream, the new one taken from the context's pool, and nothing
    // waits (cudaFree and cudaMalloc would synchronise the whole device,
    // stalling the other streams of a serving process)
    if (!ctx->ws_pool) {
      cudaMemPoolProps props = {};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = ctx->device;
      if (cudaMemPoolCreate(&ctx->ws_pool, &props) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;   // freed blocks stay in the pool for the next, larger request
        cudaMemPoolSetAttribute(ctx->ws_pool, cudaMemPoolAttrReleaseThreshold, &keep);
      } else {
        cudaGetLastError();
        ctx->ws_pool = nullptr;
      }
    }
    if (ctx->ws_pool) {
      if (ctx->ws) {
        if (ctx->ws_pooled) cudaFreeAsync(ctx->ws, ctx->stream);
        else {
          SB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
          cudaFree(ctx->ws);
        }
      }
      ctx->ws = nullptr;
      ctx->ws_bytes = 0;
      cudaError_t e = cudaErrorMemoryAllocation;
      if (grow > bytes) {
        e = cudaMallocFromPoolAsync((void**)&ctx->ws, grow, ctx->ws_pool, ctx->stream);
        if (e == cudaSuccess) bytes = grow;
        else cudaGetLastError();
      }
      if (e != cudaSuccess) e = cudaMallocFromPoolAsync((void**)&ctx->ws, bytes, ctx->ws_pool, ctx->stream);
      if (e == cudaSuccess) {
        ctx->ws_bytes = bytes;
        ctx->ws_pooled = true;
        return SB_OK;
      }
      cudaGetLastError();
      ctx->ws = nullptr;
      // the pool could not serve it: return its cached blocks and take the plain path
      SB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      cudaMemPoolTrimTo(ctx->ws_pool, 0);
    }
  }
  SB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (ctx->ws) {
    if (ctx->ws_pooled) cudaFreeAsync(ctx->ws, ctx->stream);
    else cudaFree(ctx->ws);
    SB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  ctx->ws = nullptr;
  ctx->ws_bytes = 0;
  ctx->ws_pooled = false;
  cudaError_t e = cudaErrorMemoryAllocation;
  if (grow > bytes) {
    e = cudaMalloc(&ctx->ws, grow);
    if (e == cudaSuccess) bytes = grow;
    else cudaGetLastError();   // no room for the margin: take the exact size
  }
  if (e != cudaSuccess) e = cudaMalloc(&ctx->ws, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, SB_ERR_OOM, "cudaMalloc of %zu workspace bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  ctx->ws_bytes = bytes;
  return SB_OK;
}

template <class T>
const T* upload(sb_context* ctx, const std::vector<T>& v, sb_status* st) {
  if (ctx->sink == 1) {
    const size_t off = al(ctx->blob.size()), bytes = v.size() * sizeof(T);
    ctx->blob.resize(off + al(bytes ? bytes : 1));
    if (bytes) memcpy(ctx->blob.data() + off, v.data(), bytes);
    *st = SB_OK;
    return (const T*)(ctx->blob_dev + off);
  }
  cudaError_t e = cudaSuccess;
  void* d = ctx->up.put(v.data(), v.size() * sizeof(T), ctx->stream, &e);
  if (e != cudaSuccess || !d) { *st = cuda_fail(ctx, e == cudaSuccess ? cudaErrorMemoryAllocation : e, "job upload"); return nullptr; }
  ++ctx->launches;   // the gather kernel
  *st = SB_OK;
  return (const T*)d;
}

bool geometry_ok(sb_context* ctx, int w, int h, int D, int block, sb_status* st) {
  if (block < 1 || block > 63 || (block & 1) == 0) { *st = fail(ctx, SB_ERR_INVALID_ARG, "block must be odd in [1, 63], got %d", block); return false; }
  if (D < 0 || D > 1023) { *st = fail(ctx, SB_ERR_INVALID_ARG, "max_disp must be in [0, 1023], got %d", D); return false; }
  if (w < D + block + 1 || h < block) { *st = fail(ctx, SB_ERR_INVALID_ARG, "image %dx%d too small for max_disp %d and block %d (need w >= D+block+1, h >= block)", w, h, D, block); return false; }
  if ((int64_t)w * h >= (int64_t)1 << 31) { *st = fail(ctx, SB_ERR_INVALID_ARG, "image of %dx%d pixels is too large", w, h); return false; }
  return true;
}

bool params_ok(sb_context* ctx, int w, int h, const sb_params& p, sb_status* st) {
  if (!geometry_ok(ctx, w, h, p.max_disp, p.block, st)) return false;
  if (p.k < 1 || p.k > 255) { *st = fail(ctx, SB_ERR_INVALID_ARG, "k must be in [1, 255], got %d", p.k); return false; }
  if (!(p.sigma > 0.0f && p.sigma <= 32.0f)) { *st = fail(ctx, SB_ERR_INVALID_ARG, "sigma must be in (0, 32]"); return false; }
  if (p.n_ranges < 0 || p.n_ranges > SB_MAX_RANGES) { *st = fail(ctx, SB_ERR_INVALID_ARG, "n_ranges must be in [0, %d]", SB_MAX_RANGES); return false; }
  if (p.morph_mode != SB_MORPH_FILL_REMOVE && p.morph_mode != SB_MORPH_OPEN_CLOSE) { *st = fail(ctx, SB_ERR_INVALID_ARG, "unknown morph_mode %d", p.morph_mode); return false; }
  if (!(p.cc_remove_fraction >= 0.0 && p.cc_remove_fraction <= 1.0)) { *st = fail(ctx, SB_ERR_INVALID_ARG, "cc_remove_fraction must be in [0, 1]"); return false; }
  if (p.kmeans_max_iter < 0 || p.kmeans_max_iter > 100000) { *st = fail(ctx, SB_ERR_INVALID_ARG, "kmeans_max_iter must be in [0, 100000]"); return false; }
  if (p.sad_variant < SB_SAD_AUTO || p.sad_variant > SB_SAD_BOXSUM) { *st = fail(ctx, SB_ERR_INVALID_ARG, "unknown sad_variant %d", p.sad_variant); return false; }
  if (p.peek_mode != SB_PEEK_SNAPSHOT && p.peek_mode != SB_PEEK_INPLACE) { *st = fail(ctx, SB_ERR_INVALID_ARG, "unknown peek_mode %d", p.peek_mode); return false; }
  if (p.view != SB_VIEW_LEFT && p.view != SB_VIEW_RIGHT) { *st = fail(ctx, SB_ERR_INVALID_ARG, "unknown view %d", p.view); return false; }
  return true;
}

// --------------------------------------------------------------- tuner
// The direct kernel pays off only when N_b B^2 is small against |Omega| (the
// cost model is sad_direct_limit).  The count N_b exists only on the device
// once the boundary map does, so the host passes the limit with each job and
// the kernels compare it with the pair's own count (no read-back, and a
// replayed graph re-decides for every new frame).
// (nb, nb_direct_max) of a job; *direct_possible / *box_possible say which
// kernels may serve it.
void sad_choice(const Geo& g, const int64_t* nb, SadJob* j, bool* direct_possible, bool* box_possible) {
  if (g.p.sad_variant == SB_SAD_DIRECT || g.p.sad_variant == SB_SAD_BOXSUM) {
    const bool dir = g.p.sad_variant == SB_SAD_DIRECT;
    j->nb = nullptr;
    j->nb_direct_max = dir ? 1 : -1;
    *direct_possible = dir;
    *box_possible = !dir;
    return;
  }
  const int64_t m = sad_direct_limit(g.w, g.h, g.p.max_disp, g.p.block);
  j->nb = m >= 0 ? nb : nullptr;
  j->nb_direct_max = m;
  *direct_possible = m >= 0;
  *box_possible = true;
}

// Box-sum work items: (pair, strip, disparity chunk, row band); bands are cut
// so that a small batch still fills the GPU.
void sad_items(const std::vector<std::pair<int, Geo>>& pairs, int64_t target, int sms, std::vector<SadItem>* items,
               std::vector<SadItem>* tail) {
  int64_t base = 0, tail_strips = 0;
  for (auto& pg : pairs) {
    const Geo& g = pg.second;
    const int r = (g.p.block - 1) / 2, D = g.p.max_disp;
    const int TX = sad_boxsum_strip(r);
    const int ncols = g.w - D - 2 * r;
    const int chunks = sad_has_tail(D) ? sad_tail_first(D) / kSadChunk : (D + 1 + kSadChunk - 1) / kSadChunk;
    base += (int64_t)((ncols + TX - 1) / TX) * chunks;
    if (sad_has_tail(D)) tail_strips += (ncols + sad_tail_strip(r) - 1) / sad_tail_strip(r);
  }
  // (cost, item): cost = rows including the 2r warm-up rows x the strip's columns
  std::vector<std::pair<int64_t, SadItem>> list;
  for (auto& pg : pairs) {
    const Geo& g = pg.second;
    const int r = (g.p.block - 1) / 2, D = g.p.max_disp;
    const int TX = sad_boxsum_strip(r);
    const int xo0 = D + r, xo1 = g.w - 1 - r, yo0 = r, yo1 = g.h - 1 - r;
    const int rows = yo1 - yo0 + 1;
    const int dend = sad_has_tail(D) ? sad_tail_first(D) : D + 1;   // box-sum chunks cover d < dend
    // row bands: enough items for `target` (bands of at least max(8r, 64) rows, so the
    // 2r warm-up rows stay a small share); where that still leaves CTA slots of the
    // persistent grid (two per SM) idle — a single small pair — the count, with bands of
    // at least 8 rows, that minimises (rounds of the grid) x (band rows + r), r weighing
    // the warm-up rows, which run the vertical pass only: the pair's time is then the
    // walk down one band
    const int64_t box_slots = (int64_t)sms * 2;
    const int64_t per_target = std::max<int64_t>(1, (target + base - 1) / std::max<int64_t>(base, 1));
    int bands = (int)std::min<int64_t>(per_target, std::max(1, rows / std::max(8 * r, 64)));
    if (base * bands < box_slots) {
      const int cap = (int)std::min<int64_t>(per_target, std::max(1, rows / 8));
      int64_t best_cost = -1;
      for (int t = 1; t <= cap; ++t) {
        const int64_t c = (base * t + box_slots - 1) / box_slots * ((rows + t - 1) / t + r);
        if (best_cost < 0 || c < best_cost) { best_cost = c; bands = t; }
      }
    }
    for (int b = 0; b < bands; ++b) {
      const int ya = yo0 + (int)((int64_t)rows * b / bands), yb = yo0 + (int)((int64_t)rows * (b + 1) / bands) - 1;
      if (ya > yb) continue;
      const int64_t cost = (int64_t)(yb - ya + 1 + 2 * r) * (TX + 2 * r);
      for (int x0 = xo0; x0 <= xo1; x0 += TX)
        for (int d0 = 0; d0 < dend; d0 += kSadChunk) list.push_back({cost, SadItem{pg.first, x0, d0, ya, yb}});
    }
    if (sad_has_tail(D)) {
      // tail items: the band count that minimises (rounds of the persistent
      // grid, six 256-thread CTAs per SM) x (band rows + 2r warm-up rows)
      const int TT = sad_tail_strip(r);
      const int64_t slots = (int64_t)sms * 6;
      int tb = 1;
      int64_t best = -1;
      for (int t = 1; t <= 16 && t <= rows; ++t) {
        const int64_t rounds = (tail_strips * t + slots - 1) / slots;
        const int64_t c = rounds * ((rows + t - 1) / t + 2 * r);
        if (best < 0 || c < best) { best = c; tb = t; }
      }
      for (int b = 0; b < tb; ++b) {
        const int ya = yo0 + (int)((int64_t)rows * b / tb), yb = yo0 + (int)((int64_t)rows * (b + 1) / tb) - 1;
        if (ya > yb) continue;
        for (int x0 = xo0; x0 <= xo1; x0 += TT) tail->push_back(SadItem{pg.first, x0, sad_tail_first(D), ya, yb});
      }
    }
  }
  // largest first, so the persistent kernel ends on short items (ties keep generation order)
  std::stable_sort(list.begin(), list.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
  // the last grid's worth of items (two resident CTAs per SM) is cut into four
  // row bands each, so that the grid drains on quarter items instead of
  // waiting on whole ones; only where the list holds several rounds and every
  // band keeps at least max(8r, 64) rows
  const size_t slots = (size_t)sms * 2;
  size_t keep = list.size();
  std::vector<SadItem> tail_parts;
  if (list.size() >= 4 * slots) {
    std::map<int, int> radius;
    for (auto& pg : pairs) radius[pg.first] = (pg.second.p.block - 1) / 2;
    for (size_t k = list.size() - slots; k < list.size(); ++k) {
      const SadItem& it = list[k].second;
      const int rows = it.y1 - it.y0 + 1;
      if (rows < 4 * std::max(8 * radius[it.job], 64)) { tail_parts.clear(); break; }
      for (int b = 0; b < 4; ++b)
        tail_parts.push_back(SadItem{it.job, it.x0, it.d0, it.y0 + rows * b / 4, it.y0 + rows * (b + 1) / 4 - 1});
    }
    if (!tail_parts.empty()) keep = list.size() - slots;
    // and the last grid's worth of those quarters into halves again (eighth
    // items), where a half keeps at least max(8r, 64) rows: a launch of a
    // few pairs (a host-streaming chunk) spends its last round on them
    if (tail_parts.size() >= 2 * slots) {
      std::vector<SadItem> halves;
      for (size_t k = tail_parts.size() - slots; k < tail_parts.size(); ++k) {
        const SadItem& it = tail_parts[k];
        const int rows = it.y1 - it.y0 + 1;
        if (rows < 2 * std::max(8 * radius[it.job], 64)) { halves.clear(); break; }
        halves.push_back(SadItem{it.job, it.x0, it.d0, it.y0, it.y0 + rows / 2 - 1});
        halves.push_back(SadItem{it.job, it.x0, it.d0, it.y0 + rows / 2, it.y1});
      }
      if (!halves.empty()) {
        tail_parts.resize(tail_parts.size() - slots);
        tail_parts.insert(tail_parts.end(), halves.begin(), halves.end());
      }
    }
  }
  for (size_t k = 0; k < keep; ++k) items->push_back(list[k].second);
  for (auto& it : tail_parts) items->push_back(it);
}

// NVTX ranges (host side, the default domain): "sb:run" around each sb_run
// and one range per pipeline stage, "sb:<stage>", open while the stage's
// work is enqueued, so a profiler that follows NVTX (ncu --nvtx) attributes
// the stage's launches to it.  In the graph form they mark the capture; a
// replay is a single graph launch inside "sb:run".
const char* const kStageRange[SB_N_STAGES] = {"sb:lightness", "sb:kmeans", "sb:refine", "sb:cca",
                                              "sb:sad",       "sb:sad_rest", "sb:recon", "sb:blur"};

void nvtx_stage(sb_context* ctx, int i) {
  if (ctx->nvtx_open) nvtxRangePop();
  ctx->nvtx_open = i < SB_N_STAGES;
  if (ctx->nvtx_open) nvtxRangePushA(kStageRange[i]);
}

// Closes a stage range still open when the enqueuing returns early.
struct StageRanges {
  sb_context* ctx;
  ~StageRanges() {
    if (ctx->nvtx_open) nvtx_stage(ctx, SB_N_STAGES);
  }
};

// Stage boundary marks: the NVTX stage ranges, and for sb_profile_read CUDA
// events (external records inside captures).
sb_status mark(sb_context* ctx, int i) {
  if (!ctx->dry) nvtx_stage(ctx, i);
  if (!ctx->prof_on || ctx->dry) return SB_OK;
  cudaError_t e = ctx->capturing ? cudaEventRecordWithFlags(ctx->prof_ev[i], ctx->stream, cudaEventRecordExternal)
                                 : cudaEventRecord(ctx->prof_ev[i], ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaEventRecord");
  if (i == SB_N_STAGES) ctx->prof_recorded = true;
  return SB_OK;
}

#define SB_MARK(ctx, i)                          \
  do {                                           \
    sb_status m_ = mark(ctx, i);                 \
    if (m_ != SB_OK) return m_;                  \
  } while (0)

// ------------------------------------------------------------ pipeline
struct PairRun {
  const uint8_t *left, *right;
  uint8_t* out_rgb;
  uint16_t* out_disp;
  Geo g;
  PairWs ws;
};

// Launch-group shape for the autotune cache: every pair's size, disparity
// range and block (what the box-sum work split depends on).
std::string shape_key(const Geo* geos, int n) {
  std::string key;
  for (int i = 0; i < n; ++i) {
    const int32_t v[5] = {geos[i].w, geos[i].h, geos[i].p.max_disp, geos[i].p.block,
                          (int32_t)ceil(3.0 * (double)geos[i].p.sigma)};
    key.append((const char*)v, sizeof v);
  }
  return key;
}

// A shape key whose pairs all have one geometry: that geometry's record, else
// an empty string.
std::string uniform_record(const std::string& key) {
  constexpr size_t kRec = 5 * sizeof(int32_t);
  if (key.size() < kRec || key.size() % kRec) return std::string();
  for (size_t o = kRec; o < key.size(); o += kRec)
    if (key.compare(o, kRec, key, 0, kRec) != 0) return std::string();
  return key.substr(0, kRec);
}

// Blur tile height: the candidate being timed, else the tuned value, else the
// value tuned for another batch of the same single geometry (host-buffer
// streaming cuts a tuned batch into chunks of other sizes; every form gives
// the same bytes, so only the speed of the choice is borrowed), else 112.
int blur_rows(const sb_context* ctx, const std::string& key) {
  if (ctx->blur_by_override > 0) return ctx->blur_by_override;
  auto it = ctx->tuned_blur.find(key);
  if (it != ctx->tuned_blur.end()) return it->second;
  const std::string rec = uniform_record(key);
  if (!rec.empty()) {
    int best = 0;
    size_t best_n = 0;
    for (const auto& t : ctx->tuned_blur)   // the largest tuned batch of this geometry
      if (t.first.size() > best_n && uniform_record(t.first) == rec) best = t.second, best_n = t.first.size();
    if (best) return best;
  }
  return 112;
}

// Box-sum work items a launch aims for: the candidate being timed, else the
// tuned value for this shape, else three waves of the persistent grid.
int64_t sad_target(const sb_context* ctx, const std::string& key) {
  if (ctx->sad_target_override > 0) return ctx->sad_target_override;
  auto it = ctx->tuned.find(key);
  if (it != ctx->tuned.end()) return it->second;
  return (int64_t)ctx->sms * 2 * 3;
}

// Enqueues the whole pipeline for `runs` (one launch per stage over all of
// them).  Job descriptors go to `jobs_dev` when given (graph form), else
// through the upload ring.
sb_status enqueue_pipeline(sb_context* ctx, std::vector<PairRun>& runs) {
  StageRanges ranges{ctx};
  cudaStream_t s = ctx->stream;
  sb_status st = SB_OK;
  const int n = (int)runs.size();
  if (n == 0) return SB_OK;
  int max_w = 0, max_h = 0, max_R = 0, max_nseg = 0;
  int64_t max_px = 0;
  for (auto& r : runs) {
    max_w = std::max(max_w, r.g.w);
    max_h = std::max(max_h, r.g.h);
    max_px = std::max<int64_t>(max_px, (int64_t)r.g.w * r.g.h);
    max_nseg = std::max(max_nseg, r.ws.nseg);
  }
  // zero the per-pair accumulators
  for (auto& r : runs) {
    SB_MEMSET(ctx, (r.ws.hist, 0, 256 * 4, s));
    SB_MEMSET(ctx, (r.ws.cut, 0, 8 * 8, s));
  }
  // CTAs per lightness job: one per 4096 pixels, but no more than 16 waves of the
  // whole batch (8 CTAs per SM) in all: each CTA first copies 16.5 KB of tables into
  // shared memory, which a large batch would otherwise repeat hundreds of thousands of times
  const int64_t n_light = 2 * (int64_t)runs.size();
  const int64_t light_cap = std::max<int64_t>(1, (16 * 8 * (int64_t)ctx->sms + n_light - 1) / n_light);
  const int bpj = (int)std::min<int64_t>(std::min<int64_t>(std::max<int64_t>(1, max_px / (256 * 16)), 592), light_cap);
  SB_MARK(ctx, SB_STAGE_LIGHTNESS);
  // 1. lightness of both images (+ histogram of the left)
  {
    std::vector<LightJob> J;
    for (auto& r : runs) {
      const int64_t N = (int64_t)r.g.w * r.g.h;
      // right view: the mirrored right image is the reference, the mirrored left the search image
      const bool rv = r.g.p.view == SB_VIEW_RIGHT;
      J.push_back(LightJob{rv ? r.right : r.left, r.ws.Ll, r.ws.hist, N, r.g.w, rv ? 1 : 0});
      J.push_back(LightJob{rv ? r.left : r.right, r.ws.Lr, nullptr, N, r.g.w, rv ? 1 : 0});
    }
    const LightJob* d = upload(ctx, J, &st);
    if (!d) return st;
    if (!ctx->dry) {
      launch_lightness(d, (int)J.size(), bpj, t_lin(ctx), t_ct(ctx), s);
      SB_LAUNCHED(ctx, 1);
    }
  }
  SB_MARK(ctx, SB_STAGE_KMEANS);
  // 2. histogram K-means
  {
    std::vector<KmeansJob> J;
    for (auto& r : runs) J.push_back(KmeansJob{r.ws.hist, r.ws.centroids, r.ws.lut, r.ws.iters, r.g.p.k, r.g.p.kmeans_max_iter});
    const KmeansJob* d = upload(ctx, J, &st);
    if (!d) return st;
    if (!ctx->dry) {
      launch_kmeans(d, n, s);
      SB_LAUNCHED(ctx, 1);
    }
  }
  SB_MARK(ctx, SB_STAGE_REFINE);
  // 3. boundary + refinement (grouped by mode)
  for (int mode = 0; mode < 2; ++mode) {
    std::vector<MorphJob> J;
    int mw = 0, mh = 0;
    for (auto& r : runs)
      if (r.g.p.morph_mode == mode) {
        J.push_back(MorphJob{r.ws.Ll, r.ws.lut, r.ws.refined, r.g.w, r.g.h, mode});
        mw = std::max(mw, r.g.w);
        mh = std::max(mh, r.g.h);
      }
    if (J.empty()) continue;
    const MorphJob* d = upload(ctx, J, &st);
    if (!d) return st;
    if (!ctx->dry) {
      launch_boundary_morph(d, (int)J.size(), mw, mh, mode, s);
      SB_LAUNCHED(ctx, 1);
    }
  }
  SB_MARK(ctx, SB_STAGE_CCA);
  // 4. CCA and small-component removal
  {
    std::vector<CcaJob> J;
    for (auto& r : runs) {
      SB_MEMSET(ctx, (r.ws.shist, 0, (size_t)r.ws.shist_len * 4, s));
      SB_MEMSET(ctx, (r.ws.rowcnt, 0, (size_t)r.g.h * 4, s));
      J.push_back(CcaJob{r.ws.refined, r.ws.lab16, r.ws.node, r.ws.shist, r.ws.rowcnt, r.ws.cut, r.ws.filtered,
                         r.ws.roots, nullptr, r.g.w, r.g.h, r.ws.shist_len, r.g.p.cc_remove_fraction,
                         ctx->union_limit});
    }
    const CcaJob* d = upload(ctx, J, &st);
    if (!d) return st;
    if (!ctx->dry) {
      launch_cca(d, n, max_w, max_h, ctx->dev_err, s);
      SB_LAUNCHED(ctx, 2);
    }
    if (!ctx->dry) {
      launch_cc_filter(d, n, max_w, max_h, ctx->dev_err, s);
      SB_LAUNCHED(ctx, 6);
    }
  }
  // 5. SAD at the anchors
  {
    std::vector<SadJob> J;
    std::vector<std::pair<int, Geo>> box;
    uint32_t direct_nw = 0;   // bit k: some pair the direct kernel may serve has a k-word window
    int dir_r = 0, dir_D = 0;
    for (int i = 0; i < n; ++i) {
      auto& r = runs[i];
      const size_t N = (size_t)r.g.w * r.g.h;
      SB_MEMSET(ctx, (r.ws.size_key, 0xFF, N * 4, s));
      SadJob sj{r.ws.Ll, r.ws.Lr, r.ws.filtered, r.ws.size_key, r.ws.sparse, nullptr, r.g.w, r.g.h,
                r.g.p.max_disp, (r.g.p.block - 1) / 2, nullptr, -1};
      bool dp = false, bp = true;
      sad_choice(r.g, r.ws.cut, &sj, &dp, &bp);   // cut[0]: boundary pixels of the refined map
      J.push_back(sj);
      if (dp) {
        direct_nw |= 1u << sad_direct_words(r.g.p.block);
        dir_r = std::max(dir_r, (r.g.p.block - 1) / 2);
        dir_D = std::max(dir_D, r.g.p.max_disp);
      }
      if (bp) box.push_back({i, r.g});
    }
    const SadJob* d = upload(ctx, J, &st);
    if (!d) return st;
    SB_MARK(ctx, SB_STAGE_SAD);
    if (!box.empty()) {
      std::vector<Geo> geos;
      for (auto& r : runs) geos.push_back(r.g);
      std::vector<SadItem> items, tail;
      sad_items(box, sad_target(ctx, shape_key(geos.data(), n)), ctx->sms, &items, &tail);
      const SadItem* di = upload(ctx, items, &st);
      if (!di) return st;
      const SadItem* dt = tail.empty() ? nullptr : upload(ctx, tail, &st);
      if (!tail.empty() && !dt) return st;
      int max_r = 0, uniform_r = (box[0].second.p.block - 1) / 2;
      int max_rem = 1;
      bool w16 = true;   // every box-sum pair's width a multiple of 16
      for (auto& b : box) {
        max_r = std::max(max_r, (b.second.p.block - 1) / 2);
        if ((b.second.p.block - 1) / 2 != uniform_r) uniform_r = -1;
        w16 = w16 && b.second.w % 16 == 0;
        if (sad_has_tail(b.second.p.max_disp))
          max_rem = std::max(max_rem, b.second.p.max_disp + 1 - sad_tail_first(b.second.p.max_disp));
      }
      SB_MEMSET(ctx, (ctx->sad_queue, 0, 8, s));
      if (!ctx->dry) {
        launch_sad_boxsum(d, di, (int)items.size(), max_r, uniform_r, w16, ctx->sad_queue, s);
        SB_LAUNCHED(ctx, 1);
      }
      SB_MARK(ctx, SB_STAGE_SAD_REST);
      if (!tail.empty() && !ctx->dry) {
        launch_sad_tail(d, dt, (int)tail.size(), max_rem, ctx->sad_queue + 1, s);
        SB_LAUNCHED(ctx, 1);
      }
    } else {
      SB_MARK(ctx, SB_STAGE_SAD_REST);
    }
    for (int nw = 1; nw <= 17 && !ctx->dry; ++nw)
      if (direct_nw & (1u << nw)) {
        launch_sad_direct(d, n, nw, dir_r, dir_D, s);
        SB_LAUNCHED(ctx, 1);
      }
    // the argmin keys go straight to Algorithm 1 (its kernel decodes them), so
    // the pipeline needs no key-to-disparity pass
  }
  SB_MARK(ctx, SB_STAGE_RECON);
  // 6. reconstruction (Algorithms 1 and 2)
  {
    std::vector<ReconJob> J;
    int modes = 0;
    for (auto& r : runs) {
      uint16_t* out = r.out_disp ? r.out_disp : r.ws.disp;
      const int inplace = r.g.p.peek_mode == SB_PEEK_INPLACE;
      modes |= inplace ? 2 : 1;
      J.push_back(ReconJob{r.ws.sparse, r.ws.size_key, r.ws.filled, out, r.ws.seg_top, r.ws.seg_bot, r.g.w, r.g.h,
                           r.g.p.max_disp, (r.g.p.block - 1) / 2, r.g.p.disp_threshold, kSegRows, inplace,
                           r.g.p.view == SB_VIEW_RIGHT ? 1 : 0});
    }
    const ReconJob* d = upload(ctx, J, &st);
    if (!d) return st;
    if (!ctx->dry) {
      launch_recon(d, n, max_w, max_h, max_nseg, modes, s);
      SB_LAUNCHED(ctx, recon_launches(modes));
    }
  }
  SB_MARK(ctx, SB_STAGE_BLUR);
  // 7. selective blur
  {
    std::vector<BlurJob> J;
    for (auto& r : runs) {
      int R;
      std::vector<float> taps = gauss_taps(r.g.p.sigma, &R);
      max_R = std::max(max_R, R);
      const float* dtaps = upload(ctx, taps, &st);
      if (!dtaps) return st;
      BlurJob b{};
      b.rgb = r.g.p.view == SB_VIEW_RIGHT ? r.right : r.left;   // the reference image
      b.disp = r.out_disp ? r.out_disp : r.ws.disp;
      b.out = r.out_rgb;
      b.taps = dtaps;
      b.w = r.g.w;
      b.h = r.g.h;
      b.R = R;
      b.n_ranges = r.g.p.n_ranges;
      for (int i = 0; i < r.g.p.n_ranges; ++i) { b.lo[i] = r.g.p.ranges[i].lo; b.hi[i] = r.g.p.ranges[i].hi; }
      J.push_back(b);
    }
    const BlurJob* d = upload(ctx, J, &st);
    if (!d) return st;
    if (!ctx->dry) {
      std::vector<Geo> geos;
      for (auto& r : runs) geos.push_back(r.g);
      launch_blur(d, n, max_w, max_h, max_R, blur_rows(ctx, shape_key(geos.data(), n)), s);
      SB_LAUNCHED(ctx, 1);
    }
  }
  SB_MARK(ctx, SB_N_STAGES);
  return SB_OK;
}

}  // namespace

// =================================================================== C ABI
namespace sb {
SB_CHECKS_UNIT(api)
}  // namespace sb

// The first failed bounds check of any unit (each unit's word is read and
// cleared); 0 when none failed or the build has no checks.
static uint32_t first_check_site() {
  uint32_t (*const units[])() = {checks_api, checks_noalloc, checks_segment, checks_morph,
                                 checks_cca, checks_sad, checks_recon, checks_blur};
  uint32_t first = 0;
  for (auto u : units) {
    const uint32_t v = u();
    if (v && !first) first = v;
  }
  return first;
}

static const char* check_site_stage(uint32_t site) {
  switch (site / 100) {
    case 0: return "probe";
    case 1: return "lightness / k-means";
    case 2: return "boundary refinement";
    case 3: return "connected components";
    case 4: return "SAD";
    case 5: return "reconstruction";
    case 6: return "blur";
    default: return "allocation-free SAD";
  }
}

namespace {
__global__ void k_check_probe(int trip) {
  if (SB_CHECK(trip == 0, 1u)) return;
}
}  // namespace

extern "C" {

void sb_default_params(sb_params* p) {
  if (!p) return;
  memset(p, 0, sizeof *p);
  p->k = 10;
  p->max_disp = 64;
  p->block = 9;
  p->disp_threshold = 1;
  p->morph_mode = SB_MORPH_FILL_REMOVE;
  p->kmeans_max_iter = 100;
  p->cc_remove_fraction = 0.04;
  p->sigma = 3.0f;
  p->n_ranges = 0;
  p->sad_variant = SB_SAD_AUTO;
  p->peek_mode = SB_PEEK_SNAPSHOT;
  p->view = SB_VIEW_LEFT;
}

sb_status sb_create(int device, size_t mem_budget_bytes, void* cuda_stream, sb_context** out) {
  if (!out) return SB_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return SB_ERR_INVALID_ARG;
  }
  std::unique_ptr<sb_context> ctx(new sb_context());
  ctx->device = device;
  ctx->budget = mem_budget_bytes;
  ctx->stream = (cudaStream_t)cuda_stream;
  if (cudaSetDevice(device) != cudaSuccess) return SB_ERR_CUDA;
  if (build_tables(ctx.get()) != SB_OK) return SB_ERR_CUDA;
  if (cudaMalloc(&ctx->dev_err, 4) != cudaSuccess || cudaMemset(ctx->dev_err, 0, 4) != cudaSuccess) return SB_ERR_CUDA;
  if (cudaHostAlloc(&ctx->err_host, 16, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer(reinterpret_cast<void**>(&ctx->err_host_dev), ctx->err_host, 0) != cudaSuccess)
    return SB_ERR_CUDA;
  if (cudaMalloc(&ctx->sad_queue, 8) != cudaSuccess) return SB_ERR_CUDA;   // box-sum and tail cursors
  if (cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) ctx->sms = 148;
  if (ctx->up.init(8 << 20) != cudaSuccess) return SB_ERR_OOM;
  *out = ctx.release();
  return SB_OK;
}

void sb_destroy(sb_context* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  ctx->up.release();
  ctx->drop_graphs();
  if (ctx->blob_dev) cudaFree(ctx->blob_dev);
  if (ctx->blob_host) cudaFreeHost(ctx->blob_host);
  if (ctx->blob_ev) cudaEventDestroy(ctx->blob_ev);
  for (int i = 0; i <= SB_N_STAGES; ++i)
    if (ctx->prof_ev[i]) cudaEventDestroy(ctx->prof_ev[i]);
  if (ctx->tables) cudaFree(ctx->tables);
  if (ctx->dev_err) cudaFree(ctx->dev_err);
  if (ctx->err_host) cudaFreeHost(ctx->err_host);
  if (ctx->sad_queue) cudaFree(ctx->sad_queue);
  if (ctx->ws) {
    if (ctx->ws_pooled) {
      cudaFreeAsync(ctx->ws, ctx->stream);
      cudaStreamSynchronize(ctx->stream);
    } else {
      cudaFree(ctx->ws);
    }
  }
  if (ctx->ws_pool) cudaMemPoolDestroy(ctx->ws_pool);
  if (ctx->stage) cudaFree(ctx->stage);
  if (ctx->s_in) cudaStreamDestroy(ctx->s_in);
  if (ctx->s_out) cudaStreamDestroy(ctx->s_out);
  delete ctx;
}

sb_status sb_set_stream(sb_context* ctx, void* cuda_stream) {
  if (!ctx) return SB_ERR_INVALID_ARG;
  ctx->stream = (cudaStream_t)cuda_stream;
  return SB_OK;
}

const char* sb_last_error(const sb_context* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

size_t sb_workspace_bytes(const sb_context* ctx) { return ctx ? ctx->ws_bytes : 0; }

uint64_t sb_launch_count(const sb_context* ctx) { return ctx ? ctx->launches : 0; }

sb_status sb_profile_enable(sb_context* ctx, int on) {
  if (!ctx) return SB_ERR_INVALID_ARG;
  if (on && !ctx->prof_ev[0])
    for (int i = 0; i <= SB_N_STAGES; ++i) SB_CUDA(ctx, cudaEventCreate(&ctx->prof_ev[i]));
  if (ctx->prof_on != (on != 0)) ctx->drop_graphs();  // captured graphs hold (or lack) the marks
  ctx->prof_on = on != 0;
  ctx->prof_recorded = false;
  return SB_OK;
}

int32_t sb_profile_read(sb_context* ctx, float* ms, int32_t max_stages) {
  if (!ctx || !ms || !ctx->prof_recorded) return -1;
  if (cudaEventSynchronize(ctx->prof_ev[SB_N_STAGES]) != cudaSuccess) return -1;
  const int n = std::min<int>(max_stages, SB_N_STAGES);
  for (int i = 0; i < n; ++i) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, ctx->prof_ev[i], ctx->prof_ev[i + 1]) != cudaSuccess) { cudaGetLastError(); t = -1.f; }
    ms[i] = t;
  }
  return n;
}

sb_status sb_synchronize(sb_context* ctx) {
  if (!ctx) return SB_ERR_INVALID_ARG;
  // the error word comes back through mapped host memory (see gather_h2d)
  k_read_word<<<1, 1, 0, ctx->stream>>>(ctx->dev_err, ctx->err_host_dev);
  ++ctx->launches;
  SB_CUDA(ctx, cudaGetLastError());
  SB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const uint32_t e = *reinterpret_cast<volatile uint32_t*>(ctx->err_host);
  if (e) {
    cudaMemset(ctx->dev_err, 0, 4);
    if (e & DEV_ERR_CCA_ITER)
      return fail(ctx, SB_ERR_TIMEOUT, "connected components: a union-find search or union reached its limit of %d "
                  "(sb_set_union_limit); the run's results are not valid", ctx->union_limit);
    return fail(ctx, SB_ERR_CUDA, "device-side check failed (flags 0x%x)", e);
  }
  const uint32_t site = first_check_site();
  if (site)
    return fail(ctx, SB_ERR_CHECK, "bounds check failed at site %u (%s); the run's results are not valid", site,
                check_site_stage(site));
  return SB_OK;
}

sb_status sb_check_probe(sb_context* ctx, int32_t trip) {
  if (!ctx) return SB_ERR_INVALID_ARG;
#ifdef SB_CHECKS
  k_check_probe<<<1, 32, 0, ctx->stream>>>(trip);
  SB_LAUNCHED(ctx, 1);
  return SB_OK;
#else
  (void)trip;
  return fail(ctx, SB_ERR_UNSUPPORTED, "check_probe: this library was built without SB_CHECKS (libsb_checks.so has them)");
#endif
}

int32_t sb_checks_built(void) {
#ifdef SB_CHECKS
  return 1;
#else
  return 0;
#endif
}

sb_status sb_rgb_to_lightness(sb_context* ctx, const uint8_t* rgb, int32_t w, int32_t h, uint8_t* L, uint32_t* hist) {
  if (!ctx) return SB_ERR_INVALID_ARG;
  if (!rgb || !L || w <= 0 || h <= 0) return fail(ctx, SB_ERR_INVALID_ARG, "rgb_to_lightness: null pointer or empty image");
  sb_status st;
  if (hist) SB_CUDA(ctx, cudaMemsetAsync(hist, 0, 256 * 4, ctx->stream));
  std::vector<LightJob> J{LightJob{rgb, L, hist, (int64_t)w * h, w, 0}};
  const LightJob* d = upload(ctx, J, &st);
  if (!d) return st;
  const int bpj = (int)std::min<int64_t>(std::max<int64_t>(1, (int64_t)w * h / (256 * 16)), 592);
  launch_lightness(d, 1, bpj, t_lin(ctx), t_ct(ctx), ctx->stream);
  SB_LAUNCHED(ctx, 1);
  return SB_OK;
}

sb_status sb_kmeans_segment(sb_context* ctx, const uint8_t* L_left, int32_t w, int32_t h, int32_t k, int32_t max_iter,
                            uint8_t* labels, double* centroids, uint8_t* bin2cluster, int32_t* iters) {
  if (!ctx) return SB_ERR_INVALID_ARG;
  if (!L_left || w <= 0 || h <= 0) return fail(ctx, SB_ERR_INVALID_ARG, "kmeans_segment: null pointer or empty image");
  if (k < 1 || k > 255) return fail(ctx, SB_ERR_INVALID_ARG, "k must be in [1, 255], got %d", k);
  if (max_iter < 0 || max_iter > 100000) return fail(ctx, SB_ERR_INVALID_ARG, "max_iter must be in [0, 100000]");
  sb_status st = ensure_ws(ctx, al(256 * 4) + al(256 * 8) + al(256) + al(8));
  if (st != SB_OK) return st;
  uint32_t* hist = (uint32_t*)ctx->ws;
  double* cent = centroids ? centroids : (double*)(ctx->ws + al(256 * 4));
  uint8_t* lut = bin2cluster ? bin2cluster : ctx->ws + al(256 * 4) + al(256 * 8);
  int32_t* it = iters ? iters : (int32_t*)(ctx->ws + al(256 * 4) + al(256 * 8) + al(256));
  SB_CUDA(ctx, cudaMemsetAsync(hist, 0, 256 * 4, ctx->stream));
  launch_histogram_u8(L_left, (int64_t)w * h, hist, ctx->stream);
  SB_LAUNCHED(ctx, 1);
  std::vector<KmeansJob> J{KmeansJob{hist, cent, lut, it, k, max_iter}};
  const KmeansJob* d = upload(ctx, J, &st);
  if (!d) return st;
  launch_kmeans(d, 1, ctx->stream);
  SB_LAUNCHED(ctx, 1);
  if (labels) {
    std::vector<LabelJob> LJ{LabelJob{L_left, lut, labels, (int64_t)w * h}};
    const LabelJob* dl = upload(ctx, LJ, &st);
    if (!dl) return st;
    const int bpj = (int)std::min<int64_t>(std::max<int64_t>(1, (int64_t)w * h / (256 * 16)), 592);
    launch_labels(dl, 1, bpj, ctx->stream);
    SB_LAUNCHED(ctx, 1);
  }
  return SB_OK;
}

sb_status sb_refine_boundaries(sb_context* ctx, const uint8_t* labels, int32_t w, int32_t h, int32_t morph_mode,
                               double cc_remove_fraction, uint8_t* boundary, uint8_t* refined, int32_t* cc_labels) {
  if (!ctx) return SB_ERR_INVALID_ARG;
  if (!labels || !boundary || w <= 0 || h <= 0) return fail(ctx, SB_ERR_INVALID_ARG, "refine_boundaries: null pointer or empty image");
  if (morph_mode != SB_MORPH_FILL_REMOVE && morph_mode != SB_MORPH_OPEN_CLOSE) return fail(ctx, SB_ERR_INVALID_ARG, "unknown morph_mode %d", morph_mode);
  if (!(cc_remove_fraction >= 0.0 && cc_remove_fraction <= 1.0)) return fail(ctx, SB_ERR_INVALID_ARG, "cc_remove_fraction must be in [0, 1]");
  if ((int64_t)w * h >= (int64_t)1 << 31) return fail(ctx, SB_ERR_INVALID_ARG, "image too large");
  const size_t N = (size_t)w * h;
  const size_t shist = (size_t)floor(cc_remove_fraction * (double)N) + 2;
  const size_t need = al(N) + al(N * 8) + al(N * 2) + al(shist * 4) + al((size_t)h * 4) + al(64) + al(N + w + h + 1);
  sb_status st = ensure_ws(ctx, need);
  if (st != SB_OK) return st;
  uint8_t* o = ctx->ws;
  uint8_t* ref = refined ? refined : o;
  o += al(N);
  int32_t* node = (int32_t*)o;
  o += al(N * 8);
  uint16_t* lab16 = (uint16_t*)o;
  o += al(N * 2);
  uint32_t* sh = (uint32_t*)o;
  o += al(shist * 4);
  uint32_t* rowcnt = (uint32_t*)o;
  o += al((size_t)h * 4);
  int64_t* cut = (int64_t*)o;
  o += al(64);
  int32_t* roots = (int32_t*)o;
  cudaStream_t s = ctx->stream;
  std::vector<MorphJob> MJ{MorphJob{labels, nullptr, ref, w, h, morph_mode}};
  const MorphJob* dm = upload(ctx, MJ, &st);
  if (!dm) return st;
  launch_boundary_morph(dm, 1, w, h, morph_mode, s);
  SB_LAUNCHED(ctx, 1);
  SB_CUDA(ctx, cudaMemsetAsync(sh, 0, shist * 4, s));
  SB_CUDA(ctx, cudaMemsetAsync(cut, 0, 64, s));
  SB_CUDA(ctx, cudaMemsetAsync(rowcnt, 0, (size_t)h * 4, s));
  std::vector<CcaJob> CJ{CcaJob{ref, lab16, node, sh, rowcnt, cut, boundary, roots, cc_labels, w, h, (int32_t)shist,
                                cc_remove_fraction, ctx->union_limit}};
  const CcaJob* dc = upload(ctx, CJ, &st);
  if (!dc) return st;
  launch_cca(dc, 1, w, h, ctx->dev_err, s);
  SB_LAUNCHED(ctx, 2);
  launch_cc_filter(dc, 1, w, h, ctx->dev_err, s);
  SB_LAUNCHED(ctx, 6);
  return SB_OK;
}

sb_status sb_boundary_sad(sb_context* ctx, const uint8_t* L_left, const uint8_t* L_right, const uint8_t* boundary,
                          int32_t w, int32_t h, int32_t max_disp, int32_t block, int32_t variant, uint16_t* disp,
                          uint32_t* cost) {
  if (!ctx) return SB_ERR_INVALID_ARG;
  if (!L_left || !L_right || !boundary || !disp) return fail(ctx, SB_ERR_INVALID_ARG, "boundary_sad: null pointer");
  sb_status st = SB_OK;
  if (!geometry_ok(ctx, w, h, max_disp, block, &st)) return st;
  if (variant < SB_SAD_AUTO || variant > SB_SAD_BOXSUM) return fail(ctx, SB_ERR_INVALID_ARG, "unknown SAD variant %d", variant);
  const size_t N = (size_t)w * h;
  st = ensure_ws(ctx, al(N * 4) + al(8));
  if (st != SB_OK) return st;
  uint32_t* key = (uint32_t*)ctx->ws;
  int64_t* count = (int64_t*)(ctx->ws + al(N * 4));
  cudaStream_t s = ctx->stream;
  SB_CUDA(ctx, cudaMemsetAsync(key, 0xFF, N * 4, s));
  Geo g{w, h, {}};
  sb_default_params(&g.p);
  g.p.max_disp = max_disp;
  g.p.block = block;
  g.p.sad_variant = variant;
  SadJob job{L_left, L_right, boundary, key, disp, cost, w, h, max_disp, (block - 1) / 2, nullptr, -1};
  bool dp = false, bp = true;
  sad_choice(g, count, &job, &dp, &bp);
  if (dp && bp) {   // both possible: count the boundary pixels on the device
    SB_CUDA(ctx, cudaMemsetAsync(count, 0, 8, s));
    const uint8_t* const* dm = upload(ctx, std::vector<const uint8_t*>{boundary}, &st);
    if (!dm) return st;
    const int64_t* dn = upload(ctx, std::vector<int64_t>{(int64_t)N}, &st);
    if (!dn) return st;
    launch_count_nonzero(dm, dn, count, 1, s);
    SB_LAUNCHED(ctx, 1);
  }
  const SadJob* d = upload(ctx, std::vector<SadJob>{job}, &st);
  if (!d) return st;
  if (bp) {
    std::vector<SadItem> items, tail;
    sad_items({{0, g}}, sad_target(ctx, shape_key(&g, 1)), ctx->sms, &items, &tail);
    const SadItem* di = upload(ctx, items, &st);
    if (!di) return st;
    const SadItem* dt = tail.empty() ? nullptr : upload(ctx, tail, &st);
    if (!tail.empty() && !dt) return st;
    SB_CUDA(ctx, cudaMemsetAsync(ctx->sad_queue, 0, 8, s));
    launch_sad_boxsum(d, di, (int)items.size(), (block - 1) / 2, (block - 1) / 2, w % 16 == 0, ctx->sad_queue, s);
    SB_LAUNCHED(ctx, 1);
    if (!tail.empty()) {
      launch_sad_tail(d, dt, (int)tail.size(), max_disp + 1 - sad_tail_first(max_disp), ctx->sad_queue + 1, s);
      SB_LAUNCHED(ctx, 1);
    }
  }
  if (dp) {
    launch_sad_direct(d, 1, sad_direct_words(block), (block - 1) / 2, max_disp, s);
    SB_LAUNCHED(ctx, 1);
  }
  launch_sad_finalize(d, 1, w, h, s);
  SB_LAUNCHED(ctx, 1);
  return SB_OK;
}

sb_status sb_reconstruct_disparity(sb_context* ctx, uint16_t* disp, int32_t w, int32_t h, int32_t max_disp,
                                   int32_t block, int32_t disp_threshold, int32_t peek_mode, uint16_t* filled) {
  if (!ctx) return SB_ERR_INVALID_ARG;
  if (!disp) return fail(ctx, SB_ERR_INVALID_ARG, "reconstruct_disparity: null pointer");
  if (peek_mode != SB_PEEK_SNAPSHOT && peek_mode != SB_PEEK_INPLACE)
    return fail(ctx, SB_ERR_INVALID_ARG, "unknown peek_mode %d", peek_mode);
  sb_status st = SB_OK;
  if (!geometry_ok(ctx, w, h, max_disp, block, &st)) return st;
  const size_t N = (size_t)w * h;
  if (filled && (uintptr_t)filled < (uintptr_t)(disp + N) && (uintptr_t)disp < (uintptr_t)(filled + N))
    return fail(ctx, SB_ERR_INVALID_ARG, "reconstruct_disparity: filled overlaps disp");
  const int nseg = (h + kSegRows - 1) / kSegRows;
  st = ensure_ws(ctx, al(N * 2) + al((size_t)nseg * w * 2) * 2);
  if (st != SB_OK) return st;
  uint16_t* fl = filled ? filled : (uint16_t*)ctx->ws;
  uint16_t* top = (uint16_t*)(ctx->ws + al(N * 2));
  uint16_t* bot = (uint16_t*)(ctx->ws + al(N * 2) + al((size_t)nseg * w * 2));
  const int inplace = peek_mode == SB_PEEK_INPLACE;
  std::vector<ReconJob> J{ReconJob{disp, nullptr, fl, disp, top, bot, w, h, max_disp, (block - 1) / 2, disp_threshold,
                                   kSegRows, inplace, 0}};
  const ReconJob* d = upload(ctx, J, &st);
  if (!d) return st;
  launch_recon(d, 1, w, h, nseg, inplace ? 2 : 1, ctx->stream);
  SB_LAUNCHED(ctx, recon_launches(inplace ? 2 : 1));
  return SB_OK;
}

sb_status sb_lr_consistency(sb_context* ctx, const uint16_t* dL, const uint16_t* dR, int32_t w, int32_t h,
                            int32_t tol, uint8_t* ok, int64_t* count) {
  if (!ctx) return SB_ERR_INVALID_ARG;
  if (!dL || !dR || !ok) return fail(ctx, SB_ERR_INVALID_ARG, "lr_consistency: null pointer");
  if (w < 1 || h < 1 || (int64_t)w * h >= (int64_t)1 << 31) return fail(ctx, SB_ERR_INVALID_ARG, "bad image size %dx%d", w, h);
  cudaSetDevice(ctx->device);
  if (count) SB_CUDA(ctx, cudaMemsetAsync(count, 0, 8, ctx->stream));
  launch_lr_consistency(dL, dR, w, h, tol, ok, reinterpret_cast<unsigned long long*>(count), ctx->stream);
  SB_LAUNCHED(ctx, 1);
  SB_CUDA(ctx, cudaGetLastError());
  return SB_OK;
}

sb_status sb_selective_blur(sb_context* ctx, const uint8_t* rgb, const uint16_t* disp, int32_t w, int32_t h,
                            const sb_range* ranges, int32_t n_ranges, float sigma, uint8_t* out_rgb) {
  if (!ctx) return SB_ERR_INVALID_ARG;
  if (!rgb || !disp || !out_rgb || w <= 0 || h <= 0) return fail(ctx, SB_ERR_INVALID_ARG, "selective_blur: null pointer or empty image");
  if (n_ranges < 0 || n_ranges > SB_MAX_RANGES || (n_ranges > 0 && !ranges)) return fail(ctx, SB_ERR_INVALID_ARG, "n_ranges must be in [0, %d] with a host array", SB_MAX_RANGES);
  if (!(sigma > 0.0f && sigma <= 32.0f)) return fail(ctx, SB_ERR_INVALID_ARG, "sigma must be in (0, 32]");
  int R;
  std::vector<float> taps = gauss_taps(sigma, &R);
  sb_status st = SB_OK;
  const float* dt = upload(ctx, taps, &st);
  if (!dt) return st;
  BlurJob b{};
  b.rgb = rgb;
  b.disp = disp;
  b.out = out_rgb;
  b.taps = dt;
  b.w = w;
  b.h = h;
  b.R = R;
  b.n_ranges = n_ranges;
  for (int i = 0; i < n_ranges; ++i) { b.lo[i] = ranges[i].lo; b.hi[i] = ranges[i].hi; }
  std::vector<BlurJob> J{b};
  const BlurJob* d = upload(ctx, J, &st);
  if (!d) return st;
  launch_blur(d, 1, w, h, R, ctx->blur_by_override > 0 ? ctx->blur_by_override : 112, ctx->stream);
  SB_LAUNCHED(ctx, 1);
  return SB_OK;
}

sb_status sb_set_host_chunk(sb_context* ctx, size_t first_bytes, size_t max_bytes) {
  if (!ctx) return SB_ERR_INVALID_ARG;
  if (first_bytes == 0 && max_bytes == 0) {
    ctx->host_first = (size_t)64 << 20;
    ctx->host_cap = (size_t)1024 << 20;
    return SB_OK;
  }
  if (first_bytes == 0 || max_bytes < first_bytes)
    return fail(ctx, SB_ERR_INVALID_ARG, "host chunk sizes: need 0 < first_bytes <= max_bytes (got %zu, %zu)",
                first_bytes, max_bytes);
  ctx->host_first = first_bytes;
  ctx->host_cap = max_bytes;
  return SB_OK;
}

int32_t sb_host_io_chunks(const sb_context* ctx) { return ctx ? ctx->host_chunks : 0; }

sb_status sb_set_union_limit(sb_context* ctx, int32_t limit) {
  if (!ctx) return SB_ERR_INVALID_ARG;
  if (limit < 0) return fail(ctx, SB_ERR_INVALID_ARG, "union limit must be >= 0 (0: the default), got %d", limit);
  ctx->union_limit = limit == 0 ? kUnionLimitDefault : limit;
  return SB_OK;
}

sb_status sb_set_blur_form(sb_context* ctx, int32_t form) {
  if (!ctx) return SB_ERR_INVALID_ARG;
  if (form != SB_BLUR_AUTO && form != SB_BLUR_STRIP && form != SB_BLUR_TILES_64 && form != SB_BLUR_TILES_112)
    return fail(ctx, SB_ERR_INVALID_ARG, "blur form must be 0, 32, 64 or 112, got %d", form);
  ctx->blur_by_override = form;
  return SB_OK;
}

}  // extern "C"

// ------------------------------------------------------------------- sb_run
namespace {

sb_status run_device(sb_context* ctx, const sb_pair* pairs, int n, bool batched) {
  std::vector<Geo> geos(n);
  for (int i = 0; i < n; ++i) geos[i] = Geo{pairs[i].w, pairs[i].h, pairs[i].p};
  sb_status st;
  if (!batched) {
    size_t need = 0;
    for (int i = 0; i < n; ++i) need = std::max(need, pair_ws_bytes(geos[i], pairs[i].out_disp == nullptr));
    if ((st = ensure_ws(ctx, need)) != SB_OK) return st;
    for (int i = 0; i < n; ++i) {
      std::vector<PairRun> runs{PairRun{pairs[i].left_rgb, pairs[i].right_rgb, pairs[i].out_rgb, pairs[i].out_disp, geos[i],
                                        carve(ctx->ws, geos[i], pairs[i].out_disp == nullptr)}};
      if ((st = enqueue_pipeline(ctx, runs)) != SB_OK) return st;
    }
    return SB_OK;
  }
  size_t need = 0;
  std::vector<size_t> offs(n);
  for (int i = 0; i < n; ++i) {
    offs[i] = need;
    need += pair_ws_bytes(geos[i], pairs[i].out_disp == nullptr);
  }
  if ((st = ensure_ws(ctx, need)) != SB_OK) return st;
  std::vector<PairRun> runs;
  for (int i = 0; i < n; ++i)
    runs.push_back(PairRun{pairs[i].left_rgb, pairs[i].right_rgb, pairs[i].out_rgb, pairs[i].out_disp, geos[i],
                           carve(ctx->ws + offs[i], geos[i], pairs[i].out_disp == nullptr)});
  return enqueue_pipeline(ctx, runs);
}

// Record-only pass (`pass` enqueues with ctx->dry set: uploads only, into the
// host blob), then one copy of the blob to the device on the context stream.
// A later pass run with ctx->sink = 1 (blob cleared) makes the same uploads
// in the same order and so gets the same device offsets.
sb_status record_and_upload_blob(sb_context* ctx, const std::function<sb_status()>& pass) {
  sb_status st = SB_OK;
  for (int attempt = 0; attempt < 2; ++attempt) {
    ctx->blob.clear();
    ctx->sink = 1;
    ctx->dry = true;
    st = pass();
    ctx->dry = false;
    ctx->sink = 0;
    if (st != SB_OK) return st;
    if (ctx->blob.size() <= ctx->blob_cap) break;
    // grow the blob (its address is baked into captured graphs: drop them)
    SB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->drop_graphs();
    if (ctx->blob_dev) cudaFree(ctx->blob_dev);
    if (ctx->blob_host) cudaFreeHost(ctx->blob_host);
    ctx->blob_dev = ctx->blob_host = ctx->blob_host_dev = nullptr;
    ctx->blob_cap = 0;
    const size_t cap = al(ctx->blob.size() * 2);   // a multiple of 16: the gather copies whole 16-byte words
    SB_CUDA(ctx, cudaMalloc(&ctx->blob_dev, cap));
    SB_CUDA(ctx, cudaHostAlloc(&ctx->blob_host, cap, cudaHostAllocMapped));
    SB_CUDA(ctx, cudaHostGetDevicePointer(reinterpret_cast<void**>(&ctx->blob_host_dev), ctx->blob_host, 0));
    ctx->blob_cap = cap;
  }
  if (!ctx->blob_ev) SB_CUDA(ctx, cudaEventCreateWithFlags(&ctx->blob_ev, cudaEventDisableTiming));
  SB_CUDA(ctx, cudaEventSynchronize(ctx->blob_ev));  // the previous blob copy has been read
  memcpy(ctx->blob_host, ctx->blob.data(), ctx->blob.size());
  SB_CUDA(ctx, gather_h2d(ctx->blob_dev, ctx->blob_host_dev, ctx->blob.size(), ctx->stream));
  ++ctx->launches;
  SB_CUDA(ctx, cudaEventRecord(ctx->blob_ev, ctx->stream));
  return SB_OK;
}

// Graph form: the batched pipeline is captured once per batch shape (sizes,
// parameters, workspace) and replayed.  Kernels read their job descriptors
// from a device blob owned by the context; each call rebuilds the blob for
// the caller's current pointers with a record-only pass and uploads it ahead
// of the replay, so new buffers of the same shape need no new capture.
sb_status run_graph(sb_context* ctx, const sb_pair* pairs, int n) {
  size_t need = 0;
  for (int i = 0; i < n; ++i) need += pair_ws_bytes(Geo{pairs[i].w, pairs[i].h, pairs[i].p}, pairs[i].out_disp == nullptr);
  sb_status st = ensure_ws(ctx, need);
  if (st != SB_OK) return st;
  std::string key((const char*)&ctx->ws, sizeof ctx->ws);
  {
    std::vector<Geo> geos;
    for (int i = 0; i < n; ++i) geos.push_back(Geo{pairs[i].w, pairs[i].h, pairs[i].p});
    const int64_t target = sad_target(ctx, shape_key(geos.data(), n));
    key.append((const char*)&target, sizeof target);
    const int32_t by = blur_rows(ctx, shape_key(geos.data(), n));
    key.append((const char*)&by, sizeof by);
  }
  for (int i = 0; i < n; ++i) {
    const sb_pair& q = pairs[i];
    key.append((const char*)&q.w, sizeof q.w);
    key.append((const char*)&q.h, sizeof q.h);
    key.append((const char*)&q.p, sizeof q.p);
    key.push_back(q.out_disp ? 1 : 0);
  }
  // record-only pass: the blob for the current pointers, uploaded ahead of the replay
  st = record_and_upload_blob(ctx, [&]() { return run_device(ctx, pairs, n, true); });
  if (st != SB_OK) return st;
  auto found = ctx->graphs.find(key);
  if (found == ctx->graphs.end()) {
    if (ctx->graphs.size() >= kGraphCacheMax) {   // evict the least recently used graph
      auto old = ctx->graphs.begin();
      for (auto it = ctx->graphs.begin(); it != ctx->graphs.end(); ++it)
        if (it->second.used < old->second.used) old = it;
      cudaGraphExecDestroy(old->second.exec);
      ctx->graphs.erase(old);
    }
    cudaStream_t cap = ctx->stream;
    bool own = false;
    if (cap == nullptr) {  // the legacy default stream cannot be captured
      SB_CUDA(ctx, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
      own = true;
    }
    cudaStream_t saved = ctx->stream;
    ctx->stream = cap;
    ctx->blob.clear();
    ctx->sink = 1;  // same uploads, same offsets: the captured kernels read the blob
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    const uint64_t before = ctx->launches;
    ctx->capturing = true;
    if (e == cudaSuccess) st = run_device(ctx, pairs, n, true);
    ctx->capturing = false;
    const uint64_t kernels = ctx->launches - before;
    ctx->launches = before;
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(cap, &graph) : e;
    ctx->sink = 0;
    ctx->stream = saved;
    if (own) cudaStreamDestroy(cap);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamBeginCapture");
    if (st != SB_OK) { if (graph) cudaGraphDestroy(graph); return st; }
    if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
    found = ctx->graphs.emplace(key, sb_context::GraphEntry{exec, kernels, 0}).first;
  }
  found->second.used = ++ctx->graph_clock;
  cudaError_t e = cudaGraphLaunch(found->second.exec, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphLaunch");
  ctx->launches += found->second.kernels;
  return SB_OK;
}

// Host-buffer streaming: pairs move through device staging in chunks; the
// copy-in of chunk k+1 and the copy-out of chunk k-1 overlap chunk k's compute.
sb_status run_host_io(sb_context* ctx, const sb_pair* pairs, int n, bool batched) {
  if (!ctx->s_in) SB_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->s_in, cudaStreamNonBlocking));
  if (!ctx->s_out) SB_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->s_out, cudaStreamNonBlocking));
  // chunking: up to host_cap bytes of inputs per chunk (1 GB by default), at
  // least one pair; the chunk size grows by half per chunk from host_first
  // (64 MB) at the start and shrinks the same way at the end, so the first
  // upload (nothing to overlap it with yet) and the last download are short,
  // and each chunk's upload (about 1.0 ms per pair on a shared link) stays
  // shorter than the compute of the chunk before it (about 1.6 ms per pair)
  std::vector<std::pair<int, int>> chunks;
  if (!batched) {
    for (int i = 0; i < n; ++i) chunks.push_back({i, i + 1});
  } else {
    std::vector<std::pair<int, int>> head, tail;
    int lo = 0, hi = n;
    const size_t cap = ctx->host_cap;
    for (int k = 0; lo < hi; ++k) {
      const size_t target = std::min(cap, (size_t)((double)ctx->host_first * std::pow(1.5, std::min(k, 16))));
      size_t acc = 0;
      const int a = lo;
      while (lo < hi && (acc < target || lo == a)) acc += (size_t)pairs[lo].w * pairs[lo].h * 6, ++lo;
      head.push_back({a, lo});
      if (lo >= hi) break;
      acc = 0;
      const int b = hi;
      while (hi > lo && (acc < target || hi == b)) --hi, acc += (size_t)pairs[hi].w * pairs[hi].h * 6;
      tail.push_back({hi, b});
    }
    chunks = head;
    chunks.insert(chunks.end(), tail.rbegin(), tail.rend());
  }
  ctx->host_chunks = (int)chunks.size();
  // staging per slot: left, right, out_rgb, out_disp for the largest chunk
  size_t slot = 0;
  for (auto& c : chunks) {
    size_t b = 0;
    for (int i = c.first; i < c.second; ++i) {
      const size_t N = (size_t)pairs[i].w * pairs[i].h;
      b += al(N * 3) * 3 + al(N * 2);
    }
    slot = std::max(slot, b);
  }
  // three staging slots: the upload of chunk k waits for the download of
  // chunk k-3, so a chunk's download and the next upload (longer together than
  // one chunk's compute when the link carries both directions) do not stall it
  constexpr int kSlots = 3;
  if (ctx->stage_bytes < kSlots * slot) {
    SB_CUDA(ctx, cudaDeviceSynchronize());
    if (ctx->stage) cudaFree(ctx->stage);
    ctx->stage = nullptr;
    ctx->stage_bytes = 0;
    cudaError_t e = cudaMalloc(&ctx->stage, kSlots * slot);
    if (e != cudaSuccess) { cudaGetLastError(); return fail(ctx, SB_ERR_OOM, "staging of %zu bytes failed", kSlots * slot); }
    ctx->stage_bytes = kSlots * slot;
  }
  // device-side pairs of every chunk (slot k % kSlots of the staging)
  std::vector<std::vector<sb_pair>> dps(chunks.size());
  for (size_t k = 0; k < chunks.size(); ++k) {
    uint8_t* base = ctx->stage + (k % kSlots) * slot;
    size_t o = 0;
    for (int i = chunks[k].first; i < chunks[k].second; ++i) {
      const size_t N = (size_t)pairs[i].w * pairs[i].h;
      sb_pair q = pairs[i];
      q.left_rgb = base + o; o += al(N * 3);
      q.right_rgb = base + o; o += al(N * 3);
      q.out_rgb = base + o; o += al(N * 3);
      q.out_disp = (uint16_t*)(base + o); o += al(N * 2);
      dps[k].push_back(q);
    }
  }
  // the workspace for the largest chunk first: the recorded descriptors hold
  // workspace addresses, so it must not move between the record pass and the run
  {
    size_t need = 0;
    for (auto& dp : dps) {
      size_t b = 0;
      for (auto& q : dp) {
        const size_t pb = pair_ws_bytes(Geo{q.w, q.h, q.p}, q.out_disp == nullptr);
        b = batched ? b + pb : std::max(b, pb);
      }
      need = std::max(need, b);
    }
    sb_status s0 = ensure_ws(ctx, need);
    if (s0 != SB_OK) return s0;
  }
  // every chunk's job descriptors in one upload ahead of the bulk copies:
  // small uploads on the compute stream would otherwise queue behind the next
  // chunk's bulk copy on the same copy engine and hold up the compute
  sb_status st = record_and_upload_blob(ctx, [&]() {
    for (size_t k = 0; k < chunks.size(); ++k) {
      sb_status s2 = run_device(ctx, dps[k].data(), (int)dps[k].size(), batched);
      if (s2 != SB_OK) return s2;
    }
    return SB_OK;
  });
  if (st != SB_OK) return st;
  std::vector<cudaEvent_t> ev_in(chunks.size()), ev_comp(chunks.size()), ev_out(chunks.size());
  for (size_t k = 0; k < chunks.size(); ++k) {
    cudaEventCreateWithFlags(&ev_in[k], cudaEventDisableTiming);
    cudaEventCreateWithFlags(&ev_comp[k], cudaEventDisableTiming);
    cudaEventCreateWithFlags(&ev_out[k], cudaEventDisableTiming);
  }
  ctx->blob.clear();
  ctx->sink = 1;   // the same uploads as the record pass: offsets into the uploaded blob
  for (size_t k = 0; k < chunks.size() && st == SB_OK; ++k) {
    if (k >= (size_t)kSlots) {  // the slot's previous chunk must be computed and copied out
      cudaStreamWaitEvent(ctx->s_in, ev_comp[k - kSlots], 0);
      cudaStreamWaitEvent(ctx->s_in, ev_out[k - kSlots], 0);
    }
    for (size_t j = 0; j < dps[k].size(); ++j) {
      const sb_pair& hp = pairs[chunks[k].first + j];
      const size_t N = (size_t)hp.w * hp.h;
      cudaMemcpyAsync((void*)dps[k][j].left_rgb, hp.left_rgb, N * 3, cudaMemcpyHostToDevice, ctx->s_in);
      cudaMemcpyAsync((void*)dps[k][j].right_rgb, hp.right_rgb, N * 3, cudaMemcpyHostToDevice, ctx->s_in);
    }
    cudaEventRecord(ev_in[k], ctx->s_in);
    cudaStreamWaitEvent(ctx->stream, ev_in[k], 0);
    st = run_device(ctx, dps[k].data(), (int)dps[k].size(), batched);
    cudaEventRecord(ev_comp[k], ctx->stream);
    cudaStreamWaitEvent(ctx->s_out, ev_comp[k], 0);
    for (size_t j = 0; j < dps[k].size(); ++j) {
      const sb_pair& hp = pairs[chunks[k].first + j];
      const size_t N = (size_t)hp.w * hp.h;
      cudaMemcpyAsync(hp.out_rgb, dps[k][j].out_rgb, N * 3, cudaMemcpyDeviceToHost, ctx->s_out);
      if (hp.out_disp) cudaMemcpyAsync(hp.out_disp, dps[k][j].out_disp, N * 2, cudaMemcpyDeviceToHost, ctx->s_out);
    }
    cudaEventRecord(ev_out[k], ctx->s_out);
  }
  ctx->sink = 0;
  // the caller's stream sees the end of the copies
  if (!chunks.empty()) cudaStreamWaitEvent(ctx->stream, ev_out.back(), 0);
  for (size_t k = 0; k < chunks.size(); ++k) {
    cudaEventDestroy(ev_in[k]);
    cudaEventDestroy(ev_comp[k]);
    cudaEventDestroy(ev_out[k]);
  }
  cudaError_t e = cudaGetLastError();
  if (st == SB_OK && e != cudaSuccess) return cuda_fail(ctx, e, "host-buffer streaming");
  return st;
}

}  // namespace

extern "C" sb_status sb_autotune(sb_context* ctx, const sb_pair* pairs, int32_t n_pairs, uint32_t flags,
                                 float* ms_out, int32_t* sad_items_out, int32_t* blur_rows_out) {
  if (!ctx) return SB_ERR_INVALID_ARG;
  if (n_pairs <= 0 || !pairs) return fail(ctx, SB_ERR_INVALID_ARG, "sb_autotune: no pairs");
  if (ctx->capturing) return fail(ctx, SB_ERR_INVALID_ARG, "sb_autotune cannot run inside a stream capture");
  if (flags & SB_RUN_HOST_IO)
    return fail(ctx, SB_ERR_INVALID_ARG, "sb_autotune takes device pairs (host-buffer runs split into their own groups)");
  cudaSetDevice(ctx->device);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SB_CUDA(ctx, cudaEventCreate(&e0));
  SB_CUDA(ctx, cudaEventCreate(&e1));
  // one candidate: a warm-up run (and graph capture), then a timed run
  auto time_run = [&](float* ms) -> sb_status {
    sb_status st = sb_run(ctx, pairs, n_pairs, flags);
    if (st != SB_OK) return st;
    cudaEventRecord(e0, ctx->stream);
    st = sb_run(ctx, pairs, n_pairs, flags);
    if (st != SB_OK) return st;
    cudaEventRecord(e1, ctx->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) return fail(ctx, SB_ERR_CUDA, "sb_autotune: event wait failed");
    cudaEventElapsedTime(ms, e0, e1);
    return SB_OK;
  };
  // candidates 0-3: the box-sum work split, 1, 2, 3 and 6 waves of the
  // persistent grid (blur tiles of 112 rows); candidates 4-5: blur tiles of
  // 112 and 64 rows with the chosen split
  const int waves[4] = {1, 2, 3, 6}, rows[3] = {SB_BLUR_TILES_112, SB_BLUR_TILES_64, SB_BLUR_STRIP};
  float ms[SB_AUTOTUNE_CANDIDATES] = {};
  int best_items = 0, best_rows = 112;
  float best_ms = 0.f;
  sb_status st = SB_OK;
  const int forced = ctx->blur_by_override;
  ctx->blur_by_override = 112;
  for (int c = 0; c < 4 && st == SB_OK; ++c) {
    ctx->sad_target_override = ctx->sms * 2 * waves[c];
    st = time_run(&ms[c]);
    if (st == SB_OK && (c == 0 || ms[c] < best_ms)) { best_ms = ms[c]; best_items = ctx->sad_target_override; }
  }
  for (int c = 0; c < 3 && st == SB_OK; ++c) {
    ctx->sad_target_override = best_items;
    ctx->blur_by_override = rows[c];
    st = time_run(&ms[4 + c]);
    if (st == SB_OK && (c == 0 || ms[4 + c] < best_ms)) { best_ms = ms[4 + c]; best_rows = rows[c]; }
  }
  ctx->sad_target_override = 0;
  ctx->blur_by_override = forced;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != SB_OK) return st;
  // the shape of each launch group sb_run forms with these flags
  auto keep = [&](const std::string& key) {
    ctx->tuned[key] = best_items;
    ctx->tuned_blur[key] = best_rows;
  };
  if (flags & SB_RUN_BATCHED) {
    std::vector<Geo> geos;
    for (int i = 0; i < n_pairs; ++i) geos.push_back(Geo{pairs[i].w, pairs[i].h, pairs[i].p});
    keep(shape_key(geos.data(), n_pairs));
  } else {
    for (int i = 0; i < n_pairs; ++i) {
      Geo g{pairs[i].w, pairs[i].h, pairs[i].p};
      keep(shape_key(&g, 1));
    }
  }
  if (ms_out) memcpy(ms_out, ms, sizeof ms);
  if (sad_items_out) *sad_items_out = best_items;
  if (blur_rows_out) *blur_rows_out = best_rows;
  return SB_OK;
}

extern "C" sb_status sb_run(sb_context* ctx, const sb_pair* pairs, int32_t n_pairs, uint32_t flags) {
  if (!ctx) return SB_ERR_INVALID_ARG;
  if (n_pairs < 0 || (n_pairs > 0 && !pairs)) return fail(ctx, SB_ERR_INVALID_ARG, "sb_run: bad pair array");
  if (flags & ~(uint32_t)(SB_RUN_BATCHED | SB_RUN_GRAPH | SB_RUN_HOST_IO)) return fail(ctx, SB_ERR_INVALID_ARG, "sb_run: unknown flags 0x%x", flags);
  if ((flags & SB_RUN_GRAPH) && !(flags & SB_RUN_BATCHED)) return fail(ctx, SB_ERR_INVALID_ARG, "SB_RUN_GRAPH needs SB_RUN_BATCHED");
  if ((flags & SB_RUN_GRAPH) && (flags & SB_RUN_HOST_IO)) return fail(ctx, SB_ERR_INVALID_ARG, "SB_RUN_GRAPH cannot be combined with SB_RUN_HOST_IO");
  for (int i = 0; i < n_pairs; ++i) {
    const sb_pair& q = pairs[i];
    if (!q.left_rgb || !q.right_rgb || !q.out_rgb) return fail(ctx, SB_ERR_INVALID_ARG, "pair %d: null image pointer", i);
    sb_status st = SB_OK;
    if (!params_ok(ctx, q.w, q.h, q.p, &st)) return st;
  }
  if (n_pairs == 0) return SB_OK;
  cudaSetDevice(ctx->device);
  nvtxRangePushA("sb:run");
  sb_status st;
  if (flags & SB_RUN_HOST_IO) st = run_host_io(ctx, pairs, n_pairs, (flags & SB_RUN_BATCHED) != 0);
  else if (flags & SB_RUN_GRAPH) st = run_graph(ctx, pairs, n_pairs);
  else st = run_device(ctx, pairs, n_pairs, (flags & SB_RUN_BATCHED) != 0);
  nvtxRangePop();
  return st;
}
