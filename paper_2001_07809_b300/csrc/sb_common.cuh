// Internal declarations shared by the library's CUDA translation units.
//
// Every stage kernel is written batch-first: it takes a device array of
// per-image (or per-pair) job descriptors and blockIdx.y (or .z) selects the
// job, so the per-pair path (one job) and the batched path (one launch over
// all pairs of a batch, sizes and parameters may differ per pair) are the
// same kernels.
#pragma once

#include <cuda_runtime.h>
#include <cmath>
#include <stdint.h>

#define SB_UNDET16 0xFFFFu
#define SB_KEY_DBITS 10  // SAD argmin key = (cost << 10) | d, d <= 1023

namespace sb {

// Device-side error word (bit flags) written by bounded loops: the
// connected-components union-find gave up after its link / retry limit.
enum : uint32_t { DEV_ERR_CCA_ITER = 1u };
constexpr int kUnionLimitDefault = 1 << 22;   // parent links and union retries (sb_set_union_limit)

// ------------------------------------------------------------ bounds checks
// The bounds-checked build (-DSB_CHECKS, libsb_checks.so) evaluates
// SB_CHECK(cond, site) before the accesses whose index comes from data
// (labels, parent links, root lists, work-item tables, anchor positions): a
// false condition records `site` in the translation unit's check word (the
// first failure wins), and the caller skips the access, so the kernel runs on
// without touching memory out of range.  sb_synchronize reads and clears the
// words and reports SB_ERR_CHECK with the site.  Sites: 1 the probe
// (sb_check_probe), 1xx lightness / k-means, 2xx refinement, 3xx components,
// 4xx SAD, 5xx reconstruction, 6xx blur.  In the normal build
// SB_CHECK(cond, site) is `true` and cond is not evaluated.
#ifdef SB_CHECKS
static __device__ uint32_t g_check_site;   // one per translation unit
__device__ __forceinline__ bool sb_check(bool ok, uint32_t site) {
  if (!ok) atomicCAS(&g_check_site, 0u, site);
  return ok;
}
#define SB_CHECK(cond, site) ::sb::sb_check((cond), (site))
// checks_<unit>(): this unit's check word, cleared (0: no check failed)
#define SB_CHECKS_UNIT(unit)                                                  \
  uint32_t checks_##unit() {                                                  \
    uint32_t v = 0, z = 0;                                                    \
    if (cudaMemcpyFromSymbol(&v, g_check_site, sizeof v) != cudaSuccess) return 0; \
    if (v) cudaMemcpyToSymbol(g_check_site, &z, sizeof z);                    \
    return v;                                                                 \
  }
#else
#define SB_CHECK(cond, site) true
#define SB_CHECKS_UNIT(unit) \
  uint32_t checks_##unit() { return 0; }
#endif
uint32_t checks_segment();
uint32_t checks_morph();
uint32_t checks_cca();
uint32_t checks_sad();
uint32_t checks_recon();
uint32_t checks_blur();
uint32_t checks_api();
uint32_t checks_noalloc();

// ---------------------------------------------------------------- lightness
struct LightJob {
  const uint8_t* rgb;  // n_px * 3
  uint8_t* L;          // n_px
  uint32_t* hist;      // 256 or nullptr (must be zeroed before the launch)
  int64_t n_px;
  int32_t w;           // row length (used when mirror is set)
  int32_t mirror;      // 1: write each row mirrored (pixel x of a row to w-1-x)
};
// lin: uint16[256] linear sRGB x 65535; ct: uint32[4096], entry i = L of Y = 16 i (low
// byte) | the first Y with L above that (upper 24 bits).  Both built on the host from FP64
// libm.
void launch_lightness(const LightJob* jobs, int n_jobs, int blocks_per_job, const uint16_t* lin,
                      const uint32_t* ct, cudaStream_t s);

// ------------------------------------------------------------------ k-means
struct KmeansJob {
  const uint32_t* hist;  // 256
  double* centroids;     // k
  uint8_t* lut;          // 256: bin -> cluster
  int32_t* iters;        // 1 or nullptr
  int32_t k, max_iter;
};
void launch_kmeans(const KmeansJob* jobs, int n_jobs, cudaStream_t s);

// Per-pixel label = lut[L]  (only for the optional labels output).
struct LabelJob {
  const uint8_t* L;
  const uint8_t* lut;
  uint8_t* labels;
  int64_t n_px;
};
void launch_labels(const LabelJob* jobs, int n_jobs, int blocks_per_job, cudaStream_t s);
// 256-bin histogram of an 8-bit image (hist zeroed by the caller)
void launch_histogram_u8(const uint8_t* L, int64_t n, uint32_t* hist, cudaStream_t s);

// -------------------------------------------------------------- morphology
struct MorphJob {
  const uint8_t* src;  // labels, or L when lut != nullptr
  const uint8_t* lut;  // nullptr: src holds cluster labels
  uint8_t* out;        // refined boundary map (0/1)
  int32_t w, h, mode;
};
// all jobs of one launch share the refinement mode
void launch_boundary_morph(const MorphJob* jobs, int n_jobs, int max_w, int max_h, int mode, cudaStream_t s);

// ---------------------------------------------------------------------- CCA
struct CcaJob {
  const uint8_t* b;      // refined map
  uint16_t* lab;         // tile-local labels: the pixel's local root as y * 32 + x within its 32x32 tile, 0xFFFF off the map
  int32_t* node;         // 2 per pixel, used at tile-local roots g only: [2g] parent, [2g + 1] component size
  uint32_t* shist;       // size histogram, shist_len entries (zeroed)
  uint32_t* rowcnt;      // h entries (zeroed)
  int64_t* cut;          // [0] N_b, [1] limit, [2] s*, [3] m, [4] T, [5] number of roots
  uint8_t* out;          // filtered boundary map
  int32_t* roots;        // component roots, appended by k_cc_count (count in cut[5]); room for ceil(w/2) ceil(h/2)
  int32_t* labels_out;   // nullptr or h*w component labels out (smallest linear index, -1 off the map)
  int32_t w, h;
  int32_t shist_len;
  double frac;
  int32_t union_limit;   // most parent links one root search follows, and attempts of one union
};
// A union-find search or union that reaches the limit sets DEV_ERR_CCA_ITER in *dev_err.
void launch_cca(const CcaJob* jobs, int n_jobs, int max_w, int max_h, uint32_t* dev_err, cudaStream_t s);
void launch_cc_filter(const CcaJob* jobs, int n_jobs, int max_w, int max_h, uint32_t* dev_err, cudaStream_t s);

// ---------------------------------------------------------------------- SAD
struct SadJob {
  const uint8_t* Ll;
  const uint8_t* Lr;
  const uint8_t* bmap;  // refined/filtered boundary map (0/1)
  uint32_t* key;        // h*w argmin keys (cost << 10 | d), 0xFFFFFFFF init
  uint16_t* disp;       // out
  uint32_t* cost;       // out or nullptr
  int32_t w, h, D, r;
  // Variant choice, taken on the device from the pair's own boundary count:
  // the direct kernel serves the job iff *nb <= nb_direct_max, the box-sum
  // kernel otherwise (nb null: direct iff nb_direct_max >= 0).
  const int64_t* nb;
  int64_t nb_direct_max;
};

__device__ __forceinline__ bool sad_use_direct(const SadJob& J) {
  return J.nb ? (*J.nb <= J.nb_direct_max) : (J.nb_direct_max >= 0);
}

// Cost model of the automatic SAD choice.  The direct kernel spends about
// 1/kDirectVsBox box-sum (domain pixel, disparity) steps per (anchor,
// computed disparity, window cell); it computes the disparities in passes of
// 64 plus a last pass of 32 (fitted on B300 timings of both kernels over the
// 64 pairs of mixed size, disparity range, block and boundary density of the
// uneven batch and a 4096x2304 frame).  Anchors are estimated from the
// boundary count N_b of the whole image as N_b |Omega| / (w h) plus the two
// domain-edge columns.  Returns the largest N_b for which the direct kernel
// is the cheaper one, or -1 when it never is.
constexpr double kDirectVsBox = 1.0;
inline int64_t sad_direct_limit(int w, int h, int D, int B) {
  const int r = (B - 1) / 2;
  const double omega = (double)(w - D - 2 * r) * (double)(h - 2 * r);
  const int rem = (D + 1) % 64;
  const double computed = 64.0 * ((D + 1) / 64 + (rem > 32 ? 1 : 0)) + (rem > 0 && rem <= 32 ? 32.0 : 0.0);
  const double anchors = kDirectVsBox * omega * (D + 1) / (computed * (double)B * B) - 2.0 * (h - 2 * r);
  if (!(anchors > 0.0)) return -1;
  const double lim = anchors * (double)w * h / omega;   // N_b < lim
  return (int64_t)std::ceil(lim) - 1;
}
// Box-sum variant: items = (job, column strip, disparity chunk, row band)
struct SadItem {
  int32_t job, x0, d0, y0, y1;  // output rows y0..y1 inclusive, inside Omega
};
// Tail disparities: when 1..kTailMax disparities remain past the last whole
// chunk of 64 (D + 1 = 257, 129, 65, ...), a chunk would leave most lanes idle;
// a separate kernel computes them (one box filter per disparity) and the
// box-sum work list stops at the last whole chunk.
constexpr int kTailMax = 8;
__host__ __device__ inline int sad_tail_first(int D) { return ((D + 1) / 64) * 64; }   // 64: the box-sum chunk
__host__ __device__ inline bool sad_has_tail(int D) {
  const int rem = D + 1 - sad_tail_first(D);
  return rem > 0 && rem <= kTailMax;
}
__host__ __device__ inline int sad_tail_strip(int r) { return (256 - 2 * r) & ~31; }   // outputs per tail item
// items: (job, strip x0, first tail disparity, rows y0..y1); max_rem: the most
// tail disparities among the items' jobs (sizes shared memory); queue as below
void launch_sad_tail(const SadJob* jobs, const SadItem* items, int n_items, int max_rem, unsigned* queue,
                     cudaStream_t s);
// max_r: the largest block radius among the items (sizes shared memory);
// uniform_r: the radius every item's job has, or -1 when they differ;
// w16: every job's image width is a multiple of 16 (constant row phases);
// queue: one device counter, zero before the launch (the kernel's work-item cursor)
void launch_sad_boxsum(const SadJob* jobs, const SadItem* items, int n_items, int max_r, int uniform_r, bool w16,
                       unsigned* queue,
                       cudaStream_t s);
// the direct kernel for the jobs whose window spans nw = sad_direct_words(block) words
int sad_direct_words(int block);
// (shared memory sized for the largest window radius and disparity range among them)
void launch_sad_direct(const SadJob* jobs, int n_jobs, int nw, int max_r, int max_D, cudaStream_t s);
void launch_count_nonzero(const uint8_t* const* maps, const int64_t* n, int64_t* out, int n_maps, cudaStream_t s);
int sad_boxsum_smem_bytes(int r);
void launch_sad_finalize(const SadJob* jobs, int n_jobs, int max_w, int max_h, cudaStream_t s);
// strip width of the box-sum kernel for radius r
__host__ __device__ int sad_boxsum_strip(int r);
constexpr int kSadChunk = 64;   // disparities per box-sum work item

// ----------------------------------------------------------- reconstruction
struct ReconJob {
  const uint16_t* sparse;  // SAD output: anchors, UNDET elsewhere (unused when keys is set)
  const uint32_t* keys;    // or the SAD argmin keys themselves ((cost << 10) | d, all ones off the anchors)
  uint16_t* filled;        // Algorithm 1 output
  uint16_t* out;           // Algorithm 2 output (final)
  uint16_t* seg_top;       // nseg * w
  uint16_t* seg_bot;       // nseg * w
  int32_t w, h, D, r, threshold, seg_rows;
  int32_t inplace;         // Algorithm 2 reading: 0 snapshot, 1 in-place top-down sweep
  int32_t mirror;          // 1: the final map is written mirrored (column x to w-1-x)
};
// peek_modes: bit 0 = some job uses the snapshot reading, bit 1 = some job the in-place one
void launch_recon(const ReconJob* jobs, int n_jobs, int max_w, int max_h, int max_nseg, int peek_modes,
                  cudaStream_t s);
int recon_launches(int peek_modes);

// left-right consistency: ok[p] = 1 when left pixel p's match x - dL lies in
// the image and |dL - dR there| <= tol; *count (zero on entry, or null) adds
// the consistent pixels
void launch_lr_consistency(const uint16_t* dL, const uint16_t* dR, int w, int h, int tol, uint8_t* ok,
                           unsigned long long* count, cudaStream_t s);

// --------------------------------------------------------------------- blur
struct BlurJob {
  const uint8_t* rgb;
  const uint16_t* disp;
  uint8_t* out;
  const float* taps;     // 2R+1 normalised 1-D Gaussian taps
  int32_t w, h, R, n_ranges;
  int32_t lo[8], hi[8];
};
// by: output rows per tile, 112 or 64, or kBlurStrip for the strip form
// (bands walked kSB = 32 rows at a time; used where its shared memory fits
// the largest radius, else tiles of 112 rows)
constexpr int kBlurStrip = 32;
void launch_blur(const BlurJob* jobs, int n_jobs, int max_w, int max_h, int max_R, int by, cudaStream_t s);
__host__ __device__ bool blur_strip_fits(int R);
__host__ __device__ int blur_smem_bytes(int R, int by);

}  // namespace sb
