/*
 * sb.h -- C ABI of the B300 (sm_103a) depth-based selective-blurring library.
 *
 * The library computes the data-parallel path of Mukherjee & Guddeti,
 * "Depth-based Selective Blurring in Stereo Images Using Accelerated
 * Framework" (arXiv 2001.07809), Section III: lightness conversion,
 * histogram K-means segmentation, segment-boundary detection and
 * morphological refinement, connected-components clean-up, SAD disparity at
 * the refined boundary pixels, dense disparity reconstruction (Algorithms 1
 * and 2) and the Gaussian blur of Eq. 1-2 over the depth ranges the user
 * does not want in focus.  Every stage runs in hand-written CUDA kernels.
 *
 * Conventions for every entry point
 *   - Image pointers are DEVICE pointers owned by the caller, dense row-major
 *     with no padding: RGB images are h*w*3 bytes (R,G,B interleaved),
 *     single-channel maps h*w elements.  The library never frees them.
 *   - Calls are asynchronous on the context's stream.  Argument errors are
 *     detected on the host and returned at once (SB_ERR_INVALID_ARG) with
 *     nothing launched; CUDA launch errors return SB_ERR_CUDA.  Kernel
 *     faults surface at the next synchronising call.
 *   - The context owns a device workspace grown on demand (cudaMalloc) up to
 *     the budget given to sb_create; a request beyond it returns SB_ERR_OOM.
 *   - sb_last_error() gives a message for the last failure on the context.
 *   - A context is not thread-safe; use one per host thread.
 *
 * Domain (a reading of Section III; the paper does not match near borders):
 * with r = (block-1)/2 and D = max_disp, SAD is evaluated only on
 * Omega = rows [r, h-1-r] x columns [D+r, w-1-r], where every window of every
 * candidate d in [0, D] lies inside both images.  Requirements: block odd in
 * [1, 63]; 0 <= D <= 1023; w >= D + block + 1; h >= block.
 */
#ifndef SB_H
#define SB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SB_OK = 0,
  SB_ERR_INVALID_ARG = 1,
  SB_ERR_CUDA = 2,
  SB_ERR_OOM = 3,
  SB_ERR_TIMEOUT = 4,       /* a bounded device-side loop gave up (see sb_set_union_limit) */
  SB_ERR_UNSUPPORTED = 5,
  SB_ERR_CHECK = 6          /* bounds-checked build only: a device index check failed (see sb_check_probe) */
} sb_status;

typedef struct sb_context sb_context;

/* An inclusive disparity range of INTEREST: pixels whose final disparity
 * lies in any such range stay sharp, all others are blurred (Section III,
 * "Depth-based Selective Blurring"; several discrete ranges are allowed). */
typedef struct {
  int32_t lo, hi;
} sb_range;

#define SB_MAX_RANGES 8
#define SB_UNDETERMINED 0xFFFFu

/* Boundary refinement (Section III): the paper's Fill then Remove, or a
 * 3x3 opening followed by a 3x3 closing. */
enum { SB_MORPH_FILL_REMOVE = 0, SB_MORPH_OPEN_CLOSE = 1 };

/* Algorithm 2 (Section III): an undetermined pixel is estimated from the map
 * after Algorithm 1 (SNAPSHOT, estimates do not feed each other; columns are
 * independent), or each column is swept top down writing every estimate
 * back at once (INPLACE: the pixel just above is the "nearest determined
 * pixel above"; the nearest below is the nearest one determined before the
 * step).  The paper's wording allows both. */
enum { SB_PEEK_SNAPSHOT = 0, SB_PEEK_INPLACE = 1 };

/* Reference image (Section III states the method for the left or the right
 * image).  RIGHT: the disparity map and the blurred output are the right
 * image's; pixel (x, y) of the right image is matched against (x + d, y) of
 * the left one, and the domain is rows [r, h-1-r] x columns [r, w-1-r-D].
 * The library runs the method on the mirrored pair with the roles swapped. */
enum { SB_VIEW_LEFT = 0, SB_VIEW_RIGHT = 1 };

/* SAD implementation: chosen per pair on the device from the pair's own
 * boundary-pixel count N_b and a cost model (direct iff N_b * B^2 is small
 * against w * h), exhaustive window sums at each boundary pixel, or running
 * box sums over the domain.  Both are exact and give identical results. */
enum { SB_SAD_AUTO = 0, SB_SAD_DIRECT = 1, SB_SAD_BOXSUM = 2 };

typedef struct {
  int32_t k;                  /* K-means clusters, 1..255 (Table 3 uses 10)        */
  int32_t max_disp;           /* D: candidates d = 0..D                              */
  int32_t block;              /* odd SAD block side (Table 3 uses 9)                 */
  int32_t disp_threshold;     /* Algorithm 2 threshold (Table 3 uses 0 or 1)         */
  int32_t morph_mode;         /* SB_MORPH_*                                          */
  int32_t kmeans_max_iter;    /* Lloyd update limit (100 is the usual choice)        */
  double cc_remove_fraction;  /* smallest components removed, fraction of boundary   */
                              /* pixels (Section III says about 4 %: 0.04)           */
  float sigma;                /* Gaussian sigma of Eq. 1, (0, 32]; radius ceil(3s)   */
  int32_t n_ranges;           /* 0..SB_MAX_RANGES                                    */
  sb_range ranges[SB_MAX_RANGES];
  int32_t sad_variant;        /* SB_SAD_*                                            */
  int32_t peek_mode;          /* SB_PEEK_*: reading of Algorithm 2                    */
  int32_t view;               /* SB_VIEW_*: the reference image of the pair           */
} sb_params;

/* Fills p with the defaults: K=10, block 9, threshold 1 (Table 3), Fill/Remove,
 * 100 iterations, 4 % removal, sigma 3, D = 64, no range of interest. */
void sb_default_params(sb_params* p);

/* Creates a context on CUDA device `device`.  cuda_stream is a cudaStream_t
 * (NULL = the legacy default stream) that all work is queued on; the caller
 * keeps ownership of it.  mem_budget_bytes bounds the workspace (0 = no bound). */
sb_status sb_create(int device, size_t mem_budget_bytes, void* cuda_stream, sb_context** out);
void sb_destroy(sb_context* ctx);
sb_status sb_set_stream(sb_context* ctx, void* cuda_stream);
const char* sb_last_error(const sb_context* ctx);
/* Waits for the context's stream; reports a sticky CUDA error or a device-side
 * wait that gave up (SB_ERR_TIMEOUT). */
sb_status sb_synchronize(sb_context* ctx);
/* Bytes of device workspace currently held. */
size_t sb_workspace_bytes(const sb_context* ctx);

/* Colour space conversion (Section III, "Colour Space Conversion"): CIE L*
 * of sRGB (D65), stored as round(2.55 L*) in 0..255, per pixel.
 * rgb: h*w*3 bytes; L: h*w bytes out; hist: NULL or uint32[256] out, the
 * 256-bin histogram of L (Section III, "Segmentation"). */
sb_status sb_rgb_to_lightness(sb_context* ctx, const uint8_t* rgb, int32_t w, int32_t h, uint8_t* L,
                              uint32_t* hist);

/* Segmentation (Section III): K-means on the 256-bin histogram of L_left,
 * distance |bin - centre|, each pixel takes the cluster of its bin.
 * Centres start evenly over the occupied range, c_k = Lmin + (k+1/2)(Lmax-Lmin)/K;
 * ties go to the lower cluster; an empty cluster keeps its centre; iteration
 * stops when no bin changes cluster or after max_iter updates.
 * labels: NULL or h*w bytes out; centroids: NULL or double[k] out (device);
 * bin2cluster: NULL or uint8[256] out (device); iters: NULL or int32[1] out (device). */
sb_status sb_kmeans_segment(sb_context* ctx, const uint8_t* L_left, int32_t w, int32_t h, int32_t k,
                            int32_t max_iter, uint8_t* labels, double* centroids, uint8_t* bin2cluster,
                            int32_t* iters);

/* Segment boundary detection and refinement (Section III).  A pixel is on a
 * boundary when an in-image 8-neighbour has another cluster label; then Fill
 * (a 0 with eight 1-neighbours becomes 1) and Remove (a 1 with four
 * 1-neighbours becomes 0), each one pass with outside pixels counted as 0
 * (or, with SB_MORPH_OPEN_CLOSE, a 3x3 opening then closing); then the
 * 8-connected components are ordered by (size, label) and the longest prefix
 * holding at most floor(cc_remove_fraction * N_b) pixels is removed.
 * labels: h*w cluster labels in; boundary: h*w bytes out (0/1, final map);
 * refined: NULL or h*w bytes out (map before component removal);
 * cc_labels: NULL or int32 h*w out, component label of each pixel of the
 * refined map = the smallest linear index in its component, -1 off it. */
sb_status sb_refine_boundaries(sb_context* ctx, const uint8_t* labels, int32_t w, int32_t h, int32_t morph_mode,
                               double cc_remove_fraction, uint8_t* boundary, uint8_t* refined,
                               int32_t* cc_labels);

/* Disparity of boundary pixels (Section III): at every pixel of Omega that
 * is on the boundary map, or lies in Omega's first or last column (the
 * pixels mapping to the disparity map's left and right borders), the d in
 * [0, max_disp] minimising the block x block sum of |L_left - L_right(x-d)|,
 * ties to the smaller d.  disp: uint16 h*w out, the winning d at those pixels
 * and SB_UNDETERMINED elsewhere; cost: NULL or uint32 h*w out, the winning
 * SAD at those pixels and 0 elsewhere.  variant: SB_SAD_*. */
sb_status sb_boundary_sad(sb_context* ctx, const uint8_t* L_left, const uint8_t* L_right, const uint8_t* boundary,
                          int32_t w, int32_t h, int32_t max_disp, int32_t block, int32_t variant, uint16_t* disp,
                          uint32_t* cost);

/* Disparity map reconstruction (Section III, Algorithms 1 and 2), in place.
 * In: disp as written by sb_boundary_sad (anchors = entries other than
 * SB_UNDETERMINED).  Algorithm 1: between two consecutive anchors of a row
 * with equal disparity every pixel takes it.  Algorithm 2: each pixel still
 * undetermined takes, from the nearest determined pixels above and below in
 * its column (inside Omega), the smaller if they differ by more than
 * disp_threshold, else floor of their mean; one neighbour: its value; none: 0.
 * peek_mode SB_PEEK_SNAPSHOT or SB_PEEK_INPLACE selects the reading of
 * "nearest determined pixel above" (see the enum).
 * Out: every pixel set; pixels outside Omega are 0.
 * filled: NULL or uint16 h*w out, the map after Algorithm 1 only; a buffer
 * of its own (SB_ERR_INVALID_ARG when it overlaps disp). */
sb_status sb_reconstruct_disparity(sb_context* ctx, uint16_t* disp, int32_t w, int32_t h, int32_t max_disp,
                                   int32_t block, int32_t disp_threshold, int32_t peek_mode, uint16_t* filled);

/* Depth-based selective blurring (Section III, Eq. 1 and 2): pixels whose
 * disparity lies in none of the ranges get the normalised Gaussian of
 * standard deviation sigma over a (2R+1)^2 window, R = ceil(3 sigma), of the
 * original image with replicated edges, rounded to nearest; the others are
 * copied.  ranges: HOST array of n_ranges entries.  rgb/out_rgb: h*w*3. */
sb_status sb_selective_blur(sb_context* ctx, const uint8_t* rgb, const uint16_t* disp, int32_t w, int32_t h,
                            const sb_range* ranges, int32_t n_ranges, float sigma, uint8_t* out_rgb);

/* Blur kernel form for later sb_selective_blur and sb_run calls on this
 * context: SB_BLUR_TILES_112 / SB_BLUR_TILES_64 (2-D tiles of 64 columns by
 * 112 or 64 rows, each filtering its own halo rows), SB_BLUR_STRIP (a CTA
 * walks 64-column strips down bands of 512 rows, 32 rows per step, keeping
 * the horizontally filtered rows in a ring so no row is filtered twice; taken
 * where its shared memory fits the largest radius of the launch, else tiles
 * of 112 rows), or SB_BLUR_AUTO (the form sb_autotune chose for the launch
 * shape; else, when every pair of the launch has one geometry, the form tuned
 * for the largest tuned batch of that geometry; else tiles of 112 rows).  Every form gives the same bytes.  Returns
 * SB_ERR_INVALID_ARG for any other value. */
enum { SB_BLUR_AUTO = 0, SB_BLUR_STRIP = 32, SB_BLUR_TILES_64 = 64, SB_BLUR_TILES_112 = 112 };
sb_status sb_set_blur_form(sb_context* ctx, int32_t form);

/* Chunking of SB_RUN_HOST_IO | SB_RUN_BATCHED runs on this context: pairs
 * stream through three device staging slots in chunks whose input bytes
 * (left + right RGB) start near first_bytes at both ends of the batch and
 * grow by half from one chunk to the next towards the middle, up to max_bytes
 * (at least one pair per chunk), so
 * the first upload and the last download, which nothing overlaps, stay short.
 * Defaults 64 MB and 1 GB; (0, 0) restores them; 0 < first_bytes <=
 * max_bytes, else SB_ERR_INVALID_ARG.  Smaller chunks need less staging
 * memory (three times the largest chunk's inputs and outputs). */
sb_status sb_set_host_chunk(sb_context* ctx, size_t first_bytes, size_t max_bytes);
/* Number of chunks the last SB_RUN_HOST_IO run on this context used. */
int32_t sb_host_io_chunks(const sb_context* ctx);

/* Bound of the connected-components union-find (Section III's component
 * clean-up; the paper states no bound): every root search follows at most
 * `limit` parent links and every union makes at most `limit` attempts, for
 * later sb_refine_boundaries and sb_run calls on this context.  A run that
 * reaches the bound is not valid: the next sb_synchronize returns
 * SB_ERR_TIMEOUT (and clears the flag; the context stays usable).  0 restores
 * the default, 2^22, far above any chain an image of up to 2^31 pixels
 * builds; a negative limit returns SB_ERR_INVALID_ARG. */
sb_status sb_set_union_limit(sb_context* ctx, int32_t limit);

/* Bounds-checked build.  libsb_checks.so is the same library compiled with
 * -DSB_CHECKS: before every access whose index comes from data (labels,
 * parent links, root lists, work-item tables, anchor positions) a kernel
 * checks the index; a failed check records its site number, skips the access
 * and lets the kernel finish, and the next sb_synchronize returns
 * SB_ERR_CHECK naming the first site (the record is then cleared and the
 * context stays usable).  sb_checks_built returns 1 in that library, 0 in
 * libsb.so.  sb_check_probe enqueues a kernel whose only check fails when
 * trip is nonzero (site 1), to test the reporting path; in libsb.so it
 * returns SB_ERR_UNSUPPORTED. */
int32_t sb_checks_built(void);
sb_status sb_check_probe(sb_context* ctx, int32_t trip);

/* One stereo pair for sb_run. */
typedef struct {
  const uint8_t* left_rgb;   /* h*w*3 */
  const uint8_t* right_rgb;  /* h*w*3 */
  int32_t w, h;
  sb_params p;
  uint8_t* out_rgb;          /* h*w*3 out: the selectively blurred left image */
  uint16_t* out_disp;        /* NULL or h*w out: the final disparity map      */
} sb_pair;

enum {
  SB_RUN_PLAIN = 0,          /* one pair after another, each stage one launch per pair     */
  SB_RUN_BATCHED = 1,        /* each stage one launch over all pairs (work lists per pair) */
  SB_RUN_GRAPH = 2,          /* with BATCHED: replay a captured CUDA graph of the batch    */
  SB_RUN_HOST_IO = 4         /* pair pointers are HOST memory (pinned for overlap); the    */
                             /* library streams them through device buffers, overlapping   */
                             /* host-device copies with the compute of other pairs          */
};

/* The whole pipeline of Section III for n_pairs pairs (pairs: HOST array).
 * Results are identical for every flag combination.  With SB_RUN_GRAPH the
 * first call of a batch shape (every pair's size and parameters) captures
 * and instantiates a CUDA graph; later calls of that shape replay it after
 * rebuilding its job descriptors for the current pointers.  A context keeps
 * the graphs of its 64 most recently used shapes (a graph holds no device
 * memory beyond its kernel nodes); enabling or disabling stage profiling,
 * or a growth of the descriptor blob, drops them. */
sb_status sb_run(sb_context* ctx, const sb_pair* pairs, int32_t n_pairs, uint32_t flags);

/* Boundary SAD for callers that cannot allocate device memory: a plug-in
 * inside a host application that owns all device memory through its own
 * pool, or a real-time loop that must never call cudaMalloc (it can
 * synchronise the device).  The paper has no counterpart; this is a service
 * of the library.  Same result as sb_boundary_sad, but no context: the call
 * queues its work on cuda_stream (a cudaStream_t, NULL = legacy default
 * stream) and allocates nothing.  Its scratch (one 32-bit key per pixel plus
 * the launch descriptors, about 16.25 MB) is a static device array that
 * every GPU loading the library's device code holds until the process exits.
 * CUDA loads that code lazily: the first call on a device (and the first in
 * any other CUDA context) loads it, reserves the array and looks up its
 * address, which can allocate and synchronise, so make one warm-up call
 * before a real-time loop and before any stream capture.  Images above
 * SB_STATIC_MAX_PIXELS pixels are rejected with SB_ERR_INVALID_ARG; a call
 * needing more than SB_STATIC_MAX_ITEMS work items (strips of about 200
 * columns times chunks of 64 disparities, times row bands for small images)
 * is rejected with SB_ERR_UNSUPPORTED: a 4096 x 1024 image with block 41
 * and max_disp 1023 needs about 1,000 on a 148-SM GPU, a 1048576 x 4 image
 * with block 3 and max_disp 1023 would need 74,832.  All calls share the array: calls that overlap on the GPU (other
 * streams, other threads) race and must be ordered by the caller.
 * errbuf: NULL or errbuf_len bytes that receive a message on failure. */
#define SB_STATIC_MAX_PIXELS 4194304
#define SB_STATIC_MAX_ITEMS 13094
sb_status sb_boundary_sad_static(const uint8_t* L_left, const uint8_t* L_right, const uint8_t* boundary, int32_t w,
                                 int32_t h, int32_t max_disp, int32_t block, int32_t variant, uint16_t* disp,
                                 uint32_t* cost, void* cuda_stream, char* errbuf, size_t errbuf_len);

/* Autotuning of two work shapes per launch-group shape (each pair's w, h,
 * max_disp, block and blur radius, in order): the box-sum SAD's work split
 * (how many (pair, strip, disparity chunk, row band) items a launch is cut
 * into: more items balance the persistent grid better, fewer repeat less
 * warm-up work per band; candidates 1, 2, 3 and 6 waves of the grid) and the
 * blur form (tiles of 112 rows, two CTAs per SM; tiles of 64 rows, three CTAs
 * per SM with more halo work; or strips, see sb_set_blur_form).  Runs the
 * pairs with sb_run(flags) once per candidate
 * (a warm-up run and a timed run each, so the outputs are written), keeps the
 * fastest and uses it in every later sb_run of that shape on this context.
 * Device pairs only (flags without SB_RUN_HOST_IO).  ms_out: NULL or
 * SB_AUTOTUNE_CANDIDATES timings (4 splits, then the blur forms 112, 64 and
 * strip); sad_items_out / blur_rows_out: NULL or the chosen values (the blur
 * form as in sb_set_blur_form).  A form set with sb_set_blur_form stays in
 * force over the tuned one.  Synchronises the context stream; not inside a
 * stream capture. */
#define SB_AUTOTUNE_CANDIDATES 7
sb_status sb_autotune(sb_context* ctx, const sb_pair* pairs, int32_t n_pairs, uint32_t flags, float* ms_out,
                      int32_t* sad_items_out, int32_t* blur_rows_out);

/* Left-right consistency of a left-view disparity map dL and a right-view map
 * dR of the same pair (both uint16 h*w device arrays as sb_run writes them):
 * ok[p] = 1 when left pixel p = (x, y) matches x - dL[p] inside the image and
 * |dL[p] - dR[y][x - dL[p]]| <= tol, else 0 (ok: uint8 h*w device array).
 * count: NULL or one device int64 that receives the number of consistent
 * pixels (overwritten).  The method itself has no occlusion handling; this
 * only reports agreement. */
sb_status sb_lr_consistency(sb_context* ctx, const uint16_t* dL, const uint16_t* dR, int32_t w, int32_t h,
                            int32_t tol, uint8_t* ok, int64_t* count);

/* Number of kernel launches the library has issued on this context so far
 * (a graph replay counts every kernel node it runs). */
uint64_t sb_launch_count(const sb_context* ctx);

/* Stage timing: when enabled, the pipeline records a CUDA event on the
 * context stream at each stage boundary (also inside captured graphs).
 * sb_profile_read waits for the last run and writes the milliseconds of up
 * to max_stages stages of it into ms (order: lightness, k-means, boundary
 * refinement, connected components, SAD box sums (the box-sum kernel over
 * the disparity chunks of 32), SAD rest (the tail disparities past the last
 * chunk and the direct-variant kernel), reconstruction, blur); returns the
 * number written, or -1 if nothing was recorded. */
enum { SB_STAGE_LIGHTNESS = 0, SB_STAGE_KMEANS, SB_STAGE_REFINE, SB_STAGE_CCA, SB_STAGE_SAD, SB_STAGE_SAD_REST,
       SB_STAGE_RECON, SB_STAGE_BLUR, SB_N_STAGES };
sb_status sb_profile_enable(sb_context* ctx, int on);
int32_t sb_profile_read(sb_context* ctx, float* ms, int32_t max_stages);

#ifdef __cplusplus
}
#endif

#endif /* SB_H */
