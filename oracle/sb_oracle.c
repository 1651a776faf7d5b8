/*
 * ORACLE -- test infrastructure only.
 *
 * A plain, slow, single-threaded CPU statement of what the depth-based
 * selective-blurring pipeline of Mukherjee & Guddeti (arXiv 2001.07809,
 * Section III) computes.  Only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header, table
 * or constant generator with the CUDA library: it builds its own tables from
 * FP64 libm and restates every step literally (pixel loops, an explicit-queue
 * flood fill, a sort of the components, the exhaustive SAD window sum, the
 * row scan of Algorithm 1, the column look-up of Algorithm 2 and a direct 2-D
 * Gaussian window of Eq. 1-2).  Floating point is FP64; build with
 * -ffp-contract=off so every product and sum is rounded as written.
 *
 * Where the paper is silent the oracle takes one reading and says so at the
 * function ("Reading:").  Pins that tie each function to something other than
 * itself live in tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_UNDET 0xFFFFu

/* ------------------------------------------------------------------------
 * Colour space conversion (Section III "Colour Space Conversion"; Section IV).
 * The paper converts RGB to CIE Lab with the transformations of its ref. [9]
 * and keeps L.  Reading: sRGB (IEC 61966-2-1) primaries with D65 white, CIE
 * 1976 L*, stored as an 8-bit value round(2.55 * L*) so that 256 histogram
 * bins cover it.  Per pixel the work is fixed point:
 *   lin[c]  = round(65535 * g(c/255)),  g = sRGB inverse companding
 *   Y16     = (13933 lin[R] + 46871 lin[G] + 4732 lin[B] + 32768) >> 16
 *             (Rec. 709 luminance weights x 65536, summing to 65536)
 *   L8      = floor(2.55 * L*(Y16/65535) + 0.5) clamped to [0, 255]
 *   L*(t)   = 116 t^(1/3) - 16 for t > (6/29)^3, else (29/3)^3 t
 * ------------------------------------------------------------------------ */
static uint16_t g_lin[256];
static uint8_t g_ltab[65536];
static int g_tables_ready = 0;

static double srgb_to_linear(double v) {
  return v <= 0.04045 ? v / 12.92 : pow((v + 0.055) / 1.055, 2.4);
}

static double cie_lstar(double t) {
  const double eps = (6.0 / 29.0) * (6.0 / 29.0) * (6.0 / 29.0);
  const double kappa = (29.0 / 3.0) * (29.0 / 3.0) * (29.0 / 3.0);
  return t > eps ? 116.0 * cbrt(t) - 16.0 : kappa * t;
}

static void build_tables(void) {
  if (g_tables_ready) return;
  for (int c = 0; c < 256; ++c) g_lin[c] = (uint16_t)floor(65535.0 * srgb_to_linear(c / 255.0) + 0.5);
  for (int y = 0; y < 65536; ++y) {
    double v = floor(2.55 * cie_lstar(y / 65535.0) + 0.5);
    g_ltab[y] = (uint8_t)(v < 0 ? 0 : (v > 255 ? 255 : v));
  }
  g_tables_ready = 1;
}

uint8_t or_lightness_of(uint8_t r, uint8_t g, uint8_t b) {
  build_tables();
  uint64_t y = (13933ull * g_lin[r] + 46871ull * g_lin[g] + 4732ull * g_lin[b] + 32768ull) >> 16;
  return g_ltab[y];
}

void or_rgb_to_lightness(const uint8_t* rgb, int64_t n_px, uint8_t* L) {
  build_tables();
  for (int64_t p = 0; p < n_px; ++p) L[p] = or_lightness_of(rgb[3 * p], rgb[3 * p + 1], rgb[3 * p + 2]);
}

/* ------------------------------------------------------------------------
 * Segmentation (Section III "Segmentation"; complexity in Section III): a
 * 256-bin histogram of the left image's L values, K-means on the bins, and
 * each pixel takes its bin's cluster.
 * ------------------------------------------------------------------------ */
void or_histogram(const uint8_t* L, int64_t n_px, uint32_t hist[256]) {
  memset(hist, 0, 256 * sizeof(uint32_t));
  for (int64_t p = 0; p < n_px; ++p) hist[L[p]]++;
}

static void assign_bins(const double* c, int K, uint8_t a[256]) {
  for (int b = 0; b < 256; ++b) {
    int best = 0;
    double bd = fabs((double)b - c[0]);
    for (int k = 1; k < K; ++k) {
      double dk = fabs((double)b - c[k]);
      if (dk < bd) { bd = dk; best = k; }        /* ties keep the smaller k */
    }
    a[b] = (uint8_t)best;
  }
}

/* Lloyd iterations on histogram bins, distance |b - c_k| (one absolute
 * difference, as the complexity analysis of Section III states).
 * Readings (the paper names neither): initial centres spread evenly over
 * the occupied lightness range, c_k = Lmin + ((k + 0.5)(Lmax - Lmin)) / K;
 * ties go to the smaller k; an empty cluster keeps its centre; stop when no
 * bin changes cluster or after max_iter updates.  The centre update
 * c_k = (sum h[b] b) / (sum h[b]) uses exact integer sums and one FP64
 * division.  Returns the number of updates done. */
int or_kmeans_hist(const uint32_t hist[256], int K, int max_iter, double* centroids, uint8_t bin2cluster[256]) {
  int lmin = -1, lmax = -1;
  for (int b = 0; b < 256; ++b)
    if (hist[b]) { if (lmin < 0) lmin = b; lmax = b; }
  if (lmin < 0) {
    for (int k = 0; k < K; ++k) centroids[k] = 0.0;
    memset(bin2cluster, 0, 256);
    return 0;
  }
  for (int k = 0; k < K; ++k) {
    double t = ((double)k + 0.5) * (double)(lmax - lmin);
    centroids[k] = (double)lmin + t / (double)K;
  }
  uint8_t a[256], a2[256];
  assign_bins(centroids, K, a);
  int it = 0;
  while (it < max_iter) {
    ++it;
    for (int k = 0; k < K; ++k) {
      uint64_t num = 0, den = 0;
      for (int b = 0; b < 256; ++b)
        if (a[b] == k) { num += (uint64_t)hist[b] * (uint64_t)b; den += hist[b]; }
      if (den > 0) centroids[k] = (double)num / (double)den;
    }
    assign_bins(centroids, K, a2);
    int changed = memcmp(a, a2, 256) != 0;
    memcpy(a, a2, 256);
    if (!changed) break;
  }
  memcpy(bin2cluster, a, 256);
  return it;
}

void or_label_pixels(const uint8_t* L, int64_t n_px, const uint8_t bin2cluster[256], uint8_t* labels) {
  for (int64_t p = 0; p < n_px; ++p) labels[p] = bin2cluster[L[p]];
}

/* ------------------------------------------------------------------------
 * Segment boundary detection (Section III): a pixel is on a boundary when
 * any pixel of its 8-neighbourhood (Moore neighbourhood) has another
 * cluster.  Reading: neighbours outside the image are ignored.
 * ------------------------------------------------------------------------ */
void or_boundary(const uint8_t* labels, int w, int h, uint8_t* b) {
  for (int y = 0; y < h; ++y)
    for (int x = 0; x < w; ++x) {
      uint8_t me = labels[(int64_t)y * w + x], on = 0;
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          int yy = y + dy, xx = x + dx;
          if ((dx || dy) && yy >= 0 && yy < h && xx >= 0 && xx < w && labels[(int64_t)yy * w + xx] != me) on = 1;
        }
      b[(int64_t)y * w + x] = on;
    }
}

static int px(const uint8_t* m, int w, int h, int x, int y, int outside) {
  if (x < 0 || y < 0 || x >= w || y >= h) return outside;
  return m[(int64_t)y * w + x];
}

/* Fill (Section III, the 3x3 pattern): a 0 whose eight neighbours are all 1
 * becomes 1.  Reading: one parallel pass (every output from the input map);
 * pixels outside the image count as 0, so border pixels are never filled. */
void or_morph_fill(const uint8_t* in, int w, int h, uint8_t* out) {
  for (int y = 0; y < h; ++y)
    for (int x = 0; x < w; ++x) {
      int v = in[(int64_t)y * w + x];
      if (!v) {
        int all = 1;
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx)
            if ((dx || dy) && !px(in, w, h, x + dx, y + dy, 0)) all = 0;
        v = all;
      }
      out[(int64_t)y * w + x] = (uint8_t)v;
    }
}

/* Remove (Section III): a 1 whose four 4-connected neighbours are all 1
 * becomes 0, leaving outlines.  Same one-pass and outside-is-0 reading. */
void or_morph_remove(const uint8_t* in, int w, int h, uint8_t* out) {
  for (int y = 0; y < h; ++y)
    for (int x = 0; x < w; ++x) {
      int v = in[(int64_t)y * w + x];
      if (v && px(in, w, h, x - 1, y, 0) && px(in, w, h, x + 1, y, 0) && px(in, w, h, x, y - 1, 0) &&
          px(in, w, h, x, y + 1, 0))
        v = 0;
      out[(int64_t)y * w + x] = (uint8_t)v;
    }
}

/* 3x3 square erosion (outside counts as 1) and dilation (outside counts as 0). */
static void erode3(const uint8_t* in, int w, int h, uint8_t* out) {
  for (int y = 0; y < h; ++y)
    for (int x = 0; x < w; ++x) {
      int v = 1;
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) v &= px(in, w, h, x + dx, y + dy, 1);
      out[(int64_t)y * w + x] = (uint8_t)v;
    }
}
static void dilate3(const uint8_t* in, int w, int h, uint8_t* out) {
  for (int y = 0; y < h; ++y)
    for (int x = 0; x < w; ++x) {
      int v = 0;
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) v |= px(in, w, h, x + dx, y + dy, 0);
      out[(int64_t)y * w + x] = (uint8_t)v;
    }
}

/* Alternative refinement: 3x3 opening followed by 3x3 closing. */
void or_morph_open_close(const uint8_t* in, int w, int h, uint8_t* out) {
  int64_t n = (int64_t)w * h;
  uint8_t* t = (uint8_t*)malloc(n);
  uint8_t* u = (uint8_t*)malloc(n);
  erode3(in, w, h, t);
  dilate3(t, w, h, u);   /* opening */
  dilate3(u, w, h, t);
  erode3(t, w, h, out);  /* closing */
  free(t);
  free(u);
}

/* ------------------------------------------------------------------------
 * Connected components analysis (Section III, the three-step labelling
 * with an 8-connected flood fill).  The flood fill uses an explicit queue
 * instead of recursion.  Components are found in raster order, so each
 * label is the smallest linear index in its component.  Background = -1.
 * Returns the number of components.
 * ------------------------------------------------------------------------ */
int64_t or_cca(const uint8_t* b, int w, int h, int32_t* lab) {
  int64_t n = (int64_t)w * h, ncomp = 0;
  int64_t* queue = (int64_t*)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
  for (int64_t p = 0; p < n; ++p) lab[p] = -1;
  for (int64_t p = 0; p < n; ++p) {            /* 1. search for the next unlabelled pixel */
    if (!b[p] || lab[p] >= 0) continue;
    int64_t head = 0, tail = 0;                /* 2. flood fill its component */
    lab[p] = (int32_t)p;
    queue[tail++] = p;
    while (head < tail) {
      int64_t q = queue[head++];
      int qy = (int)(q / w), qx = (int)(q % w);
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          int yy = qy + dy, xx = qx + dx;
          if ((dx || dy) && yy >= 0 && yy < h && xx >= 0 && xx < w) {
            int64_t s = (int64_t)yy * w + xx;
            if (b[s] && lab[s] < 0) { lab[s] = (int32_t)p; queue[tail++] = s; }
          }
        }
    }
    ++ncomp;                                   /* 3. repeat until all are labelled */
  }
  free(queue);
  return ncomp;
}

typedef struct { int64_t size; int64_t label; } comp_t;

static int cmp_comp(const void* a, const void* b) {
  const comp_t* x = (const comp_t*)a;
  const comp_t* y = (const comp_t*)b;
  if (x->size != y->size) return x->size < y->size ? -1 : 1;
  if (x->label != y->label) return x->label < y->label ? -1 : 1;
  return 0;
}

/* Small-component removal (Section III): order components by pixel count
 * and remove the smallest, which together hold about 4 % of the boundary
 * pixels.  Reading: sort by (size, label) ascending and remove the longest
 * prefix whose total size S satisfies S <= floor(frac * N_b), N_b = number
 * of boundary pixels before removal, frac = 0.04 by default.
 * out = b with the removed components cleared.  Returns pixels removed. */
int64_t or_cc_filter(const uint8_t* b, const int32_t* lab, int w, int h, double frac, uint8_t* out) {
  int64_t n = (int64_t)w * h, nb = 0, nc = 0;
  int64_t* size_at = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  for (int64_t p = 0; p < n; ++p)
    if (b[p]) { ++nb; if (size_at[lab[p]]++ == 0) ++nc; }
  comp_t* comps = (comp_t*)malloc(sizeof(comp_t) * (size_t)(nc > 0 ? nc : 1));
  int64_t k = 0;
  for (int64_t p = 0; p < n; ++p)
    if (size_at[p] > 0) { comps[k].size = size_at[p]; comps[k].label = p; ++k; }
  qsort(comps, (size_t)nc, sizeof(comp_t), cmp_comp);
  int64_t limit = (int64_t)floor(frac * (double)nb), S = 0, removed = 0;
  uint8_t* gone = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
  for (int64_t i = 0; i < nc; ++i) {
    if (S + comps[i].size > limit) break;
    S += comps[i].size;
    gone[comps[i].label] = 1;
  }
  for (int64_t p = 0; p < n; ++p) {
    out[p] = (uint8_t)(b[p] && !gone[lab[p]]);
    removed += b[p] && !out[p];
  }
  free(gone);
  free(comps);
  free(size_at);
  return removed;
}

/* ------------------------------------------------------------------------
 * Disparity measurement of boundary pixels (Section III; cost O(N_b w^2 d)).
 * Reading of the domain: SAD is evaluated only where every window of every
 * candidate disparity lies inside both images, Omega = rows [r, h-1-r] x
 * columns [D+r, w-1-r], r = (block-1)/2, candidates d = 0..D.  The pixels
 * that "map to the left and right borders of the disparity map" are the
 * first and last column of Omega in every Omega row; they are matched in
 * addition to the refined boundary pixels inside Omega.
 * ------------------------------------------------------------------------ */
void or_anchor_mask(const uint8_t* b, int w, int h, int max_disp, int block, uint8_t* anchor) {
  int r = (block - 1) / 2, x0 = max_disp + r, x1 = w - 1 - r;
  for (int y = 0; y < h; ++y)
    for (int x = 0; x < w; ++x) {
      int64_t p = (int64_t)y * w + x;
      int in = y >= r && y <= h - 1 - r && x >= x0 && x <= x1;
      anchor[p] = (uint8_t)(in && (b[p] || x == x0 || x == x1));
    }
}

/* SAD cost of disparity d at (x, y): sum over the block of |L_l - L_r(x - d)|. */
uint32_t or_sad_cost(const uint8_t* Ll, const uint8_t* Lr, int w, int x, int y, int d, int block) {
  int r = (block - 1) / 2;
  uint32_t s = 0;
  for (int i = -r; i <= r; ++i)
    for (int j = -r; j <= r; ++j) {
      int a = Ll[(int64_t)(y + i) * w + (x + j)];
      int c = Lr[(int64_t)(y + i) * w + (x + j - d)];
      s += (uint32_t)(a > c ? a - c : c - a);
    }
  return s;
}

/* Winner takes all: the smallest-cost disparity, ties to the smaller d. */
int or_sad_argmin(const uint8_t* Ll, const uint8_t* Lr, int w, int x, int y, int max_disp, int block, uint32_t* cost) {
  int best = 0;
  uint32_t bc = or_sad_cost(Ll, Lr, w, x, y, 0, block);
  for (int d = 1; d <= max_disp; ++d) {
    uint32_t c = or_sad_cost(Ll, Lr, w, x, y, d, block);
    if (c < bc) { bc = c; best = d; }
  }
  if (cost) *cost = bc;
  return best;
}

/* Right-referenced SAD at right-image pixel (x, y), written out directly:
 * argmin over d of sum |L_R(y+i, x+j) - L_L(y+i, x+j+d)|, ties to the
 * smallest d (Section III states the method for either image of the pair).
 * Used to check the mirrored right view. */
int or_sad_argmin_right(const uint8_t* Ll, const uint8_t* Lr, int w, int x, int y, int max_disp, int block,
                        uint32_t* cost) {
  int r = (block - 1) / 2, best = 0;
  uint32_t bc = 0xFFFFFFFFu;
  for (int d = 0; d <= max_disp; ++d) {
    uint32_t c = 0;
    for (int i = -r; i <= r; ++i)
      for (int j = -r; j <= r; ++j) {
        int a = Lr[(int64_t)(y + i) * w + (x + j)], b = Ll[(int64_t)(y + i) * w + (x + j + d)];
        c += (uint32_t)(a > b ? a - b : b - a);
      }
    if (c < bc) { bc = c; best = d; }
  }
  if (cost) *cost = bc;
  return best;
}

/* Left-right consistency of a left-referenced map dL and a right-referenced
 * map dR (both as the pipeline outputs them): left pixel (x, y) is consistent
 * when its match x - dL lies inside the image and the right map's disparity
 * there differs from dL by at most tol.  ok[p] = 1 or 0; returns the number
 * of consistent pixels. */
int64_t or_lr_consistency(const uint16_t* dL, const uint16_t* dR, int w, int h, int tol, uint8_t* ok) {
  int64_t n = 0;
  for (int y = 0; y < h; ++y)
    for (int x = 0; x < w; ++x) {
      int64_t p = (int64_t)y * w + x;
      int dl = dL[p], xr = x - dl, v = 0;
      if (xr >= 0) {
        int dr = dR[(int64_t)y * w + xr];
        v = (dl > dr ? dl - dr : dr - dl) <= tol;
      }
      ok[p] = (uint8_t)v;
      n += v;
    }
  return n;
}

/* Partial disparity map: d* at every anchor, OR_UNDET elsewhere.  cost may be NULL. */
void or_boundary_sad(const uint8_t* Ll, const uint8_t* Lr, const uint8_t* anchor, int w, int h, int max_disp,
                     int block, uint16_t* disp, uint32_t* cost) {
  for (int64_t p = 0; p < (int64_t)w * h; ++p) {
    disp[p] = OR_UNDET;
    if (cost) cost[p] = 0;
    if (anchor[p]) {
      uint32_t c;
      disp[p] = (uint16_t)or_sad_argmin(Ll, Lr, w, (int)(p % w), (int)(p / w), max_disp, block, &c);
      if (cost) cost[p] = c;
    }
  }
}

/* ------------------------------------------------------------------------
 * Disparity map reconstruction (Section III).
 * Algorithm 1 ("Fill"): scan each row left to right; when two consecutive
 * boundary (anchor) pixels have equal disparity, every pixel between them
 * takes that disparity.
 * ------------------------------------------------------------------------ */
void or_recon_fill(uint16_t* disp, const uint8_t* anchor, int w, int h) {
  for (int y = 0; y < h; ++y) {
    int prev = -1;
    for (int x = 0; x < w; ++x) {
      int64_t p = (int64_t)y * w + x;
      if (!anchor[p]) continue;
      if (prev >= 0 && disp[(int64_t)y * w + prev] == disp[p])
        for (int m = prev + 1; m < x; ++m) disp[(int64_t)y * w + m] = disp[p];
      prev = x;
    }
  }
}

/* Algorithm 2 ("Peek"): every still undetermined pixel looks at the two
 * nearest determined pixels of its column; if their range exceeds the
 * threshold it takes the smaller, else their mean.
 * Readings: "determined" means determined before this step (anchors and
 * Fill output), so estimates do not feed each other; the two nearest are
 * the nearest determined pixel above and the nearest below, inside Omega;
 * with only one of them it is used, with none the pixel gets 0; the mean is
 * the integer floor of (a+b)/2.  Pixels outside Omega get 0. */
void or_recon_peek(const uint16_t* det, int w, int h, int max_disp, int block, int threshold, uint16_t* out) {
  int r = (block - 1) / 2, x0 = max_disp + r, x1 = w - 1 - r, y0 = r, y1 = h - 1 - r;
  for (int y = 0; y < h; ++y)
    for (int x = 0; x < w; ++x) {
      int64_t p = (int64_t)y * w + x;
      if (y < y0 || y > y1 || x < x0 || x > x1) { out[p] = 0; continue; }
      if (det[p] != OR_UNDET) { out[p] = det[p]; continue; }
      int a = -1, c = -1;
      for (int yy = y - 1; yy >= y0; --yy)
        if (det[(int64_t)yy * w + x] != OR_UNDET) { a = det[(int64_t)yy * w + x]; break; }
      for (int yy = y + 1; yy <= y1; ++yy)
        if (det[(int64_t)yy * w + x] != OR_UNDET) { c = det[(int64_t)yy * w + x]; break; }
      int v;
      if (a < 0 && c < 0) v = 0;
      else if (a < 0) v = c;
      else if (c < 0) v = a;
      else {
        int range = a > c ? a - c : c - a;
        v = range > threshold ? (a < c ? a : c) : (a + c) / 2;
      }
      out[p] = (uint16_t)v;
    }
}

/* Algorithm 2 ("Peek"), in-place reading: each column of Omega is swept top
 * down and an estimate is written back before the next pixel is visited, so
 * the nearest determined pixel above an undetermined one is the pixel just
 * above it (an anchor, a Fill output or an estimate of this sweep); the
 * nearest below is the nearest anchor or Fill output below (nothing below
 * has been estimated yet).  The range test, the floor mean, the single
 * neighbour and no-neighbour cases and the pixels outside Omega are as in
 * or_recon_peek. */
void or_recon_peek_inplace(const uint16_t* det, int w, int h, int max_disp, int block, int threshold,
                           uint16_t* out) {
  int r = (block - 1) / 2, x0 = max_disp + r, x1 = w - 1 - r, y0 = r, y1 = h - 1 - r;
  for (int64_t p = 0; p < (int64_t)w * h; ++p) out[p] = 0;
  for (int x = x0; x <= x1; ++x) {
    int above = -1;                       /* the output just above, once there is one */
    for (int y = y0; y <= y1; ++y) {
      int64_t p = (int64_t)y * w + x;
      if (det[p] != OR_UNDET) { out[p] = det[p]; above = det[p]; continue; }
      int below = -1;
      for (int yy = y + 1; yy <= y1; ++yy)
        if (det[(int64_t)yy * w + x] != OR_UNDET) { below = det[(int64_t)yy * w + x]; break; }
      int v;
      if (above < 0 && below < 0) v = 0;
      else if (above < 0) v = below;
      else if (below < 0) v = above;
      else {
        int range = above > below ? above - below : below - above;
        v = range > threshold ? (above < below ? above : below) : (above + below) / 2;
      }
      out[p] = (uint16_t)v;
      above = v;
    }
  }
}

/* ------------------------------------------------------------------------
 * Depth-based selective blurring (Section III, Eq. 1 and Eq. 2).  The blur
 * map marks every pixel whose disparity lies in no range of interest; those
 * pixels get the normalised Gaussian window h = h_g / sum(h_g),
 * h_g(n1, n2) = exp(-(n1^2 + n2^2) / (2 sigma^2)), applied to the original
 * left RGB.  Readings: window radius R = ceil(3 sigma); image borders
 * replicate the edge pixel; per channel the FP64 result is rounded half up
 * and clamped to [0, 255]; ranges are inclusive.
 * ------------------------------------------------------------------------ */
int or_blur_radius(float sigma) { return (int)ceil(3.0 * (double)sigma); }

static int in_ranges(int d, const int32_t* ranges, int n_ranges) {
  for (int i = 0; i < n_ranges; ++i)
    if (d >= ranges[2 * i] && d <= ranges[2 * i + 1]) return 1;
  return 0;
}

static double* gauss2d(float sigma, int* R_out) {
  int R = or_blur_radius(sigma), n = 2 * R + 1;
  double s2 = (double)sigma * (double)sigma, tot = 0.0;
  double* wts = (double*)malloc(sizeof(double) * (size_t)n * n);
  for (int i = -R; i <= R; ++i)
    for (int j = -R; j <= R; ++j) {
      double v = exp(-((double)(i * i + j * j)) / (2.0 * s2));
      wts[(i + R) * n + (j + R)] = v;
      tot += v;
    }
  for (int k = 0; k < n * n; ++k) wts[k] /= tot;
  *R_out = R;
  return wts;
}

static void blur_pixel(const uint8_t* rgb, int w, int h, int x, int y, const double* wts, int R, uint8_t* o) {
  int n = 2 * R + 1;
  for (int ch = 0; ch < 3; ++ch) {
    double acc = 0.0;
    for (int i = -R; i <= R; ++i) {
      int yy = y + i < 0 ? 0 : (y + i >= h ? h - 1 : y + i);
      for (int j = -R; j <= R; ++j) {
        int xx = x + j < 0 ? 0 : (x + j >= w ? w - 1 : x + j);
        acc += wts[(i + R) * n + (j + R)] * (double)rgb[((int64_t)yy * w + xx) * 3 + ch];
      }
    }
    double v = floor(acc + 0.5);
    o[ch] = (uint8_t)(v < 0 ? 0 : (v > 255 ? 255 : v));
  }
}

void or_selective_blur(const uint8_t* rgb, const uint16_t* disp, int w, int h, const int32_t* ranges, int n_ranges,
                       float sigma, uint8_t* out) {
  int R;
  double* wts = gauss2d(sigma, &R);
  for (int y = 0; y < h; ++y)
    for (int x = 0; x < w; ++x) {
      int64_t p = (int64_t)y * w + x;
      if (in_ranges(disp[p], ranges, n_ranges)) {
        out[3 * p] = rgb[3 * p]; out[3 * p + 1] = rgb[3 * p + 1]; out[3 * p + 2] = rgb[3 * p + 2];
      } else {
        blur_pixel(rgb, w, h, x, y, wts, R, out + 3 * p);
      }
    }
  free(wts);
}

/* Blurred value of one pixel (for checks on large images at sampled pixels). */
void or_blur_at(const uint8_t* rgb, int w, int h, int x, int y, float sigma, uint8_t* o) {
  int R;
  double* wts = gauss2d(sigma, &R);
  blur_pixel(rgb, w, h, x, y, wts, R, o);
  free(wts);
}

/* The normalised 2-D kernel itself, (2R+1)^2 values row-major. */
int or_gauss_kernel(float sigma, double* out, int cap) {
  int R;
  double* wts = gauss2d(sigma, &R);
  int n = (2 * R + 1) * (2 * R + 1);
  if (n <= cap) memcpy(out, wts, sizeof(double) * (size_t)n);
  free(wts);
  return R;
}
