/*
 * Per-pixel core of the synthetic stereo generator, shared by the host build
 * (synth.c) and the CUDA build (synth_gpu.cu) so both produce the same bytes.
 * Integer arithmetic only.  Input generation only: none of the selective
 * blurring method's arithmetic is here.
 */
#ifndef SYNTH_CORE_H
#define SYNTH_CORE_H
#include <stdint.h>
#ifndef SYNTH_FN
#define SYNTH_FN static inline
#endif

typedef struct {
  int32_t shape;            /* 0 full frame, 1 rectangle, 2 ellipse            */
  int32_t cx, cy, hw, hh;   /* centre and half extents (px) at frame 0         */
  int32_t vx, vy;           /* translation (px/frame)                           */
  int32_t d0_q8;            /* disparity at the centre, 1/256 px, frame 0      */
  int32_t gx_q16, gy_q16;   /* disparity gradients, 1/65536 px per px          */
  int32_t dd_frame;         /* disparity drift (px/frame), reflected in range  */
  int32_t dmin, dmax;       /* drift range (px)                                 */
  uint32_t tex_seed;
  int32_t mean, contrast;   /* texture lightness mean and amplitude (0..255)   */
  int32_t tint_r, tint_g, tint_b; /* channel gains in 1/256                   */
} synth_layer;

typedef struct {
  int32_t w, h, n_layers, frame;
  int32_t noise_q8;         /* sensor noise sigma in 1/256 grey levels         */
  int32_t gain_l_q10, gain_r_q10; /* per-image gain, 1/1024                   */
  uint64_t noise_seed;
  const synth_layer* layers;
} synth_scene;

SYNTH_FN uint64_t smix(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

SYNTH_FN uint32_t lattice(uint32_t seed, int64_t i, int64_t j) {
  uint64_t k = ((uint64_t)seed << 32) ^ ((uint64_t)(uint32_t)i * 0x632BE59BD9B4E019ull) ^
               ((uint64_t)(uint32_t)j * 0x85157AF5ull);
  return (uint32_t)(smix(k) >> 56);   /* 0..255 */
}

SYNTH_FN int64_t floordiv(int64_t a, int64_t b) {
  int64_t q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
  return q;
}

/* Bilinear value noise at (u/256, v), lattice spacing s px; returns 0..255*256. */
SYNTH_FN int64_t vnoise(uint32_t seed, int64_t u_q8, int64_t v, int64_t s) {
  int64_t sq = s << 8;
  int64_t i = floordiv(u_q8, sq), fu = u_q8 - i * sq;      /* fu in [0, s*256) */
  int64_t j = floordiv(v, s), fv = v - j * s;              /* fv in [0, s)     */
  int64_t a = lattice(seed, i, j), b = lattice(seed, i + 1, j);
  int64_t c = lattice(seed, i, j + 1), d = lattice(seed, i + 1, j + 1);
  int64_t top = a * (sq - fu) + b * fu;                    /* x (s*256)        */
  int64_t bot = c * (sq - fu) + d * fu;
  int64_t val = top * (s - fv) + bot * fv;                 /* x (s*256*s)      */
  return floordiv(val, s * s);                             /* 0..255*256       */
}

/* Texture lightness (0..255) of layer L at layer-local point (u/256, v). */
SYNTH_FN int32_t texture(const synth_layer* L, int64_t u_q8, int64_t v) {
  int64_t n1 = vnoise(L->tex_seed, u_q8, v, 7);            /* coarse octave    */
  int64_t n2 = vnoise(L->tex_seed ^ 0xA5A5A5A5u, u_q8, v, 3); /* fine octave   */
  int64_t n = (2 * n1 + n2) / 3 - 128 * 256;               /* ~[-128,127]*256  */
  int64_t t = L->mean + floordiv(n * L->contrast, 128 * 256);
  if (t < 0) t = 0;
  if (t > 255) t = 255;
  return (int32_t)t;
}

typedef struct { int64_t ox, oy, d0_q8; } layer_pose;

SYNTH_FN int32_t reflect_range(int32_t v, int32_t lo, int32_t hi) {
  if (hi <= lo) return lo;
  int32_t p = 2 * (hi - lo);
  int32_t m = (v - lo) % p;
  if (m < 0) m += p;
  return lo + (m <= hi - lo ? m : p - m);
}

SYNTH_FN layer_pose pose_of(const synth_layer* L, int32_t frame) {
  layer_pose P;
  P.ox = (int64_t)L->vx * frame;
  P.oy = (int64_t)L->vy * frame;
  int32_t d0 = L->d0_q8;
  if (L->dd_frame != 0) {
    int32_t base = (d0 + 128) >> 8;
    int32_t dpx = reflect_range(base + L->dd_frame * frame, L->dmin, L->dmax);
    d0 = d0 + (dpx - base) * 256;
  }
  P.d0_q8 = d0;
  return P;
}

/* Does the layer's shape hold left point (x/256, y)?  x in 1/256 px. */
SYNTH_FN int inside(const synth_layer* L, const layer_pose* P, int64_t x_q8, int64_t y) {
  if (L->shape == 0) return 1;
  int64_t dx = x_q8 - ((L->cx + P->ox) << 8), dy = y - (L->cy + P->oy);
  int64_t hw = (int64_t)L->hw << 8, hh = L->hh;
  if (L->shape == 1) return (dx >= -hw && dx < hw && dy >= -hh && dy < hh);
  /* ellipse: (dx/hw)^2 + (dy/hh)^2 < 1, exact in integers */
  __int128 lhs = (__int128)dx * dx * hh * hh + (__int128)dy * dy * hw * hw;
  return lhs < (__int128)hw * hw * hh * hh;
}

/* disparity (1/256 px) of a layer at left point (x_q8/256, y) */
SYNTH_FN int64_t disp_q8(const synth_layer* L, const layer_pose* P, int64_t x_q8, int64_t y) {
  int64_t dx_q8 = x_q8 - ((L->cx + P->ox) << 8);
  int64_t dy = y - (L->cy + P->oy);
  return P->d0_q8 + floordiv((int64_t)L->gx_q16 * dx_q8, 65536) + floordiv((int64_t)L->gy_q16 * dy * 256, 65536);
}

/* Left point x (1/256 px) that lands at right column xr on a layer:  x = xr + d(x,y). */
SYNTH_FN int64_t left_of_right(const synth_layer* L, const layer_pose* P, int64_t xr, int64_t y) {
  int64_t cxq = (L->cx + P->ox) << 8;
  int64_t dy = y - (L->cy + P->oy);
  /* x(1 - gx) = xr + d0 - gx*cx + gy*dy   (all in 1/256 px, g in 1/65536) */
  int64_t rhs = (xr << 8) + P->d0_q8 - floordiv((int64_t)L->gx_q16 * cxq, 65536) +
                floordiv((int64_t)L->gy_q16 * dy * 256, 65536);
  return floordiv(rhs * 65536, 65536 - L->gx_q16);
}

SYNTH_FN int32_t sensor_noise(uint64_t seed, int64_t x, int64_t y, int32_t c, int32_t which, int32_t sigma_q8) {
  if (sigma_q8 == 0) return 0;
  uint64_t z = smix(seed ^ ((uint64_t)(uint32_t)x << 34) ^ ((uint64_t)(uint32_t)y << 8) ^ ((uint64_t)c << 4) ^ (uint64_t)which);
  int32_t s = 0;
  for (int k = 0; k < 8; ++k) s += (int32_t)((z >> (8 * k)) & 255);
  /* centred Irwin-Hall sum of 8 bytes: sd = sqrt(8*(256^2-1)/12) ~= 209.0 */
  int64_t v = (int64_t)(s - 1020) * sigma_q8;
  return (int32_t)floordiv(v + 209 * 128, 209 * 256);
}

SYNTH_FN uint8_t clamp8(int64_t v) { return (uint8_t)(v < 0 ? 0 : (v > 255 ? 255 : v)); }


/* One pixel (x, y) of both images and the ground truth. */
SYNTH_FN void synth_pixel(const synth_scene* sc, const synth_layer* layers, const layer_pose* pose, int64_t x, int64_t y,
                          uint8_t* left, uint8_t* right, float* gt) {
  const int32_t W = sc->w, n = sc->n_layers;
  int top = 0;
  for (int k = n - 1; k >= 0; --k)
    if (inside(&layers[k], &pose[k], x << 8, y)) { top = k; break; }
  const synth_layer* L = &layers[top];
  int32_t t = texture(L, (x << 8) - (pose[top].ox << 8), y - pose[top].oy);
  if (gt) gt[y * W + x] = (float)disp_q8(L, &pose[top], x << 8, y) / 256.0f;
  int32_t tint[3] = {L->tint_r, L->tint_g, L->tint_b};
  for (int c = 0; c < 3; ++c) {
    int64_t v = (int64_t)t * tint[c] / 256;
    v = v * sc->gain_l_q10 / 1024 + sensor_noise(sc->noise_seed, x, y, c, 0, sc->noise_q8);
    left[(y * W + x) * 3 + c] = clamp8(v);
  }
  int rtop = 0;
  int64_t xl_q8 = 0;
  for (int k = n - 1; k >= 0; --k) {
    int64_t xq = left_of_right(&layers[k], &pose[k], x, y);
    if (inside(&layers[k], &pose[k], xq, y)) { rtop = k; xl_q8 = xq; break; }
    if (k == 0) { rtop = 0; xl_q8 = xq; }
  }
  const synth_layer* R = &layers[rtop];
  int32_t tr = texture(R, xl_q8 - (pose[rtop].ox << 8), y - pose[rtop].oy);
  int32_t rt[3] = {R->tint_r, R->tint_g, R->tint_b};
  for (int c = 0; c < 3; ++c) {
    int64_t v = (int64_t)tr * rt[c] / 256;
    v = v * sc->gain_r_q10 / 1024 + sensor_noise(sc->noise_seed, x, y, c, 1, sc->noise_q8);
    right[(y * W + x) * 3 + c] = clamp8(v);
  }
}

#endif
