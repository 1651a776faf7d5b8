/*
 * Seeded synthetic rectified stereo pairs (layered and slanted-plane scenes).
 *
 * This module only makes inputs.  It holds none of the selective-blurring
 * method's arithmetic and is shared, as a pure input source, by the CPU
 * oracle tests and by the CUDA path's tests and benchmark.
 *
 * Every output byte is a pure integer function of (scene, frame, x, y): the
 * hash is splitmix64 (Steele, Lea & Flood 2014, the published finaliser), the
 * texture is bilinear value noise on two integer lattices, and the sensor
 * noise is a centred sum of eight uniform bytes (Irwin-Hall, a Gaussian
 * stand-in) scaled to the requested sigma in fixed point.  No floating point
 * is used, so any compiler on any host produces identical bytes.
 *
 * Scene model.  Layers are painted far to near (ascending disparity, the
 * caller sorts them).  A layer has a shape in left-image coordinates (full
 * frame, rectangle or ellipse), a disparity plane d(x,y) = d0 + gx*(x-cx) +
 * gy*(y-cy) in 1/256 px, a texture (mean lightness, contrast, lattice seed),
 * and an RGB tint.  Left pixel (x,y) shows the nearest layer whose shape holds
 * (x,y).  Right pixel (xr,y) shows the nearest layer whose left-image point
 * x = xr + d(x,y) lies in its shape; the layer texture is sampled there with
 * linear interpolation, so slanted planes are resampled and disoccluded
 * strips show background texture never seen in the left image.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#include "synth_core.h"

typedef struct {
  const synth_scene* sc;
  uint8_t *left, *right;
  float* gt;
  int32_t y0, y1;
} job_t;

static void render_rows(const synth_scene* sc, uint8_t* left, uint8_t* right, float* gt, int32_t y0, int32_t y1) {
  layer_pose pose[64];
  for (int k = 0; k < sc->n_layers && k < 64; ++k) pose[k] = pose_of(&sc->layers[k], sc->frame);
  for (int64_t y = y0; y < y1; ++y)
    for (int64_t x = 0; x < sc->w; ++x) synth_pixel(sc, sc->layers, pose, x, y, left, right, gt);
}

static void* job_main(void* arg) {
  job_t* j = (job_t*)arg;
  render_rows(j->sc, j->left, j->right, j->gt, j->y0, j->y1);
  return NULL;
}

/* Render one pair.  left/right: h*w*3 bytes (RGB interleaved, row-major);
 * gt: h*w float disparities of the left image (may be NULL).  Rows are split
 * over n_threads POSIX threads; the bytes do not depend on n_threads. */
int synth_render(const synth_scene* sc, uint8_t* left, uint8_t* right, float* gt, int32_t n_threads) {
  if (!sc || !left || !right || sc->w <= 0 || sc->h <= 0 || sc->n_layers < 1 || sc->n_layers > 64) return 1;
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  if (n_threads > sc->h) n_threads = sc->h;
  if (n_threads == 1) { render_rows(sc, left, right, gt, 0, sc->h); return 0; }
  pthread_t th[256];
  job_t jobs[256];
  for (int i = 0; i < n_threads; ++i) {
    jobs[i].sc = sc; jobs[i].left = left; jobs[i].right = right; jobs[i].gt = gt;
    jobs[i].y0 = (int32_t)((int64_t)sc->h * i / n_threads);
    jobs[i].y1 = (int32_t)((int64_t)sc->h * (i + 1) / n_threads);
    if (pthread_create(&th[i], NULL, job_main, &jobs[i]) != 0) { render_rows(sc, left, right, gt, jobs[i].y0, jobs[i].y1); th[i] = 0; }
  }
  for (int i = 0; i < n_threads; ++i) if (th[i]) pthread_join(th[i], NULL);
  return 0;
}

uint64_t synth_splitmix64(uint64_t z) { return smix(z); }
