// Segment boundary detection and morphological refinement (Section III),
// fused into one stencil kernel over 64x32 output tiles with the halo held in
// shared memory: labels (from L through the bin->cluster table, or given) ->
// 8-neighbour boundary -> Fill -> Remove (halo 3), or -> 3x3 erosion ->
// dilation (opening) -> dilation -> erosion (closing) (halo 5).  Each
// refinement step is one parallel pass; a neighbour outside the image reads
// as 0 for boundary, Fill, Remove and dilation, and as 1 for erosion, so the
// image border neither fills nor erodes.  HBM-bound: 1 byte in, 1 byte out.
#include "sb_common.cuh"

namespace sb {

namespace {
constexpr int TW = 64, TH = 32;

template <int HALO>
struct Tile {
  static constexpr int W = TW + 2 * HALO, H = TH + 2 * HALO;
};

// Evaluate a 3x3 stencil over the sub-region of halo `k` (k <= HALO-1):
// warps take rows, lanes take columns (no division per pixel).
template <int HALO, class F>
__device__ __forceinline__ void region(int k, F f) {
  constexpr int W = Tile<HALO>::W;
  const int i0 = HALO - k, j0 = HALO - k, ni = TH + 2 * k, nj = TW + 2 * k;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = i0 + warp; i < i0 + ni; i += blockDim.x >> 5)
    for (int j = j0 + lane; j < j0 + nj; j += 32) f(i, j, i * W + j);
}

// One tile.  INTERIOR: the tile and its halo lie inside the image, so no
// neighbour test is needed.
template <int MODE, bool INTERIOR>
__device__ __forceinline__ void morph_tile(const MorphJob& J, int tx0, int ty0, uint8_t* s_lab, uint8_t* s_a,
                                           uint8_t* s_b, const uint8_t* s_lut) {
  constexpr int HALO = MODE == 0 ? 3 : 5;
  constexpr int W = Tile<HALO>::W, H = Tile<HALO>::H;
  const int w = J.w, h = J.h;
  const int ox = tx0 - HALO, oy = ty0 - HALO;
  auto inimg = [&](int i, int j) {
    return INTERIOR || ((unsigned)(oy + i) < (unsigned)h && (unsigned)(ox + j) < (unsigned)w);
  };
  {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = warp; i < H; i += blockDim.x >> 5)
      for (int j = lane; j < W; j += 32) {
        uint8_t v = 0;
        if (inimg(i, j)) {
          const uint8_t s = J.src[(int64_t)(oy + i) * w + (ox + j)];
          v = J.lut ? s_lut[s] : s;
        }
        s_lab[i * W + j] = v;
      }
  }
  __syncthreads();
  // boundary: an in-image 8-neighbour with another label
  region<HALO>(HALO - 1, [&](int i, int j, int t) {
    uint8_t on = 0;
    if (inimg(i, j)) {
      const uint8_t me = s_lab[t];
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx)
          if ((dx | dy) && inimg(i + dy, j + dx) && s_lab[t + dy * W + dx] != me) on = 1;
    }
    s_a[t] = on;
  });
  __syncthreads();
  auto nb = [&](const uint8_t* buf, int i, int j, int t, int pad) -> int {
    return inimg(i, j) ? buf[t] : pad;
  };
  if (MODE == 0) {
    // Fill: a 0 whose eight neighbours are 1 becomes 1
    region<HALO>(HALO - 2, [&](int i, int j, int t) {
      uint8_t v = 0;
      if (inimg(i, j)) {
        v = s_a[t];
        if (!v) {
          int all = 1;
#pragma unroll
          for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx)
              if (dx | dy) all &= nb(s_a, i + dy, j + dx, t + dy * W + dx, 0);
          v = (uint8_t)all;
        }
      }
      s_b[t] = v;
    });
    __syncthreads();
    // Remove: a 1 whose four 4-neighbours are 1 becomes 0
    region<HALO>(0, [&](int i, int j, int t) {
      if (!inimg(i, j)) return;
      int v = s_b[t];
      if (v && nb(s_b, i, j - 1, t - 1, 0) && nb(s_b, i, j + 1, t + 1, 0) && nb(s_b, i - 1, j, t - W, 0) &&
          nb(s_b, i + 1, j, t + W, 0))
        v = 0;
      J.out[(int64_t)(oy + i) * w + (ox + j)] = (uint8_t)v;
    });
  } else {
    auto erode = [&](const uint8_t* in, uint8_t* out, int k) {
      region<HALO>(k, [&](int i, int j, int t) {
        int v = 1;
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
          for (int dx = -1; dx <= 1; ++dx) v &= nb(in, i + dy, j + dx, t + dy * W + dx, 1);
        out[t] = (uint8_t)v;
      });
    };
    auto dilate = [&](const uint8_t* in, uint8_t* out, int k) {
      region<HALO>(k, [&](int i, int j, int t) {
        int v = 0;
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
          for (int dx = -1; dx <= 1; ++dx) v |= nb(in, i + dy, j + dx, t + dy * W + dx, 0);
        out[t] = (uint8_t)v;
      });
    };
    erode(s_a, s_b, 3);
    __syncthreads();
    dilate(s_b, s_lab, 2);  // opening (s_lab is free now)
    __syncthreads();
    dilate(s_lab, s_a, 1);
    __syncthreads();
    region<HALO>(0, [&](int i, int j, int t) {
      if (!inimg(i, j)) return;
      int v = 1;
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) v &= nb(s_a, i + dy, j + dx, t + dy * W + dx, 1);
      J.out[(int64_t)(oy + i) * w + (ox + j)] = (uint8_t)v;  // closing
    });
  }
}
}  // namespace

template <int MODE>
__global__ void __launch_bounds__(256) k_boundary_morph(const MorphJob* __restrict__ jobs) {
  constexpr int HALO = MODE == 0 ? 3 : 5;
  constexpr int W = Tile<HALO>::W, H = Tile<HALO>::H;
  __shared__ uint8_t s_lab[H * W];
  __shared__ uint8_t s_a[H * W];
  __shared__ uint8_t s_b[H * W];
  __shared__ uint8_t s_lut[256];
  const MorphJob J = jobs[blockIdx.z];
  const int tx0 = blockIdx.x * TW, ty0 = blockIdx.y * TH;
  if (tx0 >= J.w || ty0 >= J.h) return;
  if (J.lut) {
    s_lut[threadIdx.x] = J.lut[threadIdx.x];
    __syncthreads();
  }
  const bool interior = tx0 >= HALO && ty0 >= HALO && tx0 - HALO + W <= J.w && ty0 - HALO + H <= J.h;
  if (interior)
    morph_tile<MODE, true>(J, tx0, ty0, s_lab, s_a, s_b, s_lut);
  else
    morph_tile<MODE, false>(J, tx0, ty0, s_lab, s_a, s_b, s_lut);
}

void launch_boundary_morph(const MorphJob* jobs, int n_jobs, int max_w, int max_h, int mode, cudaStream_t s) {
  if (n_jobs <= 0) return;
  dim3 grid((max_w + TW - 1) / TW, (max_h + TH - 1) / TH, n_jobs);
  if (mode == 0)
    k_boundary_morph<0><<<grid, 256, 0, s>>>(jobs);
  else
    k_boundary_morph<1><<<grid, 256, 0, s>>>(jobs);
}

}  // namespace sb
