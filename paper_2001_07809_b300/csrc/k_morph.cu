// Segment boundary detection and morphological refinement (Section III),
// fused into one stencil kernel per tile: labels (from L through the
// bin->cluster table, or given) -> 8-neighbour boundary -> Fill -> Remove
// (halo 3 rows), or -> 3x3 erosion -> dilation (opening) -> dilation ->
// erosion (closing) (halo 5 rows).  Each refinement step is one parallel pass;
// a neighbour outside the image is ignored by the boundary test, reads as 0
// for Fill, Remove and dilation, and as 1 for erosion, so the image border
// neither fills nor erodes.  1 byte in, 1 byte out per pixel.
#include "sb_common.cuh"

namespace sb {

// The stencils run on bit rows: a tile of BW words (32 columns each) by BH
// output rows; bit j of word k of a staged row is image column
// tx0 - 32 + 32k + j (one halo word on each side, HALO rows above and below).
// Labels are staged as bytes (through the bin->cluster table); the boundary
// test compares a 4-byte group with its eight shifted neighbour groups at once
// (__vcmpne4), and Fill/Remove or the openings and closings are word
// operations on the bit rows (shifts across word boundaries for x -/+ 1).
// Neighbour validity follows the byte form: a neighbour outside the image is
// ignored by the boundary test, reads 0 for Fill, Remove and dilation and 1 for
// erosion.
namespace {
constexpr int BW = 8;                 // output words per tile row (256 columns)
constexpr int BH = 32;                // output rows per tile
constexpr int NWD = BW + 2;           // words per staged row
constexpr int kBitThreads = 256;

// four bytes of 0x00 / 0xff -> bits 0..3
__device__ __forceinline__ uint32_t byte_bits(uint32_t m) { return ((m & 0x01010101u) * 0x10204080u) >> 28; }
// bits 0..3 -> four bytes of 0 / 1
__device__ __forceinline__ uint32_t nib_bytes(uint32_t n) { return (n * 0x00204081u) & 0x01010101u; }
// bytes b of a 4-pixel group at column x4 with lo <= x4 + b < hi, as 0xff
__device__ __forceinline__ uint32_t col_mask(int x4, int lo, int hi) {
  uint32_t m = 0;
#pragma unroll
  for (int b = 0; b < 4; ++b)
    if (x4 + b >= lo && x4 + b < hi) m |= 0xffu << (8 * b);
  return m;
}
// bits j of the word at column c0 with 0 <= c0 + j < w
__device__ __forceinline__ uint32_t in_bits(int c0, int w) {
  const int lo = max(0, -c0), hi = min(32, w - c0);   // bits lo .. hi-1
  if (hi <= lo) return 0u;
  const uint32_t upto = hi >= 32 ? 0xffffffffu : ((1u << hi) - 1u);
  return upto & ~((1u << lo) - 1u);
}
}  // namespace

template <int MODE>
__global__ void __launch_bounds__(kBitThreads) k_boundary_bits(const MorphJob* __restrict__ jobs) {
  constexpr int HALO = MODE == 0 ? 3 : 5;
  constexpr int R = BH + 2 * HALO;   // staged rows: image rows ty0 - HALO .. ty0 + BH + HALO - 1
  constexpr int LW = NWD * 8;        // label words (4 bytes) per staged row
  __shared__ uint32_t s_lab[R * LW];
  __shared__ uint32_t s_p[R * NWD], s_q[R * NWD], s_out[R * NWD];   // bit rows; s_out: 1 = outside the image
  __shared__ uint8_t s_lut[256];
  const MorphJob J = jobs[blockIdx.z];
  const int w = J.w, h = J.h;
  const int tx0 = blockIdx.x * BW * 32, ty0 = blockIdx.y * BH;
  if (tx0 >= w || ty0 >= h) return;
  const int tid = threadIdx.x;
  const int cx0 = tx0 - 32, ry0 = ty0 - HALO;   // image column of staged column 0, image row of staged row 0
  s_lut[tid] = J.lut ? J.lut[tid] : (uint8_t)tid;
  for (int i = tid; i < R * NWD; i += kBitThreads) {
    const int row = i / NWD, k = i - row * NWD, y = ry0 + row;
    s_out[i] = (y < 0 || y >= h) ? 0xffffffffu : ~in_bits(cx0 + 32 * k, w);
  }
  __syncthreads();
  // labels, four per word (bytes outside the image are never compared)
  for (int i = tid; i < R * LW; i += kBitThreads) {
    const int row = i / LW, x4 = cx0 + 4 * (i - row * LW), y = ry0 + row;
    uint32_t v = 0;
    if (y >= 0 && y < h) {
      const uint8_t* src = J.src + (int64_t)y * w;
      if (x4 >= 0 && x4 + 3 < w && ((reinterpret_cast<uintptr_t>(src + x4) & 3) == 0)) {
        const uint32_t raw = *reinterpret_cast<const uint32_t*>(src + x4);
        v = (uint32_t)s_lut[raw & 0xff] | ((uint32_t)s_lut[(raw >> 8) & 0xff] << 8) |
            ((uint32_t)s_lut[(raw >> 16) & 0xff] << 16) | ((uint32_t)s_lut[raw >> 24] << 24);
      } else {
#pragma unroll
        for (int b = 0; b < 4; ++b)
          if (x4 + b >= 0 && x4 + b < w) v |= (uint32_t)s_lut[src[x4 + b]] << (8 * b);
      }
    }
    s_lab[i] = v;
  }
  __syncthreads();
  // boundary bits on staged rows 1 .. R-2: an in-image 8-neighbour with another
  // label.  A thread takes one 4-pixel group (consecutive threads read
  // consecutive label words: no bank conflicts); the eight groups of a
  // 32-column bit word sit in eight consecutive lanes and are OR-ed together
  // with shuffles.  Every thread runs every round (the shuffles need all lanes).
  for (int t0 = 0; t0 < (R - 2) * LW; t0 += kBitThreads) {
    const int t = t0 + tid;
    const bool live = t < (R - 2) * LW;
    const int row = 1 + t / LW, idx = t - (row - 1) * LW, k = idx >> 3, q = idx & 7, y = ry0 + row;
    uint32_t nib = 0;
    if (live && y >= 0 && y < h) {
      const bool up = y - 1 >= 0, dn = y + 1 < h;
      const uint32_t* L0 = s_lab + row * LW;
      auto lw = [&](const uint32_t* Lr, int i) { return i >= 0 && i < LW ? Lr[i] : 0u; };
      const int c0 = cx0 + 32 * k;
      const bool interior = c0 >= 1 && c0 + 32 < w;   // every pixel and both column neighbours inside
      const uint32_t cur = L0[idx];
      auto row_diff = [&](const uint32_t* Lr, bool centre) {
        const uint32_t m = lw(Lr, idx), pv = lw(Lr, idx - 1), nx = lw(Lr, idx + 1);
        const uint32_t lft = (m << 8) | (pv >> 24), rgt = (m >> 8) | (nx << 24);
        uint32_t dl = __vcmpne4(cur, lft), dr = __vcmpne4(cur, rgt);
        if (!interior) {
          const int x4 = c0 + 4 * q;
          dl &= col_mask(x4, 1, w + 1);    // x - 1 inside
          dr &= col_mask(x4, -1, w - 1);   // x + 1 inside
        }
        return dl | dr | (centre ? 0u : __vcmpne4(cur, m));
      };
      uint32_t acc = row_diff(L0, true);
      if (up) acc |= row_diff(L0 - LW, false);
      if (dn) acc |= row_diff(L0 + LW, false);
      if (!interior) acc &= col_mask(c0 + 4 * q, 0, w);
      nib = byte_bits(acc) << (4 * q);
    }
    nib |= __shfl_xor_sync(0xffffffffu, nib, 1);
    nib |= __shfl_xor_sync(0xffffffffu, nib, 2);
    nib |= __shfl_xor_sync(0xffffffffu, nib, 4);
    if (live && q == 0) s_p[row * NWD + k] = nib;
  }
  __syncthreads();
  // word neighbours of bit rows: x - 1 and x + 1 (bits shifted in from the next words; 0 past the tile)
  auto xl = [](const uint32_t* B, int row, int k) {
    return (B[row * NWD + k] << 1) | (k > 0 ? B[row * NWD + k - 1] >> 31 : 0u);
  };
  auto xr = [](const uint32_t* B, int row, int k) {
    return (B[row * NWD + k] >> 1) | (k + 1 < NWD ? B[row * NWD + k + 1] << 31 : 0u);
  };
  // one stencil pass over staged rows [r0, r1): f(B, row, k) -> word
  auto pass = [&](const uint32_t* B, uint32_t* O, int r0, int r1, auto f) {
    for (int t = tid; t < (r1 - r0) * NWD; t += kBitThreads) {
      const int row = r0 + t / NWD, k = t - (row - r0) * NWD;
      O[row * NWD + k] = f(B, row, k);
    }
  };
  const uint32_t* res;
  if (MODE == 0) {
    // Fill: a 0 whose eight neighbours are 1 becomes 1 (outside the image reads 0)
    pass(s_p, s_q, 2, R - 2, [&](const uint32_t* B, int row, int k) {
      const uint32_t all = xl(B, row - 1, k) & B[(row - 1) * NWD + k] & xr(B, row - 1, k) & xl(B, row, k) &
                           xr(B, row, k) & xl(B, row + 1, k) & B[(row + 1) * NWD + k] & xr(B, row + 1, k);
      return (B[row * NWD + k] | all) & ~s_out[row * NWD + k];
    });
    __syncthreads();
    // Remove: a 1 whose four 4-neighbours are 1 becomes 0
    pass(s_q, s_p, HALO, HALO + BH, [&](const uint32_t* B, int row, int k) {
      const uint32_t all4 = xl(B, row, k) & xr(B, row, k) & B[(row - 1) * NWD + k] & B[(row + 1) * NWD + k];
      return B[row * NWD + k] & ~all4;
    });
    res = s_p;
  } else {
    auto erode = [&](const uint32_t* B, int row, int k) {   // outside the image reads 1
      uint32_t v = 0xffffffffu;
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy) {
        const int rr = row + dy;
        const uint32_t o = s_out[rr * NWD + k];
        const uint32_t ol = (o << 1) | (k > 0 ? s_out[rr * NWD + k - 1] >> 31 : 0xffffffffu >> 31);
        const uint32_t orr = (o >> 1) | (k + 1 < NWD ? s_out[rr * NWD + k + 1] << 31 : 0x80000000u);
        v &= (B[rr * NWD + k] | o) & (xl(B, rr, k) | ol) & (xr(B, rr, k) | orr);
      }
      return v & ~s_out[row * NWD + k];
    };
    auto dilate = [&](const uint32_t* B, int row, int k) {   // outside the image reads 0 (B is 0 there)
      uint32_t v = 0;
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy) v |= B[(row + dy) * NWD + k] | xl(B, row + dy, k) | xr(B, row + dy, k);
      return v & ~s_out[row * NWD + k];
    };
    pass(s_p, s_q, 2, R - 2, erode);            // opening: erosion
    __syncthreads();
    pass(s_q, s_p, 3, R - 3, dilate);           //          dilation
    __syncthreads();
    pass(s_p, s_q, 4, R - 4, dilate);           // closing: dilation
    __syncthreads();
    pass(s_q, s_p, HALO, HALO + BH, erode);     //          erosion
    res = s_p;
  }
  __syncthreads();
  // output: the tile's rows and words 1 .. BW as bytes 0 / 1
  for (int t = tid; t < BH * BW * 8; t += kBitThreads) {
    const int row = t / (BW * 8), rest = t - row * (BW * 8), k = 1 + rest / 8, q = rest & 7;
    const int y = ty0 + row, x4 = cx0 + 32 * k + 4 * q;
    if (y >= h || x4 >= w) continue;
    const uint32_t v = nib_bytes((res[(HALO + row) * NWD + k] >> (4 * q)) & 0xfu);
    uint8_t* dst = J.out + (int64_t)y * w + x4;
    if (x4 + 3 < w && ((reinterpret_cast<uintptr_t>(dst) & 3) == 0)) {
      *reinterpret_cast<uint32_t*>(dst) = v;
    } else {
      for (int b = 0; b < 4 && x4 + b < w; ++b) dst[b] = (uint8_t)(v >> (8 * b));
    }
  }
}

void launch_boundary_morph(const MorphJob* jobs, int n_jobs, int max_w, int max_h, int mode, cudaStream_t s) {
  if (n_jobs <= 0) return;
  dim3 grid((max_w + BW * 32 - 1) / (BW * 32), (max_h + BH - 1) / BH, n_jobs);
  if (mode == 0)
    k_boundary_bits<0><<<grid, kBitThreads, 0, s>>>(jobs);
  else
    k_boundary_bits<1><<<grid, kBitThreads, 0, s>>>(jobs);
}

SB_CHECKS_UNIT(morph)

}  // namespace sb
