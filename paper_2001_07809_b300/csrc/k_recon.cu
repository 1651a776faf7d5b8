// Disparity map reconstruction from the boundary disparities (Section III).
//
// Algorithm 1 ("Fill"): in each row, every pixel between two consecutive
// anchors of equal disparity takes that disparity.  Equivalently, a
// non-anchor pixel is filled exactly when the nearest anchor on its left and
// the nearest on its right agree.  One warp per row, four pixels per lane: a
// left-to-right pass carries the last anchor's disparity through 128-pixel
// chunks (ballot + shuffle between lanes, a scan inside each lane), a
// right-to-left pass does the same for the next anchor.
//
// Algorithm 2 ("Peek"): each pixel still undetermined after Algorithm 1
// takes, from the nearest determined pixels above and below in its column
// inside Omega, the smaller when they differ by more than the threshold and
// else the floor of their mean.  "Determined" refers to the map after
// Algorithm 1, so the columns are independent: a thread per column, and the
// column is cut into segments of seg_rows rows whose first/last determined
// values are summarised first, so a segment can start its sweeps knowing the
// nearest determined value beyond each of its ends.
//
// Algorithm 2, in-place reading: each column is swept top down and every
// estimate is written back before the next pixel, so the value above an
// undetermined pixel is the output just above it; the nearest determined
// value below is found by an upward pass first.  A thread per column.
#include <algorithm>
#include "sb_common.cuh"

namespace sb {

namespace {
constexpr uint16_t NONE = SB_UNDET16;
constexpr uint16_t kAnchorBit = 0x8000;   // Algorithm 1, between its passes: the pixel is an anchor
// the final map's entry for (y, x) of the working orientation
__device__ __forceinline__ uint16_t& out_at(const ReconJob& J, int y, int x) {
  return J.out[(int64_t)y * J.w + (J.mirror ? J.w - 1 - x : x)];
}
}

__global__ void __launch_bounds__(256) k_recon_fill(const ReconJob* __restrict__ jobs) {
  const ReconJob J = jobs[blockIdx.y];
  const int y = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (y >= J.h) return;
  const int lane = threadIdx.x & 31, w = J.w;
  const uint16_t* srow = J.sparse + (int64_t)y * w;
  const uint32_t* krow = J.keys ? J.keys + (int64_t)y * w : nullptr;
  uint16_t* dst = J.filled + (int64_t)y * w;
  // a lane owns four consecutive pixels of each 128-pixel chunk; whole rows
  // are read and written four elements at a time when they are aligned
  const bool vec = (w & 3) == 0 && ((reinterpret_cast<uintptr_t>(J.filled) & 7) == 0) &&
                   (krow ? (reinterpret_cast<uintptr_t>(J.keys) & 15) == 0 : (reinterpret_cast<uintptr_t>(J.sparse) & 7) == 0);
  // the anchor's disparity at x, or NONE: from the SAD output, or decoded from
  // the argmin keys (no real key is all ones: costs stay below 2^22)
  auto decode = [](uint32_t k) -> uint16_t {
    return k == 0xFFFFFFFFu ? NONE : (uint16_t)(k & ((1u << SB_KEY_DBITS) - 1u));
  };
  auto load4 = [&](int x, uint16_t (&v)[4]) {
    if (vec && x + 3 < w) {
      if (krow) {
        const uint4 k = *reinterpret_cast<const uint4*>(krow + x);
        v[0] = decode(k.x); v[1] = decode(k.y); v[2] = decode(k.z); v[3] = decode(k.w);
      } else {
        const uint2 q = *reinterpret_cast<const uint2*>(srow + x);
        v[0] = (uint16_t)q.x; v[1] = (uint16_t)(q.x >> 16); v[2] = (uint16_t)q.y; v[3] = (uint16_t)(q.y >> 16);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = x + j < w ? (krow ? decode(krow[x + j]) : srow[x + j]) : NONE;
    }
  };
  auto store4 = [&](int x, const uint16_t (&o)[4]) {
    if (vec && x + 3 < w) {
      *reinterpret_cast<uint2*>(dst + x) = make_uint2((uint32_t)o[0] | ((uint32_t)o[1] << 16),
                                                      (uint32_t)o[2] | ((uint32_t)o[3] << 16));
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (x + j < w) dst[x + j] = o[j];
    }
  };
  const int nchunks = (w + 127) / 128;
  // pass 1: disparity of the nearest anchor strictly to the left (NONE if
  // none); anchors are marked with bit 15 (values stay <= 1023, and NONE =
  // 0xffff has bits 10..14 set), so the second pass needs only this row
  uint16_t carry = NONE;
  for (int ci = 0; ci < nchunks; ++ci) {
    const int x = ci * 128 + 4 * lane;
    uint16_t v[4], o[4];
    load4(x, v);
    uint16_t last = NONE;   // the lane's rightmost anchor
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (v[j] != NONE) last = v[j];
    const unsigned mask = __ballot_sync(0xffffffffu, last != NONE);
    const unsigned below = mask & ((1u << lane) - 1u);
    const uint16_t from = __shfl_sync(0xffffffffu, last, below ? 31 - __clz(below) : 0);
    uint16_t cur = below ? from : carry;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const bool anc = v[j] != NONE;
      o[j] = anc ? (uint16_t)(v[j] | kAnchorBit) : cur;
      if (anc) cur = v[j];
    }
    store4(x, o);
    if (mask) carry = __shfl_sync(0xffffffffu, last, 31 - __clz(mask));
  }
  __syncwarp();
  // pass 2: nearest anchor strictly to the right; fill when both sides agree
  carry = NONE;
  for (int ci = nchunks - 1; ci >= 0; --ci) {
    const int x = ci * 128 + 4 * lane;
    uint16_t t[4], o[4];
    if (vec && x + 3 < w) {
      const uint2 q = *reinterpret_cast<const uint2*>(dst + x);
      t[0] = (uint16_t)q.x; t[1] = (uint16_t)(q.x >> 16); t[2] = (uint16_t)q.y; t[3] = (uint16_t)(q.y >> 16);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) t[j] = x + j < w ? dst[x + j] : NONE;
    }
    uint16_t first = NONE;   // the lane's leftmost anchor value
#pragma unroll
    for (int j = 3; j >= 0; --j)
      if (t[j] != NONE && (t[j] & kAnchorBit)) first = (uint16_t)(t[j] & ~kAnchorBit);
    const unsigned mask = __ballot_sync(0xffffffffu, first != NONE);
    const unsigned above = lane == 31 ? 0u : (mask & ~((2u << lane) - 1u));
    const uint16_t from = __shfl_sync(0xffffffffu, first, above ? __ffs(above) - 1 : 0);
    uint16_t cur = above ? from : carry;
#pragma unroll
    for (int j = 3; j >= 0; --j) {
      const bool anc = t[j] != NONE && (t[j] & kAnchorBit);
      const uint16_t v = anc ? (uint16_t)(t[j] & ~kAnchorBit) : t[j];   // the anchor's value, or the left carry
      o[j] = anc ? v : ((v != NONE && v == cur) ? v : NONE);
      if (anc) cur = v;
    }
    store4(x, o);
    if (mask) carry = __shfl_sync(0xffffffffu, first, __ffs(mask) - 1);
  }
}

// first / last determined value of each (segment, column) inside Omega
__global__ void __launch_bounds__(128) k_recon_peek_summary(const ReconJob* __restrict__ jobs) {
  const ReconJob J = jobs[blockIdx.z];
  if (J.inplace) return;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int seg = blockIdx.y;
  const int oy0 = J.r, oy1 = J.h - 1 - J.r;
  const int nseg = (J.h + J.seg_rows - 1) / J.seg_rows;
  if (x >= J.w || seg >= nseg) return;
  const int ya = max(seg * J.seg_rows, oy0), yb = min(seg * J.seg_rows + J.seg_rows - 1, oy1);
  uint16_t first = NONE, last = NONE;
  for (int y = ya; y <= yb; ++y) {
    const uint16_t v = J.filled[(int64_t)y * J.w + x];
    if (v != NONE) {
      if (first == NONE) first = v;
      last = v;
    }
  }
  J.seg_top[(int64_t)seg * J.w + x] = first;
  J.seg_bot[(int64_t)seg * J.w + x] = last;
}

__global__ void __launch_bounds__(128) k_recon_peek_apply(const ReconJob* __restrict__ jobs) {
  const ReconJob J = jobs[blockIdx.z];
  if (J.inplace) return;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int seg = blockIdx.y;
  const int w = J.w;
  const int nseg = (J.h + J.seg_rows - 1) / J.seg_rows;
  if (x >= w || seg >= nseg) return;
  const int oy0 = J.r, oy1 = J.h - 1 - J.r, ox0 = J.D + J.r, ox1 = w - 1 - J.r;
  const int sa = seg * J.seg_rows, sb = min(sa + J.seg_rows - 1, J.h - 1);
  const bool colin = x >= ox0 && x <= ox1;
  const int ya = max(sa, oy0), yb = min(sb, oy1);
  // rows of the segment outside Omega (or whole column outside) are 0
  for (int y = sa; y <= sb; ++y)
    if (!colin || y < oy0 || y > oy1) out_at(J, y, x) = 0;
  if (!colin || ya > yb) return;
  uint16_t above = NONE, below = NONE;
  for (int s = seg - 1; s >= 0; --s) {
    const uint16_t v = J.seg_bot[(int64_t)s * w + x];
    if (v != NONE) { above = v; break; }
  }
  for (int s = seg + 1; s < nseg; ++s) {
    const uint16_t v = J.seg_top[(int64_t)s * w + x];
    if (v != NONE) { below = v; break; }
  }
  // upward sweep: remember the nearest determined value below each pixel
  // (rows in blocks of 8 whose loads are issued together)
  const uint16_t* __restrict__ fl = J.filled + x;
  uint16_t* __restrict__ oc = J.out + (J.mirror ? w - 1 - x : x);
  uint16_t nb = below;
  int y = yb;
  for (; y - 7 >= ya; y -= 8) {
    uint16_t v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = fl[(int64_t)(y - k) * w];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (v[k] != NONE) nb = v[k];
      oc[(int64_t)(y - k) * w] = v[k] != NONE ? v[k] : nb;
    }
  }
  for (; y >= ya; --y) {
    const uint16_t v = fl[(int64_t)y * w];
    if (v != NONE) nb = v;
    oc[(int64_t)y * w] = v != NONE ? v : nb;
  }
  // downward sweep: combine with the nearest determined value above
  uint16_t na = above;
  const int T = J.threshold;
  auto combine = [T](uint16_t na_, uint16_t b) -> uint16_t {
    if (na_ == NONE && b == NONE) return 0;
    if (na_ == NONE) return b;
    if (b == NONE) return na_;
    const int a = na_, c = b;
    const int range = a > c ? a - c : c - a;
    return (uint16_t)(range > T ? min(a, c) : (a + c) / 2);
  };
  y = ya;
  for (; y + 7 <= yb; y += 8) {
    uint16_t v[8], b[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) { v[k] = fl[(int64_t)(y + k) * w]; b[k] = oc[(int64_t)(y + k) * w]; }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (v[k] != NONE) { na = v[k]; continue; }
      oc[(int64_t)(y + k) * w] = combine(na, b[k]);
    }
  }
  for (; y <= yb; ++y) {
    const uint16_t v = fl[(int64_t)y * w];
    if (v != NONE) { na = v; continue; }
    oc[(int64_t)y * w] = combine(na, oc[(int64_t)y * w]);
  }
}

__global__ void __launch_bounds__(128) k_recon_peek_inplace(const ReconJob* __restrict__ jobs) {
  const ReconJob J = jobs[blockIdx.y];
  if (!J.inplace) return;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int w = J.w, h = J.h;
  if (x >= w) return;
  const int oy0 = J.r, oy1 = h - 1 - J.r, ox0 = J.D + J.r, ox1 = w - 1 - J.r;
  const bool colin = x >= ox0 && x <= ox1;
  for (int y = 0; y < h; ++y)
    if (!colin || y < oy0 || y > oy1) out_at(J, y, x) = 0;
  if (!colin) return;
  // upward: the nearest value determined before the step at or below each pixel
  uint16_t nb = NONE;
  for (int y = oy1; y >= oy0; --y) {
    const int64_t p = (int64_t)y * w + x;
    const uint16_t v = J.filled[p];
    if (v != NONE) nb = v;
    out_at(J, y, x) = nb;
  }
  // downward, in place: the output just above is the value above
  uint16_t na = NONE;
  const int T = J.threshold;
  for (int y = oy0; y <= oy1; ++y) {
    const int64_t p = (int64_t)y * w + x;
    const uint16_t v = J.filled[p];
    if (v != NONE) { na = v; continue; }   // the output already holds v
    const uint16_t b = out_at(J, y, x);
    uint16_t o;
    if (na == NONE && b == NONE) o = 0;
    else if (na == NONE) o = b;
    else if (b == NONE) o = na;
    else {
      const int a = na, c = b;
      const int range = a > c ? a - c : c - a;
      o = (uint16_t)(range > T ? min(a, c) : (a + c) / 2);
    }
    out_at(J, y, x) = o;
    na = o;
  }
}

void launch_recon(const ReconJob* jobs, int n_jobs, int max_w, int max_h, int max_nseg, int peek_modes,
                  cudaStream_t s) {
  if (n_jobs <= 0) return;
  k_recon_fill<<<dim3((max_h + 7) / 8, n_jobs), 256, 0, s>>>(jobs);
  if (peek_modes & 1) {
    dim3 g((max_w + 127) / 128, max_nseg, n_jobs);
    k_recon_peek_summary<<<g, 128, 0, s>>>(jobs);
    k_recon_peek_apply<<<g, 128, 0, s>>>(jobs);
  }
  if (peek_modes & 2) k_recon_peek_inplace<<<dim3((max_w + 127) / 128, n_jobs), 128, 0, s>>>(jobs);
}

__global__ void __launch_bounds__(256) k_lr_consistency(const uint16_t* __restrict__ dL, const uint16_t* __restrict__ dR,
                                                        int w, int h, int tol, uint8_t* __restrict__ ok,
                                                        unsigned long long* count) {
  const int64_t n = (int64_t)w * h;
  unsigned long long mine = 0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t y = p / w;
    const int x = (int)(p - y * w), dl = dL[p], xr = x - dl;
    int v = 0;
    if (xr >= 0) {
      const int dr = dR[y * w + xr];
      v = (dl > dr ? dl - dr : dr - dl) <= tol;
    }
    ok[p] = (uint8_t)v;
    mine += v;
  }
  if (count) {
    for (int o = 16; o; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(count, mine);
  }
}

void launch_lr_consistency(const uint16_t* dL, const uint16_t* dR, int w, int h, int tol, uint8_t* ok,
                           unsigned long long* count, cudaStream_t s) {
  const int64_t n = (int64_t)w * h;
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 148 * 8);
  k_lr_consistency<<<std::max(grid, 1), 256, 0, s>>>(dL, dR, w, h, tol, ok, count);
}

// kernels launch_recon issues for the given peek_modes
int recon_launches(int peek_modes) { return 1 + ((peek_modes & 1) ? 2 : 0) + ((peek_modes & 2) ? 1 : 0); }

SB_CHECKS_UNIT(recon)

}  // namespace sb
