// Disparity of boundary pixels (Section III): winner-takes-all SAD over
// d = 0..D of block x block windows of L, cost O(N_b w^2 d).  Two exact
// implementations share the key encoding key = (cost << 10) | d, so the
// smallest key is the smallest cost with ties to the smallest d.
//
// Box-sum variant (dense over the domain, O(|Omega| d) with a few integer
// operations per pixel and disparity): a CTA owns a strip of TX output
// columns, a band of rows and a chunk of 64 disparities.
//   Stage A: thread t owns column c = x0 - r + t and keeps the 64 vertical
//     window sums V_d(y, c) = sum_{|i|<=r} |L(y+i, c) - R(y+i, c-d)| in
//     registers as 32 packed u16 pairs, sliding down one row per step.  Four
//     disparities at a time: one packed |L - R| of four bytes for the
//     entering row and one for the leaving row (vabsdiff4), split into even
//     and odd bytes (lop3 / prmt), and lane-wise u16 add-subtract (iadd3).
//     Rows are staged with cp.async into a shared-memory ring one group of
//     rows ahead, so every byte is read from HBM once per CTA and the copy
//     overlaps the arithmetic.
//   Stage B: lanes = disparity pairs (one 32-bit word of a column slot holds
//     a lane's two u16 column sums); a warp slides the horizontal sums along
//     its row segment in blocks of 8 outputs with two running words (the
//     packed pair and the upper window sum, from which the lower one is
//     recovered exactly at anchors; a zero column before each row of column
//     sums lets every output use the same add-entering / drop-leaving
//     update).  At anchor pixels (warp-uniform bits, one uniform jump per four
//     outputs) it reduces (S << 10 | d) over the warp with redux.sync; the
//     minimum of output o of the 32-output span goes to word o of a per-warp
//     shared row, and lane o keeps it in the per-pixel key with one atomicMin.
// Tail kernel: the 1..8 disparities past the last whole chunk of 64 (one
// disparity at D = 2^n), a thread per column with the vertical sums and a
// warp prefix sum per row for the horizontal ones, so the box-sum work list
// need not spend a mostly idle chunk on them.
// Direct variant (for low boundary density and small blocks): a warp per
// anchor, lanes = disparities, vabsdiff4.add over the re-aligned 4-byte
// words of each window row.
#include <algorithm>
#include "sb_common.cuh"

namespace sb {

namespace {
constexpr int kThreads = 256;
constexpr int kG = 2;                           // output rows per Stage A -> Stage B hand-off
constexpr int kSegs = 4;                        // Stage B segments per row: warp = (row of the group, segment)
constexpr int kMaxCols = 248;                   // column slots per row: a zero column, then TX + 2r columns
constexpr int kColBytes = 144;                  // bytes per column: 64 u16 sums + 16 (conflict-free STS.128)
constexpr int kLBytes = 272;                    // staged L bytes per row (240 + 16-byte alignment slack)
constexpr int kRBytes = 352;                    // staged R bytes per row (TX + 2r + 63 + look-ahead + slack)
constexpr int kRowBytes = kLBytes + kRBytes;    // 624, a multiple of 16
constexpr int kBBytes = 272;                    // staged boundary-map bytes per output row
static_assert(kSadChunk == 64, "the box-sum kernel covers 64 disparities per item");

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Copy 16-byte chunk `ch` of the image segment that starts at absolute byte
// offset a16 (a multiple of 16, possibly outside the image) into dst.  Bytes
// outside the image buffer of n bytes are never used by the caller: a chunk
// that starts before the buffer is read from offset 0 instead, a chunk that
// runs past its end is copied byte by byte with the index clamped.  `fast`
// (16-byte aligned image base) selects cp.async for whole in-buffer chunks.
__device__ __forceinline__ void stage_chunk(uint8_t* dst, const uint8_t* img, int64_t n, int64_t a16, int ch,
                                            bool fast) {
  int64_t src = a16 + 16 * (int64_t)ch;
  if (src < 0) src = 0;
  if (fast && src + 16 <= n) {
    cp_async16(dst + 16 * ch, img + src);
  } else {
#pragma unroll 1
    for (int k = 0; k < 16; ++k) {
      const int64_t q = src + k < n ? src + k : n - 1;
      dst[16 * ch + k] = img[q];
    }
  }
}
}  // namespace

__host__ __device__ int sad_boxsum_strip(int r) { return (kMaxCols - 1 - 2 * r) & ~31; }
__host__ __device__ static inline int box_vcols(int r) { return sad_boxsum_strip(r) + 2 * r + 1; }

namespace {
// Anchor emission for four consecutive outputs K0 .. K0+3 of a block whose
// anchor bits are the compile-time nibble NIB.  Lane p holds the packed
// running sums of its disparity pair (dlo, dhi) after output K: T = Slo +
// 65536 Shi (mod 2^32) and H = Shi, so Slo = T - (Shi << 16).  The lane's
// two keys (S << 10 | d) are reduced in the lane, then over the warp (redux.sync) for
// every anchor of the nibble first, so that the reductions' latencies
// overlap; the warp minimum of output o of the 32-output span goes to word o
// of the warp's slot row `sbest` (one uniform store: every lane writes the
// same value to the same word), from which lane o takes it for one atomicMin
// per anchor at the end of the span.  Disparities past D carry
// all-ones low bits, which makes their key all ones (never the minimum).
template <unsigned NIB, int K0>
__device__ __forceinline__ void emit_nibble(const uint32_t (&Tv)[8], const uint32_t (&Hv)[8], uint32_t dlo,
                                            uint32_t dhi, uint32_t* sbest) {
  uint32_t m[4];
#pragma unroll
  for (int b = 0; b < 4; ++b)
    if (NIB & (1u << b)) {
      const uint32_t shi = Hv[K0 + b];
      const uint32_t slo = Tv[K0 + b] - (shi << 16);
      const uint32_t k = min((slo << SB_KEY_DBITS) | dlo, (shi << SB_KEY_DBITS) | dhi);
      m[b] = __reduce_min_sync(0xffffffffu, k);
    }
#pragma unroll
  for (int b = 0; b < 4; ++b)
    if (NIB & (1u << b)) sbest[K0 + b] = m[b];
}

// one case per non-empty nibble value: the bits are warp-uniform, so the
// switch is a uniform jump and every case's code is straight-line
template <int K0>
__device__ __forceinline__ void emit_block_half(unsigned nib, const uint32_t (&Tv)[8], const uint32_t (&Hv)[8],
                                                uint32_t dlo, uint32_t dhi, uint32_t* sbest) {
  switch (nib) {
#define SB_EMIT_CASE(v) \
  case v: emit_nibble<v, K0>(Tv, Hv, dlo, dhi, sbest); break;
    SB_EMIT_CASE(1) SB_EMIT_CASE(2) SB_EMIT_CASE(3) SB_EMIT_CASE(4) SB_EMIT_CASE(5)
    SB_EMIT_CASE(6) SB_EMIT_CASE(7) SB_EMIT_CASE(8) SB_EMIT_CASE(9) SB_EMIT_CASE(10)
    SB_EMIT_CASE(11) SB_EMIT_CASE(12) SB_EMIT_CASE(13) SB_EMIT_CASE(14) SB_EMIT_CASE(15)
#undef SB_EMIT_CASE
    default: break;
  }
}

// Vertical step of one row for strip column tid: the entering row (L byte at
// rin[li], R words from Ri at bit shift shi) is added and the leaving row (rout,
// lo, Ro, sho) subtracted in the 32 packed u16 pairs.  Byte b of the realigned
// R word g is disparity d0 + 63 - 4g - b; Ve[g] holds its even bytes (b = 0, 2),
// Vo[g] its odd bytes (b = 1, 3), as u16 lanes: the sums stay in [0, 63 * 255],
// so no carry or borrow crosses a lane.
__device__ __forceinline__ void vertical_row(uint32_t (&Ve)[16], uint32_t (&Vo)[16], const uint8_t* rin, int li,
                                             const uint32_t* Ri, int shi, const uint8_t* rout, int lo,
                                             const uint32_t* Ro, int sho) {
  const uint32_t Lin = (uint32_t)rin[li] * 0x01010101u;
  const uint32_t Lout = (uint32_t)rout[lo] * 0x01010101u;
  uint32_t wi = Ri[0], wo = Ro[0];
#pragma unroll
  for (int g = 0; g < 16; ++g) {
    const uint32_t wi2 = Ri[g + 1], wo2 = Ro[g + 1];
    const uint32_t ri = __funnelshift_r(wi, wi2, shi), ro = __funnelshift_r(wo, wo2, sho);
    wi = wi2;
    wo = wo2;
    const uint32_t ai = __vabsdiffu4(Lin, ri), ao = __vabsdiffu4(Lout, ro);
    Ve[g] = Ve[g] + (ai & 0x00FF00FFu) - (ao & 0x00FF00FFu);
    Vo[g] = Vo[g] + __byte_perm(ai, 0u, 0x4341) - __byte_perm(ao, 0u, 0x4341);
  }
}
}  // namespace

// Persistent: each CTA takes the next work item from the queue counter (zero
// before the launch) until the list is exhausted; items come in the order of
// the list, which the host sorts largest first.  W16: every job's width is a
// multiple of 16, so the 16-byte phase of a strip column is the same in every
// row and the vertical pass of the rows past the warm-up uses the item's
// constant offsets.
template <bool W16, int RC>
__global__ void __launch_bounds__(kThreads, 2) k_sad_boxsum(const SadJob* __restrict__ jobs,
                                                            const SadItem* __restrict__ items, int n_items,
                                                            unsigned* __restrict__ queue) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ int s_item;
  __shared__ uint32_t s_best[kThreads];   // per warp: the span's 32 anchor keys
  for (;;) {
    __syncthreads();  // every thread is done with the previous item (and has read s_item)
    if (threadIdx.x == 0) s_item = (int)atomicAdd(queue, 1u);
    __syncthreads();
    if (s_item >= n_items) break;
    const SadItem it = items[s_item];
    const SadJob J = jobs[it.job];
    if (sad_use_direct(J)) continue;                        // the direct kernel serves this pair
    // a work item inside Omega, on a chunk of the disparity range
    if (!SB_CHECK(it.y0 >= J.r && it.y0 <= it.y1 && it.y1 <= J.h - 1 - J.r && it.x0 >= J.D + J.r &&
                  it.x0 < J.w - J.r && it.d0 >= 0 && it.d0 <= J.D && it.d0 % kSadChunk == 0, 401u))
      continue;
    const int r = RC > 0 ? RC : J.r, D = J.D, w = J.w;     // RC: every job's radius, known at compile time
    const int64_t npx = (int64_t)w * J.h;
    const int ring = 2 * r + 1 + 2 * kG;                    // + one group staged ahead
    const int VC = box_vcols(r);
    uint8_t* s_ring = smem;                                 // ring rows: [L | R]
    uint8_t* s_zero = s_ring + ring * kRowBytes;            // zero row (warm-up leaving rows)
    uint8_t* s_bm = s_zero + kRowBytes;                     // 2 x kG boundary-map rows
    uint8_t* s_vs = s_bm + 2 * kG * kBBytes;                // kG x VC x kColBytes
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int TX = sad_boxsum_strip(r);
    const int NC = TX + 2 * r;
    const int x0 = it.x0, d0 = it.d0;
    const int xo0 = D + r, xo1 = w - 1 - r;                 // Omega columns
    const int cstart = x0 - r;                              // strip column 0
    const int rstart = cstart - d0 - (kSadChunk - 1);       // first R byte any thread needs
    const int y_first = it.y0, y_last = it.y1;              // output rows of the band
    const bool fast = (((uintptr_t)J.Ll | (uintptr_t)J.Lr | (uintptr_t)J.bmap) & 15) == 0;
    const int nchL = (15 + NC + 15) / 16, nchR = (15 + NC + kSadChunk - 1 + 4 + 15) / 16, nchB = (15 + TX + 15) / 16;

    for (int i = tid; i < kRowBytes / 4; i += kThreads) reinterpret_cast<uint32_t*>(s_zero)[i] = 0u;
    for (int i = tid; i < kG * (kColBytes / 4); i += kThreads)   // column 0 of every row slot is zero
      reinterpret_cast<uint32_t*>(s_vs + (i / (kColBytes / 4)) * VC * kColBytes)[i % (kColBytes / 4)] = 0u;

    // stage the entering rows of the group starting at virtual output row yg, and
    // the boundary-map rows of its real output rows, into buffer `buf`; thread
    // tid copies chunk (tid & 127) of ring row (tid >> 7) and chunk (tid & 31) of
    // boundary row (tid >> 5): at most 17 + 21 chunks per ring row, 16 per map row
    const int per = nchL + nchR;
    auto stage = [&](int yg, int slot_first, int buf) {
      const int ng = min(kG, y_last - yg + 1);
      {
        const int k = tid >> 7, ch = tid & 127;
        if (k < ng && ch < per) {
          const int yin = yg + k + r;
          const int sl = slot_first + k < ring ? slot_first + k : slot_first + k - ring;
          uint8_t* row = s_ring + sl * kRowBytes;
          const int64_t ro = (int64_t)yin * w;
          if (ch < nchL) stage_chunk(row, J.Ll, npx, (ro + cstart) & ~(int64_t)15, ch, fast);
          else stage_chunk(row + kLBytes, J.Lr, npx, (ro + rstart) & ~(int64_t)15, ch - nchL, fast);
        }
      }
      {
        const int k = tid >> 5, ch = tid & 31;
        const int y = yg + k;
        if (k < ng && ch < nchB && y >= y_first)
          stage_chunk(s_bm + (buf * kG + k) * kBBytes, J.bmap, npx, ((int64_t)y * w + x0) & ~(int64_t)15, ch, fast);
      }
      cp_async_commit();
    };

    // Stage A state: 64 vertical window sums as 32 packed u16 pairs
    uint32_t Ve[16], Vo[16];
#pragma unroll
    for (int g = 0; g < 16; ++g) Ve[g] = Vo[g] = 0u;

    // Stage B: lane p reads word p of a column slot.  Words 4m .. 4m+3 hold
    // Ve[2m], Vo[2m], Ve[2m+1], Vo[2m+1], so lane p = 4m + q carries the pair
    // dlo = d0 + 63 - 4g' - (q & 1), dhi = dlo - 2 with g' = 2m + (q >> 1)
    uint32_t dlo, dhi;
    {
      const int m = lane >> 2, q = lane & 3, gp = 2 * m + (q >> 1);
      const int lo = d0 + kSadChunk - 1 - 4 * gp - (q & 1), hi = lo - 2;
      dlo = lo <= D ? (uint32_t)lo : 0xFFFFFFFFu;
      dhi = hi <= D ? (uint32_t)hi : 0xFFFFFFFFu;
    }

    // ring slot and 16-byte alignment offsets of the first entering row of the
    // current group, advanced incrementally (no division in the row loop).  The
    // leaving row y - r - 1 is 2r + 1 rows before the entering row y + r, which
    // is 2*kG slots ahead in the ring.
    const int wm = w & 15, back = ((2 * r + 1) * w) & 15;
    int slot = (y_first - r) % ring;
    int offL = (int)(((int64_t)(y_first - r) * w + cstart) & 15);
    int offR = (int)(((int64_t)(y_first - r) * w + rstart) & 15);
    // W16: the offsets of every row are these
    const int aL = offL + tid, aR = kLBytes + ((offR + tid) >> 2) * 4, shA = ((offR + tid) & 3) * 8;
    int k_iter = 0;
    stage(y_first - 2 * r, slot, 0);
    // virtual output rows run from y_first - 2r (warm-up) to y_last
    for (int yg = y_first - 2 * r; yg <= y_last; yg += kG, ++k_iter) {
      const int ng = min(kG, y_last - yg + 1);
      const int buf = k_iter & 1;
      cp_async_wait_all();
      __syncthreads();  // this group's rows have landed; the previous Stage B is done
      const int slot_next = slot + kG < ring ? slot + kG : slot + kG - ring;
      if (yg + kG <= y_last) stage(yg + kG, slot_next, buf ^ 1);
      // Stage A: ng row steps
      if (tid < NC) {
        if (W16 && yg >= y_first + 1) {
          // every row of the group has a real leaving row and stores its sums
          int sin = slot;
#pragma unroll
          for (int k = 0; k < kG; ++k) {
            if (k < ng) {
              int sout = sin + 2 * kG;
              if (sout >= ring) sout -= ring;
              const uint8_t* rin = s_ring + sin * kRowBytes;
              const uint8_t* rout = s_ring + sout * kRowBytes;
              vertical_row(Ve, Vo, rin, aL, reinterpret_cast<const uint32_t*>(rin + aR), shA, rout, aL,
                           reinterpret_cast<const uint32_t*>(rout + aR), shA);
              uint4* dst = reinterpret_cast<uint4*>(s_vs + (k * VC + tid + 1) * kColBytes);
#pragma unroll
              for (int m = 0; m < 8; ++m) dst[m] = make_uint4(Ve[2 * m], Vo[2 * m], Ve[2 * m + 1], Vo[2 * m + 1]);
              sin = sin + 1 < ring ? sin + 1 : 0;
            }
          }
        } else {
          int sin = slot, offLi = offL, offRi = offR;
#pragma unroll 1
          for (int k = 0; k < ng; ++k) {
            const int y = yg + k;
            const bool real_out = y - r - 1 >= y_first - r;
            int sout = sin + 2 * kG;
            if (sout >= ring) sout -= ring;
            const uint8_t* rin = s_ring + sin * kRowBytes;
            const uint8_t* rout = real_out ? s_ring + sout * kRowBytes : s_zero;
            const int offLo = real_out ? ((offLi - back) & 15) : 0, offRo = real_out ? ((offRi - back) & 15) : 0;
            const int ji = tid + offRi, jo = tid + offRo;
            vertical_row(Ve, Vo, rin, offLi + tid, reinterpret_cast<const uint32_t*>(rin + kLBytes) + (ji >> 2),
                         (ji & 3) * 8, rout, offLo + tid,
                         reinterpret_cast<const uint32_t*>(rout + kLBytes) + (jo >> 2), (jo & 3) * 8);
            if (y >= y_first) {
              uint4* dst = reinterpret_cast<uint4*>(s_vs + (k * VC + tid + 1) * kColBytes);
#pragma unroll
              for (int m = 0; m < 8; ++m) dst[m] = make_uint4(Ve[2 * m], Vo[2 * m], Ve[2 * m + 1], Vo[2 * m + 1]);
            }
            sin = sin + 1 < ring ? sin + 1 : 0;
            offLi = (offLi + wm) & 15;
            offRi = (offRi + wm) & 15;
          }
        }
      }
      slot = slot_next;
      offL = (offL + kG * wm) & 15;
      offR = (offR + kG * wm) & 15;
      if (yg + ng - 1 < y_first) continue;  // still warming up
      __syncthreads();
      // Stage B: warp -> (row g of the group, segment of TX / kSegs outputs);
      // lane -> disparity pair.  The column sums of a pair are one 32-bit word
      // (lo | hi << 16, each below 2^14), so one load serves two disparities.
      // The horizontal window slides by entering - leaving: T adds it (mod 2^32;
      // the packed pair of window sums, whose lanes are exact once the true sums
      // are known to fit), and H adds the upper lane of delta = entering -
      // leaving + 0x4000 taken as a signed number (arithmetic shift): the lower
      // u16 lane of delta is the lower difference plus 0x4000, in
      // [0x4000 - 16065, 0x4000 + 16065], so it never borrows from the upper
      // lane, which is then exactly the upper difference; H is the upper window
      // sum itself, and T and H give both window sums exactly.
      {
        const int g = warp / kSegs, seg = warp % kSegs;
        const int y = yg + g;
        if (g < ng && y >= y_first) {
          const int SW = TX / kSegs;                              // a multiple of 8
          const int xa = seg * SW, xb = xa + SW;
          constexpr int CW = kColBytes / 4;                       // words per column slot
          const uint32_t* vcol = reinterpret_cast<const uint32_t*>(s_vs + g * VC * kColBytes) + lane;
          const uint8_t* bm = s_bm + (buf * kG + g) * kBBytes + (int)(((int64_t)y * w + x0) & 15);
          uint32_t* krow = J.key + (int64_t)y * w + x0;
          // anchor test of strip-relative output column xi, given its map byte
          auto anchor = [&](int xi, uint8_t b) -> bool {
            const int xl = x0 + xi;
            return xi < xb && xl >= xo0 && xl <= xo1 && (xl == xo0 || xl == xo1 || b);
          };
          // warm-up: the window of output xa - 1 (slot columns xa .. xa + 2r), in
          // four independent partial sums
          uint32_t T = 0, H = 0;
          {
            uint32_t T1 = 0, T2 = 0, T3 = 0, H1 = 0, H2 = 0, H3 = 0;
            const uint32_t* p = vcol + xa * CW;
            int j = 0;
#pragma unroll(RC > 0 ? 16 : 1)
            for (; j + 4 <= 2 * r + 1; j += 4, p += 4 * CW) {
              const uint32_t v0 = p[0], v1 = p[CW], v2 = p[2 * CW], v3 = p[3 * CW];
              T += v0; H += v0 >> 16;
              T1 += v1; H1 += v1 >> 16;
              T2 += v2; H2 += v2 >> 16;
              T3 += v3; H3 += v3 >> 16;
            }
#pragma unroll(RC > 0 ? 4 : 1)
            for (; j <= 2 * r; ++j, p += CW) {
              const uint32_t v = p[0];
              T += v;
              H += v >> 16;
            }
            T += T1 + T2 + T3;
            H += H1 + H2 + H3;
          }
          // the map bytes of the next 32 outputs are read one chunk ahead
          uint8_t bcur = xa + lane < xb ? bm[xa + lane] : (uint8_t)0;
          for (int xbase = xa; xbase < xb; xbase += 32) {
            const uint8_t bnext = xbase + 32 + lane < xb ? bm[xbase + 32 + lane] : (uint8_t)0;
            const unsigned mask = __ballot_sync(0xffffffffu, anchor(xbase + lane, bcur));
            const int n = min(32, xb - xbase);
            const uint32_t* pin = vcol + (xbase + 2 * r + 1) * CW;  // slot column of strip column x + 2r
            const uint32_t* pout = vcol + xbase * CW;             // slot column of x - 1
            uint32_t* sbest = s_best + warp * 32;                 // word o: the key of output xbase + o
#pragma unroll 1
            for (int i = 0; i < n; i += 8) {
              uint32_t Tv[8], Hv[8];
#pragma unroll
              for (int k = 0; k < 8; ++k) {
                const uint32_t e = pin[(i + k) * CW], l = pout[(i + k) * CW];
                T += e - l;
                H += (uint32_t)((int32_t)(e - l + 0x4000u) >> 16);
                Tv[k] = T;
                Hv[k] = H;
              }
              const unsigned bits = (mask >> i) & 0xFFu;
              emit_block_half<0>(bits & 15u, Tv, Hv, dlo, dhi, sbest + i);
              emit_block_half<4>(bits >> 4, Tv, Hv, dlo, dhi, sbest + i);
            }
            __syncwarp();   // the span's uniform stores are visible to every lane
            if ((mask >> lane) & 1u) atomicMin(krow + xbase + lane, sbest[lane]);   // one per anchor of the span
            __syncwarp();   // read before the next span overwrites
            bcur = bnext;
          }
        }
      }
    }
  }  // next work item
}

// Tail disparities (see sad_has_tail): a persistent grid over work items
// (pair, strip of sad_tail_strip(r) outputs, row band).  Thread t owns strip
// column c = x0 - r + t and keeps, per tail disparity d = dt0 + k, the vertical
// window sum V_k of |L(., c) - R(., c - d)| sliding down the band.  Rows are
// taken in groups: first the 2r warm-up rows, 16 at a time, then groups of
// kTailRows output rows.  A group's rows (the entering rows y + r and leaving
// rows y - r of both images, the right one over the strip's columns shifted by
// dt0 with kTailMax - 1 more columns on the left, and the anchor-map rows) are
// copied with cp.async into one of two shared-memory buffers while the
// previous group is computed:
//   vertical: per output row V_k += entering cell, store V_k as that row's
//     column sums, V_k -= leaving cell;
//   horizontal: one warp per (row, disparity) line turns the line's column
//     sums into prefix sums P in place (8 values per lane and a warp scan),
//     and the window sum at strip output l is P[l + 2r] - P[l - 1]; anchors
//     keep (S << 10 | d) with atomicMin into the argmin keys.
constexpr int kTailRows = 8;                    // output rows per group
constexpr int kTailSlots = 2 * kTailRows;       // staged image rows per group
constexpr int kTailL = 272, kTailR = 288, kTailB = 272;   // staged bytes per row: 17, 18, 17 chunks
constexpr int kTailBuf = kTailSlots * (kTailL + kTailR) + kTailRows * kTailB;
__host__ __device__ inline int tail_smem_bytes(int max_rem) { return kTailRows * max_rem * 1024 + 2 * kTailBuf; }

// REM: the most tail disparities among the launch's jobs (static loop bounds)
template <int REM>
__global__ void __launch_bounds__(256, 6) k_sad_tail(const SadJob* __restrict__ jobs,
                                                     const SadItem* __restrict__ items, int n_items,
                                                     unsigned* __restrict__ queue) {
  extern __shared__ __align__(16) uint8_t t_smem[];
  uint32_t* s_v = reinterpret_cast<uint32_t*>(t_smem);            // [kTailRows][REM][256] column sums
  uint8_t* s_stage = t_smem + kTailRows * REM * 1024;              // 2 x {L rows, R rows, anchor rows}
  __shared__ int s_item;
  __shared__ uint16_t s_ph[2][kTailSlots];   // per staged row: 16-byte phase of its L run | R run << 8
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (;;) {
    __syncthreads();
    if (tid == 0) s_item = (int)atomicAdd(queue, 1u);
    __syncthreads();
    if (s_item >= n_items) break;
    const SadItem it = items[s_item];
    const SadJob J = jobs[it.job];
    if (sad_use_direct(J)) continue;
    // a work item inside Omega, on the disparities past the last whole chunk
    if (!SB_CHECK(it.y0 >= J.r && it.y0 <= it.y1 && it.y1 <= J.h - 1 - J.r && it.x0 >= J.D + J.r &&
                  it.x0 < J.w - J.r && it.d0 == sad_tail_first(J.D) && J.D + 1 - it.d0 <= kTailMax, 402u))
      continue;
    const int r = J.r, D = J.D, w = J.w, w15 = w & 15;
    const int64_t npx = (int64_t)w * J.h;
    const int dt0 = it.d0, rem = D + 1 - dt0;
    const int TX = sad_tail_strip(r), NC = TX + 2 * r;
    const int x0 = it.x0, cstart = x0 - r;
    // every thread keeps column sums, also past the strip (tid >= NC) or the
    // image (column > w - 1): no window of an output reads those, and their
    // staged bytes lie inside the staging rows
    const int cr0 = cstart - dt0 - (kTailMax - 1);         // right-image column of staged byte 0
    const int xo0 = D + r, xo1 = w - 1 - r;
    const bool fast = (((uintptr_t)J.Ll | (uintptr_t)J.Lr | (uintptr_t)J.bmap) & 15) == 0;
    const int nchL = (15 + NC + 15) / 16, nchR = (15 + NC + kTailMax - 1 + 15) / 16, nchB = (15 + TX + 15) / 16;
    const int nwarm = (2 * r + kTailSlots - 1) / kTailSlots;
    const int ngroups = nwarm + (it.y1 - it.y0 + kTailRows) / kTailRows;
    // 16-byte phase of image row `row` at column c (row * w + c mod 16, in 32-bit arithmetic)
    auto phase = [&](int row, int c) { return (row * w15 + c) & 15; };
    // group gi: image rows per staging slot (entering / warm-up rows in slots
    // 0.., leaving rows in slots kTailRows..); warps take rows, lanes chunks
    auto issue = [&](int gi, int buf) {
      uint8_t* B = s_stage + buf * kTailBuf;
      int nrows, row0 = 0, yg = 0, G = 0;
      if (gi < nwarm) {
        row0 = it.y0 - r + kTailSlots * gi;
        nrows = min(kTailSlots, it.y0 + r - row0);
      } else {
        yg = it.y0 + kTailRows * (gi - nwarm);
        G = min(kTailRows, it.y1 - yg + 1);
        nrows = 2 * G;
      }
      // one flat index over (row, chunk) so that every thread copies a chunk:
      // the image rows' L and R chunks first, then the anchor-map rows'
      const int per = nchL + nchR, nimg = nrows * per;
      for (int idx = tid; idx < nimg + G * nchB; idx += 256) {
        if (idx < nimg) {
          const int i = idx / per, ch = idx - i * per;
          const int q = gi < nwarm ? i : (i < G ? i : kTailRows + i - G);
          const int row = gi < nwarm ? row0 + i : (i < G ? yg + i + r : yg + (i - G) - r);
          const int64_t rb = (int64_t)row * w;
          if (ch == 0) s_ph[buf][q] = (uint16_t)(phase(row, cstart) | (phase(row, cr0) << 8));
          if (ch < nchL) stage_chunk(B + q * kTailL, J.Ll, npx, (rb + cstart) & ~(int64_t)15, ch, fast);
          else stage_chunk(B + kTailSlots * kTailL + q * kTailR, J.Lr, npx, (rb + cr0) & ~(int64_t)15, ch - nchL, fast);
        } else {
          const int j = (idx - nimg) / nchB, ch = idx - nimg - j * nchB;
          stage_chunk(B + kTailSlots * (kTailL + kTailR) + j * kTailB, J.bmap, npx,
                      ((int64_t)(yg + j) * w + x0) & ~(int64_t)15, ch, fast);
        }
      }
      cp_async_commit();
    };
    uint32_t V[REM];
#pragma unroll
    for (int k = 0; k < REM; ++k) V[k] = 0u;
    // V_k += sign * |L - R| of the image row staged in slot q of buffer b
    auto accumulate = [&](const uint8_t* B, int b, int q, bool add) {
      const unsigned ph = s_ph[b][q];
      const unsigned lv = B[q * kTailL + (ph & 15u) + tid];
      const uint8_t* rp = B + kTailSlots * kTailL + q * kTailR + (ph >> 8) + tid + kTailMax - 1;
#pragma unroll
      for (int k = 0; k < REM; ++k)
        if (k < rem) {
          const unsigned rv = rp[-k];
          V[k] = add ? __usad(lv, rv, V[k]) : V[k] - __usad(lv, rv, 0u);
        }
    };
    issue(0, 0);
    for (int gi = 0; gi < ngroups; ++gi) {
      cp_async_wait_all();
      __syncthreads();   // group gi has landed; every thread is done with group gi - 1
      if (gi + 1 < ngroups) issue(gi + 1, (gi + 1) & 1);
      const uint8_t* B = s_stage + (gi & 1) * kTailBuf;
      if (gi < nwarm) {
        const int row0 = it.y0 - r + kTailSlots * gi, n = min(kTailSlots, it.y0 + r - row0);
        for (int q = 0; q < n; ++q) accumulate(B, gi & 1, q, true);
        continue;
      }
      const int yg = it.y0 + kTailRows * (gi - nwarm), G = min(kTailRows, it.y1 - yg + 1);
#pragma unroll
      for (int j = 0; j < kTailRows; ++j) {
        if (j < G) {
          accumulate(B, gi & 1, j, true);
#pragma unroll
          for (int k = 0; k < REM; ++k)
            if (k < rem) s_v[(j * REM + k) * 256 + tid] = V[k];
          accumulate(B, gi & 1, kTailRows + j, false);
        }
      }
      __syncthreads();
      const uint8_t* sb = B + kTailSlots * (kTailL + kTailR);
      for (int line = warp; line < G * rem; line += 8) {
        const int j = REM == 1 ? line : line / rem, k = line - j * rem;
        uint32_t* P = s_v + (j * REM + k) * 256;
        uint4 a = reinterpret_cast<uint4*>(P)[2 * lane], b = reinterpret_cast<uint4*>(P)[2 * lane + 1];
        a.y += a.x; a.z += a.y; a.w += a.z;
        b.x += a.w; b.y += b.x; b.z += b.y; b.w += b.z;
        uint32_t t = b.w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t u = __shfl_up_sync(0xffffffffu, t, o);
          if (lane >= o) t += u;
        }
        const uint32_t ex = t - b.w;   // sum of the lanes before this one
        a.x += ex; a.y += ex; a.z += ex; a.w += ex;
        b.x += ex; b.y += ex; b.z += ex; b.w += ex;
        reinterpret_cast<uint4*>(P)[2 * lane] = a;
        reinterpret_cast<uint4*>(P)[2 * lane + 1] = b;
        __syncwarp();
        const int y = yg + j;
        const uint8_t* bm = sb + j * kTailB + phase(y, x0);
        uint32_t* krow = J.key + (int64_t)y * w + x0;
        const uint32_t dk = (uint32_t)(dt0 + k);
        for (int xl = lane; xl < TX; xl += 32) {
          const int x = x0 + xl;
          const bool anc = (x <= xo1) & ((x == xo0) | (x == xo1) | (bm[xl] != 0));
          const uint32_t S = P[xl + 2 * r] - (xl > 0 ? P[xl - 1] : 0u);
          if (anc) atomicMin(&krow[xl], (S << SB_KEY_DBITS) | dk);
        }
        __syncwarp();
      }
    }
  }
  cp_async_wait_all();
}

template <int REM>
void launch_tail_rem(const SadJob* jobs, const SadItem* items, int n_items, unsigned* queue, cudaStream_t s) {
  const int smem = tail_smem_bytes(REM);
  cudaFuncSetAttribute(k_sad_tail<REM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  int dev = 0, sms = 148, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sad_tail<REM>, 256, smem);
  const int grid = std::min(n_items, sms * std::max(1, per_sm));
  k_sad_tail<REM><<<grid, 256, smem, s>>>(jobs, items, n_items, queue);
}

void launch_sad_tail(const SadJob* jobs, const SadItem* items, int n_items, int max_rem, unsigned* queue,
                     cudaStream_t s) {
  if (n_items <= 0) return;
  switch (max_rem) {
    case 1: launch_tail_rem<1>(jobs, items, n_items, queue, s); break;
    case 2: launch_tail_rem<2>(jobs, items, n_items, queue, s); break;
    case 3: case 4: launch_tail_rem<4>(jobs, items, n_items, queue, s); break;
    default: launch_tail_rem<kTailMax>(jobs, items, n_items, queue, s); break;
  }
}

int sad_boxsum_smem_bytes(int r) {
  const int ring = 2 * r + 1 + 2 * kG;
  return (ring + 1) * kRowBytes + 2 * kG * kBBytes + kG * box_vcols(r) * kColBytes;
}

template <bool W16, int RC>
static void launch_box(const SadJob* jobs, const SadItem* items, int n_items, int smem, unsigned* queue,
                       cudaStream_t s) {
  cudaFuncSetAttribute(k_sad_boxsum<W16, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  int dev = 0, sms = 148, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sad_boxsum<W16, RC>, kThreads, smem);
  const int grid = std::min(n_items, sms * std::max(1, per_sm));
  k_sad_boxsum<W16, RC><<<grid, kThreads, smem, s>>>(jobs, items, n_items, queue);
}

template <bool W16>
static void launch_box_r(const SadJob* jobs, const SadItem* items, int n_items, int smem, int uniform_r,
                         unsigned* queue, cudaStream_t s) {
  // instances with the radius of the benchmark blocks (15, 31 and 41) built in, so the
  // horizontal warm-up over 2r + 1 columns is unrolled; any other radius, or a launch
  // mixing radii, takes the radius from each job
  switch (uniform_r) {
    case 7: launch_box<W16, 7>(jobs, items, n_items, smem, queue, s); break;
    case 15: launch_box<W16, 15>(jobs, items, n_items, smem, queue, s); break;
    case 20: launch_box<W16, 20>(jobs, items, n_items, smem, queue, s); break;
    default: launch_box<W16, 0>(jobs, items, n_items, smem, queue, s); break;
  }
}

void launch_sad_boxsum(const SadJob* jobs, const SadItem* items, int n_items, int max_r, int uniform_r, bool w16,
                       unsigned* queue, cudaStream_t s) {
  if (n_items <= 0) return;
  const int smem = sad_boxsum_smem_bytes(max_r);
  if (w16) launch_box_r<true>(jobs, items, n_items, smem, uniform_r, queue, s);
  else launch_box_r<false>(jobs, items, n_items, smem, uniform_r, queue, s);
}

// ----------------------------------------------------------------- direct
namespace {
// Direct window sums (the paper's own formulation).  A CTA takes a tile of
// kDirRows output rows x kDirCols output columns of one pair and stages, with
// cp.async, the rows its windows read: the left image over the tile's columns
// plus the window margin, the right image over the same columns shifted left
// by up to D.  Warps then take the tile's anchors, one warp per anchor.  For
// each window row the warp realigns the anchor's B left-image bytes once
// (funnel shifts of aligned words, L' below) and reuses them for every
// disparity.  Lane (c, g) = (lane & 3, lane >> 2) takes the disparity pair
// d, d + 4 with d = 64p + c + 8g in pass p (64 disparities per pass); both
// start at the same alignment within a 4-byte word, so NW + 1 aligned words
// of the right image serve both: d + 4 uses the same words one position
// earlier.  Bytes outside the window are masked to zero in both operands, so
// every vabsdiff4.add adds only window cells.  A last pass of one disparity
// per lane covers a remainder of at most 32 disparities.  Passes run in
// groups of four with the window rows re-read per group.  NW = (B + 6) / 4
// is the number of words a B-byte window spans at any alignment.  The argmin
// over the warp is one redux.sync.
constexpr int kPassGroup = 4;   // 64-disparity passes accumulated together (D < 256: one group)
constexpr int kDirRows = 8;     // output rows per tile
constexpr int kDirCols = 256;   // output columns per tile (8 warps x 32)

// staged bytes per row of the left and right image for window radius r and max disparity D
__host__ __device__ inline int dir_lbytes(int r) { return ((kDirCols + 2 * r + 16 + 15) + 15) & ~15; }
__host__ __device__ inline int dir_rbytes(int r, int D) { return ((kDirCols + 2 * r + D + 13 + 15) + 15) & ~15; }
__host__ __device__ inline int dir_smem_bytes(int r, int D) {
  return (kDirRows + 2 * r) * (dir_lbytes(r) + dir_rbytes(r, D));
}

// bytes [0, n) of a word set, n clamped to [0, 4]
__device__ __forceinline__ uint32_t low_bytes(int n) {
  return (uint32_t)((1ull << (8 * min(max(n, 0), 4))) - 1ull);
}
// valid bytes of word k of a window that starts `off` bytes into word 0 and
// spans B bytes: [off - 4k, off + B - 4k) within the word
__device__ __forceinline__ uint32_t win_mask(int k, int off, int B) {
  return low_bytes(off + B - 4 * k) & ~low_bytes(off - 4 * k);
}

__device__ __forceinline__ uint32_t lds32(const uint8_t* p) { return *reinterpret_cast<const uint32_t*>(p); }

// One anchor (y, xa) of the tile whose first output row is y0 and first output
// column x0; sL / sR hold staged row t = image row y0 - r + t from absolute
// byte aL(t) / aR(t) on (multiples of 16, so word alignment is preserved).
template <int NW>
__device__ __forceinline__ void direct_anchor(const SadJob& J, int y0, int x0, const uint8_t* sL,
                                              const uint8_t* sR, int lb, int rbytes, int y, int xa, int lane,
                                              int n2, bool p1) {
  const int r = J.r, B = 2 * r + 1, D = J.D, w = J.w;
  const int c = lane & 3, g = lane >> 2;
  // largest disparity <= D of this lane's class (d = c mod 4): where a lane
  // past D reads instead, so that every read stays inside the staged rows
  const int dcap = D >= c ? D - ((D - c) & 3) : c;
  const int ngroups = max((n2 + kPassGroup - 1) / kPassGroup, 1);
  uint32_t best = 0xFFFFFFFFu;
  for (int gi = 0; gi < ngroups; ++gi) {
    const bool last = gi == ngroups - 1;
    uint32_t acc2[kPassGroup][2], acc1 = 0;
#pragma unroll
    for (int q = 0; q < kPassGroup; ++q) acc2[q][0] = acc2[q][1] = 0;
    for (int iy = -r; iy <= r; ++iy) {
      const int t = y + iy - (y0 - r);                       // staged row
      const int64_t rb = (int64_t)(y + iy) * w;
      const int64_t aL = (rb + x0 - r - 6) & ~(int64_t)15, aR = (rb + x0 - r - D - 7) & ~(int64_t)15;
      const uint8_t* Lrow = sL + t * lb - aL;                  // index by absolute byte
      const uint8_t* Rrow = sR + t * rbytes - aR;
      const int off = (int)((rb + xa - r - c) & 3);           // window start within its word, d = c mod 4
      const int64_t s = rb + xa - r - off;                    // L' starts off bytes before the window
      const int64_t sa = s & ~(int64_t)3;
      const int sh = (int)(s - sa) * 8;
      uint32_t Lp[NW], mk[NW];
      uint32_t prev = lds32(Lrow + sa);
#pragma unroll
      for (int k = 0; k < NW; ++k) {
        const uint32_t nx = lds32(Lrow + sa + 4 * k + 4);
        mk[k] = (k == 0 || k >= NW - 2) ? win_mask(k, off, B) : 0xFFFFFFFFu;
        Lp[k] = __funnelshift_r(prev, nx, sh) & mk[k];
        prev = nx;
      }
#pragma unroll
      for (int q = 0; q < kPassGroup; ++q) {
        const int p = gi * kPassGroup + q;
        if (p < n2) {
          const int d0 = min(64 * p + c + 8 * g, dcap);
          const uint8_t* ra = Rrow + (rb + xa - r - d0 - off - 4);  // word-aligned; d0 + 4 starts here
          uint32_t R[NW + 1];
#pragma unroll
          for (int k = 0; k <= NW; ++k) R[k] = lds32(ra + 4 * k);
          // even and odd words into separate sums: twice the independent chains
          uint32_t s0 = acc2[q][0], s1 = acc2[q][1], t0 = 0, t1 = 0;
#pragma unroll
          for (int k = 0; k < NW; ++k) {
            const uint32_t r0 = (k == 0 || k >= NW - 2) ? (R[k + 1] & mk[k]) : R[k + 1];
            const uint32_t r1 = (k == 0 || k >= NW - 2) ? (R[k] & mk[k]) : R[k];
            if (k & 1) {
              asm("vabsdiff4.u32.u32.u32.add %0, %1, %2, %0;" : "+r"(t0) : "r"(Lp[k]), "r"(r0));
              asm("vabsdiff4.u32.u32.u32.add %0, %1, %2, %0;" : "+r"(t1) : "r"(Lp[k]), "r"(r1));
            } else {
              asm("vabsdiff4.u32.u32.u32.add %0, %1, %2, %0;" : "+r"(s0) : "r"(Lp[k]), "r"(r0));
              asm("vabsdiff4.u32.u32.u32.add %0, %1, %2, %0;" : "+r"(s1) : "r"(Lp[k]), "r"(r1));
            }
          }
          acc2[q][0] = s0 + t0;
          acc2[q][1] = s1 + t1;
        }
      }
      if (last && p1) {
        const int d = min(64 * n2 + lane, dcap);
        const uint8_t* ra = Rrow + (rb + xa - r - d - off);
        uint32_t s1 = acc1;
#pragma unroll
        for (int k = 0; k < NW; ++k) {
          uint32_t rw = lds32(ra + 4 * k);
          if (k == 0 || k >= NW - 2) rw &= mk[k];
          asm("vabsdiff4.u32.u32.u32.add %0, %1, %2, %0;" : "+r"(s1) : "r"(Lp[k]), "r"(rw));
        }
        acc1 = s1;
      }
    }
    // this group's argmin over the lane's disparities; lanes past D never win
#pragma unroll
    for (int q = 0; q < kPassGroup; ++q) {
      const int p = gi * kPassGroup + q;
      if (p < n2) {
        const int d0 = 64 * p + c + 8 * g;
        if (d0 <= D) best = min(best, (acc2[q][0] << SB_KEY_DBITS) | (uint32_t)d0);
        if (d0 + 4 <= D) best = min(best, (acc2[q][1] << SB_KEY_DBITS) | (uint32_t)(d0 + 4));
      }
    }
    if (last && p1 && 64 * n2 + lane <= D) best = min(best, (acc1 << SB_KEY_DBITS) | (uint32_t)(64 * n2 + lane));
  }
  best = __reduce_min_sync(0xffffffffu, best);
  if (lane == 0 && SB_CHECK(y >= 0 && y < J.h && xa >= 0 && xa < w, 403u)) J.key[(int64_t)y * w + xa] = best;
}

// Persistent grid over the tiles of the jobs whose window spans NW words and
// that the direct variant serves.
template <int NW>
__global__ void __launch_bounds__(256) k_sad_direct(const SadJob* __restrict__ jobs, int n_jobs) {
  extern __shared__ __align__(16) uint8_t dsm[];
  __shared__ uint16_t s_list[kDirRows * kDirCols];   // the tile's anchors: row * kDirCols + column
  __shared__ int s_na;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int j = 0; j < n_jobs; ++j) {
    const SadJob J = jobs[j];
    if ((2 * J.r + 1 + 6) / 4 != NW || !sad_use_direct(J)) continue;
    const int r = J.r, D = J.D, w = J.w, h = J.h;
    const int xo0 = D + r, xo1 = w - 1 - r, yo0 = r, yo1 = h - 1 - r;
    const int tcols = (xo1 - xo0 + kDirCols) / kDirCols, trows = (yo1 - yo0 + kDirRows) / kDirRows;
    const int64_t npx = (int64_t)w * h;
    const int n2 = (D + 1) / 64 + ((D + 1) % 64 > 32 ? 1 : 0);
    const bool p1 = (D + 1) % 64 != 0 && (D + 1) % 64 <= 32;
    const bool fast = (((uintptr_t)J.Ll | (uintptr_t)J.Lr) & 15) == 0;
    const int lb = dir_lbytes(r), rbytes = dir_rbytes(r, D), nrows = kDirRows + 2 * r;
    const int nchL = lb / 16, nchR = rbytes / 16;
    uint8_t* sL = dsm;
    uint8_t* sR = dsm + nrows * lb;
    for (int tile = blockIdx.x; tile < tcols * trows; tile += gridDim.x) {
      const int y0 = yo0 + (tile / tcols) * kDirRows, x0 = xo0 + (tile % tcols) * kDirCols;
      __syncthreads();  // the previous tile's windows are done
      if (tid == 0) s_na = 0;
      // stage rows y0 - r .. y0 + kDirRows - 1 + r (all inside the image: y0 >= r)
      const int last_row = min(y0 + kDirRows - 1, yo1) + r;
      for (int i = tid; i < nrows * (nchL + nchR); i += 256) {
        const int t = i / (nchL + nchR), ch = i - t * (nchL + nchR);
        const int yy = y0 - r + t;
        if (yy > last_row) continue;
        const int64_t rb = (int64_t)yy * w;
        if (ch < nchL)
          stage_chunk(sL + t * lb, J.Ll, npx, (rb + x0 - r - 6) & ~(int64_t)15, ch, fast);
        else
          stage_chunk(sR + t * rbytes, J.Lr, npx, (rb + x0 - r - D - 7) & ~(int64_t)15, ch - nchL, fast);
      }
      cp_async_commit();
      cp_async_wait_all();
      __syncthreads();
      // the tile's anchors into a shared list (warp wid scans column chunk wid
      // of every output row), then the warps take them in turn: every anchor
      // costs the same, so the warps stay balanced even when the anchors
      // cluster (the domain's edge columns are anchors in every row)
      for (int i = 0; i < kDirRows; ++i) {
        const int y = y0 + i;
        if (y > yo1) break;
        const int x = x0 + wid * 32 + lane;
        bool anc = false;
        if (x <= xo1) anc = (x == xo0) || (x == xo1) || J.bmap[(int64_t)y * w + x];
        const uint32_t mask = __ballot_sync(0xffffffffu, anc);
        int base = 0;
        if (lane == 0 && mask) base = atomicAdd(&s_na, __popc(mask));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (anc) s_list[base + __popc(mask & ((1u << lane) - 1))] = (uint16_t)(i * kDirCols + (x - x0));
      }
      __syncthreads();
      const int na = s_na;
      for (int a = wid; a < na; a += 8) {
        const int v = s_list[a];
        direct_anchor<NW>(J, y0, x0, sL, sR, lb, rbytes, y0 + v / kDirCols, x0 + v % kDirCols, lane, n2, p1);
      }
    }
  }
}

template <int NW>
void launch_direct_nw(const SadJob* jobs, int n_jobs, int smem, cudaStream_t s) {
  cudaFuncSetAttribute(k_sad_direct<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  int dev = 0, sms = 148, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sad_direct<NW>, 256, smem);
  k_sad_direct<NW><<<sms * std::max(1, per_sm), 256, smem, s>>>(jobs, n_jobs);
}
}  // namespace

int sad_direct_words(int block) { return (block + 6) / 4; }

void launch_sad_direct(const SadJob* jobs, int n_jobs, int nw, int max_r, int max_D, cudaStream_t s) {
  if (n_jobs <= 0) return;
  const int smem = dir_smem_bytes(max_r, max_D);
  switch (nw) {
    case 1: launch_direct_nw<1>(jobs, n_jobs, smem, s); break;
    case 2: launch_direct_nw<2>(jobs, n_jobs, smem, s); break;
    case 3: launch_direct_nw<3>(jobs, n_jobs, smem, s); break;
    case 4: launch_direct_nw<4>(jobs, n_jobs, smem, s); break;
    case 5: launch_direct_nw<5>(jobs, n_jobs, smem, s); break;
    case 6: launch_direct_nw<6>(jobs, n_jobs, smem, s); break;
    case 7: launch_direct_nw<7>(jobs, n_jobs, smem, s); break;
    case 8: launch_direct_nw<8>(jobs, n_jobs, smem, s); break;
    case 9: launch_direct_nw<9>(jobs, n_jobs, smem, s); break;
    case 10: launch_direct_nw<10>(jobs, n_jobs, smem, s); break;
    case 11: launch_direct_nw<11>(jobs, n_jobs, smem, s); break;
    case 12: launch_direct_nw<12>(jobs, n_jobs, smem, s); break;
    case 13: launch_direct_nw<13>(jobs, n_jobs, smem, s); break;
    case 14: launch_direct_nw<14>(jobs, n_jobs, smem, s); break;
    case 15: launch_direct_nw<15>(jobs, n_jobs, smem, s); break;
    case 16: launch_direct_nw<16>(jobs, n_jobs, smem, s); break;
    case 17: launch_direct_nw<17>(jobs, n_jobs, smem, s); break;
    default: break;
  }
}

// Nonzero bytes of each map (the boundary count the variant choice reads);
// out[i] must be zero on entry.
__global__ void __launch_bounds__(256) k_count_nonzero(const uint8_t* const* __restrict__ maps,
                                                       const int64_t* __restrict__ n, int64_t* __restrict__ out) {
  const uint8_t* m = maps[blockIdx.y];
  const int64_t N = n[blockIdx.y];
  unsigned long long c = 0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < N; i += (int64_t)gridDim.x * 256) c += m[i] != 0;
  for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  __shared__ unsigned long long s_c[8];
  if ((threadIdx.x & 31) == 0) s_c[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int i = 0; i < 8; ++i) t += s_c[i];
    if (t) atomicAdd(reinterpret_cast<unsigned long long*>(&out[blockIdx.y]), t);
  }
}

void launch_count_nonzero(const uint8_t* const* maps, const int64_t* n, int64_t* out, int n_maps, cudaStream_t s) {
  if (n_maps <= 0) return;
  k_count_nonzero<<<dim3(148, n_maps), 256, 0, s>>>(maps, n, out);
}

// keys -> disparity (uint16, UNDET off the anchors) and cost; grid = (column
// blocks of 256, rows, jobs)
__global__ void __launch_bounds__(256) k_sad_finalize(const SadJob* __restrict__ jobs) {
  const SadJob J = jobs[blockIdx.z];
  const int w = J.w, h = J.h, r = J.r;
  const int y = blockIdx.y, x = blockIdx.x * 256 + threadIdx.x;
  if (y >= h || x >= w) return;
  const int xo0 = J.D + r, xo1 = w - 1 - r;
  const int64_t p = (int64_t)y * w + x;
  const bool in = y >= r && y <= h - 1 - r && x >= xo0 && x <= xo1;
  const bool anc = in && (x == xo0 || x == xo1 || J.bmap[p]);
  uint16_t dv = SB_UNDET16;
  uint32_t cv = 0;
  if (anc) {
    const uint32_t k = J.key[p];
    dv = (uint16_t)(k & ((1u << SB_KEY_DBITS) - 1));
    cv = k >> SB_KEY_DBITS;
  }
  J.disp[p] = dv;
  if (J.cost) J.cost[p] = cv;
}

void launch_sad_finalize(const SadJob* jobs, int n_jobs, int max_w, int max_h, cudaStream_t s) {
  if (n_jobs <= 0) return;
  k_sad_finalize<<<dim3((max_w + 255) / 256, max_h, n_jobs), 256, 0, s>>>(jobs);
}

SB_CHECKS_UNIT(sad)

}  // namespace sb
