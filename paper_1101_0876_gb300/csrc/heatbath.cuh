// Heat-bath colour pass: the same plane layout, walk, Philox words and
// reductions as the Metropolis pass (pass_u8.cuh), with the single-site
// rule replaced.  Heat bath is one of the other single-flip algorithms the
// paper proposes for this lattice code (Sec. 6).
//
// Rule.  Given its four neighbours (up, down, left, right), a site takes
// state x with probability W[n_x] / Z, n_x = number of neighbours in state
// x, W[n] = round(2^m exp(beta n)) (W[0] = 2^m exactly), Z = sum over the q
// states.  Each weight is the base 2^m plus the excess W[n_x] - W[0] (zero
// for a state no neighbour holds), and [0, Z) is laid out as: first the
// excesses of the distinct neighbour states in the order they first appear
// in (up, down, left, right), then q intervals of width 2^m, one per state
// in increasing order.  The new spin is the state whose interval holds
// r = floor(u Z / 2^32), u the site's Philox word: a neighbour's state when
// r falls in its excess, else (r - excesses) >> m.  The host picks m so that
// Z < 2^32 for every neighbour configuration, so all of it is 32-bit.
#pragma once
#include <cstdint>

#include "pass_u8.cuh"

namespace potts {

// W[0..4] as above (W[5..7] zero, unused).
struct HeatTable {
  uint32_t W[8];
  uint32_t m;
};

// Shared table of a heat-bath launch: W[0..7], then one 4-word entry per
// equality pattern of the four neighbours.  The pattern code of a site has
// bit 0..5 = [up == down], [up == left], [up == right], [down == left],
// [down == right], [left == right]; the interval bounds s1..s4 (cumulative
// excesses of the neighbours' states, a neighbour that repeats an earlier
// one adding nothing) depend on the site only through that code (and on W,
// which is fixed for a launch), and the normaliser is Z = s4 + q 2^m.
// Entry: {s1, s2, s3, s4}; r < s1 selects the up neighbour's state,
// s1 <= r < s2 the down one's, and so on, r >= s4 the state (r - s4) >> m.
// Of the 64 codes only the 15 that are transitive occur.
// Each entry is stored kHbCopies times, copy j at 16-byte slot 8 code + j,
// and a lane reads copy (lane mod 8): the eight lanes of a quarter-warp,
// which share one 128-bit shared-memory wavefront, then always hit eight
// different bank groups, whatever codes they hold (with one copy, codes
// equal mod 4 collide, and the common codes 0, 4, 8, 16, 32 all do).
constexpr int kHbCopies = 8;
constexpr int kHbTableWords = 8 + 64 * kHbCopies * 4;

// Fills entry `code` (all copies) from W (sW[0..7], already in shared
// memory).
__device__ __forceinline__ void hb_pattern_entry(uint32_t *sW,
                                                 uint32_t code) {
  const uint32_t e01 = code & 1u, e02 = (code >> 1) & 1u,
                 e03 = (code >> 2) & 1u, e12 = (code >> 3) & 1u,
                 e13 = (code >> 4) & 1u, e23 = (code >> 5) & 1u;
  const uint32_t f1 = e01 ^ 1u, f2 = (e02 | e12) ^ 1u,
                 f3 = (e03 | e13 | e23) ^ 1u;
  const uint32_t c0 = 1u + e01 + e02 + e03;
  const uint32_t c1 = f1 ? 1u + e12 + e13 : 5u;
  const uint32_t c2 = f2 ? 1u + e23 : 5u;
  const uint32_t c3 = f3 ? 1u : 5u;
  // excess of a class of c equal neighbours (c = 5: a repeat, none)
  auto ex = [&](uint32_t c) { return c <= 4u ? sW[c] - sW[0] : 0u; };
  const uint32_t s1 = ex(c0), s2 = s1 + ex(c1), s3 = s2 + ex(c2),
                 s4 = s3 + ex(c3);
  uint4 *e = reinterpret_cast<uint4 *>(sW + 8) + kHbCopies * code;
  for (int j = 0; j < kHbCopies; ++j) e[j] = make_uint4(s1, s2, s3, s4);
}

// The lane's copy of entry 0, as a byte pointer: entry `code` is at
// + 128 code.
__device__ __forceinline__ const uint8_t *hb_lane_table(const uint32_t *sW) {
  return reinterpret_cast<const uint8_t *>(sW + 8) + 16u * (threadIdx.x & 7u);
}

// Whole table: W from the launch, then the 64 entries.  Every thread of the
// CTA calls it; it ends with a barrier.
__device__ __forceinline__ void hb_build_table(uint32_t *sW, const uint32_t *W,
                                               uint32_t tid) {
  if (tid < 8) sW[tid] = W[tid];
  __syncthreads();
  if (tid < 64) hb_pattern_entry(sW, tid);
  __syncthreads();
}

// New spin of one site.  t0..t3: neighbours (up, down, left, right); u: the
// site's word; sW: the table in shared memory.
__device__ __forceinline__ uint32_t hb_site(uint32_t t0, uint32_t t1,
                                            uint32_t t2, uint32_t t3,
                                            uint32_t u, uint32_t q,
                                            const uint32_t *sW, uint32_t m) {
  const uint32_t code = (uint32_t)(t0 == t1) | (uint32_t)(t0 == t2) << 1 |
                        (uint32_t)(t0 == t3) << 2 | (uint32_t)(t1 == t2) << 3 |
                        (uint32_t)(t1 == t3) << 4 | (uint32_t)(t2 == t3) << 5;
  const uint4 sb =
      *reinterpret_cast<const uint4 *>(hb_lane_table(sW) + 128u * code);
  const uint32_t r = __umulhi(u, sb.w + (q << m));
  uint32_t s = (r - sb.w) >> m;
  s = r < sb.w ? t3 : s;
  s = r < sb.z ? t2 : s;
  s = r < sb.y ? t1 : s;
  s = r < sb.x ? t0 : s;
  // s < q already; the clamp keeps the shared histogram in bounds whatever
  // the spins in memory hold
  return min(s, q - 1u);
}

__device__ __forceinline__ uint32_t hb_byte(uint32_t w, int b) {
  return __byte_perm(w, 0u, 0x4440u + (uint32_t)b);
}

// Bit FROM of every byte moved to bit TO and added to acc (the fields are
// disjoint, so the additions are ORs): a multiply-add for a left move, a
// high multiply with an addend for a right move, both on the FMA-heavy pipe.
template <int FROM, int TO>
__device__ __forceinline__ uint32_t hb_put(uint32_t x, uint32_t acc,
                                           uint32_t one) {
  if constexpr (FROM > TO)
    return __umulhi(x, 1u << (32 - (FROM - TO))) + acc;
  else
    return x * (one << (TO - FROM)) + acc;
}

// [a == b] for every byte (spins < 2^QB), as bit T of the byte, added to
// acc (whose bit T is clear).  For x = a ^ b < 2^QB and T >= QB, bit T of
// x + 2^T - 1 is [x != 0] and the sum stays inside the byte (at most
// 2^QB + 2^T - 2 < 2^(T+1) <= 256), so the test lands at bit T directly
// and one logic op masks, inverts and adds it; for T < QB it is taken at
// bit QB and moved down (hb_put).
template <int QB, int T>
__device__ __forceinline__ uint32_t hb_eq_at(uint32_t a, uint32_t b,
                                             uint32_t acc, uint32_t one) {
  if constexpr (T >= QB) {
    constexpr uint32_t K = 0x01010101u * ((1u << T) - 1u);
    constexpr uint32_t M = 0x01010101u * (1u << T);
    return (~((a ^ b) * one + K) & M) | acc;
  } else {
    constexpr uint32_t K = Swar<QB>::K, M = Swar<QB>::M;
    return hb_put<QB, T>(~((a ^ b) * one + K) & M, acc, one);
  }
}

// The four sites of one word at once (spins < 2^QB, QB <= 6): the same
// rule as hb_site, with the six neighbour equalities done per byte on whole
// words and packed into the four sites' pattern codes, the interval bounds
// and normaliser read from the pattern table per site, and the new byte
// taken from a whole-word select among the four neighbour words and the
// base state (four compares and selects a site, then one masked OR).
// U, D, Lw, Rw: neighbour words (up, down, left, right); uw: Philox words;
// ent: the lane's copy of the launch's table (hb_lane_table); qm = q << m.
// one: the run-time 1 of PassArgs.  The equality tests' additions and the
// code's bit-field moves issue as multiply-adds on the FMA-heavy pipe,
// which this pass otherwise leaves largely idle; every step is exact 32-bit
// arithmetic.
template <int QB>
__device__ __forceinline__ uint32_t hb_word(uint32_t U, uint32_t D,
                                            uint32_t Lw, uint32_t Rw,
                                            const uint32_t uw[4],
                                            const uint8_t *ent, uint32_t m,
                                            uint32_t qm, uint32_t one) {
  static_assert(QB <= 6, "byte sums below need spins < 64");
  // four times the pattern code per byte: the six equalities at bits 2..7
  // in the table's bit order, so that a site's code byte times 32 is its
  // entry's offset (128 bytes per code); the tests whose bit is at or above
  // QB need no move
  uint32_t CODE = hb_eq_at<QB, 2>(U, D, 0u, one);
  CODE = hb_eq_at<QB, 3>(U, Lw, CODE, one);
  CODE = hb_eq_at<QB, 4>(U, Rw, CODE, one);
  CODE = hb_eq_at<QB, 5>(D, Lw, CODE, one);
  CODE = hb_eq_at<QB, 6>(D, Rw, CODE, one);
  CODE = hb_eq_at<QB, 7>(Lw, Rw, CODE, one);
  const uint32_t neg = 0u - one;  // -1 at run time
  uint32_t N = 0;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const uint4 sb =
        *reinterpret_cast<const uint4 *>(ent + hb_byte(CODE, b) * 32u);
    const uint32_t r = __umulhi(uw[b], sb.w * one + qm);
    // whole-word candidates, each holding site b's answer in byte b: first
    // the state among the bases (< q when r >= s4; when r < s4 a neighbour
    // word below replaces it), then the neighbour of the first bound above r
    uint32_t t = ((sb.w * neg + r) >> m) * (one << (8 * b));
    t = r < sb.w ? Rw : t;
    t = r < sb.z ? Lw : t;
    t = r < sb.y ? D : t;
    t = r < sb.x ? U : t;
    N |= t & (0xFFu << (8 * b));
  }
  return N;
}

// One row of 16 sites (the Metropolis do_row with the heat-bath rule).
// QB <= 6: the word rule; QB 8: the per-site rule (any q <= 256).  XP: the
// cross-plane pair histogram (hist_cross, black pass only).
template <int QB, bool LEFT, bool COUNTS, bool PAIRS, int LAY, bool XP = false>
__device__ __forceinline__ void hb_row(const PassArgs &A, const PhiloxKey &ks,
                                       const uint32_t *sW, uint32_t m,
                                       Walk &w, int32_t x0, int32_t xb,
                                       int32_t xl, int32_t xr, int32_t RB,
                                       bool more, uint32_t *lane_hist,
                                       uint32_t &ne_acc) {
  using IO = Lay<LAY>;
  const int32_t L = A.L, H = A.H;
  uint32_t Dw[4];
  IO::load(w.oth_next, false, Dw);
  const uint32_t ew = IO::edge(
      __ldg(reinterpret_cast<const uint32_t *>(w.oth_cur - xb +
                                               (LEFT ? xl : xr))),
      LEFT);
  // the rule never reads the site's own spin, so the own plane is only
  // written (1 byte per site per pass instead of 1.5)
  uint8_t *own_next = (w.i + 1 == L) ? A.own + xb : w.own_cur + RB;
  const uint32_t *Cw = w.Ce;
  uint32_t Wd[4];
  if (LEFT) {
    Wd[0] = __funnelshift_l(ew, Cw[0], 8);
    Wd[1] = __funnelshift_l(Cw[0], Cw[1], 8);
    Wd[2] = __funnelshift_l(Cw[1], Cw[2], 8);
    Wd[3] = __funnelshift_l(Cw[2], Cw[3], 8);
  } else {
    Wd[0] = __funnelshift_r(Cw[0], Cw[1], 8);
    Wd[1] = __funnelshift_r(Cw[1], Cw[2], 8);
    Wd[2] = __funnelshift_r(Cw[2], Cw[3], 8);
    Wd[3] = __funnelshift_r(Cw[3], ew, 8);
  }
  const uint32_t g0 = (uint32_t)(((int64_t)(w.i + A.grow0) * H + x0) >> 2);
  uint32_t Nw[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint4 u = philox10(g0 + (uint32_t)k, A.t_lo, A.colour, A.t_hi, ks);
    const uint32_t uw[4] = {u.x, u.y, u.z, u.w};
    // left / right neighbours: the window byte x-1 (Wd) and x (Cw) when the
    // side neighbour is at x-1, else x (Cw) and x+1 (Wd)
    const uint32_t Lw = LEFT ? Wd[k] : Cw[k];
    const uint32_t Rw = LEFT ? Cw[k] : Wd[k];
    if constexpr (QB <= 6) {
      Nw[k] = hb_word<QB>(w.Up[k], Dw[k], Lw, Rw, uw, hb_lane_table(sW), m,
                          A.q << m, A.one);
    } else {
      uint32_t s[4];
#pragma unroll
      for (int b = 0; b < 4; ++b)
        s[b] = hb_site(hb_byte(w.Up[k], b), hb_byte(Dw[k], b),
                       hb_byte(Lw, b), hb_byte(Rw, b), uw[b], A.q, sW, m);
      Nw[k] = pack4(s[0], s[1], s[2], s[3]);
    }
    if (COUNTS) {
      // 16 x (neighbours unequal to the new spin) per byte
      const uint32_t nf16 = ne16_sum4<QB>(Nw[k] ^ w.Up[k], Nw[k] ^ Dw[k],
                                          Nw[k] ^ Cw[k], Nw[k] ^ Wd[k]);
      ne_acc += __umulhi(nf16, 1u << 28);
    }
  }
  IO::store(w.own_cur, Nw);
  if constexpr (XP) {
    if (COUNTS) {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        hist_cross(lane_hist - (threadIdx.x & 31u), Nw[k], Cw[k], 1u);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) hist_word<PAIRS>(lane_hist, Nw[k]);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    w.Up[k] = w.Ce[k];
    w.Ce[k] = Dw[k];
  }
  w.oth_cur = w.oth_next;
  w.oth_next = (w.i + 2 >= L) ? A.other + xb + (int64_t)(w.i + 2 - L) * RB
                              : w.oth_next + RB;
  w.own_cur = own_next;
  w.i += 1;
}

// walk_column with the heat-bath rule.
template <int QB, int COLOUR, bool COUNTS, bool PAIRS, int LAY, bool XP = false>
__device__ __forceinline__ void hb_walk_column(
    const PassArgs &A, const PhiloxKey &ks, const uint32_t *sW, uint32_t m,
    int32_t x0, int32_t i0, int32_t rows, uint32_t *lane_hist,
    uint32_t *ne_total) {
  using IO = Lay<LAY>;
  const int32_t L = A.L, H = A.H;
  const int32_t RB = IO::row_bytes(H);
  const int32_t xb = LAY == kLayoutU4 ? x0 / 2 : x0;
  const int32_t xl = (x0 == 0) ? RB - 4 : xb - 4;
  const int32_t xr = (x0 + 16 == H) ? 0 : xb + IO::kChunkBytes;
  Walk w;
  const int32_t im = (i0 == 0) ? L - 1 : i0 - 1;
  const int32_t ip = (i0 + 1 == L) ? 0 : i0 + 1;
  w.oth_cur = A.other + (int64_t)i0 * RB + xb;
  w.oth_next = A.other + (int64_t)ip * RB + xb;
  w.own_cur = A.own + (int64_t)i0 * RB + xb;
  IO::load(A.other + (int64_t)im * RB + xb, false, w.Up);
  IO::load(w.oth_cur, false, w.Ce);
  w.i = i0;
  uint32_t ne_acc = 0;
  int32_t r = 0;
  if (((i0 + A.grow0) & 1) == 0) {
    for (; r + 2 <= rows; r += 2) {
      hb_row<QB, COLOUR == 0, COUNTS, PAIRS, LAY, XP>(
          A, ks, sW, m, w, x0, xb, xl, xr, RB, true, lane_hist, ne_acc);
      hb_row<QB, COLOUR == 1, COUNTS, PAIRS, LAY, XP>(
          A, ks, sW, m, w, x0, xb, xl, xr, RB, r + 2 < rows, lane_hist,
          ne_acc);
      if (COUNTS) {
        *ne_total += (ne_acc * 0x01010101u) >> 24;
        ne_acc = 0;
      }
    }
  }
  for (; r < rows; ++r) {
    const bool left = ((w.i + A.grow0 + COLOUR) & 1) == 0;
    if (left)
      hb_row<QB, true, COUNTS, PAIRS, LAY, XP>(A, ks, sW, m, w, x0, xb, xl, xr,
                                           RB, r + 1 < rows, lane_hist, ne_acc);
    else
      hb_row<QB, false, COUNTS, PAIRS, LAY, XP>(A, ks, sW, m, w, x0, xb, xl, xr,
                                            RB, r + 1 < rows, lane_hist,
                                            ne_acc);
    if (COUNTS) {
      *ne_total += (ne_acc * 0x01010101u) >> 24;
      ne_acc = 0;
    }
  }
}

}  // namespace potts
