// Metropolis colour pass on the packed 4-bit layout (q <= 16) with the
// arithmetic done on the stored nibbles (Sec. 3.3's colour planes, two
// spins per byte).  A 32-bit word holds 8 consecutive sites of a plane row,
// site j of the word in bits 4j..4j+3 (the layout's order: site 2b in the
// low nibble of byte b, site 2b+1 in the high one), so nothing is unpacked
// or repacked: every word-wide operation serves 8 sites.
//
// Per word (8 sites):
//   - two Philox4x32-10 calls (counters as in pass_u8.cuh), eight products
//     u q giving the proposals (high words, gathered into a nibble word P)
//     and the acceptance variates (low words);
//   - neighbour compares per nibble: [S != N] for the four neighbours and
//     [P != N] likewise, by the exact zero-nibble test on x = S ^ N:
//     bit 3 of ((x & 7) + 7) | x is [x != 0]; the addition and the shift of
//     that bit down to bit 0 issue as a multiply-add and a high multiply,
//     on the FMA-heavy pipe, which has room here while the ALU pipe is the
//     busy one;
//   - idx = 4 + X - Y per nibble, X / Y the counts of neighbours unequal
//     to the proposal / the current spin, so idx = 4 + dE in 0..8;
//   - acceptance: per site one byte extraction, one shared-table load (the
//     table of pass_u8.cuh, entry k at byte 16 k) and one compare;
//   - histogram: byte b of the new word is the pair (site 2b, site 2b+1),
//     directly a pair bin;
//   - black pass: the final unequal-neighbour count per site is X where
//     accepted and Y where not.
// One thread owns 8 NWN sites (NWN = 2 or 4 words, 8 or 16 bytes) of a row
// and walks rows as the byte walk does; the side neighbour word is the
// centre row shifted by one nibble, its missing site coming from a 4-byte
// load (L1/L2 hit).
#pragma once
#include <cstdint>

#include "pass_u8.cuh"

namespace potts {

constexpr uint32_t kNib7 = 0x77777777u, kNib8 = 0x88888888u;

// [a != b] per nibble, in bit 0 of each nibble (a, b: 4-bit lanes).
__device__ __forceinline__ uint32_t nib_ne(uint32_t a, uint32_t b,
                                           uint32_t one) {
  const uint32_t x = a ^ b;
  const uint32_t t = (x & kNib7) * one + kNib7;  // bit 3: [x & 7 != 0]
  return __umulhi((t | x) & kNib8, 1u << 29);    // bit 3 -> bit 0
}

// Per-thread walk state: the three other-plane rows around the current row
// and the current own row (NWN nibble words each).
template <int NWN>
struct NibWalk {
  uint32_t Up[NWN], Ce[NWN], S[NWN];
  const uint8_t *oth_next;  // other plane, row i+1
  const uint8_t *oth_cur;   // other plane, row i
  uint8_t *own_cur;         // own plane, row i
  int32_t i;                // current plane row
  uint32_t g0;              // Philox counter word 0 of the row's first site
};

// NWN nibble words of a row from p (8 NWN / 2 bytes, aligned to them).
template <int NWN, bool STREAM>
__device__ __forceinline__ void nib_load(const uint8_t *p, uint32_t w[NWN]) {
  if constexpr (NWN == 4) {
    const uint4 v = STREAM ? __ldcs(reinterpret_cast<const uint4 *>(p))
                           : __ldg(reinterpret_cast<const uint4 *>(p));
    w[0] = v.x;
    w[1] = v.y;
    w[2] = v.z;
    w[3] = v.w;
  } else {
    const uint2 v = STREAM ? __ldcs(reinterpret_cast<const uint2 *>(p))
                           : __ldg(reinterpret_cast<const uint2 *>(p));
    w[0] = v.x;
    w[1] = v.y;
  }
}
template <int NWN>
__device__ __forceinline__ void nib_store(uint8_t *p, const uint32_t w[NWN]) {
  if constexpr (NWN == 4)
    __stcs(reinterpret_cast<uint4 *>(p), make_uint4(w[0], w[1], w[2], w[3]));
  else
    __stcs(reinterpret_cast<uint2 *>(p), make_uint2(w[0], w[1]));
}

// One row of 8 NWN sites.  LEFT: the side neighbour is at x-1, else at
// x+1.  xb: byte offset of the window in a row; xl, xr: byte offsets of the
// words holding the side sites; RB: bytes per plane row.
template <bool LEFT, bool COUNTS, bool LT0, int NWN>
__device__ __forceinline__ void nib_row(const PassArgs &A, const PhiloxKey &ks,
                                        const uint8_t *tab, NibWalk<NWN> &w,
                                        int32_t xb, int32_t xl, int32_t xr,
                                        int32_t RB, bool more,
                                        uint32_t *lane_hist,
                                        uint32_t &ne_total) {
  const int32_t L = A.L, H = A.H;
  uint32_t Dw[NWN];
  nib_load<NWN, false>(w.oth_next, Dw);
  const uint32_t ew = __ldg(reinterpret_cast<const uint32_t *>(
      w.oth_cur - xb + (LEFT ? xl : xr)));
  uint8_t *own_next = (w.i + 1 == L) ? A.own + xb : w.own_cur + RB;
  uint32_t Sn[NWN];
#pragma unroll
  for (int k = 0; k < NWN; ++k) Sn[k] = w.S[k];
  if (more) nib_load<NWN, true>(own_next, Sn);
  const uint32_t *Cw = w.Ce;
  uint32_t Wd[NWN];
  if (LEFT) {  // site x-1: the top nibble of the word before
    Wd[0] = __funnelshift_l(ew, Cw[0], 4);
#pragma unroll
    for (int k = 1; k < NWN; ++k) Wd[k] = __funnelshift_l(Cw[k - 1], Cw[k], 4);
  } else {     // site x+1: the low nibble of the word after
#pragma unroll
    for (int k = 0; k < NWN - 1; ++k)
      Wd[k] = __funnelshift_r(Cw[k], Cw[k + 1], 4);
    Wd[NWN - 1] = __funnelshift_r(Cw[NWN - 1], ew, 4);
  }
  const uint32_t one = A.one;
  uint32_t Nw[NWN], ne_acc = 0;
#pragma unroll
  for (int k = 0; k < NWN; ++k) {
    const uint4 u0 = philox10(w.g0 + 2u * k, A.t_lo, A.colour, A.t_hi, ks);
    const uint4 u1 =
        philox10(w.g0 + 2u * k + 1u, A.t_lo, A.colour, A.t_hi, ks);
    const uint32_t uw[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
    uint32_t a[8], P = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint64_t r = (uint64_t)uw[j] * A.q;
      a[j] = (uint32_t)r;
      // proposal into nibble j: a multiply-add with the run-time one (the
      // fields are disjoint), on the FMA-heavy pipe (1.117 against 1.147 ps
      // per update at L = 32768 with shifts and ORs; for the byte walk's
      // pack4 the byte permutes stay faster, 1.194 against 1.236)
      P = (uint32_t)(r >> 32) * (one << (4 * j)) + P;
    }
    const uint32_t S = w.S[k];
    const uint32_t Y = nib_ne(S, w.Up[k], one) + nib_ne(S, Dw[k], one) +
                       nib_ne(S, Cw[k], one) + nib_ne(S, Wd[k], one);
    const uint32_t X = nib_ne(P, w.Up[k], one) + nib_ne(P, Dw[k], one) +
                       nib_ne(P, Cw[k], one) + nib_ne(P, Wd[k], one);
    const uint32_t idx = X + 0x44444444u - Y;  // X + 4 >= Y: no borrow
    // 16 * idx of the even / odd sites, one per byte (the table's offsets)
    const uint32_t ev16 = (idx << 4) & 0xF0F0F0F0u, od16 = idx & 0xF0F0F0F0u;
    uint32_t m = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint32_t off =
          __byte_perm((j & 1) ? od16 : ev16, 0u, 0x4440u + (uint32_t)(j >> 1));
      const uint32_t t = *reinterpret_cast<const uint32_t *>(tab + off);
      const bool acc = LT0 ? (a[j] < t) || (off <= 64u) : a[j] <= t;
      if (acc) m |= 0xFu << (4 * j);
    }
    Nw[k] = (P & m) | (S & ~m);
    if (COUNTS) {
      const uint32_t nf = (X & m) | (Y & ~m);  // <= 4 per nibble
      ne_acc += (nf & 0x0F0F0F0Fu) + ((nf >> 4) & 0x0F0F0F0Fu);
    }
  }
  // <= 8 NWN (32) per byte, so the four bytes sum below 256
  if (COUNTS) ne_total += (ne_acc * 0x01010101u) >> 24;
  nib_store<NWN>(w.own_cur, Nw);
#pragma unroll
  for (int k = 0; k < NWN; ++k) {
#pragma unroll
    for (int b = 0; b < 4; ++b)
      bin_count(lane_hist - (threadIdx.x & 31u), Nw[k], b);
  }
#pragma unroll
  for (int k = 0; k < NWN; ++k) {
    w.Up[k] = w.Ce[k];
    w.Ce[k] = Dw[k];
    w.S[k] = Sn[k];
  }
  w.oth_cur = w.oth_next;
  w.oth_next = (w.i + 2 >= L) ? A.other + xb + (int64_t)(w.i + 2 - L) * RB
                              : w.oth_next + RB;
  w.own_cur = own_next;
  w.i += 1;
  w.g0 += (uint32_t)(H >> 2);
}

// Walks rows [i0, i0 + rows) of the 8 NWN-site column starting at site x0
// of the plane of colour COLOUR (U4 layout).  lane_hist: per-lane pair
// bins; COUNTS (black pass): *ne_total receives the unequal (site,
// neighbour) pairs after the update.
template <int COLOUR, bool COUNTS, bool LT0, int NWN = 2>
__device__ __forceinline__ void nib_walk_column(const PassArgs &A,
                                                const PhiloxKey &ks,
                                                const uint8_t *tab, int32_t x0,
                                                int32_t i0, int32_t rows,
                                                uint32_t *lane_hist,
                                                uint32_t *ne_total) {
  const int32_t L = A.L, H = A.H, RB = H / 2, xb = x0 / 2;
  const int32_t xl = (x0 == 0) ? RB - 4 : xb - 4;  // word holding site x0-1
  // word holding site x0 + 8 NWN
  const int32_t xr = (x0 + 8 * NWN == H) ? 0 : xb + 4 * NWN;
  NibWalk<NWN> w;
  const int32_t im = (i0 == 0) ? L - 1 : i0 - 1;
  const int32_t ip = (i0 + 1 == L) ? 0 : i0 + 1;
  w.oth_cur = A.other + (int64_t)i0 * RB + xb;
  w.oth_next = A.other + (int64_t)ip * RB + xb;
  w.own_cur = A.own + (int64_t)i0 * RB + xb;
  nib_load<NWN, false>(A.other + (int64_t)im * RB + xb, w.Up);
  nib_load<NWN, false>(w.oth_cur, w.Ce);
  nib_load<NWN, true>(w.own_cur, w.S);
  w.i = i0;
  w.g0 = (uint32_t)(((int64_t)(i0 + A.grow0) * H + x0) >> 2);
  int32_t r = 0;
  if (((i0 + A.grow0) & 1) == 0) {
    for (; r + 2 <= rows; r += 2) {
      nib_row<COLOUR == 0, COUNTS, LT0, NWN>(A, ks, tab, w, xb, xl, xr, RB,
                                             true, lane_hist, *ne_total);
      nib_row<COLOUR == 1, COUNTS, LT0, NWN>(A, ks, tab, w, xb, xl, xr, RB,
                                             r + 2 < rows, lane_hist,
                                             *ne_total);
    }
  }
  for (; r < rows; ++r) {
    const bool left = ((w.i + A.grow0 + COLOUR) & 1) == 0;
    if (left)
      nib_row<true, COUNTS, LT0, NWN>(A, ks, tab, w, xb, xl, xr, RB,
                                      r + 1 < rows, lane_hist, *ne_total);
    else
      nib_row<false, COUNTS, LT0, NWN>(A, ks, tab, w, xb, xl, xr, RB,
                                       r + 1 < rows, lane_hist, *ne_total);
  }
}

}  // namespace potts
