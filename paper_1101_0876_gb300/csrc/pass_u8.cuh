// One colour pass of the checkerboard Metropolis sweep on the byte-per-spin
// colour-plane layout (Sec. 3.3: white and black sites packed into separate
// contiguous arrays; here each plane is L rows x H = L/2 bytes).
//
// Plane geometry.  Colour c holds the sites (i, j) with (i + j) % 2 == c;
// the site with column j sits at byte x = j >> 1 of row i of plane c, so its
// index inside the colour class is k = i*H + x = (i*L + j) >> 1.  Its four
// neighbours are all in the other plane: rows i-1 and i+1 at the same x,
// row i at x, and row i at x-1 when (i + c) is even, x+1 when it is odd
// (all indices periodic).
//
// Work unit.  One thread owns 16 consecutive bytes (16 sites) of a row and
// walks down `rows` consecutive rows, keeping the three other-plane rows it
// needs (i-1, i, i+1) in registers, so each other-plane row is fetched from
// memory once per walk.  The one byte that lies outside the 16-byte window
// (x-1 or x+16) comes from a 4-byte load that hits L1/L2.
//
// Arithmetic is byte-SIMD on 32-bit words (4 sites per word):
//   - neighbour compares: for x = a ^ b per byte, "x != 0" is read from one
//     bit of x + (2^QB - 1) when every spin is < 2^QB (QB = 4, 5, 6, 7),
//     and from the exact zero-byte test for QB = 8; counts of unequal
//     neighbours are kept as 16 * count per byte;
//   - idx = 16 * (4 + dE) per byte, dE = n_old - n_new in -4..4;
//   - acceptance: one table load and one compare per site.
// Random numbers: one Philox4x32-10 call per 4 consecutive sites of a row,
// counter (k >> 2, t_lo, colour, t_hi), key (seed_lo, seed_hi), word k & 3.
#pragma once
#include <cstdint>

#include "philox.cuh"

namespace potts {

struct PassArgs {
  uint8_t *own;          // plane being updated (colour `colour`)
  const uint8_t *other;  // the other plane (read only in this pass)
  int32_t L;             // rows
  int32_t H;             // bytes per row = L / 2 (multiple of 16)
  uint32_t q;
  uint32_t colour;
  uint32_t t_lo, t_hi;   // global sweep index
  uint32_t key0, key1;   // seed
};

// Table of the acceptance rule, indexed by dE + 4 (0..8).
//   rule LE  : accept iff a <= tab[dE+4]   (tab = thr-1 for dE >= 1,
//                                           0xFFFFFFFF for dE <= 0);
//              valid whenever every thr[d] >= 1.
//   rule LT0 : accept iff dE <= 0 or a < tab[dE+4]  (tab = thr);
//              used when some thr[d] == 0 (very large beta).
struct AcceptTable {
  uint32_t tab[9];
  uint32_t rule_lt0;  // 1: rule LT0, 0: rule LE
};

// ---------------------------------------------------------------- SWAR

// 16 * [byte != 0] per byte of x = a ^ b, summed over four words (result
// per byte <= 64).  Every spin byte is < 2^QB.
template <int QB>
__device__ __forceinline__ uint32_t ne16_sum4(uint32_t x0, uint32_t x1,
                                              uint32_t x2, uint32_t x3) {
  if constexpr (QB == 4) {
    const uint32_t K = 0x0F0F0F0Fu, M = 0x10101010u;
    return ((x0 + K) & M) + ((x1 + K) & M) + ((x2 + K) & M) + ((x3 + K) & M);
  } else if constexpr (QB == 5) {
    const uint32_t K = 0x1F1F1F1Fu, M = 0x20202020u;
    return (((x0 + K) & M) + ((x1 + K) & M) + ((x2 + K) & M) +
            ((x3 + K) & M)) >> 1;
  } else if constexpr (QB == 6) {
    const uint32_t K = 0x3F3F3F3Fu, M = 0x40404040u;
    return ((((x0 + K) & M) + ((x1 + K) & M)) >> 2) +
           ((((x2 + K) & M) + ((x3 + K) & M)) >> 2);
  } else if constexpr (QB == 7) {
    const uint32_t K = 0x7F7F7F7Fu, M = 0x80808080u;
    return (((x0 + K) & M) >> 3) + (((x1 + K) & M) >> 3) +
           (((x2 + K) & M) >> 3) + (((x3 + K) & M) >> 3);
  } else {
    const uint32_t K = 0x7F7F7F7Fu, M = 0x80808080u;
    auto ne = [&](uint32_t x) {
      return ((((x & K) + K) | x) & M) >> 3;
    };
    return ne(x0) + ne(x1) + ne(x2) + ne(x3);
  }
}

// Updates the four sites of one 32-bit word.  S: own spins; Pw: proposals
// packed as bytes; U, D, C, W: up, down, centre and side neighbour words;
// a[b]: acceptance variates.  Returns the new word; *nf16 receives
// 16 * (number of unequal neighbours after the update) per byte.
template <int QB, bool WANT_NF, bool LT0>
__device__ __forceinline__ uint32_t update_word(
    uint32_t S, uint32_t Pw, const uint32_t a[4], uint32_t U, uint32_t D,
    uint32_t C, uint32_t W, const uint32_t *tab, uint32_t *nf16) {
  const uint32_t no = ne16_sum4<QB>(S ^ U, S ^ D, S ^ C, S ^ W);
  const uint32_t nn = ne16_sum4<QB>(Pw ^ U, Pw ^ D, Pw ^ C, Pw ^ W);
  // 16 * (4 + dE), dE = n_old - n_new = NE_new - NE_old, in 0..128
  const uint32_t idx = 0x40404040u + nn - no;
  uint32_t m = 0;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const uint32_t ib = (idx >> (8 * b)) & 0xFFu;
    const uint32_t t = tab[ib >> 4];
    bool acc;
    if (LT0)
      acc = (ib <= 64u) || (a[b] < t);
    else
      acc = a[b] <= t;
    m |= acc ? (0xFFu << (8 * b)) : 0u;
  }
  if (WANT_NF) *nf16 = no ^ ((no ^ nn) & m);
  return S ^ ((S ^ Pw) & m);
}

__device__ __forceinline__ uint32_t pack4(uint32_t p0, uint32_t p1,
                                          uint32_t p2, uint32_t p3) {
  const uint32_t lo = __byte_perm(p0, p1, 0x0040u);
  const uint32_t hi = __byte_perm(p2, p3, 0x0040u);
  return __byte_perm(lo, hi, 0x5410u);
}

// Counts state v of every byte of w into the per-lane shared histogram.
__device__ __forceinline__ void hist_word(uint32_t *s_hist, uint32_t lane,
                                          uint32_t w) {
#pragma unroll
  for (int b = 0; b < 4; ++b)
    atomicAdd(&s_hist[((w >> (8 * b)) & 0xFFu) * 32u + lane], 1u);
}

__device__ __forceinline__ uint4 ld_stream(const uint8_t *p) {
  return __ldcs(reinterpret_cast<const uint4 *>(p));
}
__device__ __forceinline__ uint4 ld_other(const uint8_t *p) {
  return __ldg(reinterpret_cast<const uint4 *>(p));
}
__device__ __forceinline__ void st_stream(uint8_t *p, uint4 v) {
  __stcs(reinterpret_cast<uint4 *>(p), v);
}

// Walks rows [i0, i0 + rows) of the 16-byte column starting at byte x0.
// COUNTS: accumulate the unequal-neighbour total of the updated sites into
// *ne_total and the final states of the updated sites and of the
// other-plane sites at the same (i, x) into s_hist.
template <int QB, bool COUNTS, bool LT0>
__device__ __forceinline__ void walk_column(const PassArgs &A,
                                            const PhiloxKey &ks,
                                            const uint32_t *tab, int32_t x0,
                                            int32_t i0, int32_t rows,
                                            uint32_t *s_hist, uint32_t lane,
                                            uint32_t *ne_total) {
  const int32_t L = A.L, H = A.H;
  const uint8_t *other = A.other;
  uint8_t *own = A.own;
  const int32_t xl = (x0 == 0) ? H - 4 : x0 - 4;    // word holding x0-1
  const int32_t xr = (x0 + 16 == H) ? 0 : x0 + 16;  // word holding x0+16

  int32_t im = (i0 == 0) ? L - 1 : i0 - 1;
  uint4 Up = ld_other(other + (int64_t)im * H + x0);
  uint4 Ce = ld_other(other + (int64_t)i0 * H + x0);
  uint4 S = ld_stream(own + (int64_t)i0 * H + x0);

  for (int32_t r = 0; r < rows; ++r) {
    const int32_t i = i0 + r;
    const int32_t ip = (i + 1 == L) ? 0 : i + 1;
    const uint4 Dn = ld_other(other + (int64_t)ip * H + x0);
    const bool left = ((i + (int32_t)A.colour) & 1) == 0;
    const uint32_t ew = __ldg(reinterpret_cast<const uint32_t *>(
        other + (int64_t)i * H + (left ? xl : xr)));
    uint4 Sn = S;
    if (r + 1 < rows) Sn = ld_stream(own + (int64_t)ip * H + x0);

    // side-neighbour words
    uint32_t Wd[4];
    const uint32_t Cw[4] = {Ce.x, Ce.y, Ce.z, Ce.w};
    if (left) {
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
    const uint32_t Uw[4] = {Up.x, Up.y, Up.z, Up.w};
    const uint32_t Dw[4] = {Dn.x, Dn.y, Dn.z, Dn.w};
    const uint32_t Sw[4] = {S.x, S.y, S.z, S.w};
    uint32_t Nw[4];
    const uint32_t g0 = (uint32_t)(((int64_t)i * H + x0) >> 2);
    uint32_t ne_acc = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const uint4 u = philox10(g0 + (uint32_t)w, A.t_lo, A.colour, A.t_hi, ks);
      const uint32_t uw[4] = {u.x, u.y, u.z, u.w};
      uint32_t p[4], a[4];
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const uint64_t prod = (uint64_t)uw[b] * A.q;
        p[b] = (uint32_t)(prod >> 32);
        a[b] = (uint32_t)prod;
      }
      const uint32_t Pw = pack4(p[0], p[1], p[2], p[3]);
      uint32_t nf16 = 0;
      Nw[w] = update_word<QB, COUNTS, LT0>(Sw[w], Pw, a, Uw[w], Dw[w], Cw[w],
                                           Wd[w], tab, &nf16);
      if (COUNTS) ne_acc += nf16 >> 4;
    }
    st_stream(own + (int64_t)i * H + x0, make_uint4(Nw[0], Nw[1], Nw[2], Nw[3]));
    if (COUNTS) {
      *ne_total += (ne_acc * 0x01010101u) >> 24;
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        hist_word(s_hist, lane, Nw[w]);
        hist_word(s_hist, lane, Cw[w]);
      }
    }
    Up = Ce;
    Ce = Dn;
    S = Sn;
  }
}

}  // namespace potts
