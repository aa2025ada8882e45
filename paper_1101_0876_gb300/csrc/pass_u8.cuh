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
// Work unit.  One thread owns 4 NW consecutive bytes (16 or 32 sites) of a
// row and walks down `rows` consecutive rows, keeping the three other-plane
// rows it needs (i-1, i, i+1) in registers, so each other-plane row is
// fetched from memory once per walk.  The one byte that lies outside the
// window (x-1 or x + 4 NW) comes from a 4-byte load that hits L1/L2.
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
  int32_t H;             // sites per plane row = L / 2 (multiple of 16)
  uint32_t q;
  uint32_t colour;
  uint32_t t_lo, t_hi;   // global sweep index
  uint32_t key0, key1;   // seed
  uint32_t layout;       // kLayoutU8 (1) or kLayoutU4 (2)
  uint32_t one;          // always 1, passed at run time (see delta_index)
  uint32_t hist_bins;    // shared histogram bins: q, or 256 when the planes
                         // come from the caller unchecked (any byte value
                         // then indexes inside the histogram)
  // Rows of the planes and their place in the lattice.  A whole lattice:
  // L rows, grow0 = 0, rows [0, L) updated, row indices periodic in L.  A
  // row strip of one lattice (rows r0 .. r0 + n - 1 of it): L = n + 2 rows,
  // row 0 and row n + 1 holding copies of the rows just above and below the
  // strip, grow0 = r0 - 1 (the lattice row of plane row 0), rows [1, n + 1)
  // updated; no row index wraps then.  The random-number counters and the
  // checkerboard parity use the lattice row grow0 + i.
  int32_t grow0;
  int32_t row_lo, row_end;
};

// Bytes of the shared acceptance table: entry k (dE + 4) at offset 16 k,
// padded so that any offset byte (0..255) stays inside it.
constexpr int kTabWords = 65;

// Acceptance rule, tabulated by dE + 4 (0..8).
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
//
// Per site the decision needs idx = 16 * (4 + dE) (dE = n_old - n_new).
// For spins < 2^QB, a = (S ^ N) + (2^QB - 1) holds [S != N] in bit QB and
// b = (P ^ N) + (2^QB - 1) holds [P != N] there, so with M = 2^QB per byte
// X = sum (b & M) = M (4 - n_new) and Y = sum (a & M) = M (4 - n_old) over
// the four neighbours, and 4 + dE = 4 + (X - Y) / M: one logic op per
// (state, neighbour) pair.  Y and X are also the mismatch counts the black
// pass needs for its bond count (old and proposed state).

template <int QB>
struct Swar {
  static constexpr uint32_t K = 0x01010101u * ((1u << QB) - 1u);
  static constexpr uint32_t M = 0x01010101u * (1u << QB);
};

// 16 * [byte != 0] per byte of x = a ^ b, summed over four words (result
// per byte <= 64).  Every spin byte is < 2^QB.  Used for QB >= 6 and for
// the unequal-neighbour count of the black pass.
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
    auto ne = [&](uint32_t x) { return ((((x & K) + K) | x) & M) >> 3; };
    return ne(x0) + ne(x1) + ne(x2) + ne(x3);
  }
}

// idx = 16 * (4 + dE) per byte for the four sites of one word.  With
// WANT_NO also *no16 = 16 * (number of neighbours unequal to S) and
// *nn16 = 16 * (number unequal to P).
// `one` is the constant 1, supplied at run time where the eight additions
// of K should issue as multiply-adds (x * one + K, which the compiler cannot
// fold back into additions) on the FMA-heavy pipe instead of the busier ALU
// pipe; a literal 1 leaves them on the ALU (the white pass with the run-time
// one: 1.55 % faster at L = 32768).
template <int QB, bool WANT_NO>
__device__ __forceinline__ uint32_t delta_index(uint32_t S, uint32_t P,
                                                uint32_t U, uint32_t D,
                                                uint32_t C, uint32_t W,
                                                uint32_t *no16, uint32_t *nn16,
                                                uint32_t one) {
  if constexpr (QB <= 5) {
    constexpr uint32_t K = Swar<QB>::K, M = Swar<QB>::M;
    const uint32_t a0 = (S ^ U) * one + K, a1 = (S ^ D) * one + K,
                   a2 = (S ^ C) * one + K, a3 = (S ^ W) * one + K;
    const uint32_t b0 = (P ^ U) * one + K, b1 = (P ^ D) * one + K,
                   b2 = (P ^ C) * one + K, b3 = (P ^ W) * one + K;
    // per byte at most 4 M = 64 (QB 4) or 128 (QB 5): no carry between bytes
    uint32_t X = (b0 & M) + (b1 & M) + (b2 & M) + (b3 & M);
    uint32_t Y = (a0 & M) + (a1 & M) + (a2 & M) + (a3 & M);
    if (QB == 5) {  // multiples of 32 per byte: the shift moves no bit across
      X >>= 1;
      Y >>= 1;
    }
    if (WANT_NO) {
      *no16 = Y;
      *nn16 = X;
    }
    return (X + 0x40404040u) - Y;  // X + 64 >= Y per byte: no borrow
  } else {
    const uint32_t no = ne16_sum4<QB>(S ^ U, S ^ D, S ^ C, S ^ W);
    const uint32_t nn = ne16_sum4<QB>(P ^ U, P ^ D, P ^ C, P ^ W);
    if (WANT_NO) {
      *no16 = no;
      *nn16 = nn;
    }
    return 0x40404040u + nn - no;
  }
}

// Acceptance of the four sites of one word: byte b of the result is 0xFF
// if site b accepts its proposal.  tab: shared table, entry for dE + 4 = k
// at byte offset 16 k (so the idx byte is the offset itself).
template <bool LT0>
__device__ __forceinline__ uint32_t accept_mask(uint32_t idx, uint32_t a0,
                                                uint32_t a1, uint32_t a2,
                                                uint32_t a3,
                                                const uint8_t *tab) {
  const uint32_t a[4] = {a0, a1, a2, a3};
  uint32_t m = 0;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const uint32_t off = __byte_perm(idx, 0u, 0x4440u + (uint32_t)b);
    const uint32_t t = *reinterpret_cast<const uint32_t *>(tab + off);
    bool acc;
    if (LT0)
      acc = (a[b] < t) || (off <= 64u);
    else
      acc = a[b] <= t;
    if (acc) m |= 0xFFu << (8 * b);
  }
  return m;
}

__device__ __forceinline__ uint32_t pack4(uint32_t p0, uint32_t p1,
                                          uint32_t p2, uint32_t p3) {
  const uint32_t lo = __byte_perm(p0, p1, 0x0040u);
  const uint32_t hi = __byte_perm(p2, p3, 0x0040u);
  return __byte_perm(lo, hi, 0x5410u);
}

// Per-lane histogram counters: lane l's counter of bin p at word
// p * kBinStride + l.  The 64-word stride lets one byte permute form a
// counter's byte offset from the bin byte and the lane (the bin in bits
// 8..15, 4 l in bits 0..6); a 32-word stride needs a shift-and-add more per
// count.
constexpr uint32_t kBinStride = 64;

// Zeroes the 32 lane counters of bins [0, bins) in the kBinStride layout
// with 16-byte stores (the other half of each bin's words is never used).
__device__ __forceinline__ void bins_zero(uint32_t *s_hist, uint32_t bins,
                                          uint32_t tid, uint32_t nthreads) {
  for (uint32_t v = tid; v < bins * 8u; v += nthreads)
    *reinterpret_cast<uint4 *>(s_hist + (v >> 3) * kBinStride + (v & 7u) * 4u) =
        make_uint4(0u, 0u, 0u, 0u);
}

// Counts bin (byte b of t) in the calling lane's counters; s_hist: the CTA's
// counters (kBinStride words a bin).
__device__ __forceinline__ void bin_count(uint32_t *s_hist, uint32_t t,
                                          int b) {
  const uint32_t lane4 = (threadIdx.x & 31u) << 2;
  const uint32_t off = __byte_perm(t, lane4, 0x5504u | ((uint32_t)b << 4));
  atomicAdd(reinterpret_cast<uint32_t *>(reinterpret_cast<uint8_t *>(s_hist) +
                                         off),
            1u);
}

// Histogram of the four spins of w into per-lane shared counters.
// PAIRS (q <= 16): the two nibble-sized spins of sites (0,1) and (2,3) form
// one 8-bit bin each, so a word costs two shared atomics; the pair bins are
// folded back to states at the end of the CTA.  WIDE: the kBinStride layout
// (bin_count), else 32 words a bin (lane_hist + 32 bin).
template <bool PAIRS, bool WIDE = true>
__device__ __forceinline__ void hist_word(uint32_t *lane_hist, uint32_t w) {
  if (PAIRS) {
    const uint32_t t = w + __umulhi(w, 1u << 28);  // byte0 = v0 | v1 << 4
    if (WIDE) {
      uint32_t *s_hist = lane_hist - (threadIdx.x & 31u);
      bin_count(s_hist, t, 0);
      bin_count(s_hist, t, 2);
    } else {
      atomicAdd(lane_hist + (t & 0xFFu) * 32u, 1u);
      atomicAdd(lane_hist + __byte_perm(t, 0u, 0x4442u) * 32u, 1u);
    }
  } else {
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      if (WIDE)
        bin_count(lane_hist - (threadIdx.x & 31u), w, b);
      else
        atomicAdd(lane_hist + __byte_perm(w, 0u, 0x4440u + (uint32_t)b) * 32u,
                  1u);
    }
  }
}

// Count of bin v summed over the 32 lanes' counters (lane l's counter of
// bin v at v * stride + l; s_hist 16-byte aligned).  Read as eight 16-byte
// chunks, chunk j ^ (v mod 8) at step j: when the threads of a warp fold
// consecutive bins, the eight lanes of a quarter-warp (one 128-bit
// wavefront) then hit eight different bank groups (in order they would all
// hit the same one).
__device__ __forceinline__ uint32_t bin_sum(const uint32_t *s_hist,
                                            uint32_t v,
                                            uint32_t stride = 32u) {
  const uint4 *row = reinterpret_cast<const uint4 *>(s_hist + v * stride);
  const uint32_t rot = v & 7u;
  uint32_t sum = 0;
#pragma unroll
  for (uint32_t j = 0; j < 8u; ++j) {
    const uint4 x = row[j ^ rot];
    sum += x.x + x.y + x.z + x.w;
  }
  return sum;
}

// Histogram of one black word's new spins paired with the white spins at
// the same plane position (q <= 16): byte b of nw + (cw << 4) is the bin
// (black spin, white spin), so four shared atomics count eight sites and
// the white pass keeps no histogram.  The white plane is final when the
// black pass runs, and the black walks read every white word of their rows
// exactly once as the centre row.  Bytes above 15 (planes the caller did
// not check) can only scramble the bins, never leave them.  one: 1, as a
// literal (the pair forms on the ALU pipe) or the run-time 1 of PassArgs
// (a multiply-add on the FMA-heavy pipe).
// s_hist: the CTA's counters (bin_count).
__device__ __forceinline__ void hist_cross(uint32_t *s_hist, uint32_t nw,
                                           uint32_t cw, uint32_t one) {
  const uint32_t t = cw * (one << 4) + nw;
#pragma unroll
  for (int b = 0; b < 4; ++b) bin_count(s_hist, t, b);
}

// ------------------------------------------------------- plane layouts
// U8: one byte per spin, 16 sites = 16 bytes per vector (one or two per
// thread-row).
// U4: two spins per byte (site 2b in the low nibble of byte b, site 2b+1 in
// the high one), 16 sites = 8 bytes, unpacked to the same four byte-words
// as U8 so that the arithmetic is shared (the heat-bath walk; the
// Metropolis pass computes on the nibbles themselves, pass_u4.cuh).
enum { kLayoutU8 = 1, kLayoutU4 = 2 };

// nibbles n0..n7 (sites 0..7) -> bytes [s0..s3], [s4..s7]
__device__ __forceinline__ void unpack8(uint32_t w, uint32_t &b0,
                                        uint32_t &b1) {
  const uint32_t lo = w & 0x0F0F0F0Fu, hi = (w >> 4) & 0x0F0F0F0Fu;
  b0 = __byte_perm(lo, hi, 0x5140u);
  b1 = __byte_perm(lo, hi, 0x7362u);
}
__device__ __forceinline__ uint32_t pack8(uint32_t b0, uint32_t b1) {
  const uint32_t lo = __byte_perm(b0, b1, 0x6420u);  // s0 s2 s4 s6
  const uint32_t hi = __byte_perm(b0, b1, 0x7531u);  // s1 s3 s5 s7
  return lo | (hi << 4);
}

template <int LAY>
struct Lay {
  static constexpr int kChunkBytes = LAY == kLayoutU4 ? 8 : 16;
  __device__ static __forceinline__ int32_t row_bytes(int32_t H) {
    return LAY == kLayoutU4 ? H / 2 : H;
  }
  __device__ static __forceinline__ void load(const uint8_t *p, bool stream,
                                              uint32_t w[4]) {
    if constexpr (LAY == kLayoutU4) {
      const uint2 v = stream ? __ldcs(reinterpret_cast<const uint2 *>(p))
                             : __ldg(reinterpret_cast<const uint2 *>(p));
      unpack8(v.x, w[0], w[1]);
      unpack8(v.y, w[2], w[3]);
    } else {
      const uint4 v = stream ? __ldcs(reinterpret_cast<const uint4 *>(p))
                             : __ldg(reinterpret_cast<const uint4 *>(p));
      w[0] = v.x;
      w[1] = v.y;
      w[2] = v.z;
      w[3] = v.w;
    }
  }
  __device__ static __forceinline__ void store(uint8_t *p,
                                               const uint32_t w[4]) {
    if constexpr (LAY == kLayoutU4)
      __stcs(reinterpret_cast<uint2 *>(p),
             make_uint2(pack8(w[0], w[1]), pack8(w[2], w[3])));
    else
      __stcs(reinterpret_cast<uint4 *>(p), make_uint4(w[0], w[1], w[2], w[3]));
  }
  // The 4-byte word holding the side site, as a U8 word whose top byte
  // (LEFT: the site before the window) or low byte (right: the site after
  // it) is that site.
  __device__ static __forceinline__ uint32_t edge(uint32_t raw, bool left) {
    if constexpr (LAY == kLayoutU4)
      return left ? (raw >> 28) << 24 : raw & 0xFu;
    else
      return raw;
  }
};

// NW consecutive words (4 NW sites) of one plane row as byte words: U8
// loads them as 16-byte vectors; U4 (NW = 4 only) loads 8 bytes and unpacks.
template <int LAY, int NW>
__device__ __forceinline__ void load_words(const uint8_t *p, bool stream,
                                           uint32_t w[NW]) {
  if constexpr (LAY == kLayoutU4) {
    static_assert(NW == 4, "the unpacking walk takes 16 sites per row");
    Lay<LAY>::load(p, stream, w);
  } else {
#pragma unroll
    for (int v = 0; v < NW / 4; ++v) Lay<LAY>::load(p + 16 * v, stream, w + 4 * v);
  }
}
template <int LAY, int NW>
__device__ __forceinline__ void store_words(uint8_t *p, const uint32_t w[NW]) {
  if constexpr (LAY == kLayoutU4) {
    Lay<LAY>::store(p, w);
  } else {
#pragma unroll
    for (int v = 0; v < NW / 4; ++v) Lay<LAY>::store(p + 16 * v, w + 4 * v);
  }
}

// Per-thread walk state: the three other-plane rows around the current row
// and the current own row (as byte words), plus pointers to the next rows.
template <int NW>
struct WalkT {
  uint32_t Up[NW], Ce[NW], S[NW];
  const uint8_t *oth_next;  // other plane, row i+1
  const uint8_t *oth_cur;   // other plane, row i
  uint8_t *own_cur;         // own plane, row i
  int32_t i;                // current row
  uint32_t g0;              // Philox counter word 0 of the window's first site
};
using Walk = WalkT<4>;

// One row: update the 4 NW sites of the own row i against Up (i-1), Ce (i),
// the freshly loaded row i+1 and the side byte.  LEFT: the side neighbour
// is at x-1 (row parity + colour even), else at x+1.  xb: byte offset of
// the window in a row; xl, xr: byte offsets of the words holding the side
// sites; RB: bytes per plane row; lane_hist: the lane's histogram counters
// (not null).  XP: the cross-plane pair histogram (hist_cross) instead of
// one of the updated sites per pass.
template <int QB, bool LEFT, bool COUNTS, bool PAIRS, bool LT0, int LAY,
          int NW = 4, bool XP = false>
__device__ __forceinline__ void do_row(const PassArgs &A, const PhiloxKey &ks,
                                       const uint8_t *tab, WalkT<NW> &w,
                                       int32_t x0, int32_t xb, int32_t xl,
                                       int32_t xr, int32_t RB, bool more,
                                       uint32_t *lane_hist,
                                       uint32_t &ne_acc) {
  using IO = Lay<LAY>;
  const int32_t L = A.L, H = A.H;
  uint32_t Dw[NW];
  load_words<LAY, NW>(w.oth_next, false, Dw);
  const uint32_t ew = IO::edge(
      __ldg(reinterpret_cast<const uint32_t *>(w.oth_cur - xb +
                                               (LEFT ? xl : xr))),
      LEFT);
  uint8_t *own_next = (w.i + 1 == L) ? A.own + xb : w.own_cur + RB;
  uint32_t Sn[NW];
#pragma unroll
  for (int k = 0; k < NW; ++k) Sn[k] = w.S[k];
  if (more) load_words<LAY, NW>(own_next, true, Sn);

  const uint32_t *Cw = w.Ce;
  uint32_t Wd[NW];
  if (LEFT) {
    Wd[0] = __funnelshift_l(ew, Cw[0], 8);
#pragma unroll
    for (int k = 1; k < NW; ++k) Wd[k] = __funnelshift_l(Cw[k - 1], Cw[k], 8);
  } else {
#pragma unroll
    for (int k = 0; k < NW - 1; ++k) Wd[k] = __funnelshift_r(Cw[k], Cw[k + 1], 8);
    Wd[NW - 1] = __funnelshift_r(Cw[NW - 1], ew, 8);
  }
  uint32_t Nw[NW];
#pragma unroll
  for (int k = 0; k < NW; ++k) {
    const uint4 u = philox10(w.g0 + (uint32_t)k, A.t_lo, A.colour, A.t_hi, ks);
    const uint64_t r0 = (uint64_t)u.x * A.q, r1 = (uint64_t)u.y * A.q;
    const uint64_t r2 = (uint64_t)u.z * A.q, r3 = (uint64_t)u.w * A.q;
    const uint32_t P = pack4((uint32_t)(r0 >> 32), (uint32_t)(r1 >> 32),
                             (uint32_t)(r2 >> 32), (uint32_t)(r3 >> 32));
    uint32_t no16 = 0, nn16 = 0;
    // the white pass moves its additions to the FMA-heavy pipe; the black
    // pass, whose counts already add multiply-adds, keeps them on the ALU
    // (1.2930 against 1.2893 ps per update at L = 32768 with a histogram per
    // pass), except with the cross-plane histogram (XP), whose extra ALU
    // work tips it the other way (1.1993 against 1.2062 ps)
    const uint32_t idx =
        delta_index<QB, COUNTS>(w.S[k], P, w.Up[k], Dw[k], Cw[k], Wd[k], &no16,
                                &nn16, (COUNTS && !XP) ? 1u : A.one);
    const uint32_t m = accept_mask<LT0>(idx, (uint32_t)r0, (uint32_t)r1,
                                        (uint32_t)r2, (uint32_t)r3, tab);
    Nw[k] = (P & m) | (w.S[k] & ~m);
    if (COUNTS) {
      // unequal neighbours after the update: those of P where accepted
      const uint32_t nf16 = (nn16 & m) | (no16 & ~m);
      ne_acc += __umulhi(nf16, 1u << 28);  // += nf16 >> 4 (<= 4 per byte)
    }
  }
  store_words<LAY, NW>(w.own_cur, Nw);
  if constexpr (XP) {
    if (COUNTS) {
#pragma unroll
      for (int k = 0; k < NW; ++k)
        hist_cross(lane_hist - (threadIdx.x & 31u), Nw[k], Cw[k], 1u);
    }
  } else {
#pragma unroll
    for (int k = 0; k < NW; ++k) hist_word<PAIRS>(lane_hist, Nw[k]);
  }
  // advance
#pragma unroll
  for (int k = 0; k < NW; ++k) {
    w.Up[k] = w.Ce[k];
    w.Ce[k] = Dw[k];
    w.S[k] = Sn[k];
  }
  w.oth_cur = w.oth_next;
  w.oth_next = (w.i + 2 >= L) ? A.other + xb + (int64_t)(w.i + 2 - L) * RB
                              : w.oth_next + RB;
  w.own_cur = own_next;
  w.i += 1;
  w.g0 += (uint32_t)(H >> 2);  // walks never wrap past the last row
}

// Walks rows [i0, i0 + rows) of the 4 NW-site column starting at site x0 of
// the plane of colour COLOUR.  lane_hist: per-lane histogram counters of the
// updated sites (XP: of both planes' sites in pairs, on the black pass
// only).  COUNTS (black pass): *ne_total receives
// the number of unequal (site, neighbour) pairs after the update.
template <int QB, int COLOUR, bool COUNTS, bool PAIRS, bool LT0,
          int LAY = kLayoutU8, int NW = 4, bool XP = false>
__device__ __forceinline__ void walk_column(const PassArgs &A,
                                            const PhiloxKey &ks,
                                            const uint8_t *tab, int32_t x0,
                                            int32_t i0, int32_t rows,
                                            uint32_t *lane_hist,
                                            uint32_t *ne_total) {
  using IO = Lay<LAY>;
  const int32_t L = A.L, H = A.H;
  const int32_t RB = IO::row_bytes(H);
  const int32_t xb = LAY == kLayoutU4 ? x0 / 2 : x0;
  const int32_t xl = (x0 == 0) ? RB - 4 : xb - 4;  // word holding site x0-1
  const int32_t xr = (x0 + 4 * NW == H) ? 0
                                        : xb + IO::kChunkBytes * (NW / 4);
  WalkT<NW> w;
  const int32_t im = (i0 == 0) ? L - 1 : i0 - 1;
  const int32_t ip = (i0 + 1 == L) ? 0 : i0 + 1;
  w.oth_cur = A.other + (int64_t)i0 * RB + xb;
  w.oth_next = A.other + (int64_t)ip * RB + xb;
  w.own_cur = A.own + (int64_t)i0 * RB + xb;
  load_words<LAY, NW>(A.other + (int64_t)im * RB + xb, false, w.Up);
  load_words<LAY, NW>(w.oth_cur, false, w.Ce);
  load_words<LAY, NW>(w.own_cur, true, w.S);
  w.i = i0;
  w.g0 = (uint32_t)(((int64_t)(i0 + A.grow0) * H + x0) >> 2);
  uint32_t ne_acc = 0;
  int32_t r = 0;
  // Side neighbour at x-1 when (lattice row + colour) is even.  Walks start
  // on even lattice rows when rows is even, so pairs of rows have a fixed
  // pattern.  The black pass's byte counts (at most 4 per word and byte, so
  // 4 NW per row) are summed across the four bytes by one multiply, whose
  // top byte must stay below 256: every pair of rows for NW = 4, every row
  // for NW = 8.
  auto fold = [&]() {
    if (COUNTS) {
      *ne_total += (ne_acc * 0x01010101u) >> 24;
      ne_acc = 0;
    }
  };
  if (((i0 + A.grow0) & 1) == 0) {
    for (; r + 2 <= rows; r += 2) {
      do_row<QB, COLOUR == 0, COUNTS, PAIRS, LT0, LAY, NW, XP>(
          A, ks, tab, w, x0, xb, xl, xr, RB, true, lane_hist, ne_acc);
      if (NW > 4) fold();
      do_row<QB, COLOUR == 1, COUNTS, PAIRS, LT0, LAY, NW, XP>(
          A, ks, tab, w, x0, xb, xl, xr, RB, r + 2 < rows, lane_hist, ne_acc);
      fold();
    }
  }
  for (; r < rows; ++r) {
    const bool left = ((w.i + A.grow0 + COLOUR) & 1) == 0;
    if (left)
      do_row<QB, true, COUNTS, PAIRS, LT0, LAY, NW, XP>(
          A, ks, tab, w, x0, xb, xl, xr, RB, r + 1 < rows, lane_hist, ne_acc);
    else
      do_row<QB, false, COUNTS, PAIRS, LT0, LAY, NW, XP>(
          A, ks, tab, w, x0, xb, xl, xr, RB, r + 1 < rows, lane_hist, ne_acc);
    fold();
  }
}

}  // namespace potts
