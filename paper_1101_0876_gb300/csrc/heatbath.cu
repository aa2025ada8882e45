// Kernel of the heat-bath colour pass (heatbath.cuh holds the rule and the
// walk) and the host side of its weight table.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "heatbath.cuh"
#include "internal.cuh"

namespace potts {

namespace {

constexpr int kHbPairBins = 256;

// Resident CTAs per SM asked of the compiler: the heat-bath rule keeps more
// values live than the Metropolis one.  3 CTAs (up to 168 registers, no
// spills); 4 CTAs fit the word rule without spills too and measured the
// same (1.585 against 1.587 ps per update at L = 32768, q = 9).
#ifndef POTTS_HB_MINB
#define POTTS_HB_MINB 3
#endif

// Same grid, walk and reductions as the Metropolis pass kernel (XP: the
// histogram of both planes in (black, white) pair bins, black pass only).
template <int QB, int COLOUR, bool PAIRS, int LAY, bool XP = false>
__global__ void __launch_bounds__(kPassThreads, POTTS_HB_MINB)
    hb_pass_kernel(PassArgs A, HeatTable T, TileGeom G,
                   unsigned long long *rec) {
  constexpr bool COUNTS = COLOUR == 1;
  constexpr bool HIST = !XP || COUNTS;
  constexpr bool PBINS = PAIRS || XP;
  extern __shared__ __align__(16) uint32_t s_hist[];
  __shared__ __align__(16) uint32_t s_W[kHbTableWords];
  __shared__ uint32_t s_sat;
  __shared__ uint32_t s_fold[16];
  const uint32_t tid = threadIdx.x;
  constexpr uint32_t STRIDE = kBinStride;  // words per bin (bin_count)
  const uint32_t bins = PBINS ? (uint32_t)kHbPairBins : A.hist_bins;
  if (HIST)
    bins_zero(s_hist, bins, tid, kPassThreads);
  if (tid < 16) s_fold[tid] = 0;
  if (tid == 0) s_sat = 0;
  hb_build_table(s_W, T.W, tid);  // ends with a barrier
  pdl_wait_previous();

  const PhiloxKey ks = philox_schedule(A.key0, A.key1);
  const int32_t cx = (int32_t)tid % G.CX, rg = (int32_t)tid / G.CX;
  const int32_t chunk = (int32_t)blockIdx.x * G.CX + cx;
  uint32_t ne = 0, rows_done = 0;
  if (rg < G.RG && chunk * 16 < A.H) {
    for (int32_t tile = blockIdx.y; tile < G.ty; tile += gridDim.y) {
      const int32_t i0 = A.row_lo + (tile * G.RG + rg) * G.TR;
      if (i0 >= A.row_end) continue;
      const int32_t rows = min(G.TR, A.row_end - i0);
      hb_walk_column<QB, COLOUR, COUNTS, PAIRS, LAY, XP>(
          A, ks, s_W, T.m, chunk * 16, i0, rows, s_hist + (tid & 31u), &ne);
      rows_done += (uint32_t)rows;
    }
  }
  pdl_release_next();
  if (COUNTS) {
    uint32_t sat = 64u * rows_done - ne;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sat += __shfl_xor_sync(0xFFFFFFFFu, sat, o);
    if ((tid & 31u) == 0 && sat) atomicAdd(&s_sat, sat);
  }
  __syncthreads();
  if (COUNTS && tid == 0 && s_sat) atomicAdd(rec, (unsigned long long)s_sat);
  if (!HIST) return;
  if (PBINS) {
    for (uint32_t p = tid; p < (uint32_t)kHbPairBins; p += kPassThreads) {
      const uint32_t sum = bin_sum(s_hist, p, STRIDE);
      if (sum) {
        atomicAdd(&s_fold[p & 15u], sum);
        atomicAdd(&s_fold[p >> 4], sum);
      }
    }
    __syncthreads();
    if (tid < A.q && s_fold[tid])
      atomicAdd(rec + 1 + tid, (unsigned long long)s_fold[tid]);
  } else {
    for (uint32_t v = tid; v < A.q; v += kPassThreads) {
      const uint32_t sum = bin_sum(s_hist, v, STRIDE);
      if (sum) atomicAdd(rec + 1 + v, (unsigned long long)sum);
    }
  }
}

template <int QB, int COLOUR, bool PAIRS, int LAY, bool XP = false>
cudaError_t launch_hb_c(const PassArgs &A, const HeatTable &T,
                        const TileGeom &G, unsigned long long *rec,
                        cudaStream_t st) {
  dim3 grid(G.gx, G.gy), block(kPassThreads);
  const size_t bins = (PAIRS || XP) ? kHbPairBins : A.hist_bins;
  const size_t smem = (XP && COLOUR == 0)
                          ? 0
                          : bins * kBinStride * sizeof(uint32_t);
  return launch_pdl(hb_pass_kernel<QB, COLOUR, PAIRS, LAY, XP>, grid, block,
                    smem, st, A, T, G, rec);
}

template <int QB, int LAY>
cudaError_t launch_hb_lay(const PassArgs &A, const HeatTable &T,
                          const TileGeom &G, unsigned long long *rec,
                          cudaStream_t st) {
  if constexpr (QB == 4) {
    if (G.pairs == 2)
      return A.colour ? launch_hb_c<4, 1, false, LAY, true>(A, T, G, rec, st)
                      : launch_hb_c<4, 0, false, LAY, true>(A, T, G, rec, st);
    if (G.pairs)
      return A.colour ? launch_hb_c<4, 1, true, LAY>(A, T, G, rec, st)
                      : launch_hb_c<4, 0, true, LAY>(A, T, G, rec, st);
  }
  return A.colour ? launch_hb_c<QB, 1, false, LAY>(A, T, G, rec, st)
                  : launch_hb_c<QB, 0, false, LAY>(A, T, G, rec, st);
}

// Largest normaliser over the ways four neighbours split into k distinct
// states with counts c_1..c_k: Z = sum W[c] + (q - k) W[0].
uint64_t zmax_of(const uint64_t w[5], int32_t q) {
  const int split[5][4] = {
      {4, 0, 0, 0}, {3, 1, 0, 0}, {2, 2, 0, 0}, {2, 1, 1, 0}, {1, 1, 1, 1}};
  uint64_t best = 0;
  for (const auto &sp : split) {
    int k = 0;
    uint64_t z = 0;
    for (int c : sp) {
      if (c == 0) continue;
      z += w[c];
      ++k;
    }
    if (k > q) continue;
    z += (uint64_t)(q - k) * w[0];
    best = std::max(best, z);
  }
  return best;
}

}  // namespace

bool heatbath_table(double beta, int32_t q, uint64_t W[5], int32_t *m) {
  if (!(beta >= 0.0) || !std::isfinite(beta) || q < 2 || q > 256) return false;
  for (int32_t e = 31; e >= 0; --e) {
    uint64_t w[5];
    bool ok = true;
    for (int n = 0; n <= 4 && ok; ++n) {
      const double x = std::ldexp(std::exp(beta * (double)n), e);
      if (!(x < 4294967296.0))
        ok = false;
      else
        w[n] = (uint64_t)std::floor(x + 0.5);
    }
    if (!ok || zmax_of(w, q) > 0xFFFFFFFFull) continue;
    std::memcpy(W, w, sizeof w);
    *m = e;
    return true;
  }
  return false;
}

HeatTable heat_table(const uint64_t W[5], int32_t m) {
  HeatTable T;
  for (int n = 0; n < 8; ++n) T.W[n] = n < 5 ? (uint32_t)W[n] : 0u;
  T.m = (uint32_t)m;
  return T;
}

cudaError_t launch_pass_hb(const PassArgs &A, const HeatTable &T,
                           const TileGeom &G, unsigned long long *rec,
                           cudaStream_t st) {
  if (!rec) return cudaErrorInvalidValue;
  if (A.layout == kLayoutU4) {
    if (A.q > 16) return cudaErrorInvalidValue;
    return launch_hb_lay<4, kLayoutU4>(A, T, G, rec, st);
  }
  switch (qbits_for((int32_t)A.q)) {
    case 4: return launch_hb_lay<4, kLayoutU8>(A, T, G, rec, st);
    case 5: return launch_hb_lay<5, kLayoutU8>(A, T, G, rec, st);
    case 6: return launch_hb_lay<6, kLayoutU8>(A, T, G, rec, st);
    default: return launch_hb_lay<8, kLayoutU8>(A, T, G, rec, st);
  }
}

}  // namespace potts

using namespace potts;

extern "C" int potts_heatbath_weights(double beta, int32_t q,
                                      uint64_t out_W[5], int32_t *out_m) {
  if (!out_W || !out_m) return fail(POTTS_EINVAL, "NULL argument");
  if (!heatbath_table(beta, q, out_W, out_m))
    return fail(POTTS_EINVAL,
                "no heat-bath weights for beta=%g, q=%d (beta must be finite, "
                ">= 0 and small enough that exp(4 beta) + q - 1 < 2^32)",
                beta, q);
  clear_error();
  return POTTS_OK;
}
