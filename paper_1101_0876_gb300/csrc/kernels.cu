// Kernels of the single-lattice path: the colour pass (white pass, and the
// black pass fused with the per-sweep counts), the random start and a full
// recount.  The per-thread work is in pass_u8.cuh (byte words) and
// pass_u4.cuh (nibble words, the packed 4-bit layout).
#include <algorithm>

#include "internal.cuh"
#include "pass_u4.cuh"

namespace potts {

// ------------------------------------------------------------ the pass
// Grid: (gx, gy) CTAs of 128 threads.  Thread t of CTA (bx, by) owns chunk
// bx*CX + t%CX (16 or 32 sites) and rows starting at (by*RG + t/CX)*TR.
// Each pass histograms the sites it updated (their final values for this
// sweep), except with the cross-plane pair bins (XP), where the black pass
// histograms both planes' sites; the black pass also reduces the
// satisfied-bond count of the black sites against the final white spins,
// which counts every bond once
// (Sec. 3.4: per-block energies and state counters, here summed with warp
// shuffles and shared atomics and added with one 64-bit atomic per
// non-empty bin per CTA, without a second kernel or a CPU-side sum).
constexpr int kPairBins = 256;

// Resident CTAs per SM the pass kernels are compiled for: 128 threads x
// 80 registers for 16 sites per thread, 168 for 32 (the longer rows save
// per-row work), and 128 for the nibble pass.
constexpr int kMinb32 = 3, kMinbNib = 4;

// XP (q <= 16): the histogram of both planes in (black, white) pair bins,
// kept by the black pass alone (hist_cross); the white pass keeps none.
cudaError_t allow_dynamic_smem(const void *kernel, size_t smem) {
  // Set before every such launch, and always to the same cap: the attribute
  // belongs to the kernel in the current context, and one value for every
  // launch keeps threads that launch the same kernel with different sizes
  // from lowering it under each other (a cache keyed by size did exactly
  // that: a later, larger launch then failed).
  if (smem > (size_t)kDynSmemCap) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(
      kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmemCap);
}

template <int QB, int COLOUR, bool PAIRS, bool LT0, int LAY, int NW,
          bool XP = false>
__global__ void __launch_bounds__(kPassThreads,
                                  NW == 8 ? kMinb32 : POTTS_PASS_MINB)
    pass_kernel(PassArgs A, AcceptTable Tin, TileGeom G,
                unsigned long long *rec) {
  constexpr bool COUNTS = COLOUR == 1;
  constexpr bool HIST = !XP || COUNTS;     // this pass keeps a histogram
  constexpr bool PBINS = PAIRS || XP;      // 256 pair bins, folded at the end
  extern __shared__ __align__(16) uint32_t s_hist[];  // bins * 32 (bins = 256 or q)
  __shared__ __align__(16) uint32_t s_tab[kTabWords];
  __shared__ uint32_t s_sat;
  __shared__ uint32_t s_fold[16];
  const uint32_t tid = threadIdx.x;
  constexpr uint32_t STRIDE = kBinStride;  // words per bin (bin_count)
  const uint32_t bins = PBINS ? (uint32_t)kPairBins : A.hist_bins;
  for (uint32_t i = tid; i < (uint32_t)kTabWords; i += kPassThreads)
    s_tab[i] = (i % 4u == 0 && i / 4u < 9u) ? Tin.tab[i / 4u] : 0u;
  if (HIST)
    bins_zero(s_hist, bins, tid, kPassThreads);
  if (tid < 16) s_fold[tid] = 0;
  if (tid == 0) s_sat = 0;
  __syncthreads();
  pdl_wait_previous();  // the other plane is the previous pass's output

  const PhiloxKey ks = philox_schedule(A.key0, A.key1);
  const int32_t cx = (int32_t)tid % G.CX, rg = (int32_t)tid / G.CX;
  const int32_t chunk = (int32_t)blockIdx.x * G.CX + cx;
  uint32_t ne = 0, rows_done = 0;
  if (rg < G.RG && chunk * 4 * NW < A.H) {
    for (int32_t tile = blockIdx.y; tile < G.ty; tile += gridDim.y) {
      const int32_t i0 = A.row_lo + (tile * G.RG + rg) * G.TR;
      if (i0 >= A.row_end) continue;
      const int32_t rows = min(G.TR, A.row_end - i0);
      walk_column<QB, COLOUR, COUNTS, PAIRS, LT0, LAY, NW, XP>(
          A, ks, reinterpret_cast<const uint8_t *>(s_tab), chunk * 4 * NW, i0,
          rows, s_hist + (tid & 31u), &ne);
      rows_done += (uint32_t)rows;
    }
  }
  pdl_release_next();
  if (COUNTS) {
    uint32_t sat = 16u * NW * rows_done - ne;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sat += __shfl_xor_sync(0xFFFFFFFFu, sat, o);
    if ((tid & 31u) == 0 && sat) atomicAdd(&s_sat, sat);
  }
  __syncthreads();
  if (COUNTS && tid == 0 && s_sat) atomicAdd(rec, (unsigned long long)s_sat);
  if (!HIST) return;
  if (PBINS) {
    // fold pair bins (v0 | v1 << 4) back to the 16 states
    for (uint32_t p = tid; p < (uint32_t)kPairBins; p += kPassThreads) {
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

// The U4 Metropolis pass on nibble words (pass_u4.cuh): 8 NWN sites per
// thread and row (16 or 32), pair bins (every byte of a nibble word is a
// pair of sites).
template <int COLOUR, bool LT0, int NWN>
__global__ void __launch_bounds__(kPassThreads, NWN == 4 ? kMinb32 : kMinbNib)
    pass_u4_kernel(PassArgs A, AcceptTable Tin, TileGeom G,
                   unsigned long long *rec) {
  constexpr bool COUNTS = COLOUR == 1;
  constexpr int32_t SITES = 8 * NWN;
  extern __shared__ __align__(16) uint32_t s_hist[];  // 256 pair bins, bin_count
  __shared__ __align__(16) uint32_t s_tab[kTabWords];
  __shared__ uint32_t s_sat;
  __shared__ uint32_t s_fold[16];
  const uint32_t tid = threadIdx.x;
  for (uint32_t i = tid; i < (uint32_t)kTabWords; i += kPassThreads)
    s_tab[i] = (i % 4u == 0 && i / 4u < 9u) ? Tin.tab[i / 4u] : 0u;
  bins_zero(s_hist, kPairBins, tid, kPassThreads);
  if (tid < 16) s_fold[tid] = 0;
  if (tid == 0) s_sat = 0;
  __syncthreads();
  pdl_wait_previous();

  const PhiloxKey ks = philox_schedule(A.key0, A.key1);
  const int32_t cx = (int32_t)tid % G.CX, rg = (int32_t)tid / G.CX;
  const int32_t chunk = (int32_t)blockIdx.x * G.CX + cx;
  uint32_t ne = 0, rows_done = 0;
  if (rg < G.RG && chunk * SITES < A.H) {
    for (int32_t tile = blockIdx.y; tile < G.ty; tile += gridDim.y) {
      const int32_t i0 = A.row_lo + (tile * G.RG + rg) * G.TR;
      if (i0 >= A.row_end) continue;
      const int32_t rows = min(G.TR, A.row_end - i0);
      nib_walk_column<COLOUR, COUNTS, LT0, NWN>(
          A, ks, reinterpret_cast<const uint8_t *>(s_tab), chunk * SITES, i0,
          rows, s_hist + (tid & 31u), &ne);
      rows_done += (uint32_t)rows;
    }
  }
  pdl_release_next();
  if (COUNTS) {
    uint32_t sat = 4u * SITES * rows_done - ne;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sat += __shfl_xor_sync(0xFFFFFFFFu, sat, o);
    if ((tid & 31u) == 0 && sat) atomicAdd(&s_sat, sat);
  }
  __syncthreads();
  if (COUNTS && tid == 0 && s_sat) atomicAdd(rec, (unsigned long long)s_sat);
  for (uint32_t p = tid; p < (uint32_t)kPairBins; p += kPassThreads) {
    const uint32_t sum = bin_sum(s_hist, p, kBinStride);
    if (sum) {
      atomicAdd(&s_fold[p & 15u], sum);
      atomicAdd(&s_fold[p >> 4], sum);
    }
  }
  __syncthreads();
  if (tid < A.q && s_fold[tid])
    atomicAdd(rec + 1 + tid, (unsigned long long)s_fold[tid]);
}

template <int QB, int COLOUR, bool PAIRS, int LAY = kLayoutU8, int NW = 4,
          bool XP = false>
static cudaError_t launch_c(const PassArgs &A, const AcceptTable &T,
                            const TileGeom &G, unsigned long long *rec,
                            cudaStream_t st) {
  dim3 grid(G.gx, G.gy), block(kPassThreads);
  const size_t bins = (PAIRS || XP) ? kPairBins : A.hist_bins;
  const size_t smem = (XP && COLOUR == 0)
                          ? 0
                          : bins * kBinStride * sizeof(uint32_t);
  if (T.rule_lt0)
    return launch_pdl(pass_kernel<QB, COLOUR, PAIRS, true, LAY, NW, XP>, grid,
                      block, smem, st, A, T, G, rec);
  return launch_pdl(pass_kernel<QB, COLOUR, PAIRS, false, LAY, NW, XP>, grid,
                    block, smem, st, A, T, G, rec);
}

template <int QB>
static cudaError_t launch_qb(const PassArgs &A, const AcceptTable &T,
                             const TileGeom &G, unsigned long long *rec,
                             cudaStream_t st) {
  if constexpr (QB == 4) {
    if (G.sites == 32 && G.pairs == 2)
      return A.colour
                 ? launch_c<QB, 1, false, kLayoutU8, 8, true>(A, T, G, rec, st)
                 : launch_c<QB, 0, false, kLayoutU8, 8, true>(A, T, G, rec, st);
  }
  if (G.sites == 32)
    return A.colour ? launch_c<QB, 1, false, kLayoutU8, 8>(A, T, G, rec, st)
                    : launch_c<QB, 0, false, kLayoutU8, 8>(A, T, G, rec, st);
  if constexpr (QB == 4) {
    if (G.pairs)
      return A.colour ? launch_c<QB, 1, true>(A, T, G, rec, st)
                      : launch_c<QB, 0, true>(A, T, G, rec, st);
  }
  return A.colour ? launch_c<QB, 1, false>(A, T, G, rec, st)
                  : launch_c<QB, 0, false>(A, T, G, rec, st);
}

template <int NWN>
static cudaError_t launch_u4_n(const PassArgs &A, const AcceptTable &T,
                               const TileGeom &G, unsigned long long *rec,
                               cudaStream_t st) {
  dim3 grid(G.gx, G.gy), block(kPassThreads);
  const size_t smem = (size_t)kPairBins * kBinStride * sizeof(uint32_t);
  if (T.rule_lt0)
    return A.colour ? launch_pdl(pass_u4_kernel<1, true, NWN>, grid, block,
                                 smem, st, A, T, G, rec)
                    : launch_pdl(pass_u4_kernel<0, true, NWN>, grid, block,
                                 smem, st, A, T, G, rec);
  return A.colour ? launch_pdl(pass_u4_kernel<1, false, NWN>, grid, block,
                               smem, st, A, T, G, rec)
                  : launch_pdl(pass_u4_kernel<0, false, NWN>, grid, block,
                               smem, st, A, T, G, rec);
}

static cudaError_t launch_u4(const PassArgs &A, const AcceptTable &T,
                             const TileGeom &G, unsigned long long *rec,
                             cudaStream_t st) {
  if (G.sites == 32) return launch_u4_n<4>(A, T, G, rec, st);
  return launch_u4_n<2>(A, T, G, rec, st);
}

cudaError_t launch_pass(const PassArgs &A, const AcceptTable &T,
                        const TileGeom &G, unsigned long long *rec,
                        cudaStream_t st) {
  if (!rec) return cudaErrorInvalidValue;
  if (A.layout == kLayoutU4) {
    if (A.q > 16 || !G.nibble || (G.sites == 32 && A.H % 32))
      return cudaErrorInvalidValue;
    return launch_u4(A, T, G, rec, st);
  }
  if (G.nibble || (G.sites == 32 && A.H % 32)) return cudaErrorInvalidValue;
  switch (qbits_for((int32_t)A.q)) {
    case 4: return launch_qb<4>(A, T, G, rec, st);
    case 5: return launch_qb<5>(A, T, G, rec, st);
    case 6: return launch_qb<6>(A, T, G, rec, st);
    case 7: return launch_qb<7>(A, T, G, rec, st);
    default: return launch_qb<8>(A, T, G, rec, st);
  }
}

int qbits_for(int32_t q) {
  if (q <= 16) return 4;
  if (q <= 32) return 5;
  if (q <= 64) return 6;
  if (q <= 128) return 7;
  return 8;
}

TileGeom choose_geom(int32_t L, int32_t H, int32_t q, int32_t sm_count,
                     int32_t tr_hint, int32_t chunk, int32_t minb) {
  TileGeom g;
  g.sites = chunk;
  g.nibble = 0;
  const int32_t nchunks = H / chunk;
  g.CX = std::min(nchunks, kPassThreads);
  g.RG = kPassThreads / g.CX;
  g.gx = (nchunks + g.CX - 1) / g.CX;
  const int64_t max_ctas = (int64_t)std::max(sm_count, 1) * minb;
  // Longest walk (<= 32 rows) that still gives every resident CTA about
  // four row tiles, so that the tiles balance across CTAs.
  int32_t tr = 1;
  if (tr_hint > 0) {
    tr = tr_hint;
  } else {
    while (tr < 32) {
      const int64_t ty = (L + (int64_t)g.RG * 2 * tr - 1) / ((int64_t)g.RG * 2 * tr);
      if (ty * g.gx < 4 * max_ctas) break;
      tr *= 2;
    }
    // at least two rows: a one-row walk loads three other-plane rows for one
    // row of work and misses the two-row unrolled loop (L = 4096: 34.9
    // against 39.1 us per sweep)
    tr = std::max(tr, 2);
  }
  // no longer than needed for the row groups of one tile to cover L
  g.TR = std::max(1, std::min(tr, (L + g.RG - 1) / g.RG));
  g.ty = (L + g.RG * g.TR - 1) / (g.RG * g.TR);
  if ((int64_t)g.ty * g.gx >= 2 * max_ctas) {
    // plenty of tiles (two waves or more): one tile per CTA, the hardware
    // balances the waves (L = 4096: 34.9 us per sweep against 37.8 with
    // persistent CTAs taking three tiles each)
    g.gy = g.ty;
  } else {
    // few tiles: persistent CTAs, balanced number of tiles each
    const int64_t gy_max = std::max<int64_t>(1, max_ctas / g.gx);
    const int64_t rounds = (g.ty + gy_max - 1) / gy_max;
    g.gy = (int32_t)((g.ty + rounds - 1) / rounds);
  }
  if (g.gy > 65535) {
    g.TR = std::min<int32_t>(L, g.TR * ((g.gy + 65534) / 65535) * 2);
    g.ty = (L + g.RG * g.TR - 1) / (g.RG * g.TR);
    g.gy = std::min(g.ty, 65535);
  }
  // Pair bins (256 x 32 counters to clear and fold per CTA) pay off only
  // when a CTA updates many sites.
  const int64_t sites_per_cta = (int64_t)L * H / ((int64_t)g.gx * g.gy);
  g.pairs = (q <= 16 && sites_per_cta >= 65536) ? 1 : 0;
  return g;
}

TileGeom pass_geom(int32_t nrows, int32_t H, int32_t q, int32_t layout,
                   int32_t update, int32_t sm_count) {
  if (update == POTTS_UPDATE_HEATBATH) {
    // q <= 16: the histogram in (black, white) pair bins, black pass only
    TileGeom g = choose_geom(nrows, H, q, sm_count, 0);
    if (q <= 16) g.pairs = 2;
    return g;
  }
  // 32 sites per thread only on planes of at least 2^23 sites (L >= 4096):
  // on smaller ones the 16-site walks' twice as many threads fill the GPU
  // better (L = 1024: 7.6 against 9.6 us per sweep; L = 2048: 11.3 against
  // 11.7; the same from L = 4096 up)
  const bool wide_ok = H % 32 == 0 && (int64_t)nrows * H >= (int64_t)1 << 23;
  if (layout == kLayoutU4) {
    // 32 sites (four nibble words, one 16-byte load) per thread and row
    // where the plane allows, else 16
    TileGeom g = wide_ok
                     ? choose_geom(nrows, H, q, sm_count, 0, 32, kMinb32)
                     : choose_geom(nrows, H, q, sm_count, 0, 16, kMinbNib);
    g.pairs = 1;
    g.nibble = 1;
    return g;
  }
  if (wide_ok && q <= 16) {
    // 32 sites per thread for the cheap q <= 16 rule (1.205 against 1.232
    // ps per update at L = 32768, q = 9; at q = 96 the longer rows are 0.7 %
    // slower); the histogram in (black, white) pair bins on the black pass
    // alone (pairs of one plane's neighbouring sites bought nothing here:
    // 1.2102 against 1.2076 ps with one state per bin)
    TileGeom g = choose_geom(nrows, H, q, sm_count, 0, 32, kMinb32);
    g.pairs = 2;
    return g;
  }
  return choose_geom(nrows, H, q, sm_count, 0);
}

// -------------------------------------------------------- random start
// One thread per 16 sites of a plane (site index = byte index for U8):
// s = floor(u q / 2^32), u = Philox word of domain 2 + colour at sweep 0.
// site0: index within the colour class of the plane's first site (0 for a
// whole lattice, r0 * L / 2 for a row strip starting at lattice row r0).
__global__ void init_random_kernel(uint8_t *plane, int64_t nchunks,
                                   uint32_t q, uint32_t domain, uint32_t key0,
                                   uint32_t key1, uint32_t layout,
                                   uint32_t ctr0) {
  const PhiloxKey ks = philox_schedule(key0, key1);
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nchunks;
       c += (int64_t)gridDim.x * blockDim.x) {
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint4 u =
          philox10(ctr0 + (uint32_t)(c * 4 + j), 0u, domain, 0u, ks);
      const uint32_t p0 = (uint32_t)(((uint64_t)u.x * q) >> 32);
      const uint32_t p1 = (uint32_t)(((uint64_t)u.y * q) >> 32);
      const uint32_t p2 = (uint32_t)(((uint64_t)u.z * q) >> 32);
      const uint32_t p3 = (uint32_t)(((uint64_t)u.w * q) >> 32);
      w[j] = pack4(p0, p1, p2, p3);
    }
    if (layout == kLayoutU4)
      reinterpret_cast<uint2 *>(plane)[c] =
          make_uint2(pack8(w[0], w[1]), pack8(w[2], w[3]));
    else
      reinterpret_cast<uint4 *>(plane)[c] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

cudaError_t launch_init_random(uint8_t *plane, int64_t plane_sites,
                               uint32_t q, uint32_t colour, uint64_t seed,
                               uint32_t layout, cudaStream_t st,
                               int64_t site0) {
  if (plane_sites % 16 || site0 % 16) return cudaErrorInvalidValue;
  const int64_t nchunks = plane_sites / 16;
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((nchunks + threads - 1) / threads,
                                           (int64_t)1 << 20);
  init_random_kernel<<<(unsigned)blocks, threads, 0, st>>>(
      plane, nchunks, q, 2u + colour, (uint32_t)seed, (uint32_t)(seed >> 32),
      layout, (uint32_t)(site0 >> 2));
  return cudaGetLastError();
}

// ------------------------------------------------------------ recount
// One thread per 16-byte chunk of a black row: satisfied bonds of the 16
// black sites with their four white neighbours, and the states of those
// black sites and of the white sites at the same (i, x).  Rows
// [row_lo, row_lo + nrows) of planes with Lp rows (periodic in Lp) whose
// row 0 is lattice row grow0.
template <int LAY>
__global__ void recount_kernel(const uint8_t *white, const uint8_t *black,
                               int32_t Lp, int32_t H, int32_t row_lo,
                               int32_t nrows, int32_t grow0, uint32_t q,
                               unsigned long long *rec) {
  using IO = Lay<LAY>;
  extern __shared__ __align__(16) uint32_t s_hist[];
  __shared__ uint32_t s_sat;
  const uint32_t tid = threadIdx.x;
  for (uint32_t v = tid; v < q * 32u; v += blockDim.x) s_hist[v] = 0;
  if (tid == 0) s_sat = 0;
  __syncthreads();
  const int64_t nch = (int64_t)nrows * (H / 16);
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + tid;
  const int32_t RB = IO::row_bytes(H);
  uint32_t sat = 0;
  if (c < nch) {
    const int32_t i = row_lo + (int32_t)(c / (H / 16));
    const int32_t x0 = (int32_t)(c % (H / 16)) * 16;
    const int32_t xb = LAY == kLayoutU4 ? x0 / 2 : x0;
    const int32_t im = i == 0 ? Lp - 1 : i - 1, ip = i + 1 == Lp ? 0 : i + 1;
    uint32_t Uw[4], Dw[4], Cw[4], Sw[4];
    IO::load(white + (int64_t)im * RB + xb, false, Uw);
    IO::load(white + (int64_t)ip * RB + xb, false, Dw);
    IO::load(white + (int64_t)i * RB + xb, false, Cw);
    IO::load(black + (int64_t)i * RB + xb, false, Sw);
    // black: x-1 when lattice row + 1 is even
    const bool left = ((i + grow0 + 1) & 1) == 0;
    const int32_t xe = left ? (x0 == 0 ? RB - 4 : xb - 4)
                            : (x0 + 16 == H ? 0 : xb + IO::kChunkBytes);
    const uint32_t ew = IO::edge(
        *reinterpret_cast<const uint32_t *>(white + (int64_t)i * RB + xe),
        left);
    uint32_t Wd[4];
    if (left) {
      Wd[0] = __funnelshift_l(ew, Cw[0], 8);
      for (int k = 1; k < 4; ++k) Wd[k] = __funnelshift_l(Cw[k - 1], Cw[k], 8);
    } else {
      for (int k = 0; k < 3; ++k) Wd[k] = __funnelshift_r(Cw[k], Cw[k + 1], 8);
      Wd[3] = __funnelshift_r(Cw[3], ew, 8);
    }
    uint32_t ne = 0;
    for (int k = 0; k < 4; ++k) {
      const uint32_t n16 = ne16_sum4<8>(Sw[k] ^ Uw[k], Sw[k] ^ Dw[k],
                                        Sw[k] ^ Cw[k], Sw[k] ^ Wd[k]);
      ne += ((n16 >> 4) * 0x01010101u) >> 24;
      hist_word<false, false>(s_hist + (tid & 31u), Sw[k]);
      hist_word<false, false>(s_hist + (tid & 31u), Cw[k]);
    }
    sat = 64u - ne;
  }
  for (int o = 16; o > 0; o >>= 1) sat += __shfl_xor_sync(0xFFFFFFFFu, sat, o);
  if ((tid & 31u) == 0 && sat) atomicAdd(&s_sat, sat);
  __syncthreads();
  if (tid == 0 && s_sat) atomicAdd(rec, (unsigned long long)s_sat);
  for (uint32_t v = tid; v < q; v += blockDim.x) {
    const uint32_t sum = bin_sum(s_hist, v);
    if (sum) atomicAdd(rec + 1 + v, (unsigned long long)sum);
  }
}

cudaError_t launch_recount(const uint8_t *white, const uint8_t *black,
                           int32_t L, int32_t H, uint32_t q, uint32_t layout,
                           unsigned long long *rec, cudaStream_t st) {
  return launch_recount_rows(white, black, L, H, 0, L, 0, q, layout, rec, st);
}

cudaError_t launch_recount_rows(const uint8_t *white, const uint8_t *black,
                                int32_t Lp, int32_t H, int32_t row_lo,
                                int32_t nrows, int32_t grow0, uint32_t q,
                                uint32_t layout, unsigned long long *rec,
                                cudaStream_t st) {
  const int64_t nch = (int64_t)nrows * (H / 16);
  const int threads = 256;
  const int64_t blocks = (nch + threads - 1) / threads;
  const size_t smem = (size_t)q * 32u * 4u;
  if (layout == kLayoutU4)
    recount_kernel<kLayoutU4><<<(unsigned)blocks, threads, smem, st>>>(
        white, black, Lp, H, row_lo, nrows, grow0, q, rec);
  else
    recount_kernel<kLayoutU8><<<(unsigned)blocks, threads, smem, st>>>(
        white, black, Lp, H, row_lo, nrows, grow0, q, rec);
  return cudaGetLastError();
}

}  // namespace potts
