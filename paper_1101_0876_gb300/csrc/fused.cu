// Fused two-colour sweep: one launch per sweep instead of two passes.
//
// A CTA stages a tile of both colour planes in shared memory: the black
// tile (rows r0-2 .. r0+R+1, chunks c0-2 .. c0+TW+1) and the white tile
// (rows r0-1 .. r0+R, chunks c0-1 .. c0+TW), periodic.  It first updates
// every white site of its white tile, including the one-row and one-chunk
// halo that the neighbouring tiles also update (the same sites with the same
// Philox words and the same pre-sweep black neighbours, so the redundant
// copies agree bit for bit), then the black sites of its R x TW interior
// against the new white sites, and writes both interiors to a second pair
// of planes (a CTA's halo is another CTA's interior, so the planes a sweep
// reads must stay unchanged until every CTA has loaded them; the caller
// swaps the two pairs after each sweep).  Each plane is read once per sweep
// (plus halos, which mostly hit L2) and written once: about 2 bytes per site
// per sweep instead of 3.  Results equal the two-pass path's bit for
// bit (same words, same rule, same order of dependence: every white site
// before any black site).  U8 layout, Metropolis rule, L a multiple of 1024
// (the tile is 32 chunks = 512 sites of a plane row wide and 32 rows high).
//
// Tiles move by the copy engine (TMA): one warp issues a 1-D bulk copy
// (cp.async.bulk) per tile row segment (a row splits into at most three
// where the tile's halo wraps around the plane's ends) that completes on a
// shared-memory mbarrier, and the interiors go back with bulk stores from
// shared memory.  Every wait on the mbarrier is bounded: a CTA that gives up
// flags the sweep's record (bit 63 of B, which no real count reaches) and
// returns, and the host turns the flag into POTTS_ETIMEOUT.
#include "internal.cuh"

namespace potts {

namespace {

constexpr int kFTW = 32;  // tile width, 16-byte chunks
constexpr int kFR = 32;   // tile height, rows
constexpr int kFThreads = 256;
constexpr int kWRows = kFR + 2, kWChunks = kFTW + 2, kWStride = kWChunks * 16;
constexpr int kBRows = kFR + 4, kBChunks = kFTW + 4, kBStride = kBChunks * 16;
constexpr int kWBytes = kWRows * kWStride;
constexpr int kBBytes = kBRows * kBStride;
constexpr int kFPairBins = 256;

__device__ __forceinline__ int32_t fwrap(int32_t a, int32_t n) {
  return a < 0 ? a + n : (a >= n ? a - n : a);
}

// ------------------------------------------------------------ TMA helpers
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar),
               "r"(count)
               : "memory");
  // make the initialised barrier visible to the copy engine
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile(
      "mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar),
      "r"(bytes)
      : "memory");
}
// Bulk copy of n bytes (multiple of 16, both addresses 16-byte aligned)
// from global memory into this CTA's shared memory, completing on mbar.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src,
                                          uint32_t n, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(n), "r"(mbar)
      : "memory");
}
// Bulk store of n bytes from shared to global memory (bulk-group tracked).
__device__ __forceinline__ void bulk_store(void *dst, uint32_t src,
                                           uint32_t n) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::
                   "l"(dst),
               "r"(src), "r"(n)
               : "memory");
}
// Waits for phase `parity` of mbar; gives up after `tries` polls (each
// poll itself suspends for a bounded time).  Returns whether it completed.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity,
                                          uint32_t tries) {
  for (uint32_t i = 0; i < tries; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
constexpr uint32_t kWaitTries = 1u << 20;
constexpr unsigned long long kTimeoutFlag = 1ull << 63;

// Copies `rows` tile rows (halo `h` chunks on each side, tile width kFTW
// chunks) of a plane into shared memory at `dst` (row stride `stride`):
// lane `lane` of the issuing warp takes rows lane, lane + 32, ...; each row
// is one to three contiguous segments (the halo wraps around the plane's
// row ends).
__device__ __forceinline__ void stage_rows(uint32_t dst, int32_t stride,
                                           const uint8_t *plane, int32_t H,
                                           int32_t L, int32_t row_first,
                                           int32_t rows, int32_t c0, int32_t h,
                                           uint32_t lane, uint32_t mbar) {
  const int32_t nch = H / 16, width = kFTW + 2 * h;
  for (int32_t rr = (int32_t)lane; rr < rows; rr += 32) {
    const uint8_t *grow = plane + (int64_t)fwrap(row_first + rr, L) * H;
    int32_t start = c0 - h, done = 0;
    while (done < width) {
      const int32_t gc = start < 0 ? start + nch : (start >= nch ? start - nch
                                                                 : start);
      const int32_t len = min(width - done, nch - gc);
      bulk_load(dst + (uint32_t)(rr * stride + done * 16), grow + gc * 16,
                (uint32_t)(len * 16), mbar);
      done += len;
      start += len;
    }
  }
}

__device__ __forceinline__ void lds4(const uint8_t *p, uint32_t w[4]) {
  const uint4 v = *reinterpret_cast<const uint4 *>(p);
  w[0] = v.x;
  w[1] = v.y;
  w[2] = v.z;
  w[3] = v.w;
}

// New values of one 16-site chunk: own words S, other-plane rows U (i-1),
// C (i), D (i+1), the word holding the side site (top byte x-1 when left,
// else low byte x+16), Philox counter g0 of its first four sites.
template <int QB, bool COUNTS, bool LT0>
__device__ __forceinline__ void fused_chunk(
    const uint32_t S[4], const uint32_t U[4], const uint32_t C[4],
    const uint32_t D[4], uint32_t side, bool left, uint32_t g0,
    uint32_t colour, uint32_t t_lo, uint32_t t_hi, uint32_t q, uint32_t one,
    const PhiloxKey &ks, const uint8_t *tab, uint32_t N[4],
    uint32_t &ne_acc) {
  uint32_t Wd[4];
  if (left) {
    Wd[0] = __funnelshift_l(side, C[0], 8);
    Wd[1] = __funnelshift_l(C[0], C[1], 8);
    Wd[2] = __funnelshift_l(C[1], C[2], 8);
    Wd[3] = __funnelshift_l(C[2], C[3], 8);
  } else {
    Wd[0] = __funnelshift_r(C[0], C[1], 8);
    Wd[1] = __funnelshift_r(C[1], C[2], 8);
    Wd[2] = __funnelshift_r(C[2], C[3], 8);
    Wd[3] = __funnelshift_r(C[3], side, 8);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint4 u = philox10(g0 + (uint32_t)k, t_lo, colour, t_hi, ks);
    const uint64_t r0 = (uint64_t)u.x * q, r1 = (uint64_t)u.y * q;
    const uint64_t r2 = (uint64_t)u.z * q, r3 = (uint64_t)u.w * q;
    const uint32_t P = pack4((uint32_t)(r0 >> 32), (uint32_t)(r1 >> 32),
                             (uint32_t)(r2 >> 32), (uint32_t)(r3 >> 32));
    uint32_t no16 = 0, nn16 = 0;
    const uint32_t idx = delta_index<QB, COUNTS>(S[k], P, U[k], D[k], C[k],
                                                 Wd[k], &no16, &nn16, one);
    const uint32_t m = accept_mask<LT0>(idx, (uint32_t)r0, (uint32_t)r1,
                                        (uint32_t)r2, (uint32_t)r3, tab);
    N[k] = (P & m) | (S[k] & ~m);
    if (COUNTS) {
      const uint32_t nf16 = (nn16 & m) | (no16 & ~m);
      ne_acc += __umulhi(nf16, 1u << 28);
    }
  }
}

template <int QB, bool PAIRS, bool LT0>
__global__ void __launch_bounds__(kFThreads, 3)
    fused_sweep_kernel(const uint8_t *white, const uint8_t *black,
                       uint8_t *white_out, uint8_t *black_out, int32_t L,
                       int32_t H,
                       uint32_t q, uint32_t t_lo, uint32_t t_hi, uint32_t key0,
                       uint32_t key1, uint32_t one, AcceptTable Tin,
                       unsigned long long *rec) {
  extern __shared__ __align__(16) uint8_t f_smem[];
  uint8_t *sw = f_smem;
  uint8_t *sb = f_smem + kWBytes;
  uint32_t *s_hist = reinterpret_cast<uint32_t *>(f_smem + kWBytes + kBBytes);
  __shared__ __align__(16) uint32_t s_tab[kTabWords];
  __shared__ uint32_t s_sat;
  __shared__ uint32_t s_fold[16];
  const uint32_t tid = threadIdx.x;
  const uint32_t bins = PAIRS ? (uint32_t)kFPairBins : q;
  for (uint32_t i = tid; i < (uint32_t)kTabWords; i += kFThreads)
    s_tab[i] = (i % 4u == 0 && i / 4u < 9u) ? Tin.tab[i / 4u] : 0u;
  for (uint32_t v = tid; v < bins * 32u; v += kFThreads) s_hist[v] = 0;
  if (tid < 16) s_fold[tid] = 0;
  if (tid == 0) s_sat = 0;
  __shared__ __align__(8) unsigned long long s_mbar;
  const uint32_t mbar = smem_addr(&s_mbar);
  if (tid == 0) mbar_init(mbar, 1);
  __syncthreads();
  pdl_wait_previous();  // the planes are the previous sweep's output

  const int32_t nch = H / 16;
  const int32_t c0 = (int32_t)blockIdx.x * kFTW;
  const int32_t r0 = (int32_t)blockIdx.y * kFR;
  if (tid < 32) {
    // the whole tile pair: expected bytes first, then the copies
    if (tid == 0) mbar_expect_tx(mbar, (uint32_t)(kBBytes + kWBytes));
    __syncwarp();
    stage_rows(smem_addr(sb), kBStride, black, H, L, r0 - 2, kBRows, c0, 2,
               tid, mbar);
    stage_rows(smem_addr(sw), kWStride, white, H, L, r0 - 1, kWRows, c0, 1,
               tid, mbar);
  }
  // every thread polls; the CTA gives up as a whole if any of them did
  const bool landed = mbar_wait(mbar, 0, kWaitTries);
  if (__syncthreads_or(!landed)) {
    if (tid == 0) atomicOr(rec, kTimeoutFlag);
    if (!landed) mbar_wait(mbar, 0, kWaitTries);  // copies in flight land
    return;
  }
  (void)nch;

  const PhiloxKey ks = philox_schedule(key0, key1);
  const uint8_t *tab = reinterpret_cast<const uint8_t *>(s_tab);
  uint32_t *lh = s_hist + (tid & 31u);
  // white: every site of the white tile (halo included)
  for (int32_t it = (int32_t)tid; it < kWRows * kWChunks; it += kFThreads) {
    const int32_t rr = it / kWChunks, cc = it - rr * kWChunks;
    const int32_t gi = fwrap(r0 - 1 + rr, L), gc = fwrap(c0 - 1 + cc, nch);
    uint8_t *own = sw + rr * kWStride + cc * 16;
    const uint8_t *bc = sb + (rr + 1) * kBStride + (cc + 1) * 16;
    uint32_t S[4], U[4], C[4], D[4], N[4];
    lds4(own, S);
    lds4(bc - kBStride, U);
    lds4(bc, C);
    lds4(bc + kBStride, D);
    const bool left = (gi & 1) == 0;
    const uint32_t side = left ? *reinterpret_cast<const uint32_t *>(bc - 4)
                               : *reinterpret_cast<const uint32_t *>(bc + 16);
    uint32_t ne_unused = 0;
    fused_chunk<QB, false, LT0>(S, U, C, D, side, left,
                                (uint32_t)(((int64_t)gi * H + gc * 16) >> 2),
                                0u, t_lo, t_hi, q, one, ks, tab, N, ne_unused);
    *reinterpret_cast<uint4 *>(own) = make_uint4(N[0], N[1], N[2], N[3]);
    if (rr >= 1 && rr <= kFR && cc >= 1 && cc <= kFTW) {
#pragma unroll
      for (int k = 0; k < 4; ++k) hist_word<PAIRS, false>(lh, N[k]);
    }
  }
  __syncthreads();
  // black: the interior, against the new white sites
  uint32_t ne = 0, items = 0;
  for (int32_t it = (int32_t)tid; it < kFR * kFTW; it += kFThreads) {
    const int32_t rr = it / kFTW, cc = it - rr * kFTW;
    const int32_t gi = r0 + rr, gc = c0 + cc;
    uint8_t *own = sb + (rr + 2) * kBStride + (cc + 2) * 16;
    const uint8_t *wc = sw + (rr + 1) * kWStride + (cc + 1) * 16;
    uint32_t S[4], U[4], C[4], D[4], N[4];
    lds4(own, S);
    lds4(wc - kWStride, U);
    lds4(wc, C);
    lds4(wc + kWStride, D);
    const bool left = ((gi + 1) & 1) == 0;
    const uint32_t side = left ? *reinterpret_cast<const uint32_t *>(wc - 4)
                               : *reinterpret_cast<const uint32_t *>(wc + 16);
    uint32_t ne_acc = 0;
    fused_chunk<QB, true, LT0>(S, U, C, D, side, left,
                               (uint32_t)(((int64_t)gi * H + gc * 16) >> 2),
                               1u, t_lo, t_hi, q, one, ks, tab, N, ne_acc);
    ne += (ne_acc * 0x01010101u) >> 24;
    items += 1;
    *reinterpret_cast<uint4 *>(own) = make_uint4(N[0], N[1], N[2], N[3]);
#pragma unroll
    for (int k = 0; k < 4; ++k) hist_word<PAIRS, false>(lh, N[k]);
  }
  pdl_release_next();
  // the threads' shared-memory writes, visible to the copy engine
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  // both interiors to the output planes: one bulk store per tile row and
  // plane from shared memory (each interior row is contiguous on both sides)
  if (tid < 32) {
    for (int32_t rr = (int32_t)tid; rr < kFR; rr += 32) {
      const int64_t g = (int64_t)(r0 + rr) * H + c0 * 16;
      bulk_store(white_out + g, smem_addr(sw + (rr + 1) * kWStride + 16),
                 kFTW * 16);
      bulk_store(black_out + g, smem_addr(sb + (rr + 2) * kBStride + 32),
                 kFTW * 16);
    }
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  }
  // B of the black interior (each bond has one black end), then the counts
  uint32_t sat = 64u * items - ne;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sat += __shfl_xor_sync(0xFFFFFFFFu, sat, o);
  if ((tid & 31u) == 0 && sat) atomicAdd(&s_sat, sat);
  __syncthreads();
  if (tid == 0 && s_sat) atomicAdd(rec, (unsigned long long)s_sat);
  if (PAIRS) {
    for (uint32_t p = tid; p < (uint32_t)kFPairBins; p += kFThreads) {
      const uint32_t sum = bin_sum(s_hist, p);
      if (sum) {
        atomicAdd(&s_fold[p & 15u], sum);
        atomicAdd(&s_fold[p >> 4], sum);
      }
    }
    __syncthreads();
    if (tid < q && s_fold[tid])
      atomicAdd(rec + 1 + tid, (unsigned long long)s_fold[tid]);
  } else {
    for (uint32_t v = tid; v < q; v += kFThreads) {
      const uint32_t sum = bin_sum(s_hist, v);
      if (sum) atomicAdd(rec + 1 + v, (unsigned long long)sum);
    }
  }
  // the tiles must stay until the bulk stores have read them
  if (tid < 32) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// Largest dynamic shared memory of any launch: both tiles and 256 x 32
// histogram counters.
constexpr int kFSmemMax = kWBytes + kBBytes + kFPairBins * 32 * 4;

template <int QB, bool PAIRS, bool LT0>
cudaError_t launch_fused_k(const uint8_t *white, const uint8_t *black,
                           uint8_t *white_out, uint8_t *black_out, int32_t L,
                           int32_t H, uint32_t q, uint64_t t, uint64_t seed,
                           const AcceptTable &T, unsigned long long *rec,
                           cudaStream_t st) {
  static_assert(kFSmemMax <= kDynSmemCap, "launch_pdl's opt-in cap");
  const dim3 grid((unsigned)(H / 16 / kFTW), (unsigned)(L / kFR));
  const size_t smem = (size_t)kWBytes + kBBytes +
                      (size_t)(PAIRS ? kFPairBins : q) * 32u * 4u;
  return launch_pdl(fused_sweep_kernel<QB, PAIRS, LT0>, grid, dim3(kFThreads),
                    smem, st, white, black, white_out, black_out, L, H, q,
                    (uint32_t)t, (uint32_t)(t >> 32), (uint32_t)seed,
                    (uint32_t)(seed >> 32), 1u, T, rec);
}

template <int QB, bool PAIRS>
cudaError_t launch_fused_qb(const uint8_t *white, const uint8_t *black,
                            uint8_t *white_out, uint8_t *black_out, int32_t L,
                            int32_t H, uint32_t q, uint64_t t, uint64_t seed,
                            const AcceptTable &T, unsigned long long *rec,
                            cudaStream_t st) {
  if (T.rule_lt0)
    return launch_fused_k<QB, PAIRS, true>(white, black, white_out, black_out,
                                           L, H, q, t, seed, T, rec, st);
  return launch_fused_k<QB, PAIRS, false>(white, black, white_out, black_out,
                                          L, H, q, t, seed, T, rec, st);
}

}  // namespace

bool fused_supported(int32_t L, int32_t q, int32_t layout) {
  return layout == kLayoutU8 && L % (kFTW * 32) == 0 && L >= kFR && q <= 256;
}

cudaError_t launch_fused_sweep(const uint8_t *white, const uint8_t *black,
                               uint8_t *white_out, uint8_t *black_out,
                               int32_t L, uint32_t q, uint64_t t,
                               uint64_t seed, const AcceptTable &T,
                               unsigned long long *rec, cudaStream_t st) {
  if (!fused_supported(L, (int32_t)q, kLayoutU8) || rec == nullptr)
    return cudaErrorInvalidValue;
  const int32_t H = L / 2;
  switch (qbits_for((int32_t)q)) {
    case 4:
      return launch_fused_qb<4, true>(white, black, white_out, black_out, L, H,
                                      q, t, seed, T, rec, st);
    case 5:
      return launch_fused_qb<5, false>(white, black, white_out, black_out, L,
                                       H, q, t, seed, T, rec, st);
    default:
      return launch_fused_qb<8, false>(white, black, white_out, black_out, L,
                                       H, q, t, seed, T, rec, st);
  }
}

}  // namespace potts
