// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <string>
#include <utility>

#include "../../include/potts.h"
#include "pass_u8.cuh"

namespace potts {

// ------------------------------------------------------------- errors
int fail(int code, const char *fmt, ...);
void clear_error();

#define POTTS_CK(call)                                                     \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess)                                                 \
      return ::potts::fail(POTTS_ECUDA, "%s failed: %s (%s:%d)", #call,    \
                           cudaGetErrorString(e_), __FILE__, __LINE__);    \
  } while (0)

// Makes a handle's device current for the scope of an entry point and
// restores the caller's device afterwards (a process may hold handles on
// several devices).
class DeviceScope {
 public:
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev_) == cudaSuccess && prev_ != dev &&
        cudaSetDevice(dev) == cudaSuccess)
      return;
    prev_ = -1;
  }
  ~DeviceScope() {
    if (prev_ >= 0) cudaSetDevice(prev_);
  }
  DeviceScope(const DeviceScope &) = delete;
  DeviceScope &operator=(const DeviceScope &) = delete;

 private:
  int prev_ = -1;
};

// ---------------------------------------------------------- geometry
// CTA work shape of a colour pass.  A row tile is CX 16-byte chunks wide
// and RG row groups of TR rows high (128 threads: thread t takes chunk t%CX
// and row group t/CX, walking TR rows).  gx CTA columns cover the row; gy
// CTA rows are launched and loop over the ty row tiles (persistent CTAs, so
// per-CTA set-up such as zeroing the histogram is paid once per CTA).
struct TileGeom {
  int32_t CX, RG, TR;
  int32_t gx, gy, ty;
  int32_t pairs;  // q <= 16: 1, bins of (state, state) pairs of one plane;
                  // 2 (32-site U8 pass), (black, white) pairs of the two
                  // planes kept by the black pass alone; 0: one state a bin
  int32_t sites;  // sites per thread and row: 16, or 32 (U8 Metropolis)
  int32_t nibble; // 1: the U4 Metropolis pass on nibbles (pass_u4.cuh)
};
constexpr int kPassThreads = 128;

// Minimum resident CTAs per SM requested from the compiler for the pass
// kernels (caps registers at 65536 / (128 * POTTS_PASS_MINB) per thread).
#ifndef POTTS_PASS_MINB
#define POTTS_PASS_MINB 6
#endif

// L: rows to cover; chunk: sites per thread and row (16 or 32); minb: the
// kernel's resident CTAs per SM.
TileGeom choose_geom(int32_t L, int32_t H, int32_t q, int32_t sm_count,
                     int32_t tr_hint, int32_t chunk = 16,
                     int32_t minb = POTTS_PASS_MINB);
// The shape of the colour pass launch_pass / launch_pass_hb will run for
// nrows rows of width H: the U4 Metropolis pass on nibbles, the U8
// Metropolis pass with 32 sites per thread where H allows, else 16.
TileGeom pass_geom(int32_t nrows, int32_t H, int32_t q, int32_t layout,
                   int32_t update, int32_t sm_count);

// Programmatic dependent launch.  A colour pass is launched so that it may
// start while the previous kernel on its stream finishes: its CTAs clear
// their shared counters and load their tables, then wait for the previous
// kernel to complete (and its writes to be visible) before touching the
// lattice; each pass lets the next one start once its own walks are done,
// so the next pass's launch and set-up overlap this pass's reduction tail.
// Both calls are no-ops when a kernel was launched without the attribute.
__device__ __forceinline__ void pdl_wait_previous() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void pdl_release_next() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Opts `kernel` in to dynamic shared memory above the 48 KB that need no
// opt-in, up to kDynSmemCap (the largest any kernel here asks for: the fused
// sweep's tiles and pair bins), in the current context; launch_pdl calls it
// before each launch of more than 48 KB.  smem above the cap: invalid value.
constexpr int kDynSmemCap = 72 * 1024;
cudaError_t allow_dynamic_smem(const void *kernel, size_t smem);

// Launches kernel<<<grid, block, smem, st>>>(args...) with the programmatic
// stream serialization attribute.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block,
                       size_t smem, cudaStream_t st, Args &&...args) {
  if (smem > 48u * 1024u) {
    const cudaError_t e =
        allow_dynamic_smem(reinterpret_cast<const void *>(kernel), smem);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Spin-width class: every spin < 2^qbits.
int qbits_for(int32_t q);

// Threshold table from beta (host FP64, glibc exp):
// thr[d] = floor(2^32 exp(-beta d)), thr[0] = 2^32.
bool threshold_table(double beta, uint64_t thr[5]);
AcceptTable accept_table(const uint64_t thr[5]);

// Heat-bath weights (host FP64, glibc exp): W[n] = round(2^m exp(beta n)),
// n = 0..4, m the largest in 0..31 keeping every normaliser below 2^32.
struct HeatTable;
bool heatbath_table(double beta, int32_t q, uint64_t W[5], int32_t *m);
HeatTable heat_table(const uint64_t W[5], int32_t m);

// ----------------------------------------------------------- launches
// One colour pass of one lattice.  rec (not null) receives, added
// atomically, histogram counts and, on the black pass, B; the record
// {B, hist[q]} of a sweep must start at zero and is complete after the
// black pass.  Each pass counts its updated sites, except with G.pairs == 2,
// where the black pass counts the sites of both planes and the white pass
// none.
cudaError_t launch_pass(const PassArgs &A, const AcceptTable &T,
                        const TileGeom &G, unsigned long long *rec,
                        cudaStream_t st);
// The same colour pass with the heat-bath rule (heatbath.cuh).
cudaError_t launch_pass_hb(const PassArgs &A, const HeatTable &T,
                           const TileGeom &G, unsigned long long *rec,
                           cudaStream_t st);
// Random start of one plane of plane_sites sites: s = floor(u q / 2^32),
// u = Philox word of domain 2 + colour at sweep 0.  site0: colour-class
// index of the plane's first site (a multiple of 16; 0 for a whole
// lattice).
cudaError_t launch_init_random(uint8_t *plane, int64_t plane_sites,
                               uint32_t q, uint32_t colour, uint64_t seed,
                               uint32_t layout, cudaStream_t st,
                               int64_t site0 = 0);
// Recount {B, hist} from the planes into rec (must start at zero).
cudaError_t launch_recount(const uint8_t *white, const uint8_t *black,
                           int32_t L, int32_t H, uint32_t q, uint32_t layout,
                           unsigned long long *rec, cudaStream_t st);
// The same over rows [row_lo, row_lo + nrows) of planes of Lp rows (row
// indices periodic in Lp) whose row 0 is lattice row grow0: the bonds of
// those rows' black sites and the states of their sites.
cudaError_t launch_recount_rows(const uint8_t *white, const uint8_t *black,
                                int32_t Lp, int32_t H, int32_t row_lo,
                                int32_t nrows, int32_t grow0, uint32_t q,
                                uint32_t layout, unsigned long long *rec,
                                cudaStream_t st);

// Both colour passes of one Metropolis sweep in one launch (fused.cu):
// U8 layout, L a multiple of 1024.  Reads the planes (white, black), writes
// the swept planes to (white_out, black_out), which must not overlap them;
// rec (not null, starting at zero) receives the sweep's record {B, hist}.
bool fused_supported(int32_t L, int32_t q, int32_t layout);
cudaError_t launch_fused_sweep(const uint8_t *white, const uint8_t *black,
                               uint8_t *white_out, uint8_t *black_out,
                               int32_t L, uint32_t q, uint64_t t,
                               uint64_t seed, const AcceptTable &T,
                               unsigned long long *rec, cudaStream_t st);

int sm_count_of_current_device();

// FP64 observables of one record.
void update_obs(potts_obs *obs, const uint64_t *rec, int32_t L, int32_t q,
                bool accumulate);

// Spins between the caller's row-major L x L host bytes and the colour
// planes (layout.cu), through a device staging buffer and conversion
// kernels on stream st; both synchronise st.  upload_rowmajor writes the
// planes only if every spin is < q (else POTTS_EINVAL).  Return POTTS_*.
// nrows: rows of the block (L for a whole lattice; a row strip's own rows,
// starting at an even lattice row, with white/black at its first row).
int download_rowmajor(const uint8_t *white, const uint8_t *black, int32_t L,
                      int32_t nrows, uint32_t layout, uint8_t *out_LxL,
                      cudaStream_t st);
int upload_rowmajor(const uint8_t *in_LxL, int32_t L, int32_t nrows,
                    uint32_t q, uint32_t layout, uint8_t *white,
                    uint8_t *black, cudaStream_t st);

}  // namespace potts
