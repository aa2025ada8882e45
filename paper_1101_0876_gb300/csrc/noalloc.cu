// Sweep entry point that allocates no memory.
//
// Who needs it: callers that cannot call cudaMalloc (or anything that does)
// at the point where they want to sweep, for example code that runs while a
// CUDA graph is being captured (allocation is not allowed there), code that
// runs inside another framework whose caching allocator already reserved
// the device memory, or real-time loops where an allocation's implicit
// device synchronisation would stall other work.  They own the two colour
// planes and the output buffer; the only extra memory this path needs is
// the per-sweep record accumulator, which here is a fixed file-scope device
// array instead of a cudaMalloc'd buffer.
#include <mutex>

#include "internal.cuh"

namespace {

// Record accumulator shared by every call on a device: room for
// kNoAllocRecordWords uint64 words, i.e. nsweeps * (1 + q) <= 8192 per
// call.  Every device that loads the library holds these 64 KiB until the
// process exits.
constexpr size_t kNoAllocRecordWords = 8192;
__device__ __align__(256) unsigned long long g_noalloc_records[kNoAllocRecordWords];

constexpr int kMaxDevices = 64;
unsigned long long *g_records_addr[kMaxDevices] = {};
std::mutex g_setup_mu;

// Device address of the accumulator on the current device, looked up once
// per device (the host-side symbol is only a stand-in for it).
int records_address(unsigned long long **out) {
  int dev = 0;
  POTTS_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices)
    return potts::fail(POTTS_EINVAL, "device %d is beyond the %d supported",
                       dev, kMaxDevices);
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_records_addr[dev]) {
    void *p = nullptr;
    POTTS_CK(cudaGetSymbolAddress(&p, g_noalloc_records));
    g_records_addr[dev] = static_cast<unsigned long long *>(p);
  }
  *out = g_records_addr[dev];
  return POTTS_OK;
}

}  // namespace

using namespace potts;

extern "C" int potts_sweep_planes_noalloc(void *white, void *black, int32_t L,
                                          int32_t q, uint64_t seed,
                                          uint64_t sweep, double beta,
                                          int64_t nsweeps,
                                          uint64_t *out_counts,
                                          void *stream) {
  if (!white || !black) return fail(POTTS_EINVAL, "plane pointer is NULL");
  if (((uintptr_t)white | (uintptr_t)black) & 15u)
    return fail(POTTS_EINVAL, "planes must be 16-byte aligned");
  if (L < 32 || L > 65536 || L % 32 != 0)
    return fail(POTTS_EINVAL, "L must be a multiple of 32 in [32, 65536] (got %d)", L);
  if (q < 2 || q > 256) return fail(POTTS_EINVAL, "q must be in [2, 256] (got %d)", q);
  if (nsweeps < 0) return fail(POTTS_EINVAL, "nsweeps < 0");
  const int64_t words = nsweeps * (int64_t)(1 + q);
  if (words > (int64_t)kNoAllocRecordWords)
    return fail(POTTS_EINVAL,
                "nsweeps * (1 + q) = %lld exceeds the fixed record buffer of "
                "%zu words; split the call",
                (long long)words, kNoAllocRecordWords);
  uint64_t thr[5];
  if (!threshold_table(beta, thr))
    return fail(POTTS_EINVAL, "beta must be finite and >= 0 (got %g)", beta);
  unsigned long long *rec = nullptr;
  int rc = records_address(&rec);
  if (rc) return rc;
  if (nsweeps == 0) return POTTS_OK;

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const AcceptTable T = accept_table(thr);
  const int32_t H = L / 2;
  const TileGeom G = choose_geom(L, H, q, sm_count_of_current_device(), 0);
  PassArgs A[2];
  uint8_t *planes[2] = {static_cast<uint8_t *>(white),
                        static_cast<uint8_t *>(black)};
  for (int c = 0; c < 2; ++c) {
    A[c].own = planes[c];
    A[c].other = planes[c ^ 1];
    A[c].L = L;
    A[c].H = H;
    A[c].q = (uint32_t)q;
    A[c].colour = (uint32_t)c;
    A[c].key0 = (uint32_t)seed;
    A[c].key1 = (uint32_t)(seed >> 32);
    // the planes are the caller's and unchecked: a byte >= q must not
    // index outside the shared histogram
    A[c].one = 1u;
    A[c].hist_bins = 256u;
    A[c].layout = kLayoutU8;
  }
  // the accumulator keeps the previous call's contents: clear what is used
  POTTS_CK(cudaMemsetAsync(rec, 0, (size_t)words * 8, st));
  for (int64_t s = 0; s < nsweeps; ++s) {
    const uint64_t t = sweep + (uint64_t)s;
    for (int c = 0; c < 2; ++c) {
      A[c].t_lo = (uint32_t)t;
      A[c].t_hi = (uint32_t)(t >> 32);
      POTTS_CK(launch_pass(A[c], T, G, rec + s * (1 + q), st));
    }
  }
  if (out_counts)
    POTTS_CK(cudaMemcpyAsync(out_counts, rec, (size_t)words * 8,
                             cudaMemcpyDefault, st));
  POTTS_CK(cudaStreamSynchronize(st));
  return POTTS_OK;
}
