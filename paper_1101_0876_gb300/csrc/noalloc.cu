// Sweep entry point that allocates no memory.
//
// Who needs it: callers that must not call cudaMalloc (or anything that
// does) at the point where they sweep: code running inside another
// framework whose caching allocator has already reserved the device memory
// for itself, or loops that cannot afford the implicit device-wide
// synchronisation an allocation may cause.  They own the two colour planes
// and the output buffer; the only extra memory this path needs is the
// per-sweep record accumulator, which here is a fixed file-scope device
// array instead of a cudaMalloc'd buffer.  The call synchronises its stream
// before it returns.
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
// One lock per device, held from the first launch of a call until its
// stream has synchronised: calls from several host threads on one device
// then run one after the other instead of racing on the shared array.
std::mutex g_call_mu[kMaxDevices];

// Device address of the accumulator on the current device, looked up once
// per device (the host-side symbol is only a stand-in for it).
int records_address(int dev, unsigned long long **out) {
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
  int dev = 0;
  POTTS_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices)
    return fail(POTTS_EINVAL, "device %d is beyond the %d supported", dev,
                kMaxDevices);
  unsigned long long *rec = nullptr;
  int rc = records_address(dev, &rec);
  if (rc) return rc;
  if (nsweeps == 0) return POTTS_OK;
  std::lock_guard<std::mutex> serialise(g_call_mu[dev]);

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const AcceptTable T = accept_table(thr);
  const int32_t H = L / 2;
  const TileGeom G = pass_geom(L, H, q, kLayoutU8, POTTS_UPDATE_METROPOLIS,
                               sm_count_of_current_device());
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
    A[c].grow0 = 0;
    A[c].row_lo = 0;
    A[c].row_end = L;
  }
  // the accumulator keeps the previous call's contents: clear what is used
  rc = [&]() -> int {
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
    return POTTS_OK;
  }();
  // also after a failed launch: whatever was queued finishes before the
  // lock lets another call touch the array
  const cudaError_t es = cudaStreamSynchronize(st);
  if (rc) return rc;
  if (es != cudaSuccess)
    return fail(POTTS_ECUDA, "cudaStreamSynchronize: %s",
                cudaGetErrorString(es));
  return POTTS_OK;
}
