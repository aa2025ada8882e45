// Independent Philox4x32-10 for pinning the oracle on the CPU: PyTorch's
// header-only engine (ATen/core/PhiloxRNGEngine.h).  Its counter is
// (offset lo, offset hi, subsequence lo, subsequence hi) and its key is the
// 64-bit seed, so any counter and key can be reached.  Test code only.
#include <ATen/core/PhiloxRNGEngine.h>

#include <cstdint>

extern "C" void ref_philox(const uint32_t *ctr, const uint32_t *key,
                           uint32_t *out, int64_t n) {
  for (int64_t t = 0; t < n; ++t) {
    const uint32_t *c = ctr + 4 * t;
    const uint32_t *k = key + 2 * t;
    uint64_t seed = (uint64_t)k[0] | ((uint64_t)k[1] << 32);
    uint64_t sub = (uint64_t)c[2] | ((uint64_t)c[3] << 32);
    uint64_t off = (uint64_t)c[0] | ((uint64_t)c[1] << 32);
    at::Philox4_32 eng(seed, sub, off);
    for (int i = 0; i < 4; ++i) out[4 * t + i] = eng();
  }
}
