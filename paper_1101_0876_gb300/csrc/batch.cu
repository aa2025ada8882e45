// Batched and served paths (interim: entry points present, not available).
#include "internal.cuh"

using namespace potts;

extern "C" {
int potts_batch_create(int32_t, const int32_t *, const int32_t *,
                       const int32_t *, const uint64_t *, potts_batch_h *out) {
  if (out) *out = nullptr;
  return fail(POTTS_EINVAL, "batched path not available in this build");
}
int potts_batch_sweep(potts_batch_h, const double *, int64_t,
                      uint64_t *const *) {
  return fail(POTTS_EINVAL, "batched path not available in this build");
}
int potts_batch_get_spins(potts_batch_h, int32_t, uint8_t *) {
  return fail(POTTS_EINVAL, "batched path not available in this build");
}
int potts_batch_observables(potts_batch_h, int32_t, potts_obs *) {
  return fail(POTTS_EINVAL, "batched path not available in this build");
}
int potts_batch_destroy(potts_batch_h) {
  return fail(POTTS_EINVAL, "batched path not available in this build");
}
int potts_serve_start(const potts_serve_cfg *, potts_server_h *out) {
  if (out) *out = nullptr;
  return fail(POTTS_EINVAL, "serving path not available in this build");
}
int potts_serve_submit(potts_server_h, const potts_req *, uint64_t *) {
  return fail(POTTS_EINVAL, "serving path not available in this build");
}
int potts_serve_poll(potts_server_h, uint64_t, uint64_t *, int64_t,
                     int64_t *, int *) {
  return fail(POTTS_EINVAL, "serving path not available in this build");
}
int potts_serve_cancel(potts_server_h, uint64_t) {
  return fail(POTTS_EINVAL, "serving path not available in this build");
}
int potts_serve_stats_get(potts_server_h, potts_serve_stats *) {
  return fail(POTTS_EINVAL, "serving path not available in this build");
}
int potts_serve_stop(potts_server_h) {
  return fail(POTTS_EINVAL, "serving path not available in this build");
}
}
