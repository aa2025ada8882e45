// C ABI of the single-lattice path: create / sweep / observables / state.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "heatbath.cuh"
#include "lattice.cuh"

namespace potts {

// ---------------------------------------------------------------- errors
static thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}
void clear_error() { g_err.clear(); }

int sm_count_of_current_device() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
      cudaSuccess)
    return 1;
  return n;
}

// ------------------------------------------------------- threshold table
// Sec. 5 (CPU code): a table of Boltzmann weights per temperature.  Here the
// weight exp(-beta d) of an energy increase d = 1..4 becomes the 32-bit
// fixed-point threshold floor(2^32 exp(-beta d)), computed on the host in
// FP64 with the C library's exp.
bool threshold_table(double beta, uint64_t thr[5]) {
  if (!(beta >= 0.0) || !std::isfinite(beta)) return false;
  thr[0] = (uint64_t)1 << 32;
  for (int d = 1; d <= 4; ++d) {
    const double w = std::exp(-beta * (double)d);
    thr[d] = (uint64_t)std::floor(std::ldexp(w, 32));
  }
  return true;
}

AcceptTable accept_table(const uint64_t thr[5]) {
  AcceptTable T;
  bool any_zero = false;
  for (int d = 1; d <= 4; ++d) any_zero |= thr[d] == 0;
  T.rule_lt0 = any_zero ? 1u : 0u;
  for (int i = 0; i < 9; ++i) {
    const int dE = i - 4;
    if (any_zero) {
      // accept iff dE <= 0 or a < thr[dE]
      T.tab[i] = dE <= 0 ? 0xFFFFFFFFu
                         : (uint32_t)std::min<uint64_t>(thr[dE], 0xFFFFFFFFu);
    } else {
      // accept iff a <= thr[dE] - 1  (thr[dE] in [1, 2^32])
      T.tab[i] = dE <= 0 ? 0xFFFFFFFFu : (uint32_t)(thr[dE] - 1);
    }
  }
  return T;
}

// ---------------------------------------------------------- observables
void update_obs(potts_obs *obs, const uint64_t *rec, int32_t L, int32_t q,
                bool accumulate) {
  const double N = (double)L * (double)L;
  uint64_t nmax = 0;
  for (int v = 0; v < q; ++v) nmax = std::max(nmax, rec[1 + v]);
  obs->bonds = rec[0];
  obs->nmax = nmax;
  obs->e = -(double)rec[0] / N;
  obs->m = ((double)q * (double)nmax / N - 1.0) / ((double)q - 1.0);
  if (accumulate) {
    const double e = obs->e, m = obs->m, e2 = e * e;
    obs->nsamples += 1;
    obs->sum_e += e;
    obs->sum_e2 += e2;
    obs->sum_e4 += e2 * e2;
    obs->sum_m += m;
    obs->sum_m2 += m * m;
  }
}

}  // namespace potts

using namespace potts;

namespace potts {

int recount_into_obs(potts_h h) {
  const int32_t q = h->q;
  POTTS_CK(cudaMemsetAsync(h->d_rec, 0, (size_t)(1 + q) * 8, h->stream));
  POTTS_CK(launch_recount(h->d_planes, h->d_planes + h->plane_bytes, h->L,
                          h->H, (uint32_t)q, (uint32_t)h->layout, h->d_rec,
                          h->stream));
  POTTS_CK(cudaMemcpyAsync(h->h_rec, h->d_rec, (size_t)(1 + q) * 8,
                           cudaMemcpyDeviceToHost, h->stream));
  POTTS_CK(cudaStreamSynchronize(h->stream));
  update_obs(&h->obs, h->h_rec, h->L, q, false);
  return POTTS_OK;
}

void free_lattice(potts_h h) {
  if (!h) return;
  for (size_t i = 0; i < h->parts.size(); ++i) {
    potts_h part = h->parts[i];
    if (!part) continue;
    DeviceScope device_scope(part->device);
    if (part->stream) cudaStreamSynchronize(part->stream);
    for (int c = 0; c < 2; ++c)
      if (2 * i + c < h->pass_done.size() && h->pass_done[2 * i + c])
        cudaEventDestroy(h->pass_done[2 * i + c]);
    free_lattice(part);
  }
  if (h->d_planes) cudaFree(h->d_planes);
  if (h->d_alt) cudaFree(h->d_alt);
  if (h->d_rec) cudaFree(h->d_rec);
  if (h->h_rec) cudaFreeHost(h->h_rec);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
  delete h;
}

}  // namespace potts

extern "C" {

const char *potts_last_error(void) { return g_err.c_str(); }

int potts_version(void) { return 220; }

int potts_threshold_table(double beta, uint64_t out_thr[5]) {
  if (!out_thr) return fail(POTTS_EINVAL, "out_thr is NULL");
  if (!threshold_table(beta, out_thr))
    return fail(POTTS_EINVAL, "beta must be finite and >= 0 (got %g)", beta);
  return POTTS_OK;
}

int potts_create_ex(int32_t L, int32_t q, int32_t start, uint64_t seed,
                    int32_t layout, potts_h *out) {
  if (!out) return fail(POTTS_EINVAL, "out is NULL");
  *out = nullptr;
  if (layout == POTTS_LAYOUT_AUTO) layout = POTTS_LAYOUT_U8;
  if (layout != POTTS_LAYOUT_U8 && layout != POTTS_LAYOUT_U4)
    return fail(POTTS_EINVAL, "layout must be 0 (auto), 1 (U8) or 2 (U4)");
  if (layout == POTTS_LAYOUT_U4 && q > 16)
    return fail(POTTS_EINVAL, "the packed 4-bit layout needs q <= 16 (got %d)", q);
  if (L < 32 || L > 65536 || L % 32 != 0)
    return fail(POTTS_EINVAL, "L must be a multiple of 32 in [32, 65536] (got %d)", L);
  if (q < 2 || q > 256) return fail(POTTS_EINVAL, "q must be in [2, 256] (got %d)", q);
  if (start != POTTS_START_ORDERED && start != POTTS_START_RANDOM)
    return fail(POTTS_EINVAL, "start must be 0 (ordered) or 1 (random)");
  potts_h h = new (std::nothrow) potts_lattice();
  if (!h) return fail(POTTS_ENOMEM, "host allocation failed");
  h->L = L;
  h->q = q;
  h->H = L / 2;
  h->layout = layout;
  h->seed = seed;
  h->plane_bytes = (int64_t)L * (layout == POTTS_LAYOUT_U4 ? L / 4 : L / 2);
  int rc = POTTS_OK;
  do {
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) {
      rc = fail(POTTS_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
      break;
    }
    e = cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      rc = fail(POTTS_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
      break;
    }
    h->stream = h->own_stream;
    e = cudaMalloc(&h->d_planes, (size_t)(2 * h->plane_bytes));
    if (e != cudaSuccess) {
      cudaGetLastError();
      h->d_planes = nullptr;
      rc = fail(POTTS_ENOMEM, "cudaMalloc(%lld bytes) for the planes: %s",
                (long long)(2 * h->plane_bytes), cudaGetErrorString(e));
      break;
    }
    h->rec_cap = std::max<int64_t>(1, kRecordBytesTarget / ((1 + q) * 8));
    const size_t rec_bytes = (size_t)h->rec_cap * (1 + q) * 8;
    e = cudaMalloc(&h->d_rec, rec_bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      h->d_rec = nullptr;
      rc = fail(POTTS_ENOMEM, "cudaMalloc records: %s", cudaGetErrorString(e));
      break;
    }
    e = cudaMallocHost(&h->h_rec, rec_bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      h->h_rec = nullptr;
      rc = fail(POTTS_ENOMEM, "cudaMallocHost records: %s",
                cudaGetErrorString(e));
      break;
    }
    h->sms = sm_count_of_current_device();
    if (start == POTTS_START_ORDERED) {
      e = cudaMemsetAsync(h->d_planes, 0, (size_t)(2 * h->plane_bytes),
                          h->stream);
    } else {
      const int64_t sites = (int64_t)L * (L / 2);
      e = launch_init_random(h->d_planes, sites, (uint32_t)q, 0, seed,
                             (uint32_t)layout, h->stream);
      if (e == cudaSuccess)
        e = launch_init_random(h->d_planes + h->plane_bytes, sites,
                               (uint32_t)q, 1, seed, (uint32_t)layout,
                               h->stream);
    }
    if (e != cudaSuccess) {
      rc = fail(POTTS_ECUDA, "init: %s", cudaGetErrorString(e));
      break;
    }
    rc = recount_into_obs(h);
  } while (0);
  if (rc != POTTS_OK) {
    free_lattice(h);
    return rc;
  }
  *out = h;
  clear_error();
  return POTTS_OK;
}

int potts_create(int32_t L, int32_t q, int32_t start, uint64_t seed,
                 potts_h *out) {
  return potts_create_ex(L, q, start, seed, POTTS_LAYOUT_AUTO, out);
}

int potts_sweep(potts_h h, double beta, int64_t nsweeps, uint64_t *out_counts) {
  if (!h) return fail(POTTS_EINVAL, "handle is NULL");
  if (!h->parts.empty()) return sharded_sweep(h, beta, nsweeps, out_counts);
  if (h->strip)
    return fail(POTTS_EINVAL,
                "a row-strip handle sweeps through potts_strip_pass");
  DeviceScope device_scope(h->device);
  if (nsweeps < 0) return fail(POTTS_EINVAL, "nsweeps < 0");
  uint64_t thr[5];
  if (!threshold_table(beta, thr))
    return fail(POTTS_EINVAL, "beta must be finite and >= 0 (got %g)", beta);
  const AcceptTable T = accept_table(thr);
  const int32_t q = h->q;
  const bool hb = h->update == POTTS_UPDATE_HEATBATH;
  HeatTable HT{};
  if (hb) {
    uint64_t W[5];
    int32_t m = 0;
    if (!heatbath_table(beta, q, W, &m))
      return fail(POTTS_EINVAL,
                  "beta=%g is outside the heat-bath weights' range for q=%d",
                  beta, q);
    HT = heat_table(W, m);
  }
  const int64_t rec_len = 1 + q;
  const TileGeom G = pass_geom(h->L, h->H, q, h->layout, h->update, h->sms);
  PassArgs A[2];
  for (int c = 0; c < 2; ++c) {
    A[c].own = h->d_planes + (c ? h->plane_bytes : 0);
    A[c].other = h->d_planes + (c ? 0 : h->plane_bytes);
    A[c].L = h->L;
    A[c].H = h->H;
    A[c].q = (uint32_t)q;
    A[c].colour = (uint32_t)c;
    A[c].key0 = (uint32_t)h->seed;
    A[c].key1 = (uint32_t)(h->seed >> 32);
    A[c].one = 1u;
    A[c].hist_bins = (uint32_t)q;
    A[c].layout = (uint32_t)h->layout;
    A[c].grow0 = 0;
    A[c].row_lo = 0;
    A[c].row_end = h->L;
  }
  int64_t done = 0;
  while (done < nsweeps) {
    const int64_t n = std::min(nsweeps - done, h->rec_cap);
    POTTS_CK(cudaMemsetAsync(h->d_rec, 0, (size_t)(n * rec_len * 8), h->stream));
    for (int64_t s = 0; s < n; ++s) {
      const uint64_t t = h->sweep + (uint64_t)s;
      if (!hb && h->schedule == POTTS_SCHEDULE_FUSED) {
        const int64_t pb = h->plane_bytes;
        POTTS_CK(launch_fused_sweep(h->d_planes, h->d_planes + pb, h->d_alt,
                                    h->d_alt + pb, h->L, (uint32_t)q, t,
                                    h->seed, T, h->d_rec + s * rec_len,
                                    h->stream));
        std::swap(h->d_planes, h->d_alt);
        continue;
      }
      for (int c = 0; c < 2; ++c) {
        A[c].t_lo = (uint32_t)t;
        A[c].t_hi = (uint32_t)(t >> 32);
        if (hb)
          POTTS_CK(launch_pass_hb(A[c], HT, G, h->d_rec + s * rec_len,
                                  h->stream));
        else
          POTTS_CK(launch_pass(A[c], T, G, h->d_rec + s * rec_len,
                               h->stream));
      }
    }
    POTTS_CK(cudaMemcpyAsync(h->h_rec, h->d_rec, (size_t)(n * rec_len * 8),
                             cudaMemcpyDeviceToHost, h->stream));
    POTTS_CK(cudaStreamSynchronize(h->stream));
    // the fused sweep marks B's top bit when a tile copy did not complete
    for (int64_t s = 0; s < n; ++s)
      if (h->h_rec[s * rec_len] >> 63)
        return fail(POTTS_ETIMEOUT, "sweep %llu: a tile copy of the fused "
                    "sweep did not complete", (unsigned long long)(h->sweep + s));
    for (int64_t s = 0; s < n; ++s)
      update_obs(&h->obs, h->h_rec + s * rec_len, h->L, q, true);
    if (out_counts)
      std::memcpy(out_counts + done * rec_len, h->h_rec,
                  (size_t)(n * rec_len * 8));
    h->sweep += (uint64_t)n;
    done += n;
  }
  h->obs.sweep = h->sweep;
  return POTTS_OK;
}

int potts_set_update(potts_h h, int32_t update) {
  if (!h) return fail(POTTS_EINVAL, "handle is NULL");
  if (update != POTTS_UPDATE_METROPOLIS && update != POTTS_UPDATE_HEATBATH)
    return fail(POTTS_EINVAL, "unknown update rule %d", update);
  h->update = update;
  for (potts_h part : h->parts) part->update = update;
  return POTTS_OK;
}

int potts_set_schedule(potts_h h, int32_t schedule) {
  if (!h) return fail(POTTS_EINVAL, "handle is NULL");
  if (schedule != POTTS_SCHEDULE_TWO_PASS && schedule != POTTS_SCHEDULE_FUSED)
    return fail(POTTS_EINVAL, "unknown sweep schedule %d", schedule);
  if (schedule == POTTS_SCHEDULE_FUSED && (h->strip || !h->parts.empty()))
    return fail(POTTS_EINVAL, "row strips sweep with two colour passes");
  if (schedule == POTTS_SCHEDULE_FUSED &&
      !fused_supported(h->L, h->q, h->layout))
    return fail(POTTS_EINVAL,
                "the fused sweep needs the U8 layout and L a multiple of 1024 "
                "(L=%d, layout=%d)", h->L, h->layout);
  if (schedule == POTTS_SCHEDULE_FUSED && !h->d_alt) {
    DeviceScope device_scope(h->device);
    if (cudaMalloc(&h->d_alt, (size_t)(2 * h->plane_bytes)) != cudaSuccess) {
      h->d_alt = nullptr;
      return fail(POTTS_ENOMEM, "cannot allocate the fused sweep's planes "
                  "(%lld bytes)", (long long)(2 * h->plane_bytes));
    }
  }
  h->schedule = schedule;
  return POTTS_OK;
}

int potts_observables(potts_h h, potts_obs *out) {
  if (!h || !out) return fail(POTTS_EINVAL, "NULL argument");
  *out = h->obs;
  out->sweep = h->sweep;
  return POTTS_OK;
}

int potts_reset_averages(potts_h h) {
  if (!h) return fail(POTTS_EINVAL, "handle is NULL");
  h->obs.nsamples = 0;
  h->obs.sum_e = h->obs.sum_e2 = h->obs.sum_e4 = 0;
  h->obs.sum_m = h->obs.sum_m2 = 0;
  return POTTS_OK;
}

int potts_get_spins(potts_h h, uint8_t *out_LxL) {
  if (!h || !out_LxL) return fail(POTTS_EINVAL, "NULL argument");
  if (!h->parts.empty()) return sharded_get_spins(h, out_LxL);
  DeviceScope device_scope(h->device);
  if (h->strip)  // the strip's own rows
    return download_rowmajor(h->d_planes + h->row_bytes,
                             h->d_planes + h->plane_bytes + h->row_bytes,
                             h->L, h->nrows, (uint32_t)h->layout, out_LxL,
                             h->stream);
  return download_rowmajor(h->d_planes, h->d_planes + h->plane_bytes, h->L,
                           h->L, (uint32_t)h->layout, out_LxL, h->stream);
}

int potts_set_state(potts_h h, const uint8_t *LxL, uint64_t sweep) {
  if (!h || !LxL) return fail(POTTS_EINVAL, "NULL argument");
  if (!h->parts.empty()) return sharded_set_state(h, LxL, sweep);
  DeviceScope device_scope(h->device);
  if (h->strip) {  // the strip's own rows; no counts are kept for a strip
    const int rc = upload_rowmajor(
        LxL, h->L, h->nrows, (uint32_t)h->q, (uint32_t)h->layout,
        h->d_planes + h->row_bytes, h->d_planes + h->plane_bytes + h->row_bytes,
        h->stream);
    if (rc) return rc;
    h->sweep = sweep;
    h->obs.sweep = sweep;
    return POTTS_OK;
  }
  const int rc = upload_rowmajor(LxL, h->L, h->L, (uint32_t)h->q,
                                 (uint32_t)h->layout, h->d_planes,
                                 h->d_planes + h->plane_bytes, h->stream);
  if (rc) return rc;
  h->sweep = sweep;
  h->obs.sweep = sweep;
  return recount_into_obs(h);
}

int potts_set_stream(potts_h h, void *stream) {
  if (!h) return fail(POTTS_EINVAL, "handle is NULL");
  if (!h->parts.empty())
    return fail(POTTS_EINVAL, "a lattice split into row strips runs one "
                "stream per strip");
  // finish work queued on the old stream before switching
  POTTS_CK(cudaStreamSynchronize(h->stream));
  h->stream = stream ? (cudaStream_t)stream : h->own_stream;
  return POTTS_OK;
}

int potts_device_planes(potts_h h, void **white, void **black,
                        int64_t *row_bytes, int32_t *layout) {
  if (!h) return fail(POTTS_EINVAL, "handle is NULL");
  if (!h->parts.empty())
    return fail(POTTS_EINVAL, "a lattice split into row strips has no single "
                "pair of planes");
  if (white) *white = h->d_planes;
  if (black) *black = h->d_planes + h->plane_bytes;
  if (row_bytes)
    *row_bytes = h->layout == POTTS_LAYOUT_U4 ? h->H / 2 : h->H;
  if (layout) *layout = h->layout;
  return POTTS_OK;
}

int potts_destroy(potts_h h) {
  if (!h) return fail(POTTS_EINVAL, "handle is NULL");
  DeviceScope device_scope(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  free_lattice(h);
  return POTTS_OK;
}

}  // extern "C"
