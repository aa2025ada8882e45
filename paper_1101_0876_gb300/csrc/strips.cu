// Row-strip decomposition of one lattice (the multi-GPU extension of
// Sec. 7, on the colour-packed planes of Sec. 3.3).  Each strip owns a band
// of consecutive lattice rows of both colour planes and keeps a copy of the
// one row just above and the one row just below its band (the halo rows).
// A colour pass reads only the other colour's plane, so before the pass of
// colour c each strip refreshes the halo rows of plane 1 - c from its two
// neighbours; the pass then updates the strip's own rows of plane c.  Every
// strip adds its sites to the sweep's histogram and, on the black pass, the
// satisfied bonds of its black sites (each bond has exactly one black end),
// so the strips' partial records sum to the lattice's record.  The random
// words are keyed by the global site index, so the result does not depend
// on how the lattice is split: it equals the single-lattice sweep bit for
// bit.
//
// Two forms: potts_create_sharded splits one lattice over several strips
// held by this process (on one device or several; halo rows move by
// device-to-device copies ordered by events), and potts_strip_* expose one
// strip for a caller that runs one strip per process and moves the halo rows
// itself (e.g. with NCCL send/receive) and sums the records across
// processes.
#include <algorithm>
#include <cstring>
#include <new>

#include "heatbath.cuh"
#include "lattice.cuh"

namespace potts {
namespace {

uint8_t *plane_of(potts_h s, int c) {
  return s->d_planes + (c ? s->plane_bytes : 0);
}

int check_lattice_args(int32_t L, int32_t q, int32_t start, int32_t layout) {
  if (layout != POTTS_LAYOUT_U8 && layout != POTTS_LAYOUT_U4)
    return fail(POTTS_EINVAL, "layout must be 0 (auto), 1 (U8) or 2 (U4)");
  if (layout == POTTS_LAYOUT_U4 && q > 16)
    return fail(POTTS_EINVAL,
                "the packed 4-bit layout needs q <= 16 (got %d)", q);
  if (L < 32 || L > 65536 || L % 32 != 0)
    return fail(POTTS_EINVAL,
                "L must be a multiple of 32 in [32, 65536] (got %d)", L);
  if (q < 2 || q > 256)
    return fail(POTTS_EINVAL, "q must be in [2, 256] (got %d)", q);
  if (start != POTTS_START_ORDERED && start != POTTS_START_RANDOM)
    return fail(POTTS_EINVAL, "start must be 0 (ordered) or 1 (random)");
  return POTTS_OK;
}

// One strip handle on the current device: rows [row0, row0 + nrows) of the
// lattice, its own rows initialised (ordered or random start), halo rows
// zero until the first exchange.
int make_strip(int32_t L, int32_t q, int32_t start, uint64_t seed,
               int32_t row0, int32_t nrows, int32_t layout, potts_h *out) {
  *out = nullptr;
  potts_h h = new (std::nothrow) potts_lattice();
  if (!h) return fail(POTTS_ENOMEM, "host allocation failed");
  h->L = L;
  h->q = q;
  h->H = L / 2;
  h->layout = layout;
  h->seed = seed;
  h->strip = 1;
  h->row0 = row0;
  h->nrows = nrows;
  h->row_bytes = layout == POTTS_LAYOUT_U4 ? L / 4 : L / 2;
  h->plane_bytes = (int64_t)(nrows + 2) * h->row_bytes;
  int rc = [&]() -> int {
    POTTS_CK(cudaGetDevice(&h->device));
    POTTS_CK(cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking));
    h->stream = h->own_stream;
    if (cudaMalloc(&h->d_planes, (size_t)(2 * h->plane_bytes)) != cudaSuccess) {
      cudaGetLastError();
      h->d_planes = nullptr;
      return fail(POTTS_ENOMEM, "cudaMalloc(%lld bytes) for a strip's planes",
                  (long long)(2 * h->plane_bytes));
    }
    h->rec_cap = std::max<int64_t>(1, kRecordBytesTarget / ((1 + q) * 8));
    const size_t rec_bytes = (size_t)h->rec_cap * (1 + q) * 8;
    if (cudaMalloc(&h->d_rec, rec_bytes) != cudaSuccess) {
      cudaGetLastError();
      h->d_rec = nullptr;
      return fail(POTTS_ENOMEM, "cudaMalloc records");
    }
    if (cudaMallocHost(&h->h_rec, rec_bytes) != cudaSuccess) {
      cudaGetLastError();
      h->h_rec = nullptr;
      return fail(POTTS_ENOMEM, "cudaMallocHost records");
    }
    h->sms = sm_count_of_current_device();
    POTTS_CK(cudaMemsetAsync(h->d_planes, 0, (size_t)(2 * h->plane_bytes),
                             h->stream));
    if (start == POTTS_START_RANDOM) {
      const int64_t sites = (int64_t)nrows * h->H;
      for (int c = 0; c < 2; ++c)
        POTTS_CK(launch_init_random(plane_of(h, c) + h->row_bytes, sites,
                                    (uint32_t)q, (uint32_t)c, seed,
                                    (uint32_t)layout, h->stream,
                                    (int64_t)row0 * h->H));
    }
    POTTS_CK(cudaStreamSynchronize(h->stream));
    return POTTS_OK;
  }();
  if (rc != POTTS_OK) {
    free_lattice(h);
    return rc;
  }
  *out = h;
  return POTTS_OK;
}

// The update rule's tables for one beta.
struct Rule {
  bool heatbath = false;
  AcceptTable T{};
  HeatTable HT{};
};

int make_rule(double beta, int32_t q, int32_t update, Rule *r) {
  uint64_t thr[5];
  if (!threshold_table(beta, thr))
    return fail(POTTS_EINVAL, "beta must be finite and >= 0 (got %g)", beta);
  r->T = accept_table(thr);
  r->heatbath = update == POTTS_UPDATE_HEATBATH;
  if (r->heatbath) {
    uint64_t W[5];
    int32_t m = 0;
    if (!heatbath_table(beta, q, W, &m))
      return fail(POTTS_EINVAL,
                  "beta=%g is outside the heat-bath weights' range for q=%d",
                  beta, q);
    r->HT = heat_table(W, m);
  }
  return POTTS_OK;
}

// The colour pass of sweep s->sweep over the strip's own rows; the strip's
// partial counts are added to rec.
cudaError_t strip_pass(potts_h s, const Rule &r, int colour,
                       unsigned long long *rec) {
  PassArgs A;
  A.own = plane_of(s, colour);
  A.other = plane_of(s, colour ^ 1);
  A.L = s->nrows + 2;
  A.H = s->H;
  A.q = (uint32_t)s->q;
  A.colour = (uint32_t)colour;
  A.t_lo = (uint32_t)s->sweep;
  A.t_hi = (uint32_t)(s->sweep >> 32);
  A.key0 = (uint32_t)s->seed;
  A.key1 = (uint32_t)(s->seed >> 32);
  A.layout = (uint32_t)s->layout;
  A.one = 1u;
  A.hist_bins = (uint32_t)s->q;
  A.grow0 = s->row0 - 1;
  A.row_lo = 1;
  A.row_end = s->nrows + 1;
  const TileGeom G = pass_geom(s->nrows, s->H, s->q, s->layout,
                               r.heatbath ? POTTS_UPDATE_HEATBATH
                                          : POTTS_UPDATE_METROPOLIS,
                               s->sms);
  if (r.heatbath) return launch_pass_hb(A, r.HT, G, rec, s->stream);
  return launch_pass(A, r.T, G, rec, s->stream);
}

cudaError_t copy_row(uint8_t *dst, int dst_dev, const uint8_t *src,
                     int src_dev, int64_t n, cudaStream_t st) {
  if (dst_dev == src_dev)
    return cudaMemcpyAsync(dst, src, (size_t)n, cudaMemcpyDeviceToDevice, st);
  return cudaMemcpyPeerAsync(dst, dst_dev, src, src_dev, (size_t)n, st);
}

// Refreshes every strip's halo rows of plane p from its neighbours' own
// rows, after the neighbours' latest pass of colour p; queued on each
// strip's stream.
int exchange(potts_h h, int p) {
  const int S = (int)h->parts.size();
  for (int s = 0; s < S; ++s) {
    potts_h me = h->parts[s];
    const int ip = (s + S - 1) % S, in = (s + 1) % S;
    potts_h prev = h->parts[ip], next = h->parts[in];
    DeviceScope device_scope(me->device);
    POTTS_CK(cudaStreamWaitEvent(me->stream, h->pass_done[2 * ip + p], 0));
    POTTS_CK(cudaStreamWaitEvent(me->stream, h->pass_done[2 * in + p], 0));
    const int64_t RB = me->row_bytes;
    uint8_t *mine = plane_of(me, p);
    POTTS_CK(copy_row(mine, me->device,
                      plane_of(prev, p) + (int64_t)prev->nrows * RB,
                      prev->device, RB, me->stream));
    POTTS_CK(copy_row(mine + (int64_t)(me->nrows + 1) * RB, me->device,
                      plane_of(next, p) + RB, next->device, RB, me->stream));
  }
  return POTTS_OK;
}

// Copies n records from every strip's ring, sums them into h->h_rec.
int gather_records(potts_h h, int64_t n) {
  const int64_t words = n * (1 + h->q);
  for (potts_h part : h->parts) {
    DeviceScope device_scope(part->device);
    POTTS_CK(cudaMemcpyAsync(part->h_rec, part->d_rec, (size_t)words * 8,
                             cudaMemcpyDeviceToHost, part->stream));
  }
  std::memset(h->h_rec, 0, (size_t)words * 8);
  for (potts_h part : h->parts) {
    DeviceScope device_scope(part->device);
    POTTS_CK(cudaStreamSynchronize(part->stream));
    for (int64_t k = 0; k < words; ++k) h->h_rec[k] += part->h_rec[k];
  }
  return POTTS_OK;
}

// Halo rows of both planes, then the recount of every strip: the lattice's
// {B, hist} into the observables.
int sharded_recount(potts_h h) {
  int rc = exchange(h, 0);
  if (!rc) rc = exchange(h, 1);
  if (rc) return rc;
  for (potts_h part : h->parts) {
    DeviceScope device_scope(part->device);
    POTTS_CK(cudaMemsetAsync(part->d_rec, 0, (size_t)(1 + h->q) * 8,
                             part->stream));
    POTTS_CK(launch_recount_rows(plane_of(part, 0), plane_of(part, 1),
                                 part->nrows + 2, part->H, 1, part->nrows,
                                 part->row0 - 1, (uint32_t)h->q,
                                 (uint32_t)h->layout, part->d_rec,
                                 part->stream));
  }
  rc = gather_records(h, 1);
  if (rc) return rc;
  update_obs(&h->obs, h->h_rec, h->L, h->q, false);
  return POTTS_OK;
}

}  // namespace

int sharded_sweep(potts_h h, double beta, int64_t nsweeps,
                  uint64_t *out_counts) {
  if (nsweeps < 0) return fail(POTTS_EINVAL, "nsweeps < 0");
  Rule rule;
  int rc = make_rule(beta, h->q, h->update, &rule);
  if (rc) return rc;
  const int64_t rec_len = 1 + h->q;
  const int S = (int)h->parts.size();
  int64_t done = 0;
  while (done < nsweeps) {
    const int64_t n = std::min(nsweeps - done, h->rec_cap);
    for (potts_h part : h->parts) {
      DeviceScope device_scope(part->device);
      POTTS_CK(cudaMemsetAsync(part->d_rec, 0, (size_t)(n * rec_len * 8),
                               part->stream));
    }
    for (int64_t t = 0; t < n; ++t) {
      for (int c = 0; c < 2; ++c) {
        rc = exchange(h, c ^ 1);  // the plane this pass reads
        if (rc) return rc;
        for (int s = 0; s < S; ++s) {
          potts_h part = h->parts[s];
          DeviceScope device_scope(part->device);
          POTTS_CK(strip_pass(part, rule, c, part->d_rec + t * rec_len));
          POTTS_CK(cudaEventRecord(h->pass_done[2 * s + c], part->stream));
        }
      }
      for (potts_h part : h->parts) part->sweep += 1;
    }
    rc = gather_records(h, n);
    if (rc) return rc;
    for (int64_t t = 0; t < n; ++t)
      update_obs(&h->obs, h->h_rec + t * rec_len, h->L, h->q, true);
    if (out_counts)
      std::memcpy(out_counts + done * rec_len, h->h_rec,
                  (size_t)(n * rec_len * 8));
    h->sweep += (uint64_t)n;
    done += n;
  }
  h->obs.sweep = h->sweep;
  return POTTS_OK;
}

int sharded_get_spins(potts_h h, uint8_t *out_LxL) {
  for (potts_h part : h->parts) {
    DeviceScope device_scope(part->device);
    const int rc = download_rowmajor(
        plane_of(part, 0) + part->row_bytes, plane_of(part, 1) + part->row_bytes,
        h->L, part->nrows, (uint32_t)h->layout,
        out_LxL + (int64_t)part->row0 * h->L, part->stream);
    if (rc) return rc;
  }
  return POTTS_OK;
}

int sharded_set_state(potts_h h, const uint8_t *LxL, uint64_t sweep) {
  // every spin is checked before any strip changes
  if (h->q < 256) {
    const int64_t N = (int64_t)h->L * h->L;
    for (int64_t k = 0; k < N; ++k)
      if (LxL[k] >= h->q)
        return fail(POTTS_EINVAL, "spin %d at %lld is >= q = %d", LxL[k],
                    (long long)k, h->q);
  }
  for (potts_h part : h->parts) {
    DeviceScope device_scope(part->device);
    const int rc = upload_rowmajor(
        LxL + (int64_t)part->row0 * h->L, h->L, part->nrows, (uint32_t)h->q,
        (uint32_t)h->layout, plane_of(part, 0) + part->row_bytes,
        plane_of(part, 1) + part->row_bytes, part->stream);
    if (rc) return rc;
    part->sweep = sweep;
  }
  h->sweep = sweep;
  h->obs.sweep = sweep;
  return sharded_recount(h);
}

}  // namespace potts

using namespace potts;

extern "C" {

int potts_create_sharded(int32_t L, int32_t q, int32_t start, uint64_t seed,
                         int32_t layout, int32_t nstrips,
                         const int32_t *devices, potts_h *out) {
  if (!out) return fail(POTTS_EINVAL, "out is NULL");
  *out = nullptr;
  if (layout == POTTS_LAYOUT_AUTO) layout = POTTS_LAYOUT_U8;
  int rc = check_lattice_args(L, q, start, layout);
  if (rc) return rc;
  if (nstrips < 1 || nstrips > L / 2)
    return fail(POTTS_EINVAL,
                "nstrips must be in [1, L/2] (got %d for L=%d)", nstrips, L);
  int ndev = 0, cur = 0;
  POTTS_CK(cudaGetDeviceCount(&ndev));
  POTTS_CK(cudaGetDevice(&cur));
  if (devices)
    for (int s = 0; s < nstrips; ++s)
      if (devices[s] < 0 || devices[s] >= ndev)
        return fail(POTTS_EINVAL, "devices[%d] = %d: only %d devices", s,
                    devices[s], ndev);
  potts_h h = new (std::nothrow) potts_lattice();
  if (!h) return fail(POTTS_ENOMEM, "host allocation failed");
  h->L = L;
  h->q = q;
  h->H = L / 2;
  h->layout = layout;
  h->seed = seed;
  h->device = cur;
  h->rec_cap = std::max<int64_t>(1, kRecordBytesTarget / ((1 + q) * 8));
  rc = [&]() -> int {
    if (cudaMallocHost(&h->h_rec, (size_t)h->rec_cap * (1 + q) * 8) !=
        cudaSuccess) {
      cudaGetLastError();
      h->h_rec = nullptr;
      return fail(POTTS_ENOMEM, "cudaMallocHost records");
    }
    // strips of an even number of rows, as equal as possible
    const int32_t pairs = L / 2, base = pairs / nstrips, extra = pairs % nstrips;
    int32_t row0 = 0;
    h->parts.assign((size_t)nstrips, nullptr);
    h->pass_done.assign((size_t)(2 * nstrips), nullptr);
    for (int s = 0; s < nstrips; ++s) {
      const int dev = devices ? devices[s] : cur;
      const int32_t n = 2 * (base + (s < extra ? 1 : 0));
      DeviceScope device_scope(dev);
      int r = make_strip(L, q, start, seed, row0, n, layout, &h->parts[s]);
      if (r) return r;
      for (int c = 0; c < 2; ++c)
        POTTS_CK(cudaEventCreateWithFlags(&h->pass_done[2 * s + c],
                                          cudaEventDisableTiming));
      row0 += n;
    }
    // direct copies between the devices that hold neighbouring strips
    for (int s = 0; s < nstrips; ++s) {
      const int a = h->parts[s]->device,
                b = h->parts[(s + 1) % nstrips]->device;
      if (a == b) continue;
      int ok = 0;
      for (int k = 0; k < 2; ++k) {
        const int from = k ? b : a, to = k ? a : b;
        if (cudaDeviceCanAccessPeer(&ok, from, to) == cudaSuccess && ok) {
          DeviceScope device_scope(from);
          const cudaError_t e = cudaDeviceEnablePeerAccess(to, 0);
          if (e == cudaErrorPeerAccessAlreadyEnabled) cudaGetLastError();
          else if (e != cudaSuccess) cudaGetLastError();  // copies still work
        }
      }
    }
    return sharded_recount(h);
  }();
  if (rc != POTTS_OK) {
    free_lattice(h);
    return rc;
  }
  *out = h;
  clear_error();
  return POTTS_OK;
}

int potts_strip_create(int32_t L, int32_t q, int32_t start, uint64_t seed,
                       int32_t layout, int32_t row0, int32_t nrows,
                       potts_h *out) {
  if (!out) return fail(POTTS_EINVAL, "out is NULL");
  *out = nullptr;
  if (layout == POTTS_LAYOUT_AUTO) layout = POTTS_LAYOUT_U8;
  int rc = check_lattice_args(L, q, start, layout);
  if (rc) return rc;
  if (row0 < 0 || row0 % 2 || nrows < 2 || nrows % 2 || row0 + nrows > L)
    return fail(POTTS_EINVAL,
                "a strip needs an even first row and an even number of rows "
                "inside the lattice (row0=%d, nrows=%d, L=%d)",
                row0, nrows, L);
  rc = make_strip(L, q, start, seed, row0, nrows, layout, out);
  if (rc == POTTS_OK) clear_error();
  return rc;
}

int potts_strip_rows(potts_h h, int32_t colour, void **rows,
                     int64_t *row_bytes) {
  if (!h || !rows) return fail(POTTS_EINVAL, "NULL argument");
  if (!h->strip || !h->parts.empty())
    return fail(POTTS_EINVAL, "not a row-strip handle");
  if (colour != 0 && colour != 1)
    return fail(POTTS_EINVAL, "colour must be 0 or 1");
  uint8_t *p = plane_of(h, colour);
  const int64_t RB = h->row_bytes;
  rows[0] = p + RB;                          // first own row
  rows[1] = p + (int64_t)h->nrows * RB;      // last own row
  rows[2] = p;                               // halo: the row above
  rows[3] = p + (int64_t)(h->nrows + 1) * RB;  // halo: the row below
  if (row_bytes) *row_bytes = RB;
  return POTTS_OK;
}

int potts_strip_pass(potts_h h, double beta, int32_t colour,
                     uint64_t *d_record) {
  if (!h || !d_record) return fail(POTTS_EINVAL, "NULL argument");
  if (!h->strip || !h->parts.empty())
    return fail(POTTS_EINVAL, "not a row-strip handle");
  if (colour != 0 && colour != 1)
    return fail(POTTS_EINVAL, "colour must be 0 or 1");
  Rule rule;
  int rc = make_rule(beta, h->q, h->update, &rule);
  if (rc) return rc;
  DeviceScope device_scope(h->device);
  POTTS_CK(strip_pass(h, rule, colour,
                      reinterpret_cast<unsigned long long *>(d_record)));
  if (colour == 1) {
    h->sweep += 1;
    h->obs.sweep = h->sweep;
  }
  return POTTS_OK;
}

}  // extern "C"
