/*
 * potts.h - C ABI of libpotts, a GB300 (sm_103a) implementation of the
 * checkerboard Metropolis sweep of the two-dimensional ferromagnetic q-state
 * Potts model, fused with per-sweep energy and magnetisation reductions.
 *
 * Method: Ferrero, De Francesco, Wolovick, Cannas, "q-state Potts model
 * metastability study using optimized GPU-based Monte Carlo algorithms"
 * (Comput. Phys. Commun. 2011, arXiv:1101.0876).
 *   - Model: H = -J sum_<ij> delta(s_i, s_j), J = 1, k_B = 1, on the periodic
 *     L x L square lattice (Sec. 2.1, Eq. 1).  Spins are 0..q-1 here (the
 *     paper's 1..q shifted by -1).  The library reports B = -H, the number
 *     of satisfied bonds, as an exact integer.
 *   - Dynamics: Metropolis single-spin flips; a new state is proposed
 *     uniformly among the q states and accepted with probability
 *     min(1, exp(-beta dE)) (Sec. 2.2, Sec. 3.2).  One sweep (one MCS) is a
 *     pass over all white sites ((i+j) even) followed by a pass over all
 *     black sites (Sec. 3, "Red-Black Gauss-Seidel").  A heat-bath rule
 *     (potts_set_update) is the alternative single-flip update.
 *   - Random numbers: counter-based Philox4x32-10 (Salmon et al., SC'11),
 *     keyed by (seed, sweep, colour, site), replacing the paper's per-thread
 *     multiply-with-carry generators (Sec. 3.2).  The word of colour-c site
 *     k = (i*L + j) >> 1 in sweep t is word (k & 3) of
 *     Philox(counter = (k >> 2, t mod 2^32, c, t >> 32),
 *            key = (seed mod 2^32, seed >> 32)).
 *     With u that word: proposal s' = floor(u q / 2^32); acceptance variate
 *     a = (u q) mod 2^32; accept iff dE <= 0 or a < thr[dE] with
 *     thr[d] = floor(2^32 exp(-beta d)) (the paper's table of Boltzmann
 *     weights, Sec. 5).  Results therefore do not depend on how threads are
 *     mapped to sites, and resuming from (spins, sweep) is exact.
 *   - Counts: after every sweep the library forms the record
 *     {B, hist[0..q-1]} (Sec. 3.4), from which e = -B/N and
 *     m = (q N_max / N - 1)/(q - 1) (Eq. 7, read so that m = 1 when ordered
 *     and 0 when disordered) are computed in FP64 on the host.
 *
 * Conventions for every function:
 *   - Return value: POTTS_OK (0) or a positive POTTS_E* code.  No C++
 *     exception and no abort crosses this boundary.  potts_last_error()
 *     returns a message for the last failure on the calling thread.
 *   - Ownership: the library owns all device memory behind a handle and
 *     frees it in the matching destroy/stop call.  The caller owns every
 *     buffer passed in (host memory unless stated otherwise).
 *   - Threads: calls on one lattice or batch handle must not run
 *     concurrently.  potts_serve_submit/poll/cancel are thread-safe.
 *   - Streams: each handle runs on its own CUDA stream unless
 *     potts_set_stream() gave it one; calls that return results to host
 *     memory synchronise that stream before returning.
 *   - Device: handles are bound to the device current at creation; calls
 *     on a handle run on that device and restore the caller's current
 *     device before returning.
 *   - Version 200 (0.2.0) added the heat-bath rule (potts_set_update,
 *     potts_heatbath_weights, potts_batch_set_update, potts_req.update);
 *     version 210 the fused sweep (potts_set_schedule); version 220 row
 *     strips (potts_create_sharded, potts_strip_*).
 */
#ifndef POTTS_H
#define POTTS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  POTTS_OK = 0,
  POTTS_EINVAL = 1,     /* bad argument (L, q, beta, pointer, layout...) */
  POTTS_ENOMEM = 2,     /* device/host allocation failed or over budget */
  POTTS_ECUDA = 3,      /* a CUDA runtime call failed (message kept) */
  POTTS_ETIMEOUT = 4,   /* a bounded device or host wait gave up */
  POTTS_EBUSY = 5,      /* server queue full (non-blocking submit) */
  POTTS_ECANCELLED = 6, /* request was cancelled */
  POTTS_ENOTFOUND = 7   /* unknown request id */
};

enum { POTTS_START_ORDERED = 0, POTTS_START_RANDOM = 1 };

/* Spin storage in device memory.  U8: one byte per spin, two colour planes
 * of L rows x L/2 bytes (the paper's byte-per-spin colour-packed layout,
 * Sec. 3.3).  U4: two spins per byte (q <= 16), planes of L rows x L/4
 * bytes, site 2b of a plane row in the low nibble of byte b and site 2b+1
 * in the high nibble; half the memory traffic.  AUTO picks U8. */
enum { POTTS_LAYOUT_AUTO = 0, POTTS_LAYOUT_U8 = 1, POTTS_LAYOUT_U4 = 2 };

typedef struct potts_lattice *potts_h;
typedef struct potts_batch *potts_batch_h;
typedef struct potts_server *potts_server_h;

/* Message for the last failure on this thread ("" if none).  The pointer
 * stays valid until the next failing call on the same thread. */
const char *potts_last_error(void);

/* Library version as an integer (major*10000 + minor*100 + patch). */
int potts_version(void);

/* ---------------------------------------------------------------- lattice
 * potts_create: allocates an L x L lattice with q states on the current
 * device and initialises it: ORDERED = every spin 0 (the paper's s_i = 1,
 * Sec. 3 protocol); RANDOM = i.i.d. uniform spins drawn from the Philox
 * words of domain 2 + colour at sweep 0 (s = floor(u q / 2^32)).
 * Constraints: 32 <= L <= 65536, L % 32 == 0; 2 <= q <= 256 (U4 needs
 * q <= 16).  Both layouts give identical results.  The sweep index starts
 * at 0.
 * Errors: EINVAL, ENOMEM, ECUDA. */
int potts_create(int32_t L, int32_t q, int32_t start, uint64_t seed,
                 potts_h *out);
int potts_create_ex(int32_t L, int32_t q, int32_t start, uint64_t seed,
                    int32_t layout, potts_h *out);

/* Runs nsweeps >= 0 sweeps at inverse temperature beta (finite, >= 0).
 * out_counts: NULL, or host memory for nsweeps * (1 + q) uint64 laid out
 * as one record {B, hist[0..q-1]} per sweep, in sweep order.  The running
 * FP64 sums of potts_observables() are updated from every record.
 * Returns after all sweeps finished.  Errors: EINVAL, ECUDA. */
int potts_sweep(potts_h h, double beta, int64_t nsweeps,
                uint64_t *out_counts);

typedef struct {
  uint64_t sweep;     /* sweeps done since create (= next sweep index) */
  uint64_t bonds;     /* B of the last sweep (2N for a fresh ordered start) */
  uint64_t nmax;      /* N_max = max_s hist[s] of the last sweep */
  double e, m;        /* -B/N and (q N_max/N - 1)/(q - 1) of the last sweep */
  uint64_t nsamples;  /* sweeps accumulated in the sums below */
  double sum_e, sum_e2, sum_e4, sum_m, sum_m2;
} potts_obs;

/* Last-sweep values and running FP64 sums since create / reset. */
int potts_observables(potts_h h, potts_obs *out);
int potts_reset_averages(potts_h h);

/* Copies the spins to host memory out_LxL (L*L bytes, row-major s[i*L+j]).
 * Synchronises the handle's stream. */
int potts_get_spins(potts_h h, uint8_t *out_LxL);

/* Replaces the spins (host, L*L bytes row-major, each < q) and the sweep
 * index; the next sweep uses index `sweep`.  B and the histogram are
 * recounted.  Errors: EINVAL (a spin >= q), ECUDA. */
int potts_set_state(potts_h h, const uint8_t *LxL, uint64_t sweep);

/* The acceptance table used for beta: out_thr[d] = floor(2^32 exp(-beta d))
 * for d = 1..4, out_thr[0] = 2^32, computed on the host in FP64.
 * Errors: EINVAL for beta < 0 or not finite. */
int potts_threshold_table(double beta, uint64_t out_thr[5]);

/* Single-site update rule of potts_sweep on a handle.
 *   POTTS_UPDATE_METROPOLIS (default): the rule above (Sec. 2.2, Sec. 3.2).
 *   POTTS_UPDATE_HEATBATH: heat bath, one of the other single-flip
 *     algorithms Sec. 6 proposes: the new spin is drawn from the site's
 *     conditional Boltzmann distribution given its four neighbours,
 *     P(x) = W[n_x] / Z, n_x = neighbours in state x, with the integer
 *     weights of potts_heatbath_weights, by inverting the cumulative
 *     distribution at r = floor(u Z / 2^32) with the site's Philox word u
 *     (same counters as Metropolis).  The states are laid out on [0, Z):
 *     first the distinct neighbour states in the order they first appear
 *     among (up, down, left, right), each of width W[count], then the states
 *     no neighbour holds in increasing order, each of width W[0].
 * Records and observables are the same for both rules.  The rule applies to
 * later potts_sweep calls; a beta outside the heat-bath weights' range then
 * fails with EINVAL.  Errors: EINVAL (unknown rule). */
enum { POTTS_UPDATE_METROPOLIS = 0, POTTS_UPDATE_HEATBATH = 1 };
int potts_set_update(potts_h h, int32_t update);

/* Kernel schedule of a Metropolis sweep on a handle.
 *   POTTS_SCHEDULE_TWO_PASS (default): one kernel per colour pass (Sec. 3:
 *     the white pass completes before the black pass starts).
 *   POTTS_SCHEDULE_FUSED: both passes of a sweep in one kernel.  Each CTA
 *     stages a 32-row x 512-site tile of both colour planes, with halos, in
 *     shared memory; it updates the white sites of the tile and of a one-site
 *     halo around it (halo sites are also updated, identically, by the
 *     neighbouring tiles), then the black sites of the tile against them, and
 *     writes both planes back once.  Each plane is read and written once per
 *     sweep instead of being read twice.  Same random words, same rule:
 *     spins and records are identical to TWO_PASS.
 * FUSED allocates a second pair of planes (the sweep reads one pair and
 * writes the other; see potts_device_planes).  The heat-bath rule always
 * runs two passes.  Errors: EINVAL (unknown schedule; FUSED on a handle
 * whose layout is not U8 or whose L is not a multiple of 1024), ENOMEM. */
enum { POTTS_SCHEDULE_TWO_PASS = 0, POTTS_SCHEDULE_FUSED = 1 };
int potts_set_schedule(potts_h h, int32_t schedule);

/* Heat-bath weights for beta and q: out_W[n] = round(2^m exp(beta n)) for
 * n = 0..4 (so out_W[0] = 2^m), computed on the host in FP64, with *out_m
 * the largest m in 0..31 that keeps the normaliser Z = sum over the q
 * states of W[neighbours in that state] below 2^32 for every neighbour
 * configuration.  Errors: EINVAL for beta < 0 or not finite, q outside
 * 2..256, or beta so large that exp(4 beta) + q - 1 >= 2^32. */
int potts_heatbath_weights(double beta, int32_t q, uint64_t out_W[5],
                           int32_t *out_m);

/* Makes the handle run on `stream` (a cudaStream_t, or NULL for the
 * handle's own stream).  The caller keeps ownership of the stream. */
int potts_set_stream(potts_h h, void *stream);

/* Device pointers of the two colour planes (white = 0, black = 1), their
 * row pitch in bytes, and the layout, for callers that inspect the device
 * state directly.  Read-only view; owned by the handle.  Under the fused
 * schedule each sweep moves the planes between two buffers, so the pointers
 * hold until the next potts_sweep. */
int potts_device_planes(potts_h h, void **white, void **black,
                        int64_t *row_bytes, int32_t *layout);

int potts_destroy(potts_h h);

/* Sweeps a lattice held in caller-owned device memory without allocating
 * anything.  The paper has no counterpart: this exists for callers that
 * must not allocate device memory at the point where they sweep, such as
 * code inside a framework whose caching allocator has already reserved the
 * device memory, or loops that cannot afford the device-wide
 * synchronisation an allocation may cause.
 * white, black: device pointers (16-byte aligned) to the two colour planes
 *   in the POTTS_LAYOUT_U8 layout (L rows x L/2 bytes each, row i of the
 *   white plane holding the sites (i, j) with i + j even in order of j);
 *   read and updated in place.
 * sweep: global index of the first sweep; seed, beta as for potts_sweep.
 * out_counts: NULL, or host or device memory for nsweeps * (1 + q) uint64
 *   records {B, hist[0..q-1]}.
 * stream: a cudaStream_t or NULL (legacy default stream).  The call
 *   synchronises this stream before it returns.
 * Limit: nsweeps * (1 + q) <= 8192 per call (the records accumulate in a
 *   fixed 64 KiB device array that every device loading the library holds
 *   until exit); larger requests fail with POTTS_EINVAL.
 * Sharing: every call on a device uses that one array.  Calls that
 *   overlapped on the GPU would race on it and could return POTTS_OK with
 *   wrong records, so the library serialises its own calls per device with
 *   a host lock held from the first launch until the stream has
 *   synchronised; calls from several host threads therefore queue.
 * Set-up: the first call on a device looks up the array's device address
 *   and keeps it for the life of the process.  After cudaDeviceReset (or
 *   anything else that destroys the device's primary context) that address
 *   is stale: do not call this entry point on that device again.
 * Results equal potts_sweep's bit for bit. */
int potts_sweep_planes_noalloc(void *white, void *black, int32_t L, int32_t q,
                               uint64_t seed, uint64_t sweep, double beta,
                               int64_t nsweeps, uint64_t *out_counts,
                               void *stream);

/* ------------------------------------------------------------- row strips
 * One lattice split into bands of rows (the multi-GPU extension Sec. 7
 * proposes, on the colour-packed planes of Sec. 3.3).  A strip owns lattice
 * rows [row0, row0 + nrows) of both colour planes and keeps a copy of the
 * row just above and the row just below its band (halo rows, periodic).
 * Before the pass of colour c every strip needs fresh halo rows of plane
 * 1 - c; after the black pass the strips' partial records {B, hist} sum to
 * the lattice's record (every bond has exactly one black end).  Random words
 * are keyed by the global site index, so any split gives the single-lattice
 * result bit for bit. */

/* A lattice split into nstrips strips held by this process: strip s has an
 * even number of rows (as equal as possible, strip 0 first) and lives on
 * device devices[s] (NULL: all on the current device).  The handle works
 * with potts_sweep, potts_observables, potts_reset_averages,
 * potts_get_spins, potts_set_state, potts_set_update and potts_destroy,
 * with the same results as potts_create_ex(L, q, start, seed, layout);
 * halo rows move by device-to-device copies ordered by events, one stream
 * per strip.  Not available on it: potts_set_stream, potts_device_planes,
 * the fused schedule.  Errors: EINVAL (arguments as for potts_create_ex;
 * nstrips outside [1, L/2]; a device index out of range), ENOMEM, ECUDA. */
int potts_create_sharded(int32_t L, int32_t q, int32_t start, uint64_t seed,
                         int32_t layout, int32_t nstrips,
                         const int32_t *devices, potts_h *out);

/* One strip of an L x L lattice on the current device, for callers that
 * hold one strip per process and move the halo rows themselves (e.g. NCCL
 * send/receive between neighbouring ranks).  row0 and nrows even,
 * nrows >= 2, row0 + nrows <= L.  Its own rows start as the lattice's would
 * (ordered or random start); halo rows start at 0.  Works with potts_destroy,
 * potts_set_stream, potts_set_update, potts_device_planes (planes of
 * nrows + 2 rows, halo rows included) and, on its own rows (nrows x L
 * row-major bytes), potts_get_spins and potts_set_state (no counts are kept
 * for a strip; set_state sets the strip's sweep index).  potts_sweep
 * rejects it: it sweeps with potts_strip_pass.  Errors: EINVAL, ENOMEM,
 * ECUDA. */
int potts_strip_create(int32_t L, int32_t q, int32_t start, uint64_t seed,
                       int32_t layout, int32_t row0, int32_t nrows,
                       potts_h *out);

/* Device addresses of four rows of the strip's plane `colour` (0 white, 1
 * black), each *row_bytes long: rows[0] its first own row, rows[1] its last
 * own row (what the neighbours above and below need), rows[2] the halo row
 * above, rows[3] the halo row below (where the neighbours' rows go).  Owned
 * by the handle. */
int potts_strip_rows(potts_h h, int32_t colour, void **rows,
                     int64_t *row_bytes);

/* The pass of colour `colour` of the strip's current sweep over its own
 * rows, queued on the strip's stream.  The halo rows of plane 1 - colour
 * must hold the neighbours' rows as they stand after the neighbours' latest
 * pass of colour 1 - colour.  d_record: device memory of 1 + q uint64 the
 * strip's partial counts are added to (the histogram of its sites and the
 * satisfied bonds of its black sites, complete after the black pass: how
 * the histogram is split between the two passes depends on q and the row
 * width); the caller zeroes it per sweep and sums it over the strips.  Passes alternate white
 * (0), black (1); the black pass advances the strip's sweep index.  Does
 * not synchronise.  Errors: EINVAL (not a strip, colour, beta as for
 * potts_sweep), ECUDA. */
int potts_strip_pass(potts_h h, double beta, int32_t colour,
                     uint64_t *d_record);

/* ------------------------------------------------------------------ batch
 * n independent lattices (the paper's "several samples", Sec. 3) swept
 * together: every colour pass of every lattice runs in one persistent
 * launch over a flat (lattice, tile) work list, and k sweeps are captured in
 * one CUDA graph.  Each lattice has its own L, q, start, seed, beta and
 * sweep index; its results equal those of potts_create/potts_sweep with the
 * same arguments bit for bit.
 * Constraints per lattice as for potts_create (U8 layout).
 * Errors: EINVAL, ENOMEM, ECUDA. */
int potts_batch_create(int32_t n, const int32_t *L, const int32_t *q,
                       const int32_t *start, const uint64_t *seed,
                       potts_batch_h *out);

/* beta[n]; out_counts: NULL or an array of n host pointers, each NULL or
 * room for nsweeps * (1 + q_i) uint64 records of lattice i. */
int potts_batch_sweep(potts_batch_h b, const double *beta, int64_t nsweeps,
                      uint64_t *const *out_counts);
/* update[n]: the single-site rule of each lattice for later sweeps
 * (POTTS_UPDATE_METROPOLIS, the default, or POTTS_UPDATE_HEATBATH; see
 * potts_set_update).  Errors: EINVAL (unknown rule). */
int potts_batch_set_update(potts_batch_h b, const int32_t *update);
int potts_batch_get_spins(potts_batch_h b, int32_t i, uint8_t *out_LxL);
int potts_batch_observables(potts_batch_h b, int32_t i, potts_obs *out);
int potts_batch_destroy(potts_batch_h b);

/* -------------------------------------------------------------- serving
 * A request loop on a host thread with continuous batching: requests
 * (L, q, beta, nsweeps, seed, start) are admitted while a slot is free and
 * the device bytes in use plus the request's bytes fit the HBM budget; every
 * step advances all active lattices by up to sweeps_per_step sweeps in one
 * batched launch sequence; finished lattices free their slot and memory.
 * Per-sweep records stream back through potts_serve_poll.  A request's
 * records are identical to those of potts_create/potts_sweep with the same
 * arguments, whatever else is running. */
typedef struct {
  uint64_t hbm_budget_bytes;  /* device bytes the server may hold */
  int32_t max_slots;          /* lattices active at once */
  int32_t sweeps_per_step;    /* sweeps per batched step (>= 1) */
  int32_t queue_capacity;     /* pending requests before EBUSY (0 = 65536) */
  int32_t policy;             /* admission order: POTTS_ADMIT_FIFO (0) or
                                 POTTS_ADMIT_SMALLEST (1) */
} potts_serve_cfg;

/* Admission order of queued requests.  FIFO: oldest first; a request that
 * does not fit the free budget blocks the ones behind it.  SMALLEST: the
 * queued request with the least work (L^2 * nsweeps, ties: oldest) among
 * those that fit is admitted next, which lowers the median latency under
 * overload; a large request can wait while smaller ones keep arriving. */
enum { POTTS_ADMIT_FIFO = 0, POTTS_ADMIT_SMALLEST = 1 };

typedef struct {
  int32_t L, q, start;
  int32_t update;   /* POTTS_UPDATE_METROPOLIS (0) or POTTS_UPDATE_HEATBATH */
  double beta;
  int64_t nsweeps;
  uint64_t seed;
} potts_req;

typedef struct {
  uint64_t submitted, admitted, completed, cancelled;
  uint64_t steps, sweeps_done;    /* batched steps run, lattice-sweeps done */
  uint64_t updates_done;          /* spin updates done (sum of L^2 per sweep) */
  uint64_t bytes_in_use;          /* device bytes held by active lattices */
  int32_t active, queued;
} potts_serve_stats;

int potts_serve_start(const potts_serve_cfg *cfg, potts_server_h *out);

/* Enqueues a request; *req_id receives its id.  EBUSY if the queue is full,
 * EINVAL if the request can never be admitted (bad arguments or larger than
 * the budget). */
int potts_serve_submit(potts_server_h s, const potts_req *req,
                       uint64_t *req_id);

/* Copies up to max_sweeps new records of the request (oldest first) to
 * out_counts (room for max_sweeps * (1 + q) uint64), sets *n_ready to the
 * number copied and *done to 1 once every record of a finished request has
 * been returned (the request is then forgotten).  Never blocks.
 * Errors: ENOTFOUND, ECANCELLED (cancelled request; *done = 1). */
int potts_serve_poll(potts_server_h s, uint64_t req_id, uint64_t *out_counts,
                     int64_t max_sweeps, int64_t *n_ready, int *done);

/* Cancels a queued or running request; its slot and memory are freed at the
 * next step boundary. */
int potts_serve_cancel(potts_server_h s, uint64_t req_id);

int potts_serve_stats_get(potts_server_h s, potts_serve_stats *out);

/* Stops the loop: running requests are cancelled, all memory is freed. */
int potts_serve_stop(potts_server_h s);

#ifdef __cplusplus
}
#endif

#endif /* POTTS_H */
