/*
 * Serial CPU oracle for the checkerboard Metropolis (and heat-bath) sweep of
 * the 2D q-state Potts model (Ferrero, De Francesco, Wolovick, Cannas, "q-state Potts model
 * metastability study using optimized GPU-based Monte Carlo algorithms").
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the reference that the CUDA path is
 * checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no code, header, table or
 * constant generator with the CUDA library: everything here is written
 * independently from the paper (Sec. 2.1, Sec. 3, Sec. 3.3-3.4, Sec. 5) and,
 * for the random numbers, from the published definition of Philox4x32-10
 * (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 * SC'11).
 *
 * Lattice storage here is the plain row-major L x L array s[i*L + j] with
 * spins in 0..q-1 (the paper's 1..q labels shifted by -1).
 */
#ifndef POTTS_ORACLE_H
#define POTTS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Philox4x32 with 10 rounds on one 128-bit counter and a 64-bit key. */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                          uint32_t out[4]);

/* The 32-bit random word of site k (index within its colour class) for a
 * given domain (0 = white pass, 1 = black pass, 2/3 = random start of the
 * white/black class) and 0-based global sweep index. */
uint32_t oracle_site_word(uint64_t seed, uint64_t sweep, uint32_t domain,
                          uint64_t k);

/* thr[d] = floor(2^32 * exp(-beta*d)) for d = 0..4 (thr[0] = 2^32).
 * Returns 0, or -1 when beta is negative or not finite. */
int oracle_thresholds(double beta, uint64_t thr[5]);

/* Heat-bath weights W[n] = round(2^m exp(beta n)), n = 0..4 (W[0] = 2^m),
 * with m the largest integer in 0..31 that keeps every normaliser
 * Z = sum over the q states of W[#neighbours in that state] below 2^32.
 * Returns 0, or -1 for a bad beta or q, or when no m >= 0 fits (beta too
 * large for 32-bit weights). */
int oracle_heatbath_weights(double beta, int32_t q, uint64_t W[5],
                            int32_t *m);

/* Full recount of the satisfied-bond number B (Eq. 1 with J = 1 gives
 * H = -B) and of the q-state histogram, straight from the definition. */
void oracle_recount(const uint8_t *s, int32_t L, int32_t q, uint64_t *B,
                    uint64_t *hist);

/* Initial spins of the sites idx[n] (= i*L + j) for the given start. */
int oracle_init_sites(int32_t L, int32_t q, int32_t start, uint64_t seed,
                      int64_t nsites, const int64_t *idx, uint8_t *out);

/* Opaque lattice state. */
typedef struct oracle_lattice oracle_lattice;

/* start: 0 = ordered (all spins 0), 1 = random.  L >= 3, 2 <= q <= 256. */
oracle_lattice *oracle_create(int32_t L, int32_t q, int32_t start,
                              uint64_t seed);
void oracle_destroy(oracle_lattice *lat);

/* Runs nsweeps sweeps at inverse temperature beta.  out_counts (may be NULL)
 * receives nsweeps records of 1+q uint64 {B, hist[0..q-1]}, one after each
 * sweep.  order: 0 = raster order inside a colour class, 1 = reverse raster
 * order.  check != 0 recounts B and the histogram from scratch after every
 * sweep and returns -2 if the incremental values disagree.
 * Returns 0 on success, -1 on bad arguments. */
int oracle_sweep(oracle_lattice *lat, double beta, int64_t nsweeps,
                 uint64_t *out_counts, int32_t order, int32_t check);

/* As oracle_sweep, with the update rule chosen: update 0 = Metropolis,
 * 1 = heat bath (oracle_heatbath_weights; -1 when beta is out of its
 * range). */
int oracle_sweep_ex(oracle_lattice *lat, double beta, int64_t nsweeps,
                    uint64_t *out_counts, int32_t order, int32_t check,
                    int32_t update);

/* Copies the current spins (L*L bytes, row-major) out / in.  set_state also
 * sets the global sweep index and recomputes B and the histogram. */
void oracle_get_spins(const oracle_lattice *lat, uint8_t *out);
int oracle_set_state(oracle_lattice *lat, const uint8_t *spins,
                     uint64_t sweep);
uint64_t oracle_sweep_index(const oracle_lattice *lat);
void oracle_counts(const oracle_lattice *lat, uint64_t *B, uint64_t *hist);

/* Sampled one-sweep update.  Given the spins `pre` before sweep `sweep`
 * (row-major, even L), writes to out[n] the value site idx[n] (= i*L + j)
 * holds after that sweep.  Uses the same single-site rule as oracle_sweep. */
int oracle_sweep_sites(const uint8_t *pre, int32_t L, int32_t q,
                       uint64_t seed, uint64_t sweep, double beta,
                       int64_t nsites, const int64_t *idx, uint8_t *out);
int oracle_sweep_sites_ex(const uint8_t *pre, int32_t L, int32_t q,
                          uint64_t seed, uint64_t sweep, double beta,
                          int64_t nsites, const int64_t *idx, uint8_t *out,
                          int32_t update);

/* One colour pass over a band of rows of an L x L lattice, for the row-strip
 * decomposition of one lattice over several devices (the multi-GPU extension
 * Sec. 7 proposes).  rows: (n + 2) x L row-major bytes: row 0 holds global
 * row r0 - 1 (mod L), rows 1..n hold global rows r0 .. r0 + n - 1, row n + 1
 * holds global row r0 + n (mod L).  Every site of colour c in rows 1..n takes
 * one step of the update rule (update: 0 Metropolis, 1 heat bath) of sweep t,
 * in raster order, against its neighbours as they stand in `rows` (columns
 * periodic), with the random word of its global colour index.  partial
 * (1 + q words) is added to: partial[1 + v] += updated sites now in state v;
 * for c = 1 also partial[0] += neighbours equal to each updated site after
 * its step (every bond has exactly one black end, so over all bands the
 * black pass counts B).  L even, n >= 1, 0 <= r0, r0 + n <= L.  Returns 0,
 * or -1 for bad arguments. */
int oracle_band_pass(uint8_t *rows, int32_t n, int32_t L, int32_t q,
                     int32_t r0, uint64_t seed, uint64_t t, int32_t c,
                     double beta, int32_t update, uint64_t *partial);

#ifdef __cplusplus
}
#endif

#endif
