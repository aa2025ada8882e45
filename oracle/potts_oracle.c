/*
 * Serial CPU oracle for the checkerboard Metropolis sweep of the 2D q-state
 * Potts model.  TEST INFRASTRUCTURE ONLY: see potts_oracle.h.
 *
 * It is plain, slow and follows the method step by step:
 *   - Hamiltonian H = -J sum_<ij> delta(s_i, s_j), J = 1, k_B = 1, periodic
 *     L x L square lattice (Sec. 2.1, Eq. 1).  We track B = -H, the number of
 *     satisfied bonds.
 *   - Metropolis single-spin flip: the new state is drawn uniformly from all
 *     q states and accepted with probability min(1, exp(-beta dE))
 *     (Sec. 2.2 definition of an MCS, Sec. 3.2 on the random numbers needed).
 *   - Checkerboard order: all white sites ((i+j) even) first, then all black
 *     ones (Sec. 3); one sweep = one MCS = N trials.
 *   - Acceptance against a per-temperature table of Boltzmann weights
 *     (Sec. 5, the CPU code), here floor(2^32 exp(-beta d)) compared with a
 *     32-bit uniform word.
 *   - Energy and the q-state histogram are carried along incrementally while
 *     spins change (Sec. 7 proposes accumulating the energy change on the
 *     fly); a check mode recounts both from scratch after every sweep.
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11), one call per group
 * of four consecutive sites of one colour, one 32-bit word per site.
 *
 * Also a heat-bath single-spin update (one of the other single-flip
 * algorithms Sec. 6 proposes for this lattice code): the new spin is drawn
 * from the site's conditional Boltzmann distribution given its four
 * neighbours, by inverting an integer cumulative distribution with the same
 * 32-bit word per site.
 */
#include "potts_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------
 * Philox4x32-10, from the SC'11 definition: each round multiplies counter
 * words 0 and 2 by two fixed 32-bit constants (full 64-bit products), then
 * forms the new counter (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0).  Between
 * rounds the two key words advance by the Weyl constants (golden ratio and
 * sqrt(3)-1 scaled to 2^32).  Ten rounds, nine key bumps.
 * ------------------------------------------------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                          uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

uint32_t oracle_site_word(uint64_t seed, uint64_t sweep, uint32_t domain,
                          uint64_t k) {
  uint32_t ctr[4], key[2], out[4];
  ctr[0] = (uint32_t)(k >> 2);
  ctr[1] = (uint32_t)sweep;
  ctr[2] = domain;
  ctr[3] = (uint32_t)(sweep >> 32);
  key[0] = (uint32_t)seed;
  key[1] = (uint32_t)(seed >> 32);
  oracle_philox4x32_10(ctr, key, out);
  return out[k & 3u];
}

/* ---------------------------------------------------------------------
 * Boltzmann table (Sec. 5): probability exp(-beta d) for an energy
 * increase d = 1..4, as a 32-bit fixed-point threshold.
 * ------------------------------------------------------------------- */
int oracle_thresholds(double beta, uint64_t thr[5]) {
  if (!(beta >= 0.0) || !isfinite(beta)) return -1;
  thr[0] = (uint64_t)1 << 32;
  for (int d = 1; d <= 4; ++d) {
    double p = exp(-beta * (double)d);
    thr[d] = (uint64_t)floor(ldexp(p, 32));
  }
  return 0;
}

/* ---------------------------------------------------------------------
 * Heat-bath weights.  Given its four neighbours, a site takes state x with
 * probability exp(beta n_x) / sum_y exp(beta n_y), n_x = number of
 * neighbours in state x (H = -sum delta, Eq. 1).  Integer form:
 * W[n] = round(2^m exp(beta n)) for n = 0..4, so W[0] = 2^m, with m the
 * largest integer in 0..31 for which the normaliser Z = sum_x W[n_x] stays
 * below 2^32 for every way the four neighbours can split into states.
 * ------------------------------------------------------------------- */

/* Largest Z over the splits of four neighbours into k distinct states with
 * counts c_1..c_k: Z = sum W[c] + (q - k) W[0]. */
static uint64_t heatbath_zmax(const uint64_t w[5], int32_t q) {
  static const int splits[5][4] = {
      {4, 0, 0, 0}, {3, 1, 0, 0}, {2, 2, 0, 0}, {2, 1, 1, 0}, {1, 1, 1, 1}};
  uint64_t zmax = 0;
  for (int p = 0; p < 5; ++p) {
    int k = 0;
    uint64_t z = 0;
    for (int c = 0; c < 4; ++c) {
      if (splits[p][c] == 0) continue;
      z += w[splits[p][c]];
      k += 1;
    }
    if (k > q) continue;  /* fewer states than classes: impossible split */
    z += (uint64_t)(q - k) * w[0];
    if (z > zmax) zmax = z;
  }
  return zmax;
}

int oracle_heatbath_weights(double beta, int32_t q, uint64_t W[5],
                            int32_t *m_out) {
  if (!(beta >= 0.0) || !isfinite(beta) || q < 2 || q > 256) return -1;
  for (int32_t m = 31; m >= 0; --m) {
    uint64_t w[5];
    int fits = 1;
    for (int n = 0; n <= 4; ++n) {
      double x = ldexp(exp(beta * (double)n), m);
      if (!(x < 4294967296.0)) {
        fits = 0;
        break;
      }
      w[n] = (uint64_t)floor(x + 0.5);
    }
    if (!fits || heatbath_zmax(w, q) > 0xFFFFFFFFull) continue;
    memcpy(W, w, sizeof w);
    *m_out = m;
    return 0;
  }
  return -1;  /* beta too large for 32-bit weights */
}

/* ---------------------------------------------------------------------
 * Counts straight from the definition (Eq. 1): each site's right and down
 * bond, periodic, and the number of sites in each state (used by Eq. 7).
 * ------------------------------------------------------------------- */
void oracle_recount(const uint8_t *s, int32_t L, int32_t q, uint64_t *B,
                    uint64_t *hist) {
  uint64_t b = 0;
  for (int32_t v = 0; v < q; ++v) hist[v] = 0;
  for (int32_t i = 0; i < L; ++i) {
    for (int32_t j = 0; j < L; ++j) {
      uint8_t x = s[(int64_t)i * L + j];
      uint8_t right = s[(int64_t)i * L + (j + 1) % L];
      uint8_t down = s[(int64_t)((i + 1) % L) * L + j];
      b += (x == right);
      b += (x == down);
      hist[x] += 1;
    }
  }
  *B = b;
}

struct oracle_lattice {
  int32_t L, q;
  uint64_t seed;
  uint64_t sweep;   /* global 0-based sweep index of the next sweep */
  uint8_t *s;       /* L*L row-major */
  uint64_t B;       /* satisfied bonds, kept incrementally */
  uint64_t *hist;   /* q counters, kept incrementally */
};

static int32_t wrap(int32_t a, int32_t L) { return (a % L + L) % L; }

/* Index of site (i,j) within its colour class: (i*L + j) / 2. */
static uint64_t colour_index(int32_t L, int32_t i, int32_t j) {
  return ((uint64_t)i * (uint64_t)L + (uint64_t)j) >> 1;
}

/* The single-site Metropolis rule.  `old` is the current spin, nb[0..3] its
 * four neighbours, u the site's 32-bit random word.  Proposal
 * s' = floor(u*q / 2^32) (uniform over all q states, the current one
 * included); acceptance variate a = (u*q) mod 2^32; with H = -B the energy
 * change is dE = n_old - n_new, where n_x counts the neighbours in state x;
 * accept iff dE <= 0 or a < thr[dE].  Returns the new spin and stores the
 * change of B in *dB. */
static int metropolis_rule(int old, const int nb[4], uint32_t u, int32_t q,
                           const uint64_t thr[5], int *dB) {
  uint64_t prod = (uint64_t)u * (uint64_t)q;
  int proposal = (int)(prod >> 32);
  uint64_t a = (uint32_t)prod;
  int n_old = 0, n_new = 0;
  for (int n = 0; n < 4; ++n) {
    n_old += nb[n] == old;
    n_new += nb[n] == proposal;
  }
  int dE = n_old - n_new;
  if ((dE <= 0) || (a < thr[dE])) {
    *dB = n_new - n_old;
    return proposal;
  }
  *dB = 0;
  return old;
}

/* The four neighbours of (i,j) on the periodic lattice: up, down, left,
 * right. */
static void neighbours(const uint8_t *s, int32_t L, int32_t i, int32_t j,
                       int nb[4]) {
  nb[0] = s[(int64_t)wrap(i - 1, L) * L + j];
  nb[1] = s[(int64_t)wrap(i + 1, L) * L + j];
  nb[2] = s[(int64_t)i * L + wrap(j - 1, L)];
  nb[3] = s[(int64_t)i * L + wrap(j + 1, L)];
}

/* The single-site heat-bath rule.  nb[0..3] are the neighbours (up, down,
 * left, right), u the site's 32-bit word.  State x has weight W[n_x]
 * (n_x = neighbours in state x), written as the base W[0] = 2^m plus the
 * excess W[n_x] - W[0], which is zero for a state no neighbour holds.
 * [0, Z) is laid out as: first the excesses of the distinct neighbour
 * states, in the order they first appear in nb, then q intervals of width
 * 2^m, one per state in increasing order.  The new spin is the state whose
 * interval holds r = floor(u Z / 2^32), so state x is drawn with
 * probability W[n_x] / Z.  Returns it and stores the change of B
 * (neighbours equal to the new spin minus those equal to the old one) in
 * *dB. */
static int heatbath_rule(int old, const int nb[4], uint32_t u, int32_t q,
                         const uint64_t W[5], int32_t m, int *dB) {
  int cls[4], cnt[4], k = 0;
  for (int a = 0; a < 4; ++a) {
    int seen = -1;
    for (int b = 0; b < k; ++b)
      if (cls[b] == nb[a]) seen = b;
    if (seen >= 0) {
      cnt[seen] += 1;
    } else {
      cls[k] = nb[a];
      cnt[k] = 1;
      k += 1;
    }
  }
  uint64_t Z = (uint64_t)q * W[0];
  for (int b = 0; b < k; ++b) Z += W[cnt[b]] - W[0];
  uint64_t r = ((uint64_t)u * Z) >> 32;
  int now = -1;
  for (int b = 0; b < k && now < 0; ++b) {
    const uint64_t excess = W[cnt[b]] - W[0];
    if (r < excess)
      now = cls[b];
    else
      r -= excess;
  }
  if (now < 0) now = (int)(r >> m);  /* r < q 2^m here: one of the q bases */
  int n_old = 0, n_now = 0;
  for (int a = 0; a < 4; ++a) {
    n_old += nb[a] == old;
    n_now += nb[a] == now;
  }
  *dB = n_now - n_old;
  return now;
}

/* The update rule of a sweep: Metropolis (thr) or heat bath (W, m). */
typedef struct {
  int32_t heatbath;
  uint64_t thr[5];
  uint64_t W[5];
  int32_t m;
} update_rule;

static int rule_setup(update_rule *ur, int32_t update, double beta,
                      int32_t q) {
  memset(ur, 0, sizeof *ur);
  if (update == 0) return oracle_thresholds(beta, ur->thr);
  if (update != 1) return -1;
  ur->heatbath = 1;
  return oracle_heatbath_weights(beta, q, ur->W, &ur->m);
}

static int apply_rule(const update_rule *ur, int old, const int nb[4],
                      uint32_t u, int32_t q, int *dB) {
  if (ur->heatbath) return heatbath_rule(old, nb, u, q, ur->W, ur->m, dB);
  return metropolis_rule(old, nb, u, q, ur->thr, dB);
}

/* One trial at (i,j) during the pass of colour c of sweep t. */
static int update_site(const uint8_t *s, int32_t L, int32_t q,
                       uint64_t seed, uint64_t t, int c,
                       const update_rule *ur, int32_t i, int32_t j, int *dB) {
  int nb[4];
  neighbours(s, L, i, j, nb);
  uint32_t u = oracle_site_word(seed, t, (uint32_t)c, colour_index(L, i, j));
  return apply_rule(ur, s[(int64_t)i * L + j], nb, u, q, dB);
}

/* Initial spin of site (i,j).  Ordered start: 0 (the paper's s_i = 1,
 * Sec. 3 protocol).  Random start: i.i.d. uniform, floor(u*q / 2^32) with u
 * the site's word of domain 2 + colour at sweep 0. */
static uint8_t initial_spin(int32_t L, int32_t q, int32_t start, uint64_t seed,
                            int32_t i, int32_t j) {
  if (start == 0) return 0;
  int c = (i + j) & 1;
  uint32_t u = oracle_site_word(seed, 0, 2u + (uint32_t)c, colour_index(L, i, j));
  return (uint8_t)(((uint64_t)u * (uint64_t)q) >> 32);
}

int oracle_init_sites(int32_t L, int32_t q, int32_t start, uint64_t seed,
                      int64_t nsites, const int64_t *idx, uint8_t *out) {
  if (L < 3 || q < 2 || q > 256 || (start != 0 && start != 1)) return -1;
  for (int64_t n = 0; n < nsites; ++n) {
    if (idx[n] < 0 || idx[n] >= (int64_t)L * L) return -1;
    out[n] = initial_spin(L, q, start, seed, (int32_t)(idx[n] / L),
                          (int32_t)(idx[n] % L));
  }
  return 0;
}

oracle_lattice *oracle_create(int32_t L, int32_t q, int32_t start,
                              uint64_t seed) {
  if (L < 3 || q < 2 || q > 256 || (start != 0 && start != 1)) return NULL;
  if ((int64_t)L * L > ((int64_t)1 << 32)) return NULL;
  oracle_lattice *lat = (oracle_lattice *)calloc(1, sizeof(*lat));
  if (!lat) return NULL;
  lat->L = L;
  lat->q = q;
  lat->seed = seed;
  lat->sweep = 0;
  lat->s = (uint8_t *)malloc((size_t)L * (size_t)L);
  lat->hist = (uint64_t *)calloc((size_t)q, sizeof(uint64_t));
  if (!lat->s || !lat->hist) {
    oracle_destroy(lat);
    return NULL;
  }
  for (int32_t i = 0; i < L; ++i)
    for (int32_t j = 0; j < L; ++j)
      lat->s[(int64_t)i * L + j] = initial_spin(L, q, start, seed, i, j);
  oracle_recount(lat->s, L, q, &lat->B, lat->hist);
  return lat;
}

void oracle_destroy(oracle_lattice *lat) {
  if (!lat) return;
  free(lat->s);
  free(lat->hist);
  free(lat);
}

int oracle_sweep(oracle_lattice *lat, double beta, int64_t nsweeps,
                 uint64_t *out_counts, int32_t order, int32_t check) {
  return oracle_sweep_ex(lat, beta, nsweeps, out_counts, order, check, 0);
}

int oracle_sweep_ex(oracle_lattice *lat, double beta, int64_t nsweeps,
                    uint64_t *out_counts, int32_t order, int32_t check,
                    int32_t update) {
  update_rule ur;
  if (!lat || nsweeps < 0 || (order != 0 && order != 1)) return -1;
  if (rule_setup(&ur, update, beta, lat->q) != 0) return -1;
  const int32_t L = lat->L, q = lat->q;
  uint64_t *tmp_hist = NULL;
  if (check) {
    tmp_hist = (uint64_t *)malloc((size_t)q * sizeof(uint64_t));
    if (!tmp_hist) return -1;
  }
  for (int64_t n = 0; n < nsweeps; ++n) {
    const uint64_t t = lat->sweep;
    for (int c = 0; c < 2; ++c) {
      for (int64_t r = 0; r < (int64_t)L * L; ++r) {
        int64_t lin = order == 0 ? r : (int64_t)L * L - 1 - r;
        int32_t i = (int32_t)(lin / L), j = (int32_t)(lin % L);
        if (((i + j) & 1) != c) continue;
        int dB = 0;
        int old = lat->s[lin];
        int now = update_site(lat->s, L, q, lat->seed, t, c, &ur, i, j, &dB);
        if (now != old) {
          lat->hist[old] -= 1;
          lat->hist[now] += 1;
          lat->s[lin] = (uint8_t)now;
        }
        lat->B = (uint64_t)((int64_t)lat->B + dB);
      }
    }
    lat->sweep = t + 1;
    if (check) {
      uint64_t b;
      oracle_recount(lat->s, L, q, &b, tmp_hist);
      if (b != lat->B ||
          memcmp(tmp_hist, lat->hist, (size_t)q * sizeof(uint64_t)) != 0) {
        free(tmp_hist);
        return -2;
      }
    }
    if (out_counts) {
      uint64_t *rec = out_counts + n * (int64_t)(1 + q);
      rec[0] = lat->B;
      memcpy(rec + 1, lat->hist, (size_t)q * sizeof(uint64_t));
    }
  }
  free(tmp_hist);
  return 0;
}

void oracle_get_spins(const oracle_lattice *lat, uint8_t *out) {
  memcpy(out, lat->s, (size_t)lat->L * (size_t)lat->L);
}

int oracle_set_state(oracle_lattice *lat, const uint8_t *spins,
                     uint64_t sweep) {
  for (int64_t n = 0; n < (int64_t)lat->L * lat->L; ++n)
    if (spins[n] >= lat->q) return -1;
  memcpy(lat->s, spins, (size_t)lat->L * (size_t)lat->L);
  lat->sweep = sweep;
  oracle_recount(lat->s, lat->L, lat->q, &lat->B, lat->hist);
  return 0;
}

uint64_t oracle_sweep_index(const oracle_lattice *lat) { return lat->sweep; }

void oracle_counts(const oracle_lattice *lat, uint64_t *B, uint64_t *hist) {
  *B = lat->B;
  memcpy(hist, lat->hist, (size_t)lat->q * sizeof(uint64_t));
}

/* A site's value after the white pass of sweep t: white sites take one
 * update step against the pre-sweep black spins, black sites keep their
 * value.  Valid for even L, where same-coloured sites never touch. */
static int after_white(const uint8_t *pre, int32_t L, int32_t q,
                       uint64_t seed, uint64_t t, const update_rule *ur,
                       int32_t i, int32_t j) {
  int dB;
  if (((i + j) & 1) != 0) return pre[(int64_t)i * L + j];
  return update_site(pre, L, q, seed, t, 0, ur, i, j, &dB);
}

int oracle_sweep_sites(const uint8_t *pre, int32_t L, int32_t q,
                       uint64_t seed, uint64_t sweep, double beta,
                       int64_t nsites, const int64_t *idx, uint8_t *out) {
  return oracle_sweep_sites_ex(pre, L, q, seed, sweep, beta, nsites, idx, out,
                               0);
}

int oracle_sweep_sites_ex(const uint8_t *pre, int32_t L, int32_t q,
                          uint64_t seed, uint64_t sweep, double beta,
                          int64_t nsites, const int64_t *idx, uint8_t *out,
                          int32_t update) {
  update_rule ur;
  if ((L & 1) != 0 || L < 4 || q < 2 || q > 256) return -1;
  if (rule_setup(&ur, update, beta, q) != 0) return -1;
  for (int64_t n = 0; n < nsites; ++n) {
    int64_t lin = idx[n];
    if (lin < 0 || lin >= (int64_t)L * L) return -1;
    int32_t i = (int32_t)(lin / L), j = (int32_t)(lin % L);
    if (((i + j) & 1) == 0) {
      out[n] = (uint8_t)after_white(pre, L, q, seed, sweep, &ur, i, j);
      continue;
    }
    /* Black site: its four white neighbours as they are after the white
     * pass, then one update step against them. */
    int nb[4], dB;
    const int32_t ni[4] = {wrap(i - 1, L), wrap(i + 1, L), i, i};
    const int32_t nj[4] = {j, j, wrap(j - 1, L), wrap(j + 1, L)};
    for (int m = 0; m < 4; ++m)
      nb[m] = after_white(pre, L, q, seed, sweep, &ur, ni[m], nj[m]);
    uint32_t u = oracle_site_word(seed, sweep, 1u, colour_index(L, i, j));
    out[n] = (uint8_t)apply_rule(&ur, pre[lin], nb, u, q, &dB);
  }
  return 0;
}

/* ---------------------------------------------------------------------
 * A band of rows (row-strip decomposition, Sec. 7): the colour pass of the
 * sweep restricted to rows r0 .. r0 + n - 1, with the rows just above and
 * below supplied by the caller.  Same rule, same words, same raster order
 * as oracle_sweep_ex within the band.
 * ------------------------------------------------------------------- */
int oracle_band_pass(uint8_t *rows, int32_t n, int32_t L, int32_t q,
                     int32_t r0, uint64_t seed, uint64_t t, int32_t c,
                     double beta, int32_t update, uint64_t *partial) {
  update_rule ur;
  if ((L & 1) != 0 || L < 4 || q < 2 || q > 256 || n < 1 || r0 < 0 ||
      r0 + n > L || (c != 0 && c != 1))
    return -1;
  if (rule_setup(&ur, update, beta, q) != 0) return -1;
  for (int32_t r = 1; r <= n; ++r) {
    const int32_t gi = r0 + r - 1;
    for (int32_t j = 0; j < L; ++j) {
      if (((gi + j) & 1) != c) continue;
      int nb[4], dB;
      nb[0] = rows[(int64_t)(r - 1) * L + j];
      nb[1] = rows[(int64_t)(r + 1) * L + j];
      nb[2] = rows[(int64_t)r * L + wrap(j - 1, L)];
      nb[3] = rows[(int64_t)r * L + wrap(j + 1, L)];
      uint32_t u = oracle_site_word(seed, t, (uint32_t)c,
                                    colour_index(L, gi, j));
      int now = apply_rule(&ur, rows[(int64_t)r * L + j], nb, u, q, &dB);
      rows[(int64_t)r * L + j] = (uint8_t)now;
      partial[1 + now] += 1;
      if (c == 1)
        for (int m = 0; m < 4; ++m) partial[0] += (uint64_t)(nb[m] == now);
    }
  }
  return 0;
}
