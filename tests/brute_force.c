/*
 * Exact Boltzmann averages of the q-state Potts model on a tiny periodic
 * L x L lattice by enumerating all q^(L*L) states (test pin for the oracle;
 * shares no code with it).
 *
 * H = -sum over the 2N nearest-neighbour bonds of delta(s_i, s_j)
 * (Sec. 2.1, Eq. 1, J = k_B = 1).  The weight of a state is exp(-beta H) =
 * exp(beta B) with B the number of satisfied bonds.  For every state we also
 * form e = H/N and m = (q N_max / N - 1)/(q - 1).
 *
 * out[0..4] = Z-normalised <e>, <e^2>, <m>, <m^2>, <e^4>.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

int potts_exact_moments(int L, int q, double beta, double *out) {
  const int N = L * L;
  if (L < 3 || N > 20 || q < 2) return -1;
  double states = pow((double)q, (double)N);
  if (states > 5e8) return -1;
  int *s = (int *)calloc((size_t)N, sizeof(int));
  int *cnt = (int *)calloc((size_t)q, sizeof(int));
  if (!s || !cnt) return -1;
  /* Boltzmann weight of each possible B, accumulated per (B, N_max). */
  const int nb = 2 * N + 1;
  double *w = (double *)calloc((size_t)nb * (size_t)(N + 1), sizeof(double));
  if (!w) return -1;
  for (;;) {
    int B = 0;
    for (int v = 0; v < q; ++v) cnt[v] = 0;
    for (int i = 0; i < L; ++i)
      for (int j = 0; j < L; ++j) {
        int x = s[i * L + j];
        B += x == s[i * L + (j + 1) % L];
        B += x == s[((i + 1) % L) * L + j];
        cnt[x] += 1;
      }
    int nmax = 0;
    for (int v = 0; v < q; ++v)
      if (cnt[v] > nmax) nmax = cnt[v];
    w[B * (N + 1) + nmax] += 1.0;
    /* next state in base q */
    int pos = 0;
    while (pos < N) {
      s[pos] += 1;
      if (s[pos] < q) break;
      s[pos] = 0;
      ++pos;
    }
    if (pos == N) break;
  }
  double Z = 0, se = 0, se2 = 0, sm = 0, sm2 = 0, se4 = 0;
  for (int B = 0; B < nb; ++B)
    for (int nm = 0; nm <= N; ++nm) {
      double g = w[B * (N + 1) + nm];
      if (g == 0) continue;
      double wt = g * exp(beta * (double)B);
      double e = -(double)B / N;
      double m = ((double)q * nm / N - 1.0) / (q - 1.0);
      Z += wt;
      se += wt * e;
      se2 += wt * e * e;
      se4 += wt * e * e * e * e;
      sm += wt * m;
      sm2 += wt * m * m;
    }
  out[0] = se / Z;
  out[1] = se2 / Z;
  out[2] = sm / Z;
  out[3] = sm2 / Z;
  out[4] = se4 / Z;
  free(s);
  free(cnt);
  free(w);
  return 0;
}
