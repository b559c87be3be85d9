/*
 * xy_oracle.c -- plain CPU oracle for the embedded-cluster SW sweep of the
 * 2D XY model with M equally spaced angles (conventions in xy_oracle.h).
 *
 * TEST INFRASTRUCTURE ONLY (see xy_oracle.h).  Written for readability:
 * the steps of Wolff's embedding (Sec. 5 of the paper; Wolff, PRL 62, 361)
 * in order, single-threaded; the labelling is the Potts oracle's.
 */
#include "xy_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "sw_oracle.h"

enum { XY_DOM_SPIN = 1, XY_DOM_AXIS = 3, XY_DOM_BOND = 0 };

static uint32_t philox_word(uint64_t seed, uint64_t idx, uint32_t sweep,
                            uint32_t domain, int word) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t ctr[4] = {(uint32_t)idx, (uint32_t)(idx >> 32), sweep, domain};
  uint32_t out[4];
  orc_philox4x32_10(ctr, key, out);
  return out[word];
}

uint32_t orc_xy_axis(uint64_t seed, uint32_t sweep, uint32_t M) {
  return orc_pick(philox_word(seed, 0, sweep, XY_DOM_AXIS, 0), M);
}

/* Embedded Ising coupling of two spins is |sigma_i| |sigma_j| (J = 1), so
 * the SW probability of a satisfied embedded bond is
 * 1 - exp(-2 |sigma_i| |sigma_j| / T). */
void orc_xy_thresholds(uint32_t M, double T, uint32_t *tt) {
  const uint32_t H = M / 2;
  const double pi = acos(-1.0);
  for (uint32_t c = 0; c <= H; ++c) {
    for (uint32_t d = 0; d <= H; ++d) {
      double sc = sin(pi * (double)c / (double)M);
      double sd = sin(pi * (double)d / (double)M);
      double p = -expm1(-2.0 * sc * sd / T);
      double t = floor(p * 4294967296.0);
      uint32_t v;
      if (!(t > 0.0))
        v = 0u;
      else if (t >= 4294967295.0)
        v = 0xFFFFFFFFu;
      else
        v = (uint32_t)t;
      tt[c * (H + 1) + d] = v;
    }
  }
}

/* Sign (-1, 0, +1) and fold index c of sigma = -sin(pi a / M),
 * a = (2k - j) mod 2M. */
static void projection(uint32_t M, uint32_t k, uint32_t j, int *sign,
                       uint32_t *c) {
  int64_t a = ((int64_t)2 * k - (int64_t)j) % (int64_t)(2 * M);
  if (a < 0) a += 2 * M;
  if (a == 0 || a == (int64_t)M)
    *sign = 0;
  else
    *sign = a < (int64_t)M ? -1 : +1;
  uint32_t b = (uint32_t)(a % M);
  *c = b < M - b ? b : M - b;
}

void orc_xy_bonds(uint64_t L, uint32_t M, const uint8_t *s,
                  const uint32_t *tt, uint32_t j, uint64_t seed,
                  uint32_t sweep, uint8_t *b) {
  const uint32_t H = M / 2;
  for (uint64_t y = 0; y < L; ++y) {
    for (uint64_t x = 0; x < L; ++x) {
      uint64_t i = y * L + x;
      uint64_t nb[2] = {y * L + (x + 1) % L, ((y + 1) % L) * L + x};
      int si;
      uint32_t ci;
      projection(M, s[i], j, &si, &ci);
      uint8_t bits = 0;
      for (int dir = 0; dir < 2; ++dir) {
        int sn;
        uint32_t cn;
        projection(M, s[nb[dir]], j, &sn, &cn);
        uint32_t u = philox_word(seed, i >> 1, sweep, XY_DOM_BOND,
                                 (int)(2 * (i & 1) + dir));
        if (si != 0 && si == sn && u < tt[ci * (H + 1) + cn])
          bits |= dir == 0 ? ORC_RIGHT : ORC_DOWN;
      }
      b[i] = bits;
    }
  }
}

/* Roots come first in raster order, so a root's coin is drawn before any
 * other member of its cluster is visited; members copy it from `coin`. */
void orc_xy_flip(uint64_t L, uint32_t M, uint32_t j, uint64_t seed,
                 uint32_t sweep, const uint32_t *root, uint8_t *s) {
  uint64_t N = L * L;
  uint8_t *coin = (uint8_t *)malloc(N ? N : 1);
  if (!coin) return;
  for (uint64_t i = 0; i < N; ++i) {
    uint64_t r = root[i];
    if (r == i)
      coin[i] = (uint8_t)orc_pick(philox_word(seed, r, sweep, XY_DOM_SPIN, 0), 2);
    else
      coin[i] = coin[r];
    if (coin[i]) s[i] = (uint8_t)((j + M - s[i]) % M);
  }
  free(coin);
}

void orc_xy_measure(uint64_t L, uint32_t M, const uint8_t *s, uint64_t *D,
                    uint64_t *n) {
  const uint32_t H = M / 2;
  for (uint32_t d = 0; d <= H; ++d) D[d] = 0;
  for (uint32_t k = 0; k < M; ++k) n[k] = 0;
  for (uint64_t y = 0; y < L; ++y) {
    for (uint64_t x = 0; x < L; ++x) {
      uint64_t i = y * L + x;
      uint64_t nb[2] = {y * L + (x + 1) % L, ((y + 1) % L) * L + x};
      for (int dir = 0; dir < 2; ++dir) {
        uint32_t delta = (s[i] + M - s[nb[dir]]) % M;
        D[delta < M - delta ? delta : M - delta] += 1;
      }
      n[s[i]] += 1;
    }
  }
}

int orc_xy_run(uint64_t L, uint32_t M, double T, uint64_t seed, uint8_t *s,
               uint32_t sweep0, uint32_t nsweeps, uint64_t *D_series,
               uint64_t *n_series) {
  if (L < 2 || L > 65536 || M < 2 || M > 256 || !(T > 0.0) || !isfinite(T))
    return -1;
  const uint32_t H = M / 2;
  uint64_t N = L * L;
  uint8_t *b = (uint8_t *)malloc(N);
  uint32_t *root = (uint32_t *)malloc(N * sizeof(uint32_t));
  uint32_t *tt = (uint32_t *)malloc((size_t)(H + 1) * (H + 1) * sizeof(uint32_t));
  if (!b || !root || !tt) {
    free(b);
    free(root);
    free(tt);
    return -2;
  }
  orc_xy_thresholds(M, T, tt);
  for (uint32_t k = 0; k < nsweeps; ++k) {
    uint32_t t = sweep0 + k;
    uint32_t j = orc_xy_axis(seed, t, M);
    orc_xy_bonds(L, M, s, tt, j, seed, t, b);
    orc_label(L, b, root);
    orc_xy_flip(L, M, j, seed, t, root, s);
    if (D_series || n_series) {
      uint64_t D[129], n[256];
      orc_xy_measure(L, M, s, D, n);
      if (D_series) memcpy(D_series + (uint64_t)k * (H + 1), D, (H + 1) * sizeof(uint64_t));
      if (n_series) memcpy(n_series + (uint64_t)k * M, n, M * sizeof(uint64_t));
    }
  }
  free(b);
  free(root);
  free(tt);
  return 0;
}
