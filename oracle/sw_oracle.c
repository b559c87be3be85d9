/*
 * sw_oracle.c -- plain CPU oracle for the Swendsen-Wang sweep.
 *
 * TEST INFRASTRUCTURE ONLY (see sw_oracle.h): loaded by tests/, the smoke
 * check and the bench's CPU-baseline leg, never by the CUDA product path.
 * Written for readability, not speed: every step follows the paper's Sec. 2
 * in order, single-threaded, with no blocking or fusion.
 */
#include "sw_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---- Philox4x32-10 (Salmon et al., SC'11, "Parallel random numbers: as
 * easy as 1, 2, 3", Sec. 5).  One round: two 32x32->64 products of the
 * multipliers with counter words 0 and 2, the high halves xored with the
 * other two counter words and the round key, the words permuted; the key is
 * bumped by the Weyl constants (golden ratio, sqrt(3)-1) between rounds. */
static const uint32_t PHILOX_M0 = 0xD2511F53u;
static const uint32_t PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u;
static const uint32_t PHILOX_W1 = 0xBB67AE85u;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    if (round < 9) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void orc_philox_many(uint64_t n, const uint32_t *in, uint32_t *out) {
  for (uint64_t i = 0; i < n; ++i) orc_philox4x32_10(in + 6 * i, in + 6 * i + 4, out + 4 * i);
}

/* Philox word `word` for stream (seed; idx, sweep, domain). */
static uint32_t stream_word(uint64_t seed, uint64_t idx, uint32_t sweep,
                            uint32_t domain, int word) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t ctr[4] = {(uint32_t)idx, (uint32_t)(idx >> 32), sweep, domain};
  uint32_t out[4];
  orc_philox4x32_10(ctr, key, out);
  return out[word];
}

enum { DOM_BOND = 0, DOM_SPIN = 1, DOM_INIT = 2 };

/* Bond probability p = 1 - exp(-J/T), J = 1 (the standard SW probability
 * for H = -J sum delta; Sec. 2 step (1) gives no formula, only that the
 * activation depends on the temperature). */
uint32_t orc_threshold(double T) {
  double p = -expm1(-1.0 / T);
  double t = floor(p * 4294967296.0);
  if (!(t > 0.0)) return 0u;
  if (t >= 4294967295.0) return 0xFFFFFFFFu;
  return (uint32_t)t;
}

/* Sec. 2 step (3): a uniformly random one of the q states. */
uint32_t orc_pick(uint32_t w, uint32_t q) {
  return (uint32_t)(((uint64_t)w * q) >> 32);
}

void orc_init_spins(uint64_t L, uint32_t q, uint64_t seed, uint8_t *s) {
  uint64_t N = L * L;
  for (uint64_t i = 0; i < N; ++i)
    s[i] = (uint8_t)orc_pick(stream_word(seed, i >> 2, 0, DOM_INIT, (int)(i & 3)), q);
}

/* Sec. 2 step (1): a bond is active only between equal spins, with
 * probability p, independently per bond. */
void orc_bonds(uint64_t L, const uint8_t *s, uint32_t thr, uint64_t seed,
               uint32_t sweep, uint8_t *b) {
  for (uint64_t y = 0; y < L; ++y) {
    for (uint64_t x = 0; x < L; ++x) {
      uint64_t i = y * L + x;
      uint64_t ir = y * L + (x + 1) % L;
      uint64_t id = ((y + 1) % L) * L + x;
      uint8_t bits = 0;
      uint32_t wr = stream_word(seed, i >> 1, sweep, DOM_BOND, (int)(2 * (i & 1) + 0));
      uint32_t wd = stream_word(seed, i >> 1, sweep, DOM_BOND, (int)(2 * (i & 1) + 1));
      if (s[i] == s[ir] && wr < thr) bits |= ORC_RIGHT;
      if (s[i] == s[id] && wd < thr) bits |= ORC_DOWN;
      b[i] = bits;
    }
  }
}

/* HK: follow label[label] until it stops changing, then point every label
 * on the path straight at the proper label. */
static uint32_t hk_find(uint32_t *label, uint32_t i) {
  uint32_t r = i;
  while (label[r] != r) r = label[r];
  while (label[i] != r) {
    uint32_t next = label[i];
    label[i] = r;
    i = next;
  }
  return r;
}

/* Join two label sets: the larger proper label points to the smaller, so
 * the proper label stays the smallest label in the cluster (Sec. 2). */
static uint32_t hk_union(uint32_t *label, uint32_t a, uint32_t b) {
  uint32_t ra = hk_find(label, a), rb = hk_find(label, b);
  if (ra == rb) return ra;
  if (ra < rb) { label[rb] = ra; return ra; }
  label[ra] = rb;
  return rb;
}

/* Sec. 2 step (2) with the Hoshen-Kopelman rule.  Raster scan: a site with
 * no active bond to its left / upper neighbour starts a new label; with one,
 * it joins that cluster; with two, the two clusters are joined.  The
 * periodic wrap bonds (Sec. 2: periodic boundary conditions) are joined
 * after the scan.  Finally each site gets its proper label. */
int orc_label(uint64_t L, const uint8_t *b, uint32_t *root) {
  if (L < 2 || L > 65536) return -1;
  uint32_t *label = root; /* label[] lives in the output array */
  for (uint64_t y = 0; y < L; ++y) {
    for (uint64_t x = 0; x < L; ++x) {
      uint32_t i = (uint32_t)(y * L + x);
      int has_left = x > 0 && (b[i - 1] & ORC_RIGHT);
      int has_up = y > 0 && (b[i - L] & ORC_DOWN);
      if (!has_left && !has_up) {
        label[i] = i;
      } else if (has_left && !has_up) {
        label[i] = hk_find(label, i - 1);
      } else if (!has_left && has_up) {
        label[i] = hk_find(label, (uint32_t)(i - L));
      } else {
        label[i] = hk_union(label, i - 1, (uint32_t)(i - L));
      }
    }
  }
  for (uint64_t y = 0; y < L; ++y) {
    uint32_t i = (uint32_t)(y * L + (L - 1));
    if (b[i] & ORC_RIGHT) hk_union(label, i, (uint32_t)(y * L));
  }
  for (uint64_t x = 0; x < L; ++x) {
    uint32_t i = (uint32_t)((L - 1) * L + x);
    if (b[i] & ORC_DOWN) hk_union(label, i, (uint32_t)x);
  }
  uint64_t N = L * L;
  for (uint64_t i = 0; i < N; ++i) label[i] = hk_find(label, (uint32_t)i);
  return 0;
}

/* Sec. 2 step (3).  Roots come first in raster order (root <= i), so the
 * root's new state is already in s when a later member reads it. */
void orc_recolor(uint64_t L, uint32_t q, uint64_t seed, uint32_t sweep,
                 const uint32_t *root, uint8_t *s) {
  uint64_t N = L * L;
  for (uint64_t i = 0; i < N; ++i) {
    uint64_t r = root[i];
    if (r == i)
      s[i] = (uint8_t)orc_pick(stream_word(seed, r, sweep, DOM_SPIN, 0), q);
    else
      s[i] = s[r];
  }
}

/* Sec. 4: energy (as the satisfied-bond count) and magnetisation (as the
 * per-state occupation numbers). */
void orc_measure(uint64_t L, uint32_t q, const uint8_t *s, uint64_t *E_sat,
                 uint64_t *n) {
  uint64_t E = 0;
  for (uint32_t k = 0; k < q; ++k) n[k] = 0;
  for (uint64_t y = 0; y < L; ++y) {
    for (uint64_t x = 0; x < L; ++x) {
      uint64_t i = y * L + x;
      E += s[i] == s[y * L + (x + 1) % L];
      E += s[i] == s[((y + 1) % L) * L + x];
      n[s[i]] += 1;
    }
  }
  *E_sat = E;
}

int orc_run(uint64_t L, uint32_t q, double T, uint64_t seed, uint8_t *s,
            uint32_t sweep0, uint32_t nsweeps, uint64_t *E_series,
            uint64_t *n_series) {
  if (L < 2 || L > 65536 || q < 2 || q > 255 || !(T > 0.0) || !isfinite(T))
    return -1;
  uint64_t N = L * L;
  uint8_t *b = (uint8_t *)malloc(N);
  uint32_t *root = (uint32_t *)malloc(N * sizeof(uint32_t));
  if (!b || !root) { free(b); free(root); return -2; }
  uint32_t thr = orc_threshold(T);
  for (uint32_t k = 0; k < nsweeps; ++k) {
    uint32_t t = sweep0 + k;
    orc_bonds(L, s, thr, seed, t, b);
    orc_label(L, b, root);
    orc_recolor(L, q, seed, t, root, s);
    if (E_series || n_series) {
      uint64_t E, nn[256];
      orc_measure(L, q, s, &E, nn);
      if (E_series) E_series[k] = E;
      if (n_series) memcpy(n_series + (uint64_t)k * q, nn, q * sizeof(uint64_t));
    }
  }
  free(b);
  free(root);
  return 0;
}
