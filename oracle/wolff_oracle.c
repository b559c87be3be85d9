/*
 * wolff_oracle.c -- plain CPU oracle for the Wolff single-cluster update of
 * the 2D q-state Potts model (conventions in wolff_oracle.h).
 *
 * TEST INFRASTRUCTURE ONLY (see wolff_oracle.h).  The growth is the
 * textbook one: a FIFO queue of cluster sites, each neighbour in the old
 * state tested once through the bond that joins it.
 */
#include "wolff_oracle.h"

#include <math.h>
#include <stdlib.h>

#include "sw_oracle.h"

enum { W_DOM_SEED = 4, W_DOM_BOND = 5 };

static void words(uint64_t seed, uint64_t idx, uint32_t t, uint32_t domain,
                  uint32_t out[4]) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t ctr[4] = {(uint32_t)idx, (uint32_t)(idx >> 32), t, domain};
  orc_philox4x32_10(ctr, key, out);
}

void orc_wolff_seed(uint64_t L, uint32_t q, const uint8_t *s, uint64_t seed,
                    uint32_t t, uint64_t *i0, uint32_t *s_new) {
  uint32_t w[4];
  words(seed, 0, t, W_DOM_SEED, w);
  uint64_t N = L * L;
  *i0 = ((uint64_t)w[0] * N) >> 32;
  uint32_t old = s[*i0];
  *s_new = (old + 1 + orc_pick(w[1], q - 1)) % q;
}

/* Is the bond owned by site o in direction dir (0 right, 1 down) active? */
static int bond_active(uint64_t seed, uint32_t t, uint32_t thr, uint64_t o,
                       int dir) {
  uint32_t w[4];
  words(seed, o >> 1, t, W_DOM_BOND, w);
  return w[2 * (o & 1) + dir] < thr;
}

uint64_t orc_wolff_step(uint64_t L, uint32_t q, uint32_t thr, uint64_t seed,
                        uint32_t t, uint8_t *s) {
  uint64_t N = L * L, i0;
  uint32_t s_new;
  orc_wolff_seed(L, q, s, seed, t, &i0, &s_new);
  uint8_t s_old = s[i0];
  uint64_t *queue = (uint64_t *)malloc(N * sizeof(uint64_t));
  if (!queue) return 0;
  uint64_t head = 0, tail = 0;
  /* a site leaves state s_old when it joins, so "state s_old" also means
   * "not in the cluster yet" */
  s[i0] = (uint8_t)s_new;
  queue[tail++] = i0;
  while (head < tail) {
    uint64_t i = queue[head++];
    uint64_t y = i / L, x = i % L;
    /* the four neighbours and the (owner, direction) of the joining bond */
    uint64_t nb[4] = {y * L + (x + 1) % L, y * L + (x + L - 1) % L,
                      ((y + 1) % L) * L + x, ((y + L - 1) % L) * L + x};
    uint64_t owner[4] = {i, nb[1], i, nb[3]};
    int dir[4] = {0, 0, 1, 1};
    for (int k = 0; k < 4; ++k) {
      uint64_t j = nb[k];
      if (s[j] != s_old) continue;
      if (!bond_active(seed, t, thr, owner[k], dir[k])) continue;
      s[j] = (uint8_t)s_new;
      queue[tail++] = j;
    }
  }
  free(queue);
  return tail;
}

int orc_wolff_run(uint64_t L, uint32_t q, double T, uint64_t seed,
                  uint8_t *s, uint32_t t0, uint32_t nsteps, uint64_t *sizes) {
  if (L < 2 || L > 65536 || q < 2 || q > 255 || !(T > 0.0) || !isfinite(T))
    return -1;
  uint32_t thr = orc_threshold(T);
  for (uint32_t k = 0; k < nsteps; ++k) {
    uint64_t c = orc_wolff_step(L, q, thr, seed, t0 + k, s);
    if (c == 0) return -2;
    if (sizes) sizes[k] = c;
  }
  return 0;
}
