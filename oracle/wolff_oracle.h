/*
 * wolff_oracle.h -- plain, slow, single-threaded CPU oracle for the Wolff
 * single-cluster update of the periodic 2D q-state Potts model, the
 * comparison workload of the paper's related work (Sec. 1: Wolff's
 * single-cluster algorithm, U. Wolff, PRL 62, 361 (1989); grown on a GPU by
 * processing the newly added spins of the cluster in parallel).
 *
 * TEST INFRASTRUCTURE ONLY, like sw_oracle.h: loaded by tests/ and the
 * bench's CPU legs, never by the CUDA product path, and sharing no code,
 * header, table or constant generator with it.
 *
 * One step t:
 *   (1) a seed site i0 = floor(w0 * N / 2^32) and a new state
 *       s_new = (s_old + 1 + floor(w1 * (q-1) / 2^32)) mod q, s_old = s[i0],
 *       from words 0 and 1 of Philox counter (0, 0, t, 4);
 *   (2) the cluster is grown from i0: a neighbour in state s_old joins
 *       through the bond to a cluster site when that bond is active, i.e.
 *       u < thr with thr the SW threshold of Sec. 2 (p = 1 - exp(-1/T)) and
 *       u the bond's word of Philox counter (i>>1, t, 5), word
 *       2*(i&1)+dir, i the site owning the bond (its right / down bond);
 *   (3) every cluster site takes s_new.
 * Because every bond has one fixed word per step, the cluster is the
 * connected component of i0 among the active bonds between s_old sites,
 * whatever order the growth visits them in.  Requires N <= 2^32.
 */
#ifndef WOLFF_ORACLE_H
#define WOLFF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Step (1): seed site and new state of step t. */
void orc_wolff_seed(uint64_t L, uint32_t q, const uint8_t *s, uint64_t seed,
                    uint32_t t, uint64_t *i0, uint32_t *s_new);

/* One step (1)-(3) on s (in place); returns the cluster size. */
uint64_t orc_wolff_step(uint64_t L, uint32_t q, uint32_t thr, uint64_t seed,
                        uint32_t t, uint8_t *s);

/* Steps t0 .. t0+nsteps-1; sizes[k] (may be NULL) receives the cluster
 * size of step t0+k.  Returns 0, -1 on bad arguments, -2 on allocation
 * failure. */
int orc_wolff_run(uint64_t L, uint32_t q, double T, uint64_t seed,
                  uint8_t *s, uint32_t t0, uint32_t nsteps, uint64_t *sizes);

#ifdef __cplusplus
}
#endif
#endif
