/*
 * xy_oracle.h -- plain, slow, single-threaded CPU oracle for one
 * embedded-cluster Swendsen-Wang sweep of the 2D XY model with M equally
 * spaced angles (the M-state clock model; M = 256 stands in for the
 * continuous XY model).
 *
 * TEST INFRASTRUCTURE ONLY, like sw_oracle.h: loaded by tests/ and the
 * bench's CPU legs, never by the CUDA product path, and sharing no code,
 * header, table or constant generator with it.
 *
 * Method: Sec. 5 of Komura & Okabe names the extension of the multi-cluster
 * SW sweep to the classical XY model through Wolff's embedded clusters
 * (U. Wolff, PRL 62, 361 (1989)).  Each sweep:
 *   (0) a random unit vector r is drawn; every spin s_i is split into its
 *       component sigma_i = s_i . r along r and the rest, and the model
 *       restricted to the signs of sigma is an Ising model with couplings
 *       J_ij = |sigma_i sigma_j| (H = -sum s_i . s_j, J = 1);
 *   (1) a bond is active with probability 1 - exp(-2 beta sigma_i sigma_j)
 *       when sigma_i sigma_j > 0, never otherwise;
 *   (2) clusters of active bonds are labelled exactly as in the Potts sweep
 *       (root = smallest site index);
 *   (3) every cluster is reflected across the line perpendicular to r
 *       (s -> s - 2 (s . r) r) with probability 1/2.
 *
 * Conventions fixed here (both sides follow them bit for bit):
 *   - spin k in 0..M-1 is the angle 2 pi k / M, stored as one byte; M in
 *     2..256.
 *   - r is at angle pi j / M - pi / 2 with j = pick(w, M), w the Philox word
 *     0 of counter (0, 0, sweep, 3) (same key as every other stream).  The
 *     reflection then maps k to (j - k) mod M, so the angle set is closed
 *     under it, and sigma_i = -sin(pi a_i / M) with a_i = (2 k_i - j) mod 2M.
 *   - sign: sigma_i < 0 for 0 < a_i < M, > 0 for a_i > M, 0 for a_i in
 *     {0, M}; |sigma_i| = sin(pi c_i / M) with c_i = min(a_i mod M,
 *     M - a_i mod M) in 0..floor(M/2).
 *   - thresholds tt[c][c'] = floor((1 - exp(-2 sin(pi c/M) sin(pi c'/M) / T))
 *     * 2^32), clamped to 2^32 - 1, (floor(M/2)+1)^2 of them, row-major;
 *     a bond is active iff the two signs are equal and nonzero and
 *     u < tt[c_i][c_j], u the same Philox bond word as in the Potts sweep.
 *   - the coin of a cluster is pick(w, 2), w the word the Potts sweep uses
 *     for the new state of the same root (counter (root, sweep, 1), word 0);
 *     coin 1 reflects.
 *   - measurement of a configuration: n[k] = sites at angle k, and
 *     D[d] = bonds (right and down, 2N in all) whose angle difference is
 *     +-d mod M, d in 0..floor(M/2).  Energy E = -sum_d D[d] cos(2 pi d/M).
 */
#ifndef XY_ORACLE_H
#define XY_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Step (0): the axis index j of a sweep. */
uint32_t orc_xy_axis(uint64_t seed, uint32_t sweep, uint32_t M);

/* The bond threshold table, (M/2 + 1)^2 entries (M/2 rounded down). */
void orc_xy_thresholds(uint32_t M, double T, uint32_t *tt);

/* Step (1): b[i] = ORC_RIGHT / ORC_DOWN bits of the bonds site i owns. */
void orc_xy_bonds(uint64_t L, uint32_t M, const uint8_t *s,
                  const uint32_t *tt, uint32_t j, uint64_t seed,
                  uint32_t sweep, uint8_t *b);

/* Step (3): reflect every cluster whose root's coin is 1 (in place). */
void orc_xy_flip(uint64_t L, uint32_t M, uint32_t j, uint64_t seed,
                 uint32_t sweep, const uint32_t *root, uint8_t *s);

/* Measurement: D[0..M/2] and n[0..M-1] of configuration s. */
void orc_xy_measure(uint64_t L, uint32_t M, const uint8_t *s, uint64_t *D,
                    uint64_t *n);

/* Sweeps sweep0 .. sweep0+nsweeps-1 on s (in place); entry k of the series
 * (D_series: nsweeps x (M/2+1), n_series: nsweeps x M; either may be NULL)
 * holds the configuration after sweep sweep0+k.  Returns 0, -1 on bad
 * arguments, -2 if memory could not be allocated. */
int orc_xy_run(uint64_t L, uint32_t M, double T, uint64_t seed, uint8_t *s,
               uint32_t sweep0, uint32_t nsweeps, uint64_t *D_series,
               uint64_t *n_series);

#ifdef __cplusplus
}
#endif
#endif
