/*
 * sw_oracle.h -- plain, slow, single-threaded CPU oracle for one
 * Swendsen-Wang (SW) sweep of the periodic 2D q-state Potts model.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * bench's CPU-baseline / reference leg may load this library.  The CUDA
 * product path never links, loads or calls it, and this file shares no code,
 * header, table or constant generator with that path.
 *
 * Method (Komura & Okabe, "Multi-GPU-based Swendsen-Wang multi-cluster
 * algorithm for the simulation of two-dimensional q-state Potts model",
 * Sec. 2, Eq. 1 and the three SW steps that follow it):
 *   (1) bonds between nearest-neighbour sites are activated depending on T,
 *   (2) the active bonds partition the lattice into clusters, labelled after
 *       Hoshen and Kopelman: a cluster's label is the smallest label of
 *       its sites,
 *   (3) every cluster is set to one of the q states uniformly at random.
 * Measurement of energy and magnetisation follows Sec. 4 (the update plus
 * measurement column of Table 1).
 *
 * Conventions fixed here (the paper is silent on them; both sides follow
 * them so the GPU path must reproduce every configuration bit for bit):
 *   - H = -J sum delta(s_i, s_j), J = 1, spins stored 0..q-1 (paper's state
 *     S = s + 1; Eq. 1's "-1" only shifts H by the bond count).
 *   - site i = y*L + x; each site owns its right (+x) and down (+y) bond,
 *     periodic, so there are always 2N bonds (a multigraph for L = 2).
 *   - bond probability p = 1 - exp(-1/T); integer threshold
 *     thr = floor(p * 2^32) clamped to 2^32-1; active iff spins equal and
 *     u < thr (strict), u a 32-bit Philox word.
 *   - Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with
 *     key = (seed_lo, seed_hi) and 4-word counters:
 *       bonds  : ctr = (lo(i>>1), hi(i>>1), sweep, 0), word 2*(i&1)+dir
 *       spins  : ctr = (lo(r),    hi(r),    sweep, 1), word 0, r = root
 *       init   : ctr = (lo(i>>2), hi(i>>2), 0,     2), word i&3
 *   - a 32-bit word w picks state floor(w*q / 2^32).
 *   - the root of a cluster is its minimum site index (the Hoshen-Kopelman label).
 *   - E_sat = number of satisfied bonds (0..2N); n[s] = sites in state s.
 */
#ifndef SW_ORACLE_H
#define SW_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_RIGHT = 1, ORC_DOWN = 2 };

/* Philox4x32 with 10 rounds: out = Philox(key, ctr). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]);

/* The same for n inputs: in[6i .. 6i+3] counter, in[6i+4 .. 6i+5] key,
 * out[4i .. 4i+3] the words (one call per input, for tests). */
void orc_philox_many(uint64_t n, const uint32_t *in, uint32_t *out);

/* Integer bond threshold floor((1 - exp(-1/T)) * 2^32), clamped. */
uint32_t orc_threshold(double T);

/* Uniform pick of one of q states from a 32-bit word: floor(w*q/2^32). */
uint32_t orc_pick(uint32_t w, uint32_t q);

/* Initial spins s[i], i < L*L, drawn from the init stream. */
void orc_init_spins(uint64_t L, uint32_t q, uint64_t seed, uint8_t *s);

/* Step (1): b[i] = ORC_RIGHT / ORC_DOWN bits of the bonds site i owns. */
void orc_bonds(uint64_t L, const uint8_t *s, uint32_t thr, uint64_t seed,
               uint32_t sweep, uint8_t *b);

/* Step (2): Hoshen-Kopelman labelling of the bond field b.  On return
 * root[i] is the minimum site index of i's cluster.  Requires L*L <= 2^32.
 * Returns 0, or -1 if L is out of range. */
int orc_label(uint64_t L, const uint8_t *b, uint32_t *root);

/* Step (3): every site takes its cluster's new state, drawn once per root.
 * s is overwritten in place. */
void orc_recolor(uint64_t L, uint32_t q, uint64_t seed, uint32_t sweep,
                 const uint32_t *root, uint8_t *s);

/* Measurement: satisfied-bond count and per-state occupation counts. */
void orc_measure(uint64_t L, uint32_t q, const uint8_t *s, uint64_t *E_sat,
                 uint64_t *n);

/* Run sweeps sweep0 .. sweep0+nsweeps-1 on s (in place).  If E_series /
 * n_series are non-NULL, entry k holds the observables of the configuration
 * after sweep sweep0+k (n_series is nsweeps x q).  Returns 0, -1 on bad
 * arguments, -2 if memory could not be allocated. */
int orc_run(uint64_t L, uint32_t q, double T, uint64_t seed, uint8_t *s,
            uint32_t sweep0, uint32_t nsweeps, uint64_t *E_series,
            uint64_t *n_series);

#ifdef __cplusplus
}
#endif
#endif
