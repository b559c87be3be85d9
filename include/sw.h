/*
 * sw.h -- C ABI of the GB300 Swendsen-Wang library (libswgb.so).
 *
 * One Swendsen-Wang (SW) multi-cluster sweep of the periodic 2D q-state
 * Potts model H = -J sum_<ij> delta(s_i, s_j), J = 1 (Komura & Okabe,
 * Sec. 2, Eq. 1 up to the constant -J per bond), on one GPU:
 *   (1) bond activation between equal nearest-neighbour spins with
 *       probability p = 1 - exp(-1/T)                       (Sec. 2, step 1)
 *   (2) connected-component labelling of the bond graph; a cluster's label
 *       is its smallest site index, the Hoshen-Kopelman label          
 *                                                          (Sec. 2, step 2)
 *   (3) a uniformly random new state per cluster           (Sec. 2, step 3)
 *   (4) integer energy / magnetisation reductions (update plus measurement,
 *       Sec. 4, Table 1).
 *
 * Conventions (shared with the CPU oracle so every configuration is
 * reproduced bit for bit):
 *   - spins are uint8 in 0..q-1, row-major, site i = y*L + x, L*L bytes;
 *   - each site owns its right (+x) and down (+y) bond (periodic), so there
 *     are 2N bonds; the packed bond lattice stores 2 bits per site
 *     (bit 0 right, bit 1 down), 4 sites per byte, rows padded to
 *     ceil(L/4) bytes: byte [y*ceil(L/4) + x/4], bits 2*(x%4)..;
 *   - thr = floor(p * 2^32) clamped to 2^32-1; a bond is active iff the two
 *     spins are equal and u < thr for its Philox word u;
 *   - Philox4x32-10 (Salmon et al., SC'11), key = (seed_lo, seed_hi),
 *     counters (lo, hi, sweep, domain): bonds (i>>1, sweep, 0) word
 *     2*(i&1)+dir; new state of the cluster with root r (r, sweep, 1) word 0;
 *     initial spins (i>>2, 0, 2) word i&3; a word w picks floor(w*q/2^32);
 *   - E_sat = satisfied bonds (0..2N); the paper's energy is -E_sat (Eq. 1
 *     without the constant) and 2N - E_sat with it; n[s] = sites in state s.
 *
 * Errors: every call returns SW_OK (0) or a negative SW_ERR_* code.  Errors
 * on a handle are sticky: once a call fails with SW_ERR_CUDA / SW_ERR_DEVICE
 * the handle refuses further work; sw_strerror() names every code.
 * Ownership: the library owns all device memory of a handle (allocated at
 * create through the allocator installed with sw_set_allocator, cudaMalloc
 * by default) and frees it in sw_destroy.  Host buffers passed in are owned
 * by the caller and only read/written during the call.  Device buffers
 * passed in must stay valid until the work enqueued on the handle's stream
 * has completed.  A handle is not thread-safe; distinct handles are.
 * All work is enqueued on the handle's stream (sw_bind_stream; default: the
 * legacy default stream); calls that return host data synchronise it.
 */
#ifndef SWGB_SW_H
#define SWGB_SW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SW_OK 0
#define SW_ERR_INVAL (-1)   /* bad argument (L < 2, q not in [2,255], T <= 0 or
                               not finite, null pointer, size mismatch, ...) */
#define SW_ERR_NOMEM (-2)   /* device or host allocation failed */
#define SW_ERR_CUDA (-3)    /* a CUDA runtime call failed */
#define SW_ERR_TIMEOUT (-4) /* a bounded device loop hit its iteration cap */
#define SW_ERR_STATE (-5)   /* call not valid in the handle's state */
#define SW_ERR_DEVICE (-6)  /* a device-side consistency check failed */
#define SW_ERR_RANGE (-7)   /* requested observables are not (or no longer)
                               held in the observable ring */

#define SW_INIT_RANDOM 0u   /* spins from the init stream (default) */
#define SW_INIT_ZERO 1u     /* all spins in state 0 */

typedef struct sw_sim sw_sim;

/* Observables of one configuration (Sec. 4: energy and magnetisation). */
typedef struct {
  uint64_t config; /* configuration index = sweeps applied since create */
  uint64_t E_sat;  /* satisfied bonds, 0..2N */
  uint32_t q;      /* number of states; n[0..q-1] are valid */
  uint32_t pad_;
  uint64_t n[256]; /* sites in each state */
} sw_obs;

/* Boundary-union schedules (Sec. 2 step (2), global part; Sec. 3's
 * boundary-only stage on one GPU): SW_MERGE_KERNEL unites the clusters
 * across tile edges in a kernel of its own after the labelling;
 * SW_MERGE_FUSED has the labelling do it: of the two tiles that share an
 * edge, the one that finishes second unites across it (an atomic counter
 * per edge decides, nothing waits).  Same results; the batch autotuner
 * times both. */
#define SW_MERGE_AUTO 0u
#define SW_MERGE_KERNEL 1u
#define SW_MERGE_FUSED 2u

/* Creation parameters; zero means "default" for every optional field. */
typedef struct {
  uint64_t L;           /* linear size, >= 2 (N = L*L sites) */
  uint32_t q;           /* states, 2..255 */
  uint32_t label_bits;  /* 0 = auto (32 if L <= 32768, else 64), 32 or 64:
                           width of the cluster labels (site indices) where
                           they are written out; 32 requires L*L <= 2^32.
                           Inside a sweep the labels are the site keys of
                           the global union-find's 64-bit nodes (one per
                           open tile root, 8 B x (2 tile_h + 256) per tile),
                           whatever this width */
  double T;             /* temperature in units of J, finite, > 0 */
  uint64_t seed;        /* Philox key */
  uint32_t tile_h;      /* labelling tile height: 0 = auto (16 up to L = 32,
                           32 up to 256, 64 up to 1024, else 128), or 16, 32,
                           64 or 128 (tile width is 128 sites); results do
                           not depend on it */
  uint32_t ring;        /* observable ring capacity in configurations,
                           0 = 1024 */
  uint32_t init;        /* SW_INIT_RANDOM or SW_INIT_ZERO */
  uint32_t store_bonds; /* 1 = keep the packed bond lattice of the latest
                           sweep (sw_bonds); costs 0.25 B/site per sweep */
  uint32_t measure;     /* 0 = default (on); 2 = off: sweeps record no
                           observables (update only, Sec. 4 Table 1) */
  uint32_t walk_cap;    /* 0 = default (2^24): bound on the steps of one walk
                           through the global union-find; a sweep whose walk
                           runs into it reports SW_ERR_TIMEOUT (sw_sync,
                           sw_measure) and the handle refuses further work.
                           A small value is for tests of that path. */
  uint32_t merge;       /* boundary-union schedule, SW_MERGE_*: 0 = auto
                           (SW_MERGE_KERNEL, the faster one for a single
                           lattice on GB300), results do not depend on it */
  uint32_t reserved[1];
} sw_params;

/* Library-wide device allocator (e.g. a framework's caching allocator).
 * alloc returns a device pointer of at least `bytes` bytes (256-byte
 * aligned) or NULL; free releases it.  Applies to handles created after the
 * call.  Passing NULL for both restores cudaMalloc/cudaFree. */
typedef void *(*sw_alloc_fn)(size_t bytes, void *ctx);
typedef void (*sw_free_fn)(void *ptr, size_t bytes, void *ctx);
int sw_set_allocator(sw_alloc_fn alloc, sw_free_fn free_fn, void *ctx);

/* Create a simulation of the L x L lattice at temperature T with Philox key
 * `seed`; spins start from the init stream, the sweep counter at 0.
 * (The problem statement of Sec. 2: L, q, T, periodic boundaries.) */
int sw_create(uint64_t L, uint32_t q, double T, uint64_t seed, sw_sim **out);
/* Same with every option of sw_params. */
int sw_create_ex(const sw_params *params, sw_sim **out);
/* Free the handle and all its device memory (synchronises its stream). */
void sw_destroy(sw_sim *sim);

/* Enqueue later work on `stream` (a cudaStream_t; NULL = default stream). */
int sw_bind_stream(sw_sim *sim, void *stream);

/* Run n full SW sweeps (steps 1-3 of Sec. 2 plus the fused measurement of
 * each configuration the sweeps read).  Asynchronous on the handle's
 * stream. */
int sw_sweep(sw_sim *sim, uint64_t n);

/* Observables of the current configuration (synchronises). */
int sw_measure(sw_sim *sim, sw_obs *out);

/* Observables of configurations first .. first+count-1 (configuration c =
 * the state after c sweeps).  E receives count values, n receives count*q
 * values (row-major); either may be NULL.  Fails with SW_ERR_RANGE if a
 * configuration was not measured (created before the last sw_set_spins /
 * sw_set_sweep, swept with measurement off) or has left the ring.
 * Synchronises. */
int sw_series(sw_sim *sim, uint64_t first, uint64_t count, uint64_t *E,
              uint64_t *n);

/* Copy the L*L spins out to dst (host, or device if dst_on_device).
 * n must equal L*L.  Synchronises for a host destination. */
int sw_spins(sw_sim *sim, uint8_t *dst, uint64_t n, int dst_on_device);
/* Replace the configuration from host or device memory.  Values must be
 * < q: they are checked on the device after the copy; on failure the call
 * returns SW_ERR_INVAL and the handle refuses to sweep (SW_ERR_STATE) until
 * a valid configuration is set.  The sweep counter is unchanged; the call
 * synchronises the handle's stream (the caller may reuse src on return). */
int sw_set_spins(sw_sim *sim, const uint8_t *src, uint64_t n,
                 int src_on_device);

/* Packed bond lattice of the most recent sweep (layout above); nbytes must
 * equal L*ceil(L/4).  Requires store_bonds = 1. */
int sw_bonds(sw_sim *sim, uint8_t *dst, uint64_t nbytes, int dst_on_device);

/* One call from a host configuration to observables: uploads the N spins
 * from `src` (host memory; page-locked memory lets the upload overlap) on a
 * stream of the handle's own in at most 16 bands of tile rows (one tile row
 * first, then doubling up to an eighth of the lattice, each copy carrying
 * its band's halo row), runs `nsweeps` sweeps of which the first labels
 * each band as soon as its copy has landed, and, if `out` is not NULL,
 * fills it as sw_measure (the observables of the resulting
 * configuration).  The uploaded configuration becomes configuration `sweep`
 * (as after sw_set_spins).  The banded labelling checks every spin: a spin
 * >= q gives SW_ERR_INVAL after the call, the lattice is then undefined and
 * sweeps return SW_ERR_STATE until a valid configuration is set.  Not
 * recorded by sw_profile.  Synchronises the handle's stream. */
int sw_sweep_host(sw_sim *sim, const uint8_t *src, uint64_t n,
                  uint64_t nsweeps, sw_obs *out);

/* Sweep counter (the Philox "sweep" counter word of the next sweep); with
 * the spins it is the whole state of a run, so get + spins, then set +
 * set_spins, resumes a run bit for bit. */
int sw_get_sweep(const sw_sim *sim, uint64_t *sweep);
int sw_set_sweep(sw_sim *sim, uint64_t sweep);

/* Block until the handle's queued work is done; reports device-side errors
 * (SW_ERR_TIMEOUT / SW_ERR_DEVICE) raised by that work. */
int sw_sync(sw_sim *sim);

/* Static facts about a handle. */
typedef struct {
  uint64_t L;
  uint32_t q;
  uint32_t thr;          /* integer bond threshold in use */
  uint32_t label_bits;   /* 32 or 64 */
  uint32_t tile_w, tile_h;
  uint32_t ring;
  uint64_t device_bytes; /* device memory held by the handle */
  uint64_t tiles;
  uint32_t merge;        /* SW_MERGE_KERNEL or SW_MERGE_FUSED */
  uint32_t pad_;
} sw_info_t;
int sw_info(const sw_sim *sim, sw_info_t *out);

/* Integer bond threshold floor((1 - exp(-1/T)) * 2^32), clamped. */
int sw_threshold(double T, uint32_t *thr);

/* Step (2) alone, for a given bond lattice: label the packed bond lattice
 * `bonds` (device, layout above, L*ceil(L/4) bytes) and write, per site, the
 * smallest site index of its cluster to `roots` (device, L*L entries of
 * uint32 if label_bits == 32 (requires L*L <= 2^32), else uint64).
 * tile_h as in sw_params.  Scratch memory is taken from the allocator and
 * released before return; runs on `stream` and synchronises it. */
int sw_label_bonds(uint64_t L, const uint8_t *bonds, void *roots,
                   uint32_t label_bits, uint32_t tile_h, void *stream);

/* Per-kernel timing with CUDA events recorded on the handle's stream around
 * each launch of a sweep (bond+tile labelling, boundary merge, recolour),
 * for profiling the hot path from the caller's side.  enable = 1 starts
 * recording (clearing earlier totals), 0 stops.  sw_profile_read
 * synchronises and returns, per phase, the summed milliseconds and the
 * number of launches since recording started (arrays of `nphase` <= 3). */
int sw_profile(sw_sim *sim, int enable);
int sw_profile_read(sw_sim *sim, double *ms, uint64_t *launches, int nphase);

/* ---------------------------------------------------------------------------
 * Batched replicas (not in the paper: many independent lattices of uneven
 * L, q and T advanced together).  Every replica follows exactly the single-
 * lattice conventions above with its own Philox key, so replica r of a batch
 * reproduces sw_create(L[r], q[r], T[r], seed[r]) bit for bit.  All replicas'
 * tiles form one work list: a sweep of the whole batch is one persistent
 * labelling launch plus three short ones, replayed as a CUDA graph.
 * ------------------------------------------------------------------------- */
typedef struct sw_batch sw_batch;

typedef struct {
  uint32_t R;           /* replicas, >= 1 */
  uint32_t tile_h;      /* 0 = 64, or 16 / 32 / 64 / 128 (one tile height for
                           all) */
  const uint64_t *L;    /* host arrays of R entries: linear sizes (>= 2) */
  const uint32_t *q;    /*   states (2..255) */
  const double *T;      /*   temperatures (finite, > 0) */
  const uint64_t *seed; /*   Philox keys */
  uint32_t ring;        /* per-replica observable ring, 0 = 64 configurations */
  uint32_t init;        /* SW_INIT_RANDOM or SW_INIT_ZERO */
  uint32_t measure;     /* 0 = on, 2 = off */
  uint32_t graph;       /* 0 = replay sweeps as a CUDA graph, 2 = plain launches */
  uint32_t merge;       /* boundary-union schedule, SW_MERGE_* (0 = auto:
                           SW_MERGE_KERNEL) */
  uint32_t reserved[3];
} sw_batch_params;

typedef struct {
  uint32_t R;
  uint32_t tile_h;
  uint64_t tiles;        /* tiles of all replicas */
  uint64_t sites;        /* sum of L*L */
  uint64_t device_bytes; /* device memory held (one arena) */
  uint32_t label_bits;   /* 32, or 64 if any L > 32768 */
  uint32_t graph;        /* 1 if sweeps replay a CUDA graph */
  uint32_t merge;        /* SW_MERGE_KERNEL or SW_MERGE_FUSED */
  uint32_t pad_;
} sw_batch_info_t;

/* Create R replicas (host arrays are read during the call only); one device
 * arena from the installed allocator.  Errors as for sw_create_ex. */
int sw_batch_create(uint32_t R, const uint64_t *L, const uint32_t *q,
                    const double *T, const uint64_t *seed, sw_batch **out);
int sw_batch_create_ex(const sw_batch_params *params, sw_batch **out);
void sw_batch_destroy(sw_batch *batch);
int sw_batch_bind_stream(sw_batch *batch, void *stream);
/* n sweeps of every replica (asynchronous on the batch's stream). */
int sw_batch_sweep(sw_batch *batch, uint64_t n);
/* Per-replica observables, configuration series and spins, as sw_measure /
 * sw_series / sw_spins / sw_set_spins for replica r < R. */
int sw_batch_measure(sw_batch *batch, uint32_t r, sw_obs *out);
int sw_batch_series(sw_batch *batch, uint32_t r, uint64_t first,
                    uint64_t count, uint64_t *E, uint64_t *n);
int sw_batch_spins(sw_batch *batch, uint32_t r, uint8_t *dst, uint64_t n,
                   int dst_on_device);
int sw_batch_set_spins(sw_batch *batch, uint32_t r, const uint8_t *src,
                       uint64_t n, int src_on_device);
/* Sweeps applied to every replica since creation. */
int sw_batch_get_sweep(const sw_batch *batch, uint64_t *sweep);
int sw_batch_sync(sw_batch *batch);
int sw_batch_info(const sw_batch *batch, sw_batch_info_t *out);
/* Per-phase event timing of batch sweeps (as sw_profile; profiled sweeps
 * are launched directly, not through the graph). */
int sw_batch_profile(sw_batch *batch, int enable);
int sw_batch_profile_read(sw_batch *batch, double *ms, uint64_t *launches,
                          int nphase);
int sw_batch_last_error(const sw_batch *batch);

/* The paper's labeller (Sec. 2: label equivalence after Kalentev et al.),
 * for comparison with sw_label_bonds: every site starts labelled with its
 * own index; a scanning pass lowers label[label[i]] to the smallest label
 * among i's active-bond neighbours, an analysis pass makes every site adopt
 * the end of its label chain; both repeat until a scan changes nothing.
 * Same inputs and result as sw_label_bonds (bit-identical roots).
 * *iterations (may be NULL) receives the number of scan+analysis rounds,
 * the last one being the round that found nothing to change; more than
 * max_iter rounds (0 = no practical limit) returns SW_ERR_TIMEOUT.  Reads a
 * flag back after every round; synchronises `stream`. */
int sw_label_bonds_le(uint64_t L, const uint8_t *bonds, void *roots,
                      uint32_t label_bits, uint32_t max_iter,
                      uint32_t *iterations, void *stream);

/* The paper's multi-GPU labelling (Sec. 3), emulated on one GPU for
 * comparison: the lattice is split into (L/sub)^2 sub-lattices of sub x sub
 * sites (sub must divide L).  Stage 1 labels each sub-lattice by label
 * equivalence, ignoring bonds that leave it; stage 2 iterates scanning and
 * analysis on a label_total table over the boundary layers only (the
 * bonds crossing sub-lattice boundaries); finally every site adopts
 * label_total of its stage-1 label.  Same inputs and result as
 * sw_label_bonds (bit-identical roots).  iterations (may be NULL) receives
 * {stage-1 rounds, stage-2 rounds}; stage_ms (may be NULL) receives the
 * CUDA-event times in ms of {stage 1, stage 2, final update}, each round's
 * host convergence check included.  A scratch table of N labels is
 * allocated through the library's allocator for label_total (SW_ERR_NOMEM
 * if that fails).  Synchronises `stream`. */
int sw_label_bonds_2stage(uint64_t L, uint64_t sub, const uint8_t *bonds,
                          void *roots, uint32_t label_bits,
                          uint32_t *iterations, float *stage_ms, void *stream);

/* Step (2) alone, like sw_label_bonds, for callers that cannot allocate
 * device memory: a program whose GPU memory belongs to a framework pool it
 * cannot borrow from, or one that must not call cudaMalloc/cudaFree once
 * running (they synchronise the whole device).  The paper has no
 * counterpart; this is a deployment convenience.
 * Same inputs and result as sw_label_bonds with label_bits = 32 (bonds and
 * roots are device pointers, roots receives L*L uint32), but it allocates
 * nothing: its working memory is one fixed 8 MiB __device__ array in the
 * library, held by every GPU that loads the library until the process exits.
 * Lattices larger than SW_LABEL_STATIC_MAX_L are rejected with
 * SW_ERR_INVAL.  The first call on a device looks up that array's device
 * address (and configures the kernels); make that first call before any
 * stream capture.  All calls share the array and the call clears what must
 * start at zero, so calls that overlap on the GPU (other threads, other
 * streams) race and must be serialised by the caller.  Runs on `stream` and
 * synchronises it. */
#define SW_LABEL_STATIC_MAX_L 1024u
int sw_label_bonds_static(uint64_t L, const uint8_t *bonds, uint32_t *roots,
                          uint32_t tile_h, void *stream);

/* ---------------------------------------------------------------------------
 * XY model, embedded-cluster sweep (Sec. 5: the extension of the sweep to
 * the classical XY model through Wolff's embedded clusters), with M equally
 * spaced angles (spin k in 0..M-1 is the angle 2 pi k / M, one byte; M in
 * 2..256, M = 256 standing in for continuous angles).  H = -sum cos(theta_i
 * - theta_j), J = 1.  One sweep:
 *   (0) embedding axis r at angle pi j / M - pi / 2, j = floor(w M / 2^32)
 *       with w word 0 of Philox counter (0, 0, sweep, 3);
 *   (1) the bond (i, k) is active iff sigma_i sigma_k > 0 (sigma = s . r)
 *       and u < tt[c_i][c_k], u the Potts sweep's bond word, c the fold
 *       index of |sigma| = sin(pi c / M) and tt the sw_xy_thresholds table;
 *   (2) clusters labelled as in the Potts sweep (root = smallest index);
 *   (3) each cluster reflected, k -> (j - k) mod M, iff its coin
 *       floor(w 2 / 2^32) is 1, w the Potts state word of its root.
 * Measurement of a configuration: D[d], d in 0..M/2, bonds (right and down,
 * 2N in all) with angle difference +-d mod M, and n[k], sites at angle k;
 * E = -sum_d D[d] cos(2 pi d / M).
 * ------------------------------------------------------------------------- */
typedef struct sw_xy sw_xy;
typedef struct {
  uint64_t L;          /* linear size, 2 .. 2^20 */
  uint32_t M;          /* angles, 2 .. 256 */
  uint32_t label_bits; /* 0 = auto (32 up to L = 32768, else 64), 32, 64 */
  double T;            /* temperature > 0 */
  uint64_t seed;       /* Philox key */
  uint32_t tile_h;     /* 0 = auto (as sw_params), 16, 32, 64 or 128 */
  uint32_t ring;       /* configurations whose observables are kept (0 = 1024) */
  uint32_t init;       /* SW_INIT_RANDOM (angles from the init stream) or SW_INIT_ZERO */
  uint32_t measure;    /* 0: measure after every sweep; 2: only on request */
  uint32_t reserved[4];
} sw_xy_params;
/* Bond thresholds floor((1 - exp(-2 sin(pi c/M) sin(pi d/M) / T)) 2^32),
 * clamped to 2^32 - 1, into tt[c * (M/2+1) + d] (host array of
 * (M/2+1)^2 entries; M/2 rounded down).  Host only. */
int sw_xy_thresholds(uint32_t M, double T, uint32_t *tt);
/* Allocates the lattice (N bytes), the per-site codes (2N), the global
 * union-find (8 B per possible open tile root), per-tile records and the ring through
 * the installed allocator; uploads the threshold table; measures the
 * initial configuration (measure = 0).  SW_ERR_INVAL for parameters out of
 * range (label_bits 32 with L*L > 2^32 included), SW_ERR_NOMEM, SW_ERR_CUDA.
 * *out is NULL on failure; the handle owns all device memory. */
int sw_xy_create(const sw_xy_params *prm, sw_xy **out);
void sw_xy_destroy(sw_xy *xy);
int sw_xy_bind_stream(sw_xy *xy, void *stream);
/* n sweeps (asynchronous; with measurement on, five kernels per sweep:
 * the four of the Potts sweep in their XY form and the measurement). */
int sw_xy_sweep(sw_xy *xy, uint64_t n);
int sw_xy_sync(sw_xy *xy);
/* Observables of configurations first .. first+count-1 (configuration c is
 * the one after c sweeps): D (count x (M/2+1)) and n (count x M) host
 * arrays, either may be NULL.  SW_ERR_RANGE outside the ring window, before
 * the last sw_xy_set_spins, or (measurement off) for anything but the
 * current configuration.  Synchronises the stream. */
int sw_xy_series(sw_xy *xy, uint64_t first, uint64_t count, uint64_t *D,
                 uint64_t *n);
/* Copy the N = L*L angles out / in (host or device buffer).  set_spins
 * validates on the device: an angle >= M gives SW_ERR_INVAL and sweeps
 * return SW_ERR_STATE until a valid configuration is set. */
int sw_xy_spins(sw_xy *xy, uint8_t *dst, uint64_t n, int dst_on_device);
int sw_xy_set_spins(sw_xy *xy, const uint8_t *src, uint64_t n,
                    int src_on_device);
int sw_xy_get_sweep(const sw_xy *xy, uint64_t *sweep);
/* Per-phase CUDA-event timing of sweeps: phases labelling, merge+resolve,
 * reflection, measurement (as sw_profile). */
int sw_xy_profile(sw_xy *xy, int enable);
int sw_xy_profile_read(sw_xy *xy, double *ms, uint64_t *launches, int nphase);
int sw_xy_last_error(const sw_xy *xy);

/* ---------------------------------------------------------------------------
 * Wolff single-cluster update of the q-state Potts model (the comparison
 * workload of the paper's related work, Sec. 1: one cluster per step, grown
 * by processing the newly added spins in parallel).  One step t:
 *   (1) seed i0 = floor(w0 N / 2^32), new state s_new = (s_old + 1 +
 *       floor(w1 (q-1) / 2^32)) mod q, from words 0 and 1 of Philox counter
 *       (0, 0, t, 4) (key = seed);
 *   (2) the cluster: the connected component of i0 among the bonds between
 *       sites in state s_old whose word u < thr (thr as sw_threshold; u the
 *       word 2*(o&1)+dir of counter (o>>1, t, 5), o the site owning the bond,
 *       dir 0 right / 1 down);
 *   (3) every cluster site takes s_new.
 * L is at most 32768 (site indices below 2^30).  Three kernels per step.
 * ------------------------------------------------------------------------- */
typedef struct sw_wolff sw_wolff;
/* init: SW_INIT_RANDOM (the Potts init stream) or SW_INIT_ZERO; ring: steps
 * whose cluster sizes are kept (0 = 1024).  Allocates N spins, an N-slot
 * queue of uint32 site indices and the labelling buffers of the default
 * mode. */
int sw_wolff_create(uint64_t L, uint32_t q, double T, uint64_t seed,
                    uint32_t init, uint32_t ring, sw_wolff **out);
/* (Create: SW_ERR_INVAL for L outside 2..32768, q outside 2..255, T <= 0 or
 * not finite, a bad init; SW_ERR_NOMEM, SW_ERR_CUDA; *out NULL on failure.
 * All calls on a handle share its stream; errors from the device are sticky
 * per handle.) */
void sw_wolff_destroy(sw_wolff *w);
int sw_wolff_bind_stream(sw_wolff *w, void *stream);
/* n steps (asynchronous). */
int sw_wolff_step(sw_wolff *w, uint64_t n);
/* Reads the device error word: SW_ERR_TIMEOUT if a growth wait hit its
 * bound, SW_ERR_DEVICE on another device-side failure. */
int sw_wolff_sync(sw_wolff *w);
/* Cluster sizes of steps first .. first+count-1 (0-based) into a host
 * array; SW_ERR_RANGE outside the ring window.  Synchronises. */
int sw_wolff_sizes(sw_wolff *w, uint64_t first, uint64_t count,
                   uint64_t *sizes);
/* Copy the N spins out / in (host or device buffer); set_spins leaves the
 * lattice unchanged and returns SW_ERR_INVAL if a spin is >= q. */
int sw_wolff_spins(sw_wolff *w, uint8_t *dst, uint64_t n, int dst_on_device);
int sw_wolff_set_spins(sw_wolff *w, const uint8_t *src, uint64_t n,
                       int src_on_device);
int sw_wolff_get_step(const sw_wolff *w, uint64_t *step);
/* How the cluster is found (same result either way).  SW_WOLFF_LABEL
 * (default, tens of times faster on critical clusters): the step's active
 * bonds over the whole lattice are labelled by the SW sweep's tile
 * union-find and the sites with the seed's root flipped (the
 * connected-component route of the related work); its buffers (about 11 B
 * per site) are taken by sw_wolff_create.  SW_WOLFF_GROW: persistent warps
 * grow the cluster from a site queue, work proportional to the cluster but
 * bound by the latency of the growth front; kept as the order-independent
 * reference form of the step. */
#define SW_WOLFF_GROW 0
#define SW_WOLFF_LABEL 1
int sw_wolff_set_mode(sw_wolff *w, int mode);
/* Growth mode: the number of idle polls (each followed by a back-off of up to
 * 1 us) after which a growth warp that finds no work, while the cluster is
 * not complete, gives up; the step then reports SW_ERR_TIMEOUT (sw_wolff_sync)
 * and the handle refuses further steps.  0 restores the default (2^22).  A
 * small value is for tests of that path: no wait of the growth is unbounded. */
int sw_wolff_set_wait_limit(sw_wolff *w, uint32_t idle_polls);

/* ---------------------------------------------------------------------------
 * Surrogate network (not in the paper): a 3 -> 64 -> 64 -> 64 -> 4 tanh MLP
 * with bfloat16 weights and fp32 accumulation that maps (q, log2 L, T/T_c)
 * to standardised observables and only places temperature grids.
 * Parameters are SW_MLP_PARAMS floats, flat, in the order W1[64][3], b1[64],
 * W2[64][64], b2[64], W3[64][64], b3[64], W4[4][64], b4[4]; every parameter
 * and every layer input is rounded to bfloat16 before use.  X is B x 3,
 * outputs / targets / mask are B x 4, row-major fp32 device arrays.
 * ------------------------------------------------------------------------- */
#define SW_MLP_PARAMS 8836u
typedef struct sw_mlp sw_mlp;
/* init: host array of SW_MLP_PARAMS fp32 master weights (copied). */
int sw_mlp_create(const float *init, sw_mlp **out);
void sw_mlp_destroy(sw_mlp *mlp);
int sw_mlp_bind_stream(sw_mlp *mlp, void *stream);
/* Y = f(X) for B rows (device pointers; asynchronous).  sw_mlp_predict is
 * the same call under the name used for inference. */
int sw_mlp_forward(sw_mlp *mlp, const float *X, uint32_t B, float *Y);
int sw_mlp_predict(sw_mlp *mlp, const float *X, uint32_t B, float *Y);
/* Gradient of loss = sum(mask*(f(X)-Yt)^2)/(4B) (mask NULL = all ones) into
 * grad (device, SW_MLP_PARAMS floats) and the loss into *loss (device, may be
 * NULL); the rounding is treated as the identity in the backward pass. */
int sw_mlp_gradients(sw_mlp *mlp, const float *X, const float *Yt,
                     const float *mask, uint32_t B, float *grad, float *loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on the
 * fp32 master weights with learning rate lr; refreshes the bfloat16 copy. */
int sw_mlp_train_step(sw_mlp *mlp, const float *X, const float *Yt,
                      const float *mask, uint32_t B, float lr, float *loss);
/* Copy the fp32 master weights and/or their bfloat16 copy to host arrays
 * (either may be NULL); synchronises.  set_params also resets Adam. */
int sw_mlp_get_params(sw_mlp *mlp, float *master, uint16_t *bf16);
int sw_mlp_set_params(sw_mlp *mlp, const float *master);

/* Name of an error code. */
const char *sw_strerror(int code);
/* Last error recorded on the handle (SW_OK if none). */
int sw_last_error(const sw_sim *sim);

#ifdef __cplusplus
}
#endif
#endif /* SWGB_SW_H */
