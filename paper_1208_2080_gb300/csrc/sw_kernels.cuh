// sw_kernels.cuh -- sm_103a kernels of one Swendsen-Wang sweep.
//
// A sweep is four launches over a tiling of the L x L lattice into
// 128 x TH tiles (tile t = ty*ntx + tx, origin (128*tx, TH*ty); the last
// tile row/column is ragged when TH or 128 does not divide L):
//
//   k_label_tile  (persistent; a CTA per tile at a time)  Sec. 2 steps
//       (1)+(2), tile-local part: stage the tile's uint8 spins plus a
//       one-site right/down halo in shared memory; draw the bonds (Philox,
//       one call per two sites); measure E_sat / n[s] of the configuration
//       it reads (Sec. 4); label the tile with a shared-memory union-find:
//       horizontal runs inside a warp's 128-site row come from one
//       __ballot_sync, vertical bonds are atomicMin unions (redundant ones
//       between the same two runs skipped); a cluster that touches the tile
//       edge is "open", the others are complete and get their new state
//       here (Sec. 2 step (3)), drawn once per cluster from their root =
//       smallest site index.  Per site it writes a 16-bit code: 0x8000|state
//       for a closed cluster, the slot of its open root otherwise.  For the
//       boundary pass it writes the open slots of the four edge lines, the
//       cross-edge bond bits, and initialises the open roots' nodes of the
//       global union-find (below).
//   k_merge       Sec. 2 step (2), global part: the single-GPU analogue of
//       the paper's boundary-only inter-GPU labelling (Sec. 3): for every
//       active bond that crosses a tile edge (periodic wrap included) a
//       lock-free atomicMin union of the two open roots' nodes; lanes that
//       would repeat the same union are merged with __match_any_sync.
//   k_resolve     Sec. 2 step (3) for open clusters: each open local root
//       finds (and compresses to) its global root and draws the cluster
//       state.
//   k_recolor     every site writes its new uint8 spin from its code.
//
// The XY form (kXY; Sec. 5, Wolff's embedded clusters) is the same sweep
// with the embedded bond rule in k_label_tile and reflections in
// k_recolor; clusters draw a coin (the state draw with q = 2).
//
// Union always links the larger root under the smaller one, so the final
// root of every cluster is its smallest site index -- the Hoshen-Kopelman
// label of Sec. 2 -- independent of the order in which the GPU
// happens to process unions.  That makes the result bit-exact with the
// sequential oracle.  Every union-find walk is bounded (kFindCap); a walk
// that hits the bound sets an error bit and stops instead of spinning.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "philox.cuh"

namespace swgb {

constexpr int kTW = 128;                  // tile width (32 lanes x 4 sites)
constexpr int kThreads = 512;             // threads per tile CTA
constexpr int kWarps = kThreads / 32;
constexpr int kSpPitch = 144;             // smem spin row: 128 sites, halo; 16-byte rows
constexpr uint32_t kOpen = 0x80000000u;   // smem root flag: cluster touches tile edge
constexpr uint32_t kIdx = 0x7FFFu;        // local index bits
constexpr uint16_t kClosed = 0x8000u;     // code flag: cluster complete in tile
constexpr uint32_t kFindCap = 1u << 24;   // bound on any global union-find walk
constexpr uint32_t kLocalCap = 1u << 16;  // bound on any shared-memory walk
constexpr int kMergeThreads = 256;

// kErrSpin: a spin >= q was read by a labelling that checks its input
// (BandSrc); the host reports it as an invalid configuration.
enum : uint32_t { kErrFind = 1u, kErrUnion = 2u, kErrLocal = 4u, kErrSpin = 8u };

__host__ __device__ constexpr int align16(int x) { return (x + 15) & ~15; }

// Per-tile record sizes.
template <int TH>
struct TileRec {
  static constexpr int kEdge = 2 * TH + 2 * kTW;           // u16: right col, left col, bottom, top
  static constexpr int kRightWords = (TH + 31) / 32;       // cross-right bits
  static constexpr int kBitWords = kRightWords + kTW / 32; // + cross-down bits
  static constexpr int kOpenCap = 2 * TH + 2 * kTW;        // open roots <= edge sites
};

// Tile CTA shape: a warp owns 4 consecutive rows, so a 128 x TH tile is
// labelled by TH/4 warps.
template <int TH>
struct TileCta {
  static constexpr int kRpw = 4;                 // rows per warp
  static constexpr int kWarps = TH / kRpw;       // warps per CTA
  static constexpr int kThreads = 32 * kWarps;
  static constexpr int kMinBlocks = 128 / TH;    // keeps the register budget at 64
};

// Shared-memory layout of k_label_tile.
template <int TH>
struct LabelSmem {
  static constexpr int kNW = TileCta<TH>::kWarps;
  static constexpr int kP = 0;                                     // u32 [kTW*TH] union-find
  static constexpr int kSpBuf = align16((TH + 1) * kSpPitch);      // one staged tile of spins
  static constexpr int kSp = kP + 4 * kTW * TH;                    // u8 [2][kSpBuf] double buffer
  static constexpr int kRbn = kSp + 2 * kSpBuf;                    // u8 [TH*32] right-bond nibbles
  static constexpr int kQ = align16(kRbn + TH * 32);               // u16 [kNW*kTW] task queues
  static constexpr int kCb = align16(kQ + 2 * kNW * kTW);          // u32 cross bits
  static constexpr int kCnt = align16(kCb + 4 * TileRec<TH>::kBitWords);  // u32 [kNW]
  static constexpr int kObs = align16(kCnt + 4 * kNW);             // u32 [1 + 256]
  static constexpr int kCl = align16(kObs + 4 * 257);              // u16 [kTW*TH] root lists
  static constexpr int kBytes = align16(kCl + 2 * kTW * TH);
  // XY form only: the bond thresholds of M <= 256 angles, lower triangle
  // (129 * 130 / 2 entries), after the Potts layout
  static constexpr int kXYTab = kBytes;
  static constexpr int kXYBytes = align16(kXYTab + 4 * (129 * 130 / 2));
};

struct Lattice {
  uint64_t L;
  uint32_t ntx, nty;  // tiles across / down
  uint64_t bp;        // packed-bond row pitch in bytes, ceil(L/4)
  uint32_t vec4;      // L % 4 == 0: rows start 4-byte aligned
  uint32_t ntiles;
  uint32_t ntx_m;     // floor(2^32 / ntx) (2^32 - 1 for ntx = 1): t / ntx by a multiply
  uint32_t xb;        // bits of a column index: the least b with 2^b >= L
  uint32_t db;        // bits of a global union-find node index, 0: nodes named by open slot
};

struct Bufs {
  uint8_t* spin;              // N spins
  uint16_t* code;             // N per-site codes
  uint8_t* bonds;             // packed bonds (out, or in for the given-bond mode) or null
  uint64_t* G;                // ntiles * kOpenCap nodes of the global union-find
  uint16_t* edge;             // ntiles * kEdge open slots of the edge sites
  uint32_t* ebits;            // ntiles * kBitWords
  uint32_t* ocnt;             // ntiles
  uint8_t* nso;               // ntiles * kOpenCap: new state of each open root
  unsigned long long* acc;    // [1 + q]: E_sat, n[q] of the configuration being measured
  unsigned long long* ring;   // [ring_cap][2 + q]: tag, E_sat, n[q]
  unsigned long long* ctl;    // [0] next sweep, [1] sweep being recoloured
  uint32_t* err;              // device error bits
  uint64_t seed;
  uint32_t thr, q;
  uint32_t ring_cap;
  uint32_t measure;           // 1: k_label_tile accumulates observables of its input
  uint32_t rk[20];            // Philox round keys of `seed` (see set_round_keys)
  uint32_t walk_cap;          // bound on a global union-find walk (0: kFindCap)
  uint32_t fuse;              // 1: the labeller unites across tile edges (no k_merge)
  uint32_t* ecnt;             // fuse: 2 * ntiles edge counters (right, bottom edge of each tile)
  // XY model (embedded clusters, M angles; q = 2 coins): 0 for Potts
  uint32_t M;
  const uint32_t* tt;         // bond thresholds by |sigma| fold indices (c >= d): tt[c(c+1)/2 + d]
};

// The ten Philox round keys of a seed: (lo, hi) + r * (Weyl constants).
__host__ __device__ inline void set_round_keys(Bufs& b) {
  uint32_t k0 = (uint32_t)b.seed, k1 = (uint32_t)(b.seed >> 32);
  for (int r = 0; r < 10; ++r) {
    b.rk[2 * r] = k0;
    b.rk[2 * r + 1] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// A replica of the batched runner: its buffers, geometry and first tile in
// the concatenated tile list.
struct Rep {
  Bufs b;
  Lattice lat;
  uint32_t tile0;
  uint32_t pad_;
};

// Tile sources: which lattice (and which of its tiles) a global tile id g
// names.  SingleSrc: one lattice, g is the tile.  BatchSrc: the tiles of R
// independent replicas (each with its own L, q, T, seed and buffers)
// concatenated, so one launch sweeps all of them.
struct SingleSrc {
  Bufs b;
  Lattice lat;
  static constexpr bool kMulti = false;
  static constexpr bool kCheck = false;
  __device__ __forceinline__ uint32_t ntiles() const { return lat.ntiles; }
  __device__ __forceinline__ uint32_t nreps() const { return 1; }
  __device__ __forceinline__ uint32_t rep(uint32_t) const { return 0; }
  __device__ __forceinline__ const Bufs& bufs(uint32_t) const { return b; }
  __device__ __forceinline__ const Lattice& lattice(uint32_t) const { return lat; }
  __device__ __forceinline__ uint32_t tile0(uint32_t) const { return 0; }
};

struct BatchSrc {
  const Rep* __restrict__ reps;
  const uint32_t* __restrict__ tile_rep;  // replica of each global tile
  uint32_t total;                         // tiles of all replicas
  uint32_t nrep;
  static constexpr bool kMulti = true;
  static constexpr bool kCheck = false;
  __device__ __forceinline__ uint32_t ntiles() const { return total; }
  __device__ __forceinline__ uint32_t nreps() const { return nrep; }
  __device__ __forceinline__ uint32_t rep(uint32_t g) const { return __ldg(tile_rep + g); }
  __device__ __forceinline__ const Bufs& bufs(uint32_t r) const { return reps[r].b; }
  __device__ __forceinline__ const Lattice& lattice(uint32_t r) const { return reps[r].lat; }
  __device__ __forceinline__ uint32_t tile0(uint32_t r) const { return reps[r].tile0; }
};

// BandSrc: tiles base .. base+count-1 of one lattice (whole tile rows), for
// a labelling that starts while later rows are still being uploaded; it
// also checks that every spin it reads is < q (kErrSpin).
struct BandSrc {
  Bufs b;
  Lattice lat;
  uint32_t base, count;
  static constexpr bool kMulti = false;
  static constexpr bool kCheck = true;
  __device__ __forceinline__ uint32_t ntiles() const { return count; }
  __device__ __forceinline__ uint32_t nreps() const { return 1; }
  __device__ __forceinline__ uint32_t rep(uint32_t) const { return 0; }
  __device__ __forceinline__ const Bufs& bufs(uint32_t) const { return b; }
  __device__ __forceinline__ const Lattice& lattice(uint32_t) const { return lat; }
  __device__ __forceinline__ uint32_t tile0(uint32_t) const { return 0u - base; }  // t = g + base
};

// Tile column and row of tile t: the quotient by ntx from a multiply-high by
// floor(2^32 / ntx), which is the true quotient or one less for every 32-bit
// t, and one correction step.
__device__ __forceinline__ void tile_xy(const Lattice& lat, uint32_t t, uint32_t& tx, uint32_t& ty) {
  uint32_t qt = __umulhi(t, lat.ntx_m);
  uint32_t rt = t - qt * lat.ntx;
  if (rt >= lat.ntx) {
    ++qt;
    rt -= lat.ntx;
  }
  tx = rt;
  ty = qt;
}

__device__ __forceinline__ void tile_geom(const Lattice& lat, uint32_t t, int TH, uint64_t& x0,
                                          uint64_t& y0, int& w, int& h) {
  uint32_t tx, ty;
  tile_xy(lat, t, tx, ty);
  x0 = (uint64_t)tx * kTW;
  y0 = (uint64_t)ty * TH;
  const uint64_t rw = lat.L - x0, rh = lat.L - y0;
  w = rw < (uint64_t)kTW ? (int)rw : kTW;
  h = rh < (uint64_t)TH ? (int)rh : TH;
}

// ---------------------------------------------------------------- shared-memory union-find
// Entries are tile-local site indices and every parent is <= its child, so a
// walk strictly decreases and ends at a root (bounded anyway).  Path halving
// stores only replace a parent by one of its ancestors, which cannot undo a
// concurrent atomicMin link (the union retries with the old parent).
__device__ __forceinline__ uint32_t find_local(uint32_t* P, uint32_t x, uint32_t& bad) {
  volatile uint32_t* vp = P;
  for (uint32_t it = 0; it < kLocalCap; ++it) {
    const uint32_t p = vp[x];
    if (p == x) return x;
    const uint32_t gp = vp[p];
    if (gp == p) return p;
    vp[x] = gp;
    x = gp;
  }
  bad = 1;
  return x;
}

// Read-only walk, for the compression pass: there, every run start must end
// up pointing straight at its root, which halving stores by other threads
// could undo.
__device__ __forceinline__ uint32_t root_local(const uint32_t* P, uint32_t x, uint32_t& bad) {
  const volatile uint32_t* vp = P;
  for (uint32_t it = 0; it < kLocalCap; ++it) {
    const uint32_t p = vp[x];
    if (p == x) return x;
    x = p;
  }
  bad = 1;
  return x;
}

__device__ __forceinline__ void unite_local(uint32_t* P, uint32_t a, uint32_t b, uint32_t& bad) {
  for (uint32_t it = 0; it < kLocalCap; ++it) {
    a = find_local(P, a, bad);
    b = find_local(P, b, bad);
    if (a == b) return;
    if (a < b) {
      const uint32_t tmp = a;
      a = b;
      b = tmp;
    }
    const uint32_t old = atomicMin(&P[a], b);  // link the larger root under the smaller
    if (old == a) return;
    a = old;  // a was no longer a root: join its new parent instead
  }
  bad = 1;
}

// Root of x once all unions are done (roots may carry flag bits above
// kIdx); returns the root and its raw entry.  Halving stores touch only
// non-root entries, which carry no flags.
__device__ __forceinline__ uint32_t walk_root(uint32_t* P, uint32_t x, uint32_t& vroot, uint32_t& bad) {
  volatile uint32_t* vp = P;
  for (uint32_t it = 0; it < kLocalCap; ++it) {
    const uint32_t v = vp[x];
    const uint32_t p = v & kIdx;
    if (p == x) {
      vroot = v;
      return x;
    }
    const uint32_t v2 = vp[p];
    const uint32_t gp = v2 & kIdx;
    if (gp == p) {
      vroot = v2;
      return p;
    }
    vp[x] = gp;
    x = gp;
  }
  bad = 1;
  vroot = 0;
  return x;
}

// Read-only walk to the root, ignoring flag bits above kIdx (used while
// other threads compress starts and flag roots).
__device__ __forceinline__ uint32_t root_masked(const uint32_t* P, uint32_t x, uint32_t& bad) {
  const volatile uint32_t* vp = P;
  for (uint32_t it = 0; it < kLocalCap; ++it) {
    const uint32_t p = vp[x] & kIdx;
    if (p == x) return x;
    x = p;
  }
  bad = 1;
  return x;
}

// Warp-level compaction: lane l contributes the sites (4l+k, k in `mask`)
// of row base `rowbase`; returns the number of tasks written to q[0..n).
// The tasks are ordered by site k first, then by lane: one ballot per k
// gives every position without a prefix scan.
__device__ __forceinline__ uint32_t warp_enqueue(uint16_t* q, uint32_t mask, uint32_t rowbase,
                                                 int lane) {
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t total = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t bk = __ballot_sync(0xFFFFFFFFu, (mask >> k) & 1u);
    if ((mask >> k) & 1u) q[total + __popc(bk & lt)] = (uint16_t)(rowbase + 4 * lane + k);
    total += __popc(bk);
  }
  __syncwarp();
  return total;
}

// ---------------------------------------------------------------- global union-find
// The nodes are the open local roots of all tiles, in a dense table G:
// node d = t * kOpenCap + slot (slot: the root's place in its tile's open
// list).  A node's 64-bit word names its parent by the parent's site key
// and the parent's node,
//     word = key << db | d,   key = y << xb | x for site (x, y),
// db the bits of a node index, so a root's word names itself.  Keys order
// like site indices (row-major), so an atomicMin of whole words links the
// larger root under the smaller and every cluster's final root is its
// smallest site index -- the Hoshen-Kopelman label of Sec. 2 -- whatever
// order the unions run in.  A tile's nodes are contiguous, so the nodes
// that neighbouring edge sites and one tile's open roots touch share
// sectors, and the table holds 8 B x open slots instead of a label per site.
// Where key and node do not fit in 64 bits together (L above 2^17 with
// small tiles) the word carries the parent's open slot instead (db = 0,
// word = key << kSlotBits | slot) and the node is computed from the key.
constexpr int kSlotBits = 9;  // kOpenCap <= 512 for tiles up to 128 x 128
constexpr uint64_t kSlotMask = (1ull << kSlotBits) - 1;

// Word of node d, the tile-local site `local` of the tile at (x0, y0) whose
// open slot is `slot`.
__device__ __forceinline__ uint64_t gword(const Lattice& lat, uint64_t d, uint64_t x0, uint64_t y0, uint32_t local,
                                          uint32_t slot) {
  const uint64_t key = ((y0 + (local >> 7)) << lat.xb) | (x0 + (local & (kTW - 1)));
  return lat.db ? (key << lat.db) | d : (key << kSlotBits) | slot;
}

// The node a word names.
template <int TH>
__device__ __forceinline__ uint64_t gnode(const Lattice& lat, uint64_t w) {
  if (lat.db) return w & ((1ull << lat.db) - 1);
  const uint64_t key = w >> kSlotBits;
  const uint32_t y = (uint32_t)(key >> lat.xb), x = (uint32_t)(key & ((1ull << lat.xb) - 1));
  return ((uint64_t)(y / (uint32_t)TH) * lat.ntx + (x >> 7)) * (uint64_t)TileRec<TH>::kOpenCap + (w & kSlotMask);
}

// Site index of the node a word names (the cluster label of a root's word).
__device__ __forceinline__ uint64_t gsite(const Lattice& lat, uint64_t w) {
  const uint64_t key = w >> (lat.db ? lat.db : kSlotBits);
  return (key >> lat.xb) * lat.L + (key & ((1ull << lat.xb) - 1));
}

// A load that bypasses L1 (another SM may have changed the word).
__device__ __forceinline__ uint64_t ldcg(const uint64_t* p) {
  return (uint64_t)__ldcg(reinterpret_cast<const unsigned long long*>(p));
}

// Root word of node d, whose word w = G[d] is already loaded, with path
// halving.  The halving stores only ever replace a parent by one of its
// ancestors, so they cannot undo a concurrent link.
template <int TH>
__device__ __forceinline__ uint64_t gfind(uint64_t* G, const Lattice& lat, uint64_t d, uint64_t w, uint32_t* err,
                                          uint32_t cap) {
  for (uint32_t it = 0; it < cap; ++it) {
    const uint64_t p = gnode<TH>(lat, w);
    if (p == d) return w;
    const uint64_t wp = ldcg(G + p);
    const uint64_t gp = gnode<TH>(lat, wp);
    if (gp == p) return wp;
    G[d] = wp;
    d = gp;
    w = ldcg(G + d);
  }
  atomicOr(err, kErrFind);
  return w;
}

// Union of the clusters of nodes a and c: the larger root is linked under
// the smaller by an atomicMin of its word; a root that was linked meanwhile
// (the old word is not its own) is united again from its new parent.
template <int TH>
__device__ __forceinline__ void gunite(uint64_t* G, const Lattice& lat, uint64_t a, uint64_t c, uint32_t* err,
                                       uint32_t cap) {
  for (uint32_t it = 0; it < cap; ++it) {
    // both first words in flight at once: the common case (two roots, or
    // one step from them) costs one round trip instead of two
    const uint64_t wa = ldcg(G + a), wc = ldcg(G + c);
    uint64_t ra = gfind<TH>(G, lat, a, wa, err, cap);
    uint64_t rc = gfind<TH>(G, lat, c, wc, err, cap);
    if (ra == rc) return;
    if (ra < rc) {
      const uint64_t tmp = ra;
      ra = rc;
      rc = tmp;
    }
    const uint64_t na = gnode<TH>(lat, ra);
    const uint64_t old = (uint64_t)atomicMin(reinterpret_cast<unsigned long long*>(G + na), (unsigned long long)rc);
    if (old == ra) return;
    a = gnode<TH>(lat, old);
    c = gnode<TH>(lat, rc);
  }
  atomicOr(err, kErrUnion);
}

__device__ __forceinline__ uint64_t global_index(const Lattice& lat, uint64_t x0, uint64_t y0,
                                                 uint32_t local) {
  return (y0 + (local >> 7)) * lat.L + x0 + (local & (kTW - 1));
}

// 4-byte asynchronous global -> shared copy (completes at cp_async_wait).
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
}
// 16-byte asynchronous global -> shared copy, both addresses 16-byte aligned.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// 4-bit mask of the zero bytes of x (bit k <-> byte k).  The per-byte test
// works on 7-bit lanes, so no carry crosses a byte; the multiply gathers the
// four byte flags into bits 24..27 (all other partial products fall below
// bit 24 or beyond bit 31).
__device__ __forceinline__ uint32_t zero_bytes4(uint32_t x) {
  const uint32_t t = ~(((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x) & 0x80808080u;
  return ((t >> 7) * 0x01020408u) >> 24;
}

// Bit k = (w[k] < thr), k = 0..3: the carry-out of each subtraction w[k] -
// thr (PTX sub.cc; set when no borrow occurs, i.e. w[k] >= thr) is shifted
// into d by an add with carry-in (addc: d = 2d + carry), highest k first,
// and the four bits are inverted.
__device__ __forceinline__ uint32_t lt_mask4(const uint32_t (&w)[4], uint32_t thr) {
  uint32_t d = 0, t;
  asm("sub.cc.u32 %1, %2, %6;\n\t"
      "addc.u32 %0, %0, %0;\n\t"
      "sub.cc.u32 %1, %3, %6;\n\t"
      "addc.u32 %0, %0, %0;\n\t"
      "sub.cc.u32 %1, %4, %6;\n\t"
      "addc.u32 %0, %0, %0;\n\t"
      "sub.cc.u32 %1, %5, %6;\n\t"
      "addc.u32 %0, %0, %0;"
      : "+r"(d), "=&r"(t)
      : "r"(w[3]), "r"(w[2]), "r"(w[1]), "r"(w[0]), "r"(thr));
  return ~d & 0xFu;
}

__device__ __forceinline__ uint32_t byte_mask(uint32_t nib) {
  // 4-bit site mask -> 0xFF per selected byte
  return ((nib & 1u) ? 0x000000FFu : 0u) | ((nib & 2u) ? 0x0000FF00u : 0u) |
         ((nib & 4u) ? 0x00FF0000u : 0u) | ((nib & 8u) ? 0xFF000000u : 0u);
}

// ================================================================== k_label_tile
// Persistent: CTA c labels tiles c, c + gridDim.x, ...; while it works on one
// tile the next tile's spin rows are already in flight into the second
// shared staging buffer (cp.async).
//
// kGiven: bonds are read from b.bonds instead of drawn (labelling-only entry).
// kRoots: closed clusters keep their local root in the code (no new state).
//
// Union-find entries P[j] hold tile-local site indices j = ly*128 + lx
// (15 bits).  A site that is not the start of its horizontal run keeps
// pointing at its run start for the whole tile; only run starts take part
// in unions, so only they are compressed, and every site's root is
// P[P[j] & kIdx] & kIdx.  An open cluster's root carries kOpen until the
// root lists are built; then every root entry's high half is the 16-bit
// site code of its cluster (0x8000|state closed, the open-root slot open;
// the labelling-only form keeps kOpen on open roots and no state).  Lane l
// owns sites 4l..4l+3 of a row; its four entries are
// moved with one 16-byte shared-memory access (conflict free); unions and
// compressions are compacted into per-warp task queues so that all lanes
// stay busy.
template <int TH, typename LabelT, bool kGiven, bool kRoots, typename Src, bool kXY = false>
__global__ void __launch_bounds__(TileCta<TH>::kThreads, TileCta<TH>::kMinBlocks)
    k_label_tile(const __grid_constant__ Src src) {
  static_assert(TH % 16 == 0 && kTW * TH <= 32768, "tile shape");
  using S = LabelSmem<TH>;
  using R = TileRec<TH>;
  constexpr int kRpw = TileCta<TH>::kRpw;       // rows per warp
  constexpr int kWarps = TileCta<TH>::kWarps;    // shadows the recolour CTA shape
  constexpr int kThreads = TileCta<TH>::kThreads;
  constexpr unsigned kFull = 0xFFFFFFFFu;

  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* P = reinterpret_cast<uint32_t*>(smem + S::kP);
  uint8_t* sp = smem + S::kSp;
  uint8_t* rbn = smem + S::kRbn;
  uint16_t* wq = reinterpret_cast<uint16_t*>(smem + S::kQ);
  uint32_t* cbits = reinterpret_cast<uint32_t*>(smem + S::kCb);
  uint32_t* wcnt = reinterpret_cast<uint32_t*>(smem + S::kCnt);
  uint32_t* sobs = reinterpret_cast<uint32_t*>(smem + S::kObs);
  uint16_t* clist = reinterpret_cast<uint16_t*>(smem + S::kCl);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int lx0 = 4 * lane;
  uint16_t* q = wq + warp * kTW;
  const uint32_t total = src.ntiles();
  uint32_t bad = 0, spin_max = 0;  // spin_max: byte-wise maximum of the spins read (BandSrc)

  for (int k = tid; k < 257; k += kThreads) sobs[k] = 0;
  uint32_t* xtt = reinterpret_cast<uint32_t*>(smem + S::kXYTab);  // XY form only
  if constexpr (kXY) {
    static_assert(!Src::kMulti, "the XY form labels one lattice");
    const Bufs& b0 = src.bufs(0);
    const uint32_t H1 = (b0.M >> 1) + 1;
    for (uint32_t k = tid; k < H1 * (H1 + 1) / 2; k += kThreads) xtt[k] = __ldg(b0.tt + k);
  }
  uint32_t e_loc = 0, nsites = 0;
  uint32_t ncnt[3] = {0, 0, 0};

  // Observables accumulated so far (E_sat, and for q <= 4 the bit-plane
  // counts c1 = n1 + n3, c2 = n2 + n3, c3 = n3 in registers, else n[s] in
  // shared memory) go to the lattice's accumulator; n[0] follows from the
  // site count.  Called by all threads.
  auto flush = [&](const Bufs& fb, uint32_t fq) {
    const bool fregs = fq <= 4;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e_loc += __shfl_xor_sync(kFull, e_loc, o);
    if (lane == 0) atomicAdd(&sobs[0], e_loc);
    if (fregs) {
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ncnt[k] += __shfl_xor_sync(kFull, ncnt[k], o);
      if (lane == 0) {
        atomicAdd(&sobs[2], ncnt[0] - ncnt[2]);                // n1
        if (fq > 2) atomicAdd(&sobs[3], ncnt[1] - ncnt[2]);    // n2
        if (fq > 3) atomicAdd(&sobs[4], ncnt[2]);              // n3
      }
    }
    __syncthreads();
    if (fregs && tid == 0) {
      uint32_t rest = nsites;
      for (uint32_t st = 1; st < fq; ++st) rest -= sobs[1 + st];
      sobs[1] = rest;  // n0
    }
    __syncthreads();
    for (uint32_t k = tid; k <= fq; k += kThreads)
      if (sobs[k]) atomicAdd(&fb.acc[k], (unsigned long long)sobs[k]);
    __syncthreads();
    for (uint32_t k = tid; k <= fq; k += kThreads) sobs[k] = 0;
    e_loc = 0;
    nsites = 0;
    ncnt[0] = ncnt[1] = ncnt[2] = 0;
  };

  // ---- stage a tile's spin rows (0..h-1 and the halo row h) plus each
  // row's halo byte at column w into a shared buffer.  Rows start 4-byte
  // aligned when L % 4 == 0: then the copies are asynchronous (cp.async)
  // and the next tile is staged while this one is labelled; 16 bytes per
  // copy (8 lanes a row, 4 rows a warp) when L % 16 == 0.
  auto stage = [&](uint32_t gg, uint8_t* buf, bool async) {
    const uint32_t fr = src.rep(gg);
    const Lattice& fl = src.lattice(fr);
    const uint8_t* fspin = src.bufs(fr).spin;
    const uint64_t FL = fl.L;
    uint64_t fx0, fy0;
    int fw, fh;
    tile_geom(fl, gg - src.tile0(fr), TH, fx0, fy0, fw, fh);
    // halo row and column wrap around the lattice (x0 + w <= L, y0 + h <= L)
    const uint64_t hx = (fx0 + fw == FL) ? 0 : fx0 + fw;
    const uint64_t hy = (fy0 + fh == FL) ? 0 : fy0 + fh;
    if (async && (FL & 15u) == 0 && (reinterpret_cast<uintptr_t>(fspin) & 15u) == 0) {
      // w is a multiple of 16 here (x0 a multiple of 128, L of 16)
      const int c16 = (lane & 7) * 16;
      for (int ly = warp * 4 + (lane >> 3); ly <= fh; ly += 4 * kWarps) {
        const uint64_t gy = (ly < fh) ? (fy0 + ly) : hy;
        if (c16 < fw) cp_async16(buf + ly * kSpPitch + c16, fspin + gy * FL + fx0 + c16);
      }
      // halo column: 4 aligned bytes starting at column (x0 + w) mod L
      for (int ly = tid; ly <= fh; ly += kThreads) {
        const uint64_t gy = (ly < fh) ? (fy0 + ly) : hy;
        cp_async4(buf + ly * kSpPitch + fw, fspin + gy * FL + hx);
      }
      return;
    }
    for (int ly = warp; ly <= fh; ly += kWarps) {
      const uint64_t gy = (ly < fh) ? (fy0 + ly) : hy;
      const uint8_t* row = fspin + gy * FL;
      uint8_t* dst = buf + ly * kSpPitch;
      if (async) {
        if (lx0 < fw) cp_async4(dst + lx0, row + fx0 + lx0);
        // halo column: 4 aligned bytes starting at column (x0 + w) mod L
        if (lane == 31) cp_async4(dst + fw, row + hx);
      } else {
        uint32_t v = 0;
        if (lx0 < fw) {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (lx0 + k < fw) v |= (uint32_t)row[fx0 + lx0 + k] << (8 * k);
        }
        *reinterpret_cast<uint32_t*>(dst + lx0) = v;
        __syncwarp();
        if (lane == 0) dst[fw] = row[hx];
      }
    }
  };
  bool pre = false;  // this tile's spins were staged asynchronously
  if (!kGiven && blockIdx.x < total && src.lattice(src.rep(blockIdx.x)).vec4) {
    stage(blockIdx.x, sp, true);
    cp_async_commit();
    pre = true;
  }

  uint32_t it = 0;
  for (uint32_t g = blockIdx.x; g < total; g += gridDim.x, ++it) {
    const uint32_t rep = src.rep(g);
    const Bufs& b = src.bufs(rep);
    const Lattice& lat = src.lattice(rep);
    const uint32_t t = g - src.tile0(rep);
    const uint64_t L = lat.L;
    const uint32_t q_states = b.q;
    const bool measure = !kGiven && !kXY && b.measure;
    const uint32_t sweep = kGiven ? 0u : (uint32_t)b.ctl[0];
    const uint32_t qs = q_states <= 4 ? q_states - 1 : 0;  // states counted in registers
    uint64_t x0, y0;
    int w, h;
    tile_geom(lat, t, TH, x0, y0, w, h);
    uint8_t* spc = sp + (it & 1u) * S::kSpBuf;  // this tile's staged spins
    if (tid < R::kBitWords) cbits[tid] = 0;
    bool synced = false;  // a barrier already separates this tile from the last one
    if (!kGiven) {
      if (pre) {
        cp_async_wait();
        __syncthreads();  // every thread's copies of this tile have landed
        synced = true;
      } else {
        stage(g, spc, false);
      }
      pre = false;
      const uint32_t gn = g + gridDim.x;
      if (gn < total && src.lattice(src.rep(gn)).vec4) {
        stage(gn, sp + ((it + 1) & 1u) * S::kSpBuf, true);
        cp_async_commit();
        pre = true;
      }
    }
    if constexpr (kXY) {
      // projection class of every angle on this sweep's embedding axis
      // (Wolff's embedding): sign of sigma in bits 8-9 (1 negative,
      // 2 positive, 0 zero), fold index c of |sigma| = sin(pi c / M) below;
      // built for the CTA's first tile only (one lattice, one sweep)
      uint16_t* xcls = reinterpret_cast<uint16_t*>(sobs);
      const uint32_t M = b.M;
      const uint32_t jx = it == 0 ? pick_state(stream4_rk(b.rk, 0ull, sweep, kDomAxis).x, M) : 0u;
      for (uint32_t k = tid; it == 0 && k < M; k += kThreads) {
        const uint32_t a = (2 * k >= jx) ? 2 * k - jx : 2 * k + 2 * M - jx;  // (2k - j) mod 2M
        const uint32_t sg = (a == 0 || a == M) ? 0u : (a < M ? 1u : 2u);
        const uint32_t bm = a >= M ? a - M : a;
        xcls[k] = (uint16_t)((sg << 8) | (bm < M - bm ? bm : M - bm));
      }
    }
    if (tid == 0) nsites += (uint32_t)(w * h);
    // synchronous staging, the zeroed cross bits (labelling from given
    // bonds) or the XY class table must be visible before the bonds pass
    if (!synced || (kXY && it == 0)) __syncthreads();

    // ---- bonds, measurement, horizontal runs
    uint32_t rowbits[kRpw];  // bits 0-3 internal right, 4-7 internal down, 8-11 run starts
#pragma unroll
    for (int rr = 0; rr < kRpw; ++rr) {
      const int ly = warp * kRpw + rr;  // a warp owns a block of kRpw consecutive rows
      uint32_t vm = 0;  // valid sites of this lane's group
      if (ly < h) {
        const int nv = w - lx0;
        vm = nv >= 4 ? 0xFu : (nv > 0 ? (1u << nv) - 1u : 0u);
      }
      uint32_t br = 0, bd = 0;  // active bonds (right / down), all of them
      if (kGiven) {
        if (vm) {
          const uint32_t byte = b.bonds[(y0 + ly) * lat.bp + ((x0 + lx0) >> 2)];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            br |= ((byte >> (2 * k)) & 1u) << k;
            bd |= ((byte >> (2 * k + 1)) & 1u) << k;
          }
          br &= vm;
          bd &= vm;
        }
      } else {
        const uint32_t s = *reinterpret_cast<const uint32_t*>(spc + ly * kSpPitch + lx0);
        if constexpr (Src::kCheck) spin_max = __vmaxu4(spin_max, s & byte_mask(vm));
        const uint32_t sn = *reinterpret_cast<const uint32_t*>(spc + ly * kSpPitch + lx0 + 4);
        const uint32_t sd = *reinterpret_cast<const uint32_t*>(spc + (ly + 1) * kSpPitch + lx0);
        const uint32_t sr = __funnelshift_r(s, sn, 8);
        uint32_t eqr, eqd;  // bond candidates: equal states (Potts), equal signs of sigma (XY)
        uint32_t tr[4], td[4];
        if constexpr (kXY) {
          const uint16_t* xcls = reinterpret_cast<const uint16_t*>(sobs);
          // threshold of fold indices (c, d): lower-triangle entry of the larger
          auto thr_of = [&](uint32_t c, uint32_t d) -> uint32_t {
            const uint32_t hi = c > d ? c : d, lo = c > d ? d : c;
            return xtt[((hi * (hi + 1)) >> 1) + lo];
          };
          uint32_t cs[5], cd[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            cs[k] = xcls[(s >> (8 * k)) & 0xFFu];
            cd[k] = xcls[(sd >> (8 * k)) & 0xFFu];
          }
          cs[4] = xcls[sn & 0xFFu];
          eqr = eqd = 0;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint32_t sg = cs[k] >> 8;
            eqr |= (sg != 0u && sg == (cs[k + 1] >> 8)) ? (1u << k) : 0u;
            eqd |= (sg != 0u && sg == (cd[k] >> 8)) ? (1u << k) : 0u;
            tr[k] = thr_of(cs[k] & 0xFFu, cs[k + 1] & 0xFFu);
            td[k] = thr_of(cs[k] & 0xFFu, cd[k] & 0xFFu);
          }
          eqr &= vm;
          eqd &= vm;
        } else {
          eqr = zero_bytes4(s ^ sr) & vm;  // right neighbour has the same state
          eqd = zero_bytes4(s ^ sd) & vm;  // lower neighbour has the same state
        }
        if (!kXY && measure) {
          e_loc += __popc(eqr) + __popc(eqd);
          if (qs) {
            // bit planes of the valid sites (q <= 4): bit 0 marks states 1, 3,
            // bit 1 states 2, 3, both state 3
            const uint32_t m1 = (vm * 0x00204081u) & 0x01010101u;  // bit 0 of each valid byte
            ncnt[0] += __popc(s & m1);
            if (qs > 1) {
              const uint32_t s1 = (s >> 1) & m1;
              ncnt[1] += __popc(s1);
              ncnt[2] += __popc(s & s1);
            }
          } else {
#pragma unroll
            for (int k = 0; k < 4; ++k)
              if (vm & (1u << k)) atomicAdd(&sobs[1 + ((s >> (8 * k)) & 0xFFu)], 1u);
          }
        }
        if ((eqr | eqd) != 0u) {
          const uint64_t i0 = (y0 + ly) * L + x0 + lx0;
          const uint64_t pa = i0 >> 1;
          const Words4 A = stream4_rk(b.rk, pa, sweep, kDomBond);
          const Words4 B = stream4_rk(b.rk, pa + 1, sweep, kDomBond);
          uint32_t wr[4], wd[4];
          if ((i0 & 1u) == 0u) {
            wr[0] = A.x; wd[0] = A.y; wr[1] = A.z; wd[1] = A.w;
            wr[2] = B.x; wd[2] = B.y; wr[3] = B.z; wd[3] = B.w;
          } else {
            const Words4 C = stream4_rk(b.rk, pa + 2, sweep, kDomBond);
            wr[0] = A.z; wd[0] = A.w; wr[1] = B.x; wd[1] = B.y;
            wr[2] = B.z; wd[2] = B.w; wr[3] = C.x; wd[3] = C.y;
          }
          uint32_t ur = 0, ud = 0;  // u < thr per site
          if constexpr (kXY) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              ur |= (wr[k] < tr[k] ? 1u : 0u) << k;
              ud |= (wd[k] < td[k] ? 1u : 0u) << k;
            }
          } else {
            ur = lt_mask4(wr, b.thr);
            ud = lt_mask4(wd, b.thr);
          }
          br = eqr & ur;
          bd = eqd & ud;
        }
        if (b.bonds && vm) {
          uint32_t byte = 0;
#pragma unroll
          for (int k = 0; k < 4; ++k) byte |= (((br >> k) & 1u) << (2 * k)) | (((bd >> k) & 1u) << (2 * k + 1));
          b.bonds[(y0 + ly) * lat.bp + ((x0 + lx0) >> 2)] = (uint8_t)byte;
        }
      }
      // internal vs cross-edge bonds
      const int last = w - 1 - lx0;  // position of the tile's last column in this group
      const uint32_t rint = (last >= 4) ? 0xFu : (last > 0 ? (1u << last) - 1u : 0u);
      if (last >= 0 && last < 4 && ((br >> last) & 1u)) atomicOr(&cbits[ly >> 5], 1u << (ly & 31));
      if (ly == h - 1) {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const uint32_t v = (lane >> 3) == m ? (bd & 0xFu) << (4 * (lane & 7)) : 0u;
          const uint32_t word = __reduce_or_sync(kFull, v);
          if (lane == 0) cbits[R::kRightWords + m] = word;
        }
      }
      const uint32_t r4 = br & rint;
      const uint32_t d4 = (ly < h - 1) ? bd : 0u;
      // horizontal runs: a site whose left bond is inactive starts a run;
      // every site's provisional label is its run start (one ballot per row)
      uint32_t prev3 = __shfl_up_sync(kFull, (r4 >> 3) & 1u, 1);
      if (lane == 0) prev3 = 0;
      const uint32_t brk = (~((r4 << 1) | prev3)) & 0xFu;
      rowbits[rr] = r4 | (d4 << 4) | ((brk & vm) << 8);
      const uint32_t Bm = __ballot_sync(kFull, brk != 0u);
      const int lb = brk ? 31 - __clz(brk) : 0;
      const uint32_t below = Bm & ((1u << lane) - 1u);
      const int src = below ? 31 - __clz(below) : 0;
      const int lbs = __shfl_sync(kFull, lb, src);
      const uint32_t rowbase = (uint32_t)(ly * kTW);
      // run start of each site: itself if it breaks the run, else the start
      // of the site to its left (the first site inherits from earlier lanes)
      const uint32_t st0 = rowbase + ((brk & 1u) ? (uint32_t)lx0 : (uint32_t)(4 * src + lbs));
      const uint32_t st1 = (brk & 2u) ? rowbase + lx0 + 1 : st0;
      const uint32_t st2 = (brk & 4u) ? rowbase + lx0 + 2 : st1;
      const uint32_t st3 = (brk & 8u) ? rowbase + lx0 + 3 : st2;
      *reinterpret_cast<uint4*>(P + rowbase + lx0) = make_uint4(st0, st1, st2, st3);
      rbn[ly * 32 + lane] = (uint8_t)r4;
    }
    __syncthreads();

    // ---- vertical unions.  Each warp first links its own rows top-down,
    // one row pair at a time, so a new run is hung directly under an
    // existing root and trees stay shallow; then the kWarps-1 row pairs that
    // straddle two warps' blocks are linked.  Unions that repeat the left
    // neighbour's union of the same two runs are skipped, the rest are
    // compacted into the warp's task queue so all lanes stay busy.
    auto link_rows = [&](int ly, uint32_t r4, uint32_t d4, uint32_t rb, uint32_t pb) {
      uint32_t pd = __shfl_up_sync(kFull, (d4 >> 3) & 1u, 1);
      uint32_t pr = __shfl_up_sync(kFull, (r4 >> 3) & 1u, 1);
      if (lane == 0) pd = pr = pb = 0;
      const uint32_t skip = ((d4 << 1) | pd) & ((r4 << 1) | pr) & ((rb << 1) | pb);
      const uint32_t n = warp_enqueue(q, d4 & ~skip & 0xFu, (uint32_t)(ly * kTW), lane);
      for (uint32_t i = lane; i < n; i += 32) {
        const uint32_t a = q[i];
        unite_local(P, P[a], P[a + kTW], bad);
      }
      __syncwarp();
    };
#pragma unroll
    for (int rr = 0; rr + 1 < kRpw; ++rr) {
      const int ly = warp * kRpw + rr;
      if (ly < h - 1) {  // warp-uniform
        const uint32_t rb = rowbits[rr + 1] & 0xFu;
        const uint32_t pb = __shfl_up_sync(kFull, (rb >> 3) & 1u, 1);
        link_rows(ly, rowbits[rr] & 0xFu, (rowbits[rr] >> 4) & 0xFu, rb, pb);
      }
    }
    // no barrier: the lock-free unions are order independent, so a warp may
    // link across the block boundary while its neighbour still links inside
    {
      const int ly = warp * kRpw + kRpw - 1;
      if (warp + 1 < kWarps && ly < h - 1) {  // warp-uniform
        const uint32_t rb = rbn[(ly + 1) * 32 + lane];
        const uint32_t pb = lane > 0 ? (rbn[(ly + 1) * 32 + lane - 1] >> 3) & 1u : 0u;
        link_rows(ly, rowbits[kRpw - 1] & 0xFu, (rowbits[kRpw - 1] >> 4) & 0xFu, rb, pb);
      }
    }
    __syncthreads();

    if (tid == 0) wcnt[0] = 0;  // open-slot counter of this tile

    // ---- compress the run starts of the warp's rows (only starts can be
    // roots; all rows in one batch, listed in the root-list area, which is
    // free until the root lists), and flag clusters that touch the tile
    // edge as open (the edge sites are spread over all threads)
    {
      uint16_t* tq = clist + warp * (kRpw * kTW);
      const uint32_t jbase = (uint32_t)(warp * kRpw * kTW + lx0);
      uint32_t smask = 0;
#pragma unroll
      for (int rr = 0; rr < kRpw; ++rr)
        if (warp * kRpw + rr < h) smask |= ((rowbits[rr] >> 8) & 0xFu) << (4 * rr);
      const uint32_t mine = (uint32_t)__popc(smask);
      uint32_t inc = mine;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += y;
      }
      uint32_t pos = inc - mine;
      while (smask) {
        const int bb = __ffs(smask) - 1;
        smask &= smask - 1u;
        tq[pos++] = (uint16_t)(jbase + (bb >> 2) * kTW + (bb & 3));
      }
      const uint32_t n = __shfl_sync(kFull, inc, 31);
      __syncwarp();
      for (uint32_t i = lane; i < n; i += 32) {
        const uint32_t j = tq[i];
        const uint32_t r = root_masked(P, j, bad);
        if (r != j) P[j] = r;
      }
      __syncwarp();
    }
    {
      const int nedge = 2 * (w + h);
      for (int e = tid; e < nedge; e += kThreads) {
        int lx, ly;
        if (e < h) { lx = w - 1; ly = e; }
        else if (e < 2 * h) { lx = 0; ly = e - h; }
        else if (e < 2 * h + w) { lx = e - 2 * h; ly = 0; }
        else { lx = e - 2 * h - w; ly = h - 1; }
        const uint32_t r = root_masked(P, (uint32_t)(ly * kTW + lx), bad);
        atomicOr(&P[r], kOpen);
      }
    }
    __syncthreads();

    // ---- root lists, warp-local: a run start j is a root iff P[j] == j.
    // Closed roots fill the warp's region from the front, open ones from the
    // back.
    constexpr int kRegion = kRpw * kTW;
    uint16_t* wl = clist + warp * kRegion;
    // a lane's roots over all its rows (bit 4*rr + k), one prefix over the
    // warp for all rows, then the lane writes its closed and open roots
    uint32_t cmask = 0, omask = 0;
#pragma unroll
    for (int rr = 0; rr < kRpw; ++rr) {
      const int ly = warp * kRpw + rr;
      const uint32_t stb = (rowbits[rr] >> 8) & 0xFu;
      if (ly < h && stb) {
        const uint32_t j0 = (uint32_t)(ly * kTW + lx0);
        const uint4 v4 = *reinterpret_cast<const uint4*>(P + j0);
        const uint32_t v[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint32_t isroot = ((stb >> k) & 1u) & ((v[k] & kIdx) == j0 + k ? 1u : 0u);
          const uint32_t open = v[k] >> 31;  // kOpen
          cmask |= (isroot & (open ^ 1u)) << (4 * rr + k);
          omask |= (isroot & open) << (4 * rr + k);
        }
      }
    }
    uint32_t nclosed, nopen;  // warp-uniform
    {
      const uint32_t mine = (uint32_t)__popc(cmask) | ((uint32_t)__popc(omask) << 16);
      uint32_t inc = mine;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += y;
      }
      const uint32_t excl = inc - mine;
      uint32_t cpos = excl & 0xFFFFu, opos = excl >> 16;
      const uint32_t jbase = (uint32_t)(warp * kRpw * kTW + lx0);
      while (cmask) {
        const int bb = __ffs(cmask) - 1;
        cmask &= cmask - 1u;
        wl[cpos++] = (uint16_t)(jbase + (bb >> 2) * kTW + (bb & 3));
      }
      while (omask) {
        const int bb = __ffs(omask) - 1;
        omask &= omask - 1u;
        wl[kRegion - 1 - (opos++)] = (uint16_t)(jbase + (bb >> 2) * kTW + (bb & 3));
      }
      const uint32_t total = __shfl_sync(kFull, inc, 31);
      nclosed = total & 0xFFFFu;
      nopen = total >> 16;
    }
    // ---- new state of each complete cluster, drawn once at its root, by the
    // warp that listed it (its own rows: no other warp reads these entries
    // before the next barrier, so this needs no barrier of its own)
    __syncwarp();
    if (!kRoots) {
      for (uint32_t i = lane; i < nclosed; i += 32) {
        const uint32_t j = wl[i];
        const uint32_t stt =
            pick_state(stream4_rk(b.rk, global_index(lat, x0, y0, j), sweep, kDomSpin).x, q_states);
        P[j] = j | ((kClosed | stt) << 16);  // the high half is the site code
      }
    }
    // ---- open roots get a block of slots in the tile's open list (in
    // whatever order the warps arrive: a slot only names the root to later
    // kernels, results do not depend on it) and their node of the global
    // union-find, a root for now
    {
      uint32_t obase = 0;
      if (lane == 0 && nopen) obase = atomicAdd(&wcnt[0], nopen);
      obase = __shfl_sync(kFull, obase, 0);
      for (uint32_t i = lane; i < nopen; i += 32) {
        const uint32_t j = wl[kRegion - 1 - i];
        const uint32_t slot = obase + i;
        // the high half is the site code (the slot); the labelling-only form
        // keeps the open flag to tell open from closed roots
        P[j] = j | (kRoots ? kOpen : 0u) | (slot << 16);
        const uint64_t d = (uint64_t)t * R::kOpenCap + slot;
        b.G[d] = gword(lat, d, x0, y0, j, slot);
      }
    }
    __syncthreads();
    if (tid == 0) b.ocnt[t] = wcnt[0];

    // ---- per-site codes and the edge lines
    uint16_t* edge = b.edge + (uint64_t)t * R::kEdge;
#pragma unroll
    for (int rr = 0; rr < kRpw; ++rr) {
      const int ly = warp * kRpw + rr;
      if (ly < h && lx0 < w) {
        const uint32_t rowbase = (uint32_t)(ly * kTW);
        const uint4 v4 = *reinterpret_cast<const uint4*>(P + rowbase + lx0);
        const uint32_t v[4] = {v4.x, v4.y, v4.z, v4.w};
        uint32_t c[4];
        // four independent two-step lookups (run start, root), no branches
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint32_t x = v[k] & kIdx;  // run start, or the root for a start
          const uint32_t pr = P[x] & kIdx;
          const uint32_t pvr = P[pr];
          if constexpr (kRoots)
            c[k] = (pvr & kOpen) ? ((pvr >> 16) & 0x1FFu) : (kClosed | pr);
          else
            c[k] = pvr >> 16;
        }
        const uint64_t gi = (y0 + ly) * L + x0 + lx0;
        if (lat.vec4) {
          *reinterpret_cast<uint2*>(b.code + gi) = make_uint2(c[0] | (c[1] << 16), c[2] | (c[3] << 16));
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (lx0 + k < w) b.code[gi + k] = (uint16_t)c[k];
        }
        // edge sites belong to open clusters: their codes are open slots
        const bool edge_row = (ly == 0 || ly == h - 1);
        const int last = w - 1 - lx0;
        if (edge_row || lane == 0 || (last >= 0 && last < 4)) {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int lx = lx0 + k;
            if (lx < w) {
              if (lx == w - 1) edge[ly] = (uint16_t)c[k];
              if (lx == 0) edge[TH + ly] = (uint16_t)c[k];
              if (ly == h - 1) edge[2 * TH + lx] = (uint16_t)c[k];
              if (ly == 0) edge[2 * TH + kTW + lx] = (uint16_t)c[k];
            }
          }
        }
      }
    }
    if (tid < R::kBitWords) b.ebits[(uint64_t)t * R::kBitWords + tid] = cbits[tid];
    // no barrier here: the next tile touches shared memory that this tile
    // still reads (P, root lists) only after its own first barrier, and the
    // cross bits only through the threads that read them here
    // a replica's observables go out when the CTA's next tile belongs to
    // another replica (or there is none); until then they accumulate
    if (Src::kMulti && measure) {
      const uint32_t gn = g + gridDim.x;
      if (gn >= total || src.rep(gn) != rep) flush(b, q_states);
    }
  }

  // ---- observables of the configuration read (Sec. 4), once per CTA
  if (!Src::kMulti && !kGiven && total > 0 && blockIdx.x < total) {
    const Bufs& b0 = src.bufs(0);
    if (b0.measure) flush(b0, b0.q);
  }
  if (bad) atomicOr(src.bufs(0).err, kErrLocal);
  if constexpr (Src::kCheck) {
    const uint32_t m2 = __vmaxu4(spin_max, spin_max >> 16);
    if ((__vmaxu4(m2, m2 >> 8) & 0xFFu) >= src.bufs(0).q) atomicOr(src.bufs(0).err, kErrSpin);
  }
}

// ================================================================== boundary unions
// The crossing bond at edge position pos of tile t (0 .. TH-1: row of the
// right edge, TH .. TH+127: column of the bottom edge; the periodic wrap
// included): true if it is active, with its two nodes (t's, the
// neighbour's) and their open slots.  kCG: loads that bypass L1 (records
// another SM wrote during this launch).  The bond bit and both slots are
// loaded together; the slots of a position without an active bond are not
// used.
template <int TH, bool kCG>
__device__ __forceinline__ bool crossing_bond(const Bufs& b, const Lattice& lat, uint32_t t, int pos, uint64_t& a,
                                              uint64_t& c, uint32_t& sa, uint32_t& sc) {
  using R = TileRec<TH>;
  uint64_t x0, y0;
  int w, h;
  tile_geom(lat, t, TH, x0, y0, w, h);
  uint32_t tx, ty;
  tile_xy(lat, t, tx, ty);
  const bool right = pos < TH;
  const int k = right ? pos : pos - TH;  // row of the right edge, or column of the bottom edge
  const uint32_t tn = right ? ty * lat.ntx + (tx + 1 == lat.ntx ? 0u : tx + 1)
                            : (ty + 1 == lat.nty ? 0u : ty + 1) * lat.ntx + tx;
  const int ea = right ? k : 2 * TH + k;             // own right column / bottom row
  const int ec = right ? TH + k : 2 * TH + kTW + k;  // the neighbour's left column / top row
  const uint32_t* bw = b.ebits + (uint64_t)t * R::kBitWords + (right ? (k >> 5) : R::kRightWords + (k >> 5));
  const uint16_t* pa = b.edge + (uint64_t)t * R::kEdge + ea;
  const uint16_t* pc = b.edge + (uint64_t)tn * R::kEdge + ec;
  const uint32_t word = kCG ? __ldcg(bw) : *bw;
  sa = kCG ? __ldcg(pa) : *pa;
  sc = kCG ? __ldcg(pc) : *pc;
  a = (uint64_t)t * R::kOpenCap + sa;
  c = (uint64_t)tn * R::kOpenCap + sc;
  return k < (right ? h : w) && ((word >> (k & 31)) & 1u);
}

// End of a labelling pass: files the observables of the configuration the
// labeller read into the ring, advances the lattice's sweep counter, and
// (XY form) draws the sweep's embedding axis.
__device__ __forceinline__ void file_sweep(const Bufs& b) {
  const unsigned long long s = b.ctl[0];
  if (b.measure) {
    unsigned long long* rec = b.ring + (s % b.ring_cap) * (2ull + b.q);
    rec[0] = s;
    for (uint32_t k = 0; k <= b.q; ++k) {
      rec[1 + k] = b.acc[k];
      b.acc[k] = 0ull;
    }
  }
  b.ctl[1] = s;
  b.ctl[0] = s + 1ull;
  if (b.M) b.ctl[2] = pick_state(stream4_rk(b.rk, 0ull, (uint32_t)s, kDomAxis).x, b.M);
}

// ================================================================== k_merge
// One thread per edge position of every tile: TH right-edge rows, then the
// 128 bottom-edge columns.  The thread at position 0 of a lattice's tile 0
// also files the sweep (file_sweep).
template <int TH, typename LabelT, typename Src>
__global__ void __launch_bounds__(kMergeThreads) k_merge(const __grid_constant__ Src src) {
  constexpr int kPer = TH + kTW;
  const uint64_t item = (uint64_t)blockIdx.x * kMergeThreads + threadIdx.x;
  const uint32_t g = (uint32_t)(item / kPer);
  const int pos = (int)(item % kPer);
  uint64_t a = 0, c = 0;  // the two nodes of an active crossing bond
  uint32_t key = 0xFFFFFFFFu;  // (parity of g, edge, slot of a, slot of c): unique within a warp
  bool active = false;
  const uint32_t rep = g < src.ntiles() ? src.rep(g) : 0u;
  const Bufs& b = src.bufs(rep);
  const Lattice& lat = src.lattice(rep);
  const uint32_t t = g - src.tile0(rep);
  if (g < src.ntiles()) {
    uint32_t sa, sc;
    active = crossing_bond<TH, false>(b, lat, t, pos, a, c, sa, sc);
    key = ((g & 1u) << 19) | ((pos < TH ? 0u : 1u) << 18) | (sa << kSlotBits) | sc;
  }
  // neighbouring edge sites usually repeat the same pair of roots: one lane
  // per distinct (a, c) pair does the union.  A warp's positions lie in at
  // most two consecutive global tiles g (TH + 128 >= 32 positions each), so
  // g's parity, the edge (right or bottom) and the two open slots name the
  // pair.
  const unsigned same = __match_any_sync(0xFFFFFFFFu, active ? key : 0xFFFFFFFFu);
  if (active && (int)(threadIdx.x & 31) == __ffs(same) - 1)
    gunite<TH>(b.G, lat, a, c, b.err, b.walk_cap ? b.walk_cap : kFindCap);
  if (g < src.ntiles() && t == 0 && pos == 0) file_sweep(b);
}

// The sweep's filing when the labeller did the boundary unions (fused
// merge schedule): a thread per lattice.
template <typename Src>
__global__ void k_file(const __grid_constant__ Src src) {
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < src.nreps()) file_sweep(src.bufs(r));
}

// ================================================================== k_resolve
// Sec. 2 step (3) for open clusters: a thread per open root finds (and
// compresses to) its global root and draws the cluster's new state, keyed
// by the root's site index.  A block of kResolveThreads per tile (a tile
// has far fewer open roots than slots; a thread takes slots k, k + 256, ...
// when it has more), so the walks of the whole lattice are in flight
// together; the tile's nodes are contiguous, so a warp's first loads share
// sectors.
constexpr int kResolveThreads = 256;

template <int TH, typename LabelT, typename Src>
__global__ void __launch_bounds__(kResolveThreads) k_resolve(const __grid_constant__ Src src) {
  using R = TileRec<TH>;
  const uint32_t g = blockIdx.x;
  if (g >= src.ntiles()) return;
  const uint32_t rep = src.rep(g);
  const Bufs& b = src.bufs(rep);
  const uint32_t t = g - src.tile0(rep);
  const uint64_t d0 = (uint64_t)t * R::kOpenCap;
  // the first node's word is loaded with the tile's count (a slot past the
  // count holds a stale word that is not used)
  const uint32_t n0 = b.ocnt[t];
  uint64_t w = ldcg(b.G + d0 + threadIdx.x);
  const uint32_t n = min(n0, (uint32_t)R::kOpenCap);
  const Lattice& lat = src.lattice(rep);
  const uint32_t sweep = (uint32_t)b.ctl[1];
  const uint32_t cap = b.walk_cap ? b.walk_cap : kFindCap;
  for (uint32_t k = threadIdx.x; k < n; k += kResolveThreads) {
    if (k != threadIdx.x) w = ldcg(b.G + d0 + k);
    const uint64_t r = gfind<TH>(b.G, lat, d0 + k, w, b.err, cap);
    b.nso[d0 + k] = (uint8_t)pick_state(stream4_rk(b.rk, gsite(lat, r), sweep, kDomSpin).x, b.q);
  }
}

// ================================================================== k_recolor
// Streams codes to spins: closed clusters carry their state in the code,
// open ones index the tile's resolved open-root states.
// kRoots: write each site's global root (LabelT) to `roots` instead.
// kXY: the coin of each cluster (q = 2) says whether its spins are
// reflected, k -> (j - k) mod M, j the sweep's embedding axis.
template <int TH, typename LabelT, bool kRoots, typename Src, bool kXY = false>
__global__ void __launch_bounds__(kThreads) k_recolor(const __grid_constant__ Src src, LabelT* roots) {
  using R = TileRec<TH>;
  constexpr int kRpw = TH / kWarps;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t g = blockIdx.x;
  const uint32_t rep = src.rep(g);
  // a replica batch: the block's replica record once, through shared memory
  // (each thread reading it from the replica table would wait on a chain of
  // loads before streaming)
  __shared__ __align__(16) unsigned char srec[Src::kMulti ? sizeof(Rep) : 16];
  if constexpr (Src::kMulti) {
    const uint32_t* from = reinterpret_cast<const uint32_t*>(&src.bufs(rep));
    for (int k = tid; k < (int)(sizeof(Rep) / 4); k += kThreads)
      reinterpret_cast<uint32_t*>(srec)[k] = __ldg(from + k);
    __syncthreads();
  }
  const Bufs& b = [&]() -> const Bufs& {
    if constexpr (Src::kMulti) return reinterpret_cast<const Rep*>(srec)->b;
    else return src.bufs(rep);
  }();
  const Lattice& lat = [&]() -> const Lattice& {
    if constexpr (Src::kMulti) return reinterpret_cast<const Rep*>(srec)->lat;
    else return src.lattice(rep);
  }();
  const uint32_t t = g - src.tile0(rep);
  uint64_t x0, y0;
  int w, h;
  tile_geom(lat, t, TH, x0, y0, w, h);
  const uint64_t L = lat.L;
  const uint8_t* nso = b.nso + (uint64_t)t * R::kOpenCap;
  // kRoots: the global root of each of the tile's open roots, found once
  // (a thread per open slot) instead of once per site of its cluster
  __shared__ LabelT oroot[kRoots ? R::kOpenCap : 1];
  if constexpr (kRoots) {
    const uint32_t n = min(b.ocnt[t], (uint32_t)R::kOpenCap);
    const uint32_t cap = b.walk_cap ? b.walk_cap : kFindCap;
    for (uint32_t k = (uint32_t)tid; k < n; k += kThreads) {
      const uint64_t d = (uint64_t)t * R::kOpenCap + k;
      oroot[k] = (LabelT)gsite(lat, gfind<TH>(b.G, lat, d, ldcg(b.G + d), b.err, cap));
    }
    __syncthreads();
  }
  uint32_t jx = 0, Mx = 0;
  if constexpr (kXY) {
    jx = (uint32_t)b.ctl[2];  // the sweep's embedding axis, filed by k_merge
    Mx = b.M;
  }
  // new spin of a site with old spin k whose cluster drew st
  auto next = [&](uint32_t st, uint32_t k) -> uint32_t {
    if constexpr (kXY) return st ? (k <= jx ? jx - k : jx + Mx - k) : k;
    else return st;
  };
  if (!kRoots && (L & 7u) == 0) {
    // rows of 8-site groups: a thread reads 8 codes (16 B), writes 8 spins;
    // two rows per step, both rows' loads issued before either is used
    constexpr int kStep = kThreads / 16;
    const int lx = 8 * (tid & 15);
    for (int ly = tid >> 4; ly < h; ly += 2 * kStep) {
      const bool has2 = ly + kStep < h;
      if (lx < w) {
        const uint64_t gi = (y0 + ly) * L + x0 + lx;
        const uint64_t gi2 = gi + (uint64_t)kStep * L;
        uint4 v[2];
        uint2 old[2] = {make_uint2(0u, 0u), make_uint2(0u, 0u)};
        v[0] = __ldcs(reinterpret_cast<const uint4*>(b.code + gi));
        v[1] = has2 ? __ldcs(reinterpret_cast<const uint4*>(b.code + gi2)) : make_uint4(0u, 0u, 0u, 0u);
        if constexpr (kXY) {
          old[0] = *reinterpret_cast<const uint2*>(b.spin + gi);
          if (has2) old[1] = *reinterpret_cast<const uint2*>(b.spin + gi2);
        }
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          if (r == 1 && !has2) break;
          const uint32_t cw[4] = {v[r].x, v[r].y, v[r].z, v[r].w};
          const uint32_t ow[2] = {old[r].x, old[r].y};
          uint32_t s2[2] = {0u, 0u};
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const uint32_t c = (cw[k >> 1] >> (16 * (k & 1))) & 0xFFFFu;
            const uint32_t st = (c & kClosed) ? (c & 0xFFu) : nso[c];
            s2[k >> 2] |= next(st, (ow[k >> 2] >> (8 * (k & 3))) & 0xFFu) << (8 * (k & 3));
          }
          *reinterpret_cast<uint2*>(b.spin + (r ? gi2 : gi)) = make_uint2(s2[0], s2[1]);
        }
      }
    }
    return;
  }
  const int lx0 = 4 * lane;
#pragma unroll
  for (int rr = 0; rr < kRpw; ++rr) {
    const int ly = warp + rr * kWarps;
    if (ly < h && lx0 < w) {
      const uint64_t gi = (y0 + ly) * L + x0 + lx0;
      uint32_t c[4];
      if (lat.vec4) {
        const uint2 v = __ldcs(reinterpret_cast<const uint2*>(b.code + gi));
        c[0] = v.x & 0xFFFFu; c[1] = v.x >> 16; c[2] = v.y & 0xFFFFu; c[3] = v.y >> 16;
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) c[k] = lx0 + k < w ? b.code[gi + k] : 0u;
      }
      if (kRoots) {
        LabelT rv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
          rv[k] = (c[k] & kClosed) ? (LabelT)global_index(lat, x0, y0, c[k] & kIdx) : oroot[c[k]];
        if (lat.vec4 && lx0 + 4 <= w) {
          // four roots at once (gi is a multiple of 4 when L is)
          if constexpr (sizeof(LabelT) == 4) {
            *reinterpret_cast<uint4*>(roots + gi) = make_uint4((uint32_t)rv[0], (uint32_t)rv[1], (uint32_t)rv[2], (uint32_t)rv[3]);
          } else {
            *reinterpret_cast<ulonglong2*>(roots + gi) = make_ulonglong2(rv[0], rv[1]);
            *reinterpret_cast<ulonglong2*>(roots + gi + 2) = make_ulonglong2(rv[2], rv[3]);
          }
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (lx0 + k < w) roots[gi + k] = rv[k];
        }
      } else {
        uint32_t ok = 0;  // old spins (XY only)
        if constexpr (kXY) {
          if (lat.vec4) {
            ok = *reinterpret_cast<const uint32_t*>(b.spin + gi);
          } else {
#pragma unroll
            for (int k = 0; k < 4; ++k)
              if (lx0 + k < w) ok |= (uint32_t)b.spin[gi + k] << (8 * k);
          }
        }
        uint32_t s = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint32_t v = (c[k] & kClosed) ? (c[k] & 0xFFu) : nso[c[k]];
          s |= next(v, (ok >> (8 * k)) & 0xFFu) << (8 * k);
        }
        if (lat.vec4) {
          *reinterpret_cast<uint32_t*>(b.spin + gi) = s;
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (lx0 + k < w) b.spin[gi + k] = (uint8_t)(s >> (8 * k));
        }
      }
    }
  }
}

// ================================================================== init / measure
static __global__ void k_init_spins(uint8_t* s, uint64_t N, uint32_t q, uint64_t seed) {
  const uint64_t nq = (N + 3) >> 2;
  for (uint64_t qd = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; qd < nq;
       qd += (uint64_t)gridDim.x * blockDim.x) {
    const Words4 wv = stream4(seed, qd, 0u, kDomInit);
    const uint32_t v = pick_state(wv.x, q) | (pick_state(wv.y, q) << 8) |
                       (pick_state(wv.z, q) << 16) | (pick_state(wv.w, q) << 24);
    const uint64_t i = qd << 2;
    if (i + 3 < N) {
      *reinterpret_cast<uint32_t*>(s + i) = v;
    } else {
      for (int k = 0; i + k < N; ++k) s[i + k] = (uint8_t)(v >> (8 * k));
    }
  }
}

// Block reduction of one thread's measurement counts (E_sat, the states
// 0 .. qs-1 counted in registers, sites) into hist[] and then acc[]; q > 8
// (qs = 0) has counted its states in hist[1 + s] already.
__device__ __forceinline__ void measure_flush(uint32_t* hist, uint32_t e, uint32_t (&cnt)[7],
                                              uint32_t nsites, uint32_t qs, uint32_t q,
                                              unsigned long long* acc) {
  for (int o = 16; o > 0; o >>= 1) {
    e += __shfl_xor_sync(0xFFFFFFFFu, e, o);
    nsites += __shfl_xor_sync(0xFFFFFFFFu, nsites, o);
  }
  if (qs) {
#pragma unroll
    for (uint32_t st = 0; st < 7; ++st)
      for (int o = 16; o > 0; o >>= 1) cnt[st] += __shfl_xor_sync(0xFFFFFFFFu, cnt[st], o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&hist[0], e);
    if (qs) {
      uint32_t rest = nsites;
      for (uint32_t st = 0; st < qs; ++st) {
        atomicAdd(&hist[1 + st], cnt[st]);
        rest -= cnt[st];
      }
      atomicAdd(&hist[1 + qs], rest);
    }
  }
  __syncthreads();
  for (uint32_t k = threadIdx.x; k <= q; k += blockDim.x)
    if (hist[k]) atomicAdd(&acc[k], (unsigned long long)hist[k]);
}

// E_sat and n[s] for L a multiple of 16, streaming: thread (gx, strip)
// holds the 16 sites gx*16 .. gx*16+15 of row y in registers, loads row y+1
// (its down neighbours, then its own sites of the next step) and takes the
// right neighbour of its last site from the next lane.  A strip of
// kMeasRows rows reads each spin once plus one extra row, with kMeasAhead
// rows' loads in flight per thread.
//
// States are counted by bit planes for q <= 2^B (B = 1, 2, 3): c[T-1]
// counts the sites that have every bit of the plane set T (T = 1 .. 2^B-1)
// set, and n[s] = sum over T containing s of (-1)^(|T|-|s|) c[T-1]
// (Moebius inversion over the subsets), n[0] = sites - the rest.  B = 0:
// q > 8, every site counted in a shared histogram.
constexpr uint32_t kMeasRows = 64, kMeasAhead = 4;
template <int B>
static __global__ void __launch_bounds__(256) k_measure16(const uint8_t* s, uint64_t L, uint32_t q,
                                                   unsigned long long* acc) {
  constexpr int NC = B ? (1 << B) - 1 : 1;
  __shared__ uint32_t hist[257];
  __shared__ uint32_t bsites;
  for (int k = threadIdx.x; k < 257; k += blockDim.x) hist[k] = 0;
  if (threadIdx.x == 0) bsites = 0;
  __syncthreads();
  const uint64_t g16 = L >> 4;
  const uint64_t gx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = gx < g16;
  const uint64_t x = live ? gx * 16 : 0;
  const uint64_t xn = (x + 16 == L) ? 0 : x + 16;  // first site of the next group
  const bool edge = (threadIdx.x & 31) == 31 || gx + 1 >= g16;  // next group not in this warp
  const uint64_t y0 = (uint64_t)blockIdx.y * kMeasRows;
  const uint32_t rows = (uint32_t)(L - y0 < kMeasRows ? L - y0 : kMeasRows);
  uint32_t e = 0, nsites = 0, c[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) c[k] = 0;
  auto ld = [&](uint64_t y) -> uint4 {
    const uint64_t yy = y >= L ? y - L : y;
    return live ? __ldcs(reinterpret_cast<const uint4*>(s + yy * L + x)) : make_uint4(0, 0, 0, 0);
  };
  // bit 7 of each byte of the result: that byte of a ^ b is zero
  auto eq_hi = [](uint32_t a, uint32_t b) -> uint32_t {
    const uint32_t d = a ^ b;
    if constexpr (B != 0) return ~(d + 0x7F7F7F7Fu) & 0x80808080u;  // bytes < 128 (q <= 8)
    else return ~(((d & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | d) & 0x80808080u;
  };
  uint4 v = ld(y0);
  for (uint32_t r = 0; r < rows; r += kMeasAhead) {
    uint4 nxt[kMeasAhead];
#pragma unroll
    for (uint32_t k = 0; k < kMeasAhead; ++k)
      nxt[k] = (r + k < rows) ? ld(y0 + r + k + 1) : make_uint4(0, 0, 0, 0);
#pragma unroll
    for (uint32_t k = 0; k < kMeasAhead; ++k) {
      if (r + k >= rows) break;  // uniform over the block
      uint32_t nx = __shfl_down_sync(0xFFFFFFFFu, v.x, 1);
      if (edge && live) nx = *reinterpret_cast<const uint32_t*>(s + (y0 + r + k) * L + xn);
      if (live) {
        const uint32_t w4[5] = {v.x, v.y, v.z, v.w, nx};
        const uint32_t d4[4] = {nxt[k].x, nxt[k].y, nxt[k].z, nxt[k].w};
        // the four words' flags packed into disjoint bits, one popcount per
        // 16 sites: equal right / down neighbours of word j at bits 7-2j and
        // 6-2j of each byte, plane-set bits of word j at bit j
        uint32_t eb = 0, pc[NC];
#pragma unroll
        for (int t = 0; t < NC; ++t) pc[t] = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint32_t w = w4[j];
          eb |= (eq_hi(w, __funnelshift_r(w, w4[j + 1], 8)) | (eq_hi(w, d4[j]) >> 1)) >> (2 * j);
          if constexpr (B == 0) {
            for (int b = 0; b < 4; ++b) atomicAdd(&hist[1 + ((w >> (8 * b)) & 0xFFu)], 1u);
          } else {
            const uint32_t p0 = w & 0x01010101u;
            pc[0] |= p0 << j;
            if constexpr (B >= 2) {
              const uint32_t p1 = (w >> 1) & 0x01010101u;
              pc[1] |= p1 << j;
              pc[2] |= (p0 & p1) << j;
              if constexpr (B == 3) {
                const uint32_t p2 = (w >> 2) & 0x01010101u;
                pc[3] |= p2 << j;
                pc[4] |= (p0 & p2) << j;
                pc[5] |= (p1 & p2) << j;
                pc[6] |= (p0 & p1 & p2) << j;
              }
            }
          }
        }
        e += __popc(eb);
        if constexpr (B != 0) {
#pragma unroll
          for (int t = 0; t < NC; ++t) c[t] += __popc(pc[t]);
        }
        nsites += 16;
      }
      v = nxt[k];
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    e += __shfl_xor_sync(0xFFFFFFFFu, e, o);
    nsites += __shfl_xor_sync(0xFFFFFFFFu, nsites, o);
#pragma unroll
    for (int k = 0; k < NC; ++k) c[k] += __shfl_xor_sync(0xFFFFFFFFu, c[k], o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&hist[0], e);
    if constexpr (B != 0) {
      atomicAdd(&bsites, nsites);
      for (uint32_t st = 1; st < q; ++st) {
        int64_t n = 0;
        for (uint32_t T = st; T < (1u << B); ++T)
          if ((T & st) == st) n += ((__popc(T) - __popc(st)) & 1) ? -(int64_t)c[T - 1] : (int64_t)c[T - 1];
        atomicAdd(&hist[1 + st], (uint32_t)n);
      }
    }
  }
  __syncthreads();
  if constexpr (B != 0) {
    if (threadIdx.x == 0) {
      uint32_t rest = bsites;
      for (uint32_t st = 1; st < q; ++st) rest -= hist[1 + st];
      hist[1] = rest;  // n[0]
    }
    __syncthreads();
  }
  for (uint32_t k = threadIdx.x; k <= q; k += blockDim.x)
    if (hist[k]) atomicAdd(&acc[k], (unsigned long long)hist[k]);
}

// E_sat and n[s] of a configuration (the configuration no later sweep reads),
// any L: one thread per group of 4 sites of a row; 4-byte loads when rows
// are 4-byte aligned, per-state counts in registers for q <= 8.  Lattices
// with L a multiple of 16 take k_measure16.
static __global__ void __launch_bounds__(256) k_measure(const uint8_t* s, Lattice lat, uint32_t q,
                                                 unsigned long long* acc) {
  __shared__ uint32_t hist[257];
  for (int k = threadIdx.x; k < 257; k += blockDim.x) hist[k] = 0;
  __syncthreads();
  const uint64_t L = lat.L;
  const uint64_t groups = (L + 3) >> 2;
  const uint32_t qs = q <= 8 ? q - 1 : 0;
  uint32_t e = 0, cnt[7] = {0, 0, 0, 0, 0, 0, 0}, nsites = 0;
  // rows over blocks, 4-site groups of a row over threads
  for (uint64_t y = blockIdx.x; y < L; y += gridDim.x) {
    const uint64_t yd = (y + 1 == L) ? 0 : y + 1;
    for (uint64_t gx = threadIdx.x; gx < groups; gx += blockDim.x) {
      const uint64_t x = gx * 4;
      uint32_t v, vr, vd, vm;
      if (lat.vec4) {
        v = *reinterpret_cast<const uint32_t*>(s + y * L + x);
        const uint64_t xn = (x + 4 == L) ? 0 : x + 4;
        const uint32_t vn = *reinterpret_cast<const uint32_t*>(s + y * L + xn);
        vr = __funnelshift_r(v, vn, 8);
        vd = *reinterpret_cast<const uint32_t*>(s + yd * L + x);
        vm = 0xFFFFFFFFu;
      } else {
        v = vr = vd = vm = 0;
        for (int k = 0; k < 4 && x + k < L; ++k) {
          const uint64_t xk = x + k, xr = (xk + 1 == L) ? 0 : xk + 1;
          v |= (uint32_t)s[y * L + xk] << (8 * k);
          vr |= (uint32_t)s[y * L + xr] << (8 * k);
          vd |= (uint32_t)s[yd * L + xk] << (8 * k);
          vm |= 0xFFu << (8 * k);
        }
      }
      const uint32_t vnib = zero_bytes4(~vm);  // valid sites of the group
      e += __popc(zero_bytes4(v ^ vr) & vnib) + __popc(zero_bytes4(v ^ vd) & vnib);
      nsites += __popc(vnib);
      if (qs) {
#pragma unroll
        for (uint32_t st = 0; st < 7; ++st)
          if (st < qs) cnt[st] += __popc(zero_bytes4(v ^ (st * 0x01010101u)) & vnib);
      } else {
        for (int k = 0; k < 4; ++k)
          if ((vm >> (8 * k)) & 1u) atomicAdd(&hist[1 + ((v >> (8 * k)) & 0xFFu)], 1u);
      }
    }
  }
  measure_flush(hist, e, cnt, nsites, qs, q, acc);
}

// Sets *bad if any of the N spins is >= q (validation of a new configuration).
static __global__ void k_check_spins(const uint8_t* s, uint64_t N, uint32_t q, uint32_t* bad) {
  uint32_t any = 0;
  const uint64_t nw = N >> 2;
  const uint32_t lim = q * 0x01010101u;  // q <= 255: per-byte "value >= q" via __vcmpgeu4
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nw;
       i += (uint64_t)gridDim.x * blockDim.x)
    any |= __vcmpgeu4(reinterpret_cast<const uint32_t*>(s)[i], lim);
  if (blockIdx.x == 0)
    for (uint64_t i = (nw << 2) + threadIdx.x; i < N; i += blockDim.x) any |= (s[i] >= q);
  if (__any_sync(0xFFFFFFFFu, any != 0) && (threadIdx.x & 31) == 0) atomicOr(bad, 1u);
}

// Copies N spins from page-locked host memory (read through its device
// mapping, 16 B per load, many loads in flight) into the lattice and checks
// them on the way: *bad is set if a spin is >= q.  src and dst 16-byte
// aligned.
static __global__ void __launch_bounds__(256) k_copy_check_spins(const uint8_t* __restrict__ src,
                                                                 uint8_t* __restrict__ dst, uint64_t N,
                                                                 uint32_t q, uint32_t* bad) {
  const uint32_t lim = q * 0x01010101u;
  const uint64_t n16 = N >> 4;
  const uint4* s16 = reinterpret_cast<const uint4*>(src);
  uint4* d16 = reinterpret_cast<uint4*>(dst);
  uint32_t any = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n16; i += 4 * stride) {  // four 16-byte loads in flight per thread
    uint4 v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = s16[i + k * stride];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      any |= __vcmpgeu4(v[k].x, lim) | __vcmpgeu4(v[k].y, lim) | __vcmpgeu4(v[k].z, lim) |
             __vcmpgeu4(v[k].w, lim);
      d16[i + k * stride] = v[k];
    }
  }
  for (; i < n16; i += stride) {
    const uint4 v = s16[i];
    any |= __vcmpgeu4(v.x, lim) | __vcmpgeu4(v.y, lim) | __vcmpgeu4(v.z, lim) | __vcmpgeu4(v.w, lim);
    d16[i] = v;
  }
  if (blockIdx.x == 0)
    for (uint64_t j = (n16 << 4) + threadIdx.x; j < N; j += blockDim.x) {
      const uint8_t v = src[j];
      dst[j] = v;
      any |= (v >= q);
    }
  if (__any_sync(0xFFFFFFFFu, any != 0) && (threadIdx.x & 31) == 0) atomicOr(bad, 1u);
}

// Files the accumulated observables as configuration ctl[0].
static __global__ void k_commit(Bufs b) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const unsigned long long s = b.ctl[0];
    unsigned long long* rec = b.ring + (s % b.ring_cap) * (2ull + b.q);
    rec[0] = s;
    for (uint32_t k = 0; k <= b.q; ++k) {
      rec[1 + k] = b.acc[k];
      b.acc[k] = 0ull;
    }
  }
}

}  // namespace swgb
