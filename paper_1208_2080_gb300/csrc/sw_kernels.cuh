// sw_kernels.cuh -- sm_103a kernels of one Swendsen-Wang sweep.
//
// A sweep is four launches over a tiling of the L x L lattice into
// 128 x TH tiles (tile t = ty*ntx + tx, origin (128*tx, TH*ty); the last
// tile row/column is ragged when TH or 128 does not divide L):
//
//   k_label_rows  (sw_label.cuh; persistent, a CTA per tile at a time)
//       Sec. 2 steps (1)+(2), tile-local part: draw the bonds (Philox, one
//       call per two sites), measure E_sat / n[s] of the configuration it
//       reads (Sec. 4), label the tile with a shared-memory union-find over
//       horizontal run starts; a cluster that touches the tile edge is
//       "open", the others are complete and get their new state there
//       (Sec. 2 step (3)), drawn once per cluster from their root = smallest
//       site index.  Per site it writes a 16-bit code: 0x8000|state for a
//       closed cluster, the slot of its open root otherwise.  For the
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
// with the embedded bond rule in k_label_rows and reflections in
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

constexpr int kTW = 128;                  // tile width
constexpr int kThreads = 512;             // threads of a k_recolor block (a tile)
constexpr int kWarps = kThreads / 32;
constexpr uint32_t kIdx = 0x7FFFu;        // payload bits of a closed code
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
  uint32_t measure;           // 1: the labeller accumulates observables of its input
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
