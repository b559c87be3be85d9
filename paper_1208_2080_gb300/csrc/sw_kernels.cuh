// sw_kernels.cuh -- sm_103a kernels of one Swendsen-Wang sweep.
//
// A sweep is three launches over a tiling of the L x L lattice into
// 128 x TH tiles (tile t = ty*ntx + tx, origin (128*tx, TH*ty); the last
// tile row/column is ragged when TH or 128 does not divide L):
//
//   k_label_tile  (one CTA per tile)  Sec. 2 steps (1)+(2), tile-local part:
//       stage the tile's uint8 spins plus a one-site right/down halo in
//       shared memory; draw the bonds (Philox, one call per two sites);
//       measure E_sat / n[s] of the configuration it reads (Sec. 4); label
//       the tile with a shared-memory union-find: horizontal runs inside a
//       warp's 128-site row come from one __ballot_sync, vertical bonds are
//       atomicMin unions (redundant ones between the same two runs skipped);
//       a cluster that touches the tile edge is "open", the others are
//       complete and get their new state here (Sec. 2 step (3)), drawn once
//       per cluster from their root = smallest site index.  Per site it
//       writes a 16-bit code: 0x8000|state for a closed cluster, the local
//       root index for an open one.  For the boundary pass it writes the
//       local roots of the four edge lines, the cross-edge bond bits, the
//       list of open local roots, and initialises their global labels.
//   k_merge       Sec. 2 step (2), global part: the single-GPU analogue of
//       the paper's boundary-only inter-GPU labelling (Sec. 3): for every
//       active bond that crosses a tile edge (periodic wrap included) a
//       lock-free atomicMin union of the two open roots' global labels
//       (site indices, uint32 or uint64), lanes that would repeat the same
//       union are merged with __match_any_sync.
//   k_recolor     Sec. 2 step (3) for open clusters: each open local root
//       finds (and compresses to) its global root, draws the cluster state;
//       every site then writes its new uint8 spin.
//
// Union always links the larger root under the smaller one, so the final
// root of every cluster is its smallest site index -- the Hoshen-Kopelman
// "proper label" of Sec. 2 -- independent of the order in which the GPU
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
constexpr int kSpPitch = 132;             // smem spin row: 128 sites, halo, pad
constexpr uint32_t kOpen = 0x80000000u;   // smem root flag: cluster touches tile edge
constexpr uint32_t kIdx = 0x7FFFu;        // local index bits
constexpr uint16_t kClosed = 0x8000u;     // code flag: cluster complete in tile
constexpr uint32_t kFindCap = 1u << 24;   // bound on any global union-find walk
constexpr uint32_t kLocalCap = 1u << 16;  // bound on any shared-memory walk
constexpr int kMergeThreads = 256;

enum : uint32_t { kErrFind = 1u, kErrUnion = 2u, kErrLocal = 4u };

__host__ __device__ constexpr int align16(int x) { return (x + 15) & ~15; }

// Per-tile record sizes.
template <int TH>
struct TileRec {
  static constexpr int kEdge = 2 * TH + 2 * kTW;           // u16: right col, left col, bottom, top
  static constexpr int kRightWords = (TH + 31) / 32;       // cross-right bits
  static constexpr int kBitWords = kRightWords + kTW / 32; // + cross-down bits
  static constexpr int kOpenCap = 2 * TH + 2 * kTW;        // open roots <= edge sites
};

// Shared-memory layout of k_label_tile.
template <int TH>
struct LabelSmem {
  static constexpr int kP = 0;                                     // u32 [kTW*TH] union-find
  static constexpr int kSp = kP + 4 * kTW * TH;                    // u8 [(TH+1)*kSpPitch]
  static constexpr int kRbn = align16(kSp + (TH + 1) * kSpPitch);  // u8 [TH*32] right-bond nibbles
  static constexpr int kCb = align16(kRbn + TH * 32);              // u32 cross bits
  static constexpr int kCnt = align16(kCb + 4 * TileRec<TH>::kBitWords);  // u32 [4]
  static constexpr int kObs = align16(kCnt + 16);                  // u32 [1 + 256]
  static constexpr int kCl = align16(kObs + 4 * 257);              // u16 [kTW*TH] closed roots
  static constexpr int kBytes = align16(kCl + 2 * kTW * TH);
};

struct Lattice {
  uint64_t L;
  uint32_t ntx, nty;  // tiles across / down
  uint64_t bp;        // packed-bond row pitch in bytes, ceil(L/4)
  uint32_t vec4;      // L % 4 == 0: rows start 4-byte aligned
  uint32_t ntiles;
};

struct Bufs {
  uint8_t* spin;              // N spins
  uint16_t* code;             // N per-site codes
  uint8_t* bonds;             // packed bonds (out, or in for the given-bond mode) or null
  void* T;                    // N global labels (LabelT); only open roots are touched
  uint16_t* edge;             // ntiles * kEdge
  uint32_t* ebits;            // ntiles * kBitWords
  uint16_t* olist;            // ntiles * kOpenCap
  uint32_t* ocnt;             // ntiles
  unsigned long long* acc;    // [1 + q]: E_sat, n[q] of the configuration being measured
  unsigned long long* ring;   // [ring_cap][2 + q]: tag, E_sat, n[q]
  unsigned long long* ctl;    // [0] next sweep, [1] sweep being recoloured
  uint32_t* err;              // device error bits
  uint64_t seed;
  uint32_t thr, q;
  uint32_t ring_cap;
  uint32_t measure;           // 1: k_label_tile accumulates observables of its input
};

__device__ __forceinline__ void tile_geom(const Lattice& lat, uint32_t t, int TH, uint64_t& x0,
                                          uint64_t& y0, int& w, int& h) {
  const uint32_t tx = t % lat.ntx, ty = t / lat.ntx;
  x0 = (uint64_t)tx * kTW;
  y0 = (uint64_t)ty * TH;
  const uint64_t rw = lat.L - x0, rh = lat.L - y0;
  w = rw < (uint64_t)kTW ? (int)rw : kTW;
  h = rh < (uint64_t)TH ? (int)rh : TH;
}

// ---------------------------------------------------------------- shared-memory union-find
__device__ __forceinline__ uint32_t find_local(const uint32_t* P, uint32_t x, uint32_t& bad) {
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

// ---------------------------------------------------------------- global union-find
template <typename LabelT>
__device__ __forceinline__ LabelT ldcg(const LabelT* p);
template <>
__device__ __forceinline__ uint32_t ldcg<uint32_t>(const uint32_t* p) {
  return __ldcg(p);
}
template <>
__device__ __forceinline__ uint64_t ldcg<uint64_t>(const uint64_t* p) {
  return (uint64_t)__ldcg(reinterpret_cast<const unsigned long long*>(p));
}

__device__ __forceinline__ uint32_t atomic_min_label(uint32_t* p, uint32_t v) { return atomicMin(p, v); }
__device__ __forceinline__ uint64_t atomic_min_label(uint64_t* p, uint64_t v) {
  return (uint64_t)atomicMin(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}

// Root of x with path halving.  The halving stores only ever replace a
// parent by one of its ancestors, so they cannot undo a concurrent link.
template <typename LabelT>
__device__ __forceinline__ LabelT find_global(LabelT* T, LabelT x, uint32_t* err) {
  for (uint32_t it = 0; it < kFindCap; ++it) {
    const LabelT p = ldcg(T + x);
    if (p == x) return x;
    const LabelT gp = ldcg(T + p);
    if (gp == p) return p;
    T[x] = gp;
    x = gp;
  }
  atomicOr(err, kErrFind);
  return x;
}

template <typename LabelT>
__device__ __forceinline__ void unite_global(LabelT* T, LabelT a, LabelT b, uint32_t* err) {
  for (uint32_t it = 0; it < kFindCap; ++it) {
    a = find_global(T, a, err);
    b = find_global(T, b, err);
    if (a == b) return;
    if (a < b) {
      const LabelT tmp = a;
      a = b;
      b = tmp;
    }
    const LabelT old = atomic_min_label(T + a, b);
    if (old == a) return;
    a = old;
  }
  atomicOr(err, kErrUnion);
}

__device__ __forceinline__ uint64_t global_index(const Lattice& lat, uint64_t x0, uint64_t y0,
                                                 uint32_t local) {
  return (y0 + (local >> 7)) * lat.L + x0 + (local & (kTW - 1));
}

__device__ __forceinline__ uint32_t byte_mask(uint32_t nib) {
  // 4-bit site mask -> 0xFF per selected byte
  return ((nib & 1u) ? 0x000000FFu : 0u) | ((nib & 2u) ? 0x0000FF00u : 0u) |
         ((nib & 4u) ? 0x00FF0000u : 0u) | ((nib & 8u) ? 0xFF000000u : 0u);
}

// ================================================================== k_label_tile
// kGiven: bonds are read from b.bonds instead of drawn (labelling-only entry).
// kRoots: closed clusters keep their local root in the code (no new state).
template <int TH, typename LabelT, bool kGiven, bool kRoots>
__global__ void __launch_bounds__(kThreads) k_label_tile(const Bufs b, const Lattice lat) {
  static_assert(TH % kWarps == 0 && kTW * TH <= 32768, "tile shape");
  using S = LabelSmem<TH>;
  using R = TileRec<TH>;
  constexpr int kRpw = TH / kWarps;  // rows per warp
  constexpr unsigned kFull = 0xFFFFFFFFu;

  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* P = reinterpret_cast<uint32_t*>(smem + S::kP);
  uint8_t* sp = smem + S::kSp;
  uint8_t* rbn = smem + S::kRbn;
  uint32_t* cbits = reinterpret_cast<uint32_t*>(smem + S::kCb);
  uint32_t* cnt = reinterpret_cast<uint32_t*>(smem + S::kCnt);
  uint32_t* sobs = reinterpret_cast<uint32_t*>(smem + S::kObs);
  uint16_t* clist = reinterpret_cast<uint16_t*>(smem + S::kCl);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t t = blockIdx.x;
  uint64_t x0, y0;
  int w, h;
  tile_geom(lat, t, TH, x0, y0, w, h);
  const uint64_t L = lat.L;
  const uint32_t q = b.q;
  const bool measure = !kGiven && b.measure;
  const uint32_t sweep = kGiven ? 0u : (uint32_t)b.ctl[0];
  uint32_t bad = 0;

  for (int k = tid; k < R::kBitWords; k += kThreads) cbits[k] = 0;
  if (tid < 4) cnt[tid] = 0;
  if (measure)
    for (int k = tid; k < 257; k += kThreads) sobs[k] = 0;

  // ---- stage spins (tile rows 0..h-1 plus the halo row h and column w)
  if (!kGiven) {
    for (int ly = warp; ly <= h; ly += kWarps) {
      const uint64_t gy = (ly < h) ? (y0 + ly) : ((y0 + h) % L);
      const uint8_t* row = b.spin + gy * L + x0;
      uint32_t v = 0;
      const int lx0 = 4 * lane;
      if (lx0 < w) {
        if (lat.vec4) {
          v = *reinterpret_cast<const uint32_t*>(row + lx0);
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (lx0 + k < w) v |= (uint32_t)row[lx0 + k] << (8 * k);
        }
      }
      *reinterpret_cast<uint32_t*>(sp + ly * kSpPitch + lx0) = v;
      __syncwarp();
      if (lane == 0) sp[ly * kSpPitch + w] = b.spin[gy * L + (x0 + w) % L];
    }
  }
  __syncthreads();

  // ---- bonds, measurement, horizontal runs
  const int lx0 = 4 * lane;
  uint32_t R4[kRpw], D4[kRpw];
  uint32_t e_loc = 0;
  uint32_t ncnt[7] = {0, 0, 0, 0, 0, 0, 0};
  const uint32_t qs = q <= 8 ? q - 1 : 0;  // states counted in registers
#pragma unroll
  for (int rr = 0; rr < kRpw; ++rr) {
    const int ly = warp + rr * kWarps;
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
      const uint32_t s = *reinterpret_cast<const uint32_t*>(sp + ly * kSpPitch + lx0);
      const uint32_t sn = *reinterpret_cast<const uint32_t*>(sp + ly * kSpPitch + lx0 + 4);
      const uint32_t sd = *reinterpret_cast<const uint32_t*>(sp + (ly + 1) * kSpPitch + lx0);
      const uint32_t sr = __funnelshift_r(s, sn, 8);
      const uint32_t vb = byte_mask(vm);
      const uint32_t eqr = __vcmpeq4(s, sr) & vb;
      const uint32_t eqd = __vcmpeq4(s, sd) & vb;
      if (measure) {
        e_loc += __popc(eqr & 0x01010101u) + __popc(eqd & 0x01010101u);
        if (qs) {
#pragma unroll
          for (uint32_t st = 0; st < 7; ++st)
            if (st < qs) ncnt[st] += __popc(__vcmpeq4(s, st * 0x01010101u) & vb & 0x01010101u);
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (vm & (1u << k)) atomicAdd(&sobs[1 + ((s >> (8 * k)) & 0xFFu)], 1u);
        }
      }
      if ((eqr | eqd) != 0u) {
        const uint64_t i0 = (y0 + ly) * L + x0 + lx0;
        const uint64_t pa = i0 >> 1;
        const Words4 A = stream4(b.seed, pa, sweep, kDomBond);
        const Words4 B = stream4(b.seed, pa + 1, sweep, kDomBond);
        uint32_t wr[4], wd[4];
        if ((i0 & 1u) == 0u) {
          wr[0] = A.x; wd[0] = A.y; wr[1] = A.z; wd[1] = A.w;
          wr[2] = B.x; wd[2] = B.y; wr[3] = B.z; wd[3] = B.w;
        } else {
          const Words4 C = stream4(b.seed, pa + 2, sweep, kDomBond);
          wr[0] = A.z; wd[0] = A.w; wr[1] = B.x; wd[1] = B.y;
          wr[2] = B.z; wd[2] = B.w; wr[3] = C.x; wd[3] = C.y;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          br |= (((eqr >> (8 * k)) & 1u) & (wr[k] < b.thr ? 1u : 0u)) << k;
          bd |= (((eqd >> (8 * k)) & 1u) & (wd[k] < b.thr ? 1u : 0u)) << k;
        }
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
    R4[rr] = r4;
    D4[rr] = d4;
    // horizontal runs: a site whose left bond is inactive starts a run; every
    // site's provisional label is its run start (one ballot per row)
    uint32_t prev3 = __shfl_up_sync(kFull, (r4 >> 3) & 1u, 1);
    if (lane == 0) prev3 = 0;
    const uint32_t brk = (~((r4 << 1) | prev3)) & 0xFu;
    const uint32_t B = __ballot_sync(kFull, brk != 0u);
    const int lb = brk ? 31 - __clz(brk) : 0;
    const uint32_t below = B & ((1u << lane) - 1u);
    const int src = below ? 31 - __clz(below) : 0;
    const int lbs = __shfl_sync(kFull, lb, src);
    if (ly < TH) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t m = brk & ((2u << k) - 1u);
        const int start = m ? lx0 + 31 - __clz(m) : 4 * src + lbs;
        P[ly * kTW + lx0 + k] = (uint32_t)(ly * kTW + start);
      }
      rbn[ly * 32 + lane] = (uint8_t)r4;
    }
  }
  __syncthreads();

  // ---- vertical unions (skip the ones that repeat the left neighbour's)
#pragma unroll
  for (int rr = 0; rr < kRpw; ++rr) {
    const int ly = warp + rr * kWarps;
    if (ly < h - 1) {
      const uint32_t d4 = D4[rr], r4 = R4[rr];
      const uint32_t rb = rbn[(ly + 1) * 32 + lane];
      uint32_t pd = __shfl_up_sync(kFull, (d4 >> 3) & 1u, 1);
      uint32_t pr = __shfl_up_sync(kFull, (r4 >> 3) & 1u, 1);
      uint32_t pb = lane > 0 ? (rbn[(ly + 1) * 32 + lane - 1] >> 3) & 1u : 0u;
      if (lane == 0) pd = pr = pb = 0;
      const uint32_t skip = ((d4 << 1) | pd) & ((r4 << 1) | pr) & ((rb << 1) | pb);
      uint32_t todo = d4 & ~skip & 0xFu;
      while (todo) {
        const int k = __ffs(todo) - 1;
        todo &= todo - 1u;
        const uint32_t a = (uint32_t)(ly * kTW + lx0 + k);
        unite_local(P, a, a + kTW, bad);
      }
    }
  }
  __syncthreads();

  // ---- compress: every site points at its tile-local root
#pragma unroll
  for (int rr = 0; rr < kRpw; ++rr) {
    const int ly = warp + rr * kWarps;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t j = (uint32_t)(ly * kTW + lx0 + k);
      P[j] = find_local(P, j, bad);
    }
  }
  __syncthreads();

  // ---- mark clusters that touch the tile edge as open
#pragma unroll
  for (int rr = 0; rr < kRpw; ++rr) {
    const int ly = warp + rr * kWarps;
    if (ly < h) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int lx = lx0 + k;
        if (lx < w && (lx == 0 || lx == w - 1 || ly == 0 || ly == h - 1)) {
          const uint32_t j = (uint32_t)(ly * kTW + lx);
          atomicOr(&P[P[j] & kIdx], kOpen);
        }
      }
    }
  }
  __syncthreads();

  // ---- root lists: closed roots to smem, open roots to the tile's record
  LabelT* T = reinterpret_cast<LabelT*>(b.T);
  const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int rr = 0; rr < kRpw; ++rr) {
    const int ly = warp + rr * kWarps;
    if (ly < h) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int lx = lx0 + k;
        const uint32_t j = (uint32_t)(ly * kTW + lx);
        const uint32_t v = lx < w ? P[j] : 0u;
        const bool isroot = lx < w && (v & kIdx) == j;
        const bool open = isroot && (v & kOpen);
        const bool closed = isroot && !(v & kOpen);
        const unsigned mc = __ballot_sync(kFull, closed);
        if (mc) {
          uint32_t base = 0;
          if (lane == __ffs(mc) - 1) base = atomicAdd(&cnt[0], (uint32_t)__popc(mc));
          base = __shfl_sync(kFull, base, __ffs(mc) - 1);
          if (closed) clist[base + __popc(mc & lt_mask)] = (uint16_t)j;
        }
        const unsigned mo = __ballot_sync(kFull, open);
        if (mo) {
          uint32_t base = 0;
          if (lane == __ffs(mo) - 1) base = atomicAdd(&cnt[1], (uint32_t)__popc(mo));
          base = __shfl_sync(kFull, base, __ffs(mo) - 1);
          if (open) {
            b.olist[(uint64_t)t * R::kOpenCap + base + __popc(mo & lt_mask)] = (uint16_t)j;
            const uint64_t g = global_index(lat, x0, y0, j);
            T[g] = (LabelT)g;
          }
        }
      }
    }
  }
  __syncthreads();

  // ---- new state of each complete cluster, drawn once at its root
  if (!kRoots) {
    const uint32_t nc = cnt[0];
    for (uint32_t k = tid; k < nc; k += kThreads) {
      const uint32_t j = clist[k];
      const uint32_t st = cluster_state(b.seed, global_index(lat, x0, y0, j), sweep, q);
      P[j] = j | (st << 16);
    }
    __syncthreads();
  }

  // ---- per-site codes and the edge lines
  uint16_t* edge = b.edge + (uint64_t)t * R::kEdge;
#pragma unroll
  for (int rr = 0; rr < kRpw; ++rr) {
    const int ly = warp + rr * kWarps;
    if (ly < h && lx0 < w) {
      uint32_t c[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t j = (uint32_t)(ly * kTW + lx0 + k);
        const uint32_t r = P[j] & kIdx;
        const uint32_t vr = P[r];
        c[k] = (vr & kOpen) ? r : (kRoots ? (kClosed | r) : (kClosed | ((vr >> 16) & 0xFFu)));
      }
      const uint64_t gi = (y0 + ly) * L + x0 + lx0;
      if (lat.vec4) {
        *reinterpret_cast<uint2*>(b.code + gi) = make_uint2(c[0] | (c[1] << 16), c[2] | (c[3] << 16));
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (lx0 + k < w) b.code[gi + k] = (uint16_t)c[k];
      }
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
  for (int k = tid; k < R::kBitWords; k += kThreads) b.ebits[(uint64_t)t * R::kBitWords + k] = cbits[k];
  if (tid == 0) b.ocnt[t] = cnt[1];

  // ---- observables of the configuration read (Sec. 4)
  if (measure) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e_loc += __shfl_xor_sync(kFull, e_loc, o);
    if (lane == 0) atomicAdd(&sobs[0], e_loc);
    if (qs) {
#pragma unroll
      for (uint32_t st = 0; st < 7; ++st) {
        if (st < qs) {
          uint32_t v = ncnt[st];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
          if (lane == 0) atomicAdd(&sobs[1 + st], v);
        }
      }
    }
    __syncthreads();
    if (qs) {
      if (tid == 0) {
        uint32_t rest = (uint32_t)(w * h);
        for (uint32_t st = 0; st < qs; ++st) rest -= sobs[1 + st];
        sobs[1 + qs] = rest;
      }
      __syncthreads();
    }
    for (uint32_t k = tid; k <= q; k += kThreads)
      if (sobs[k]) atomicAdd(&b.acc[k], (unsigned long long)sobs[k]);
  }
  if (bad) atomicOr(b.err, kErrLocal);
}

// ================================================================== k_merge
// One thread per edge position of every tile: TH right-edge rows, then the
// 128 bottom-edge columns.  Block 0 / thread 0 also files the observables
// of the configuration k_label_tile read and advances the sweep counter.
template <int TH, typename LabelT>
__global__ void __launch_bounds__(kMergeThreads) k_merge(const Bufs b, const Lattice lat) {
  using R = TileRec<TH>;
  constexpr int kPer = TH + kTW;
  const uint64_t item = (uint64_t)blockIdx.x * kMergeThreads + threadIdx.x;
  const uint32_t t = (uint32_t)(item / kPer);
  const int pos = (int)(item % kPer);
  LabelT a = (LabelT)~(LabelT)0, c = (LabelT)~(LabelT)0;
  bool active = false;
  if (t < lat.ntiles) {
    uint64_t x0, y0;
    int w, h;
    tile_geom(lat, t, TH, x0, y0, w, h);
    const uint32_t tx = t % lat.ntx, ty = t / lat.ntx;
    const uint32_t* bits = b.ebits + (uint64_t)t * R::kBitWords;
    const uint16_t* edge = b.edge + (uint64_t)t * R::kEdge;
    if (pos < TH) {
      const int ly = pos;
      if (ly < h && ((bits[ly >> 5] >> (ly & 31)) & 1u)) {
        const uint32_t tn = ty * lat.ntx + (tx + 1 == lat.ntx ? 0u : tx + 1);
        uint64_t nx0, ny0;
        int nw, nh;
        tile_geom(lat, tn, TH, nx0, ny0, nw, nh);
        a = (LabelT)global_index(lat, x0, y0, edge[ly]);
        c = (LabelT)global_index(lat, nx0, ny0, b.edge[(uint64_t)tn * R::kEdge + TH + ly]);
        active = true;
      }
    } else {
      const int lx = pos - TH;
      if (lx < w && ((bits[R::kRightWords + (lx >> 5)] >> (lx & 31)) & 1u)) {
        const uint32_t tn = (ty + 1 == lat.nty ? 0u : ty + 1) * lat.ntx + tx;
        uint64_t nx0, ny0;
        int nw, nh;
        tile_geom(lat, tn, TH, nx0, ny0, nw, nh);
        a = (LabelT)global_index(lat, x0, y0, edge[2 * TH + lx]);
        c = (LabelT)global_index(lat, nx0, ny0, b.edge[(uint64_t)tn * R::kEdge + 2 * TH + kTW + lx]);
        active = true;
      }
    }
  }
  // neighbouring edge sites usually repeat the same pair of roots: one lane
  // per distinct (a, c) pair does the union
  const unsigned same = __match_any_sync(0xFFFFFFFFu, a) & __match_any_sync(0xFFFFFFFFu, c);
  if (active && (int)(threadIdx.x & 31) == __ffs(same) - 1)
    unite_global(reinterpret_cast<LabelT*>(b.T), a, c, b.err);

  if (blockIdx.x == 0 && threadIdx.x == 0) {
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
  }
}

// ================================================================== k_recolor
// kRoots: write each site's global root (LabelT) to `roots` instead of spins.
template <int TH, typename LabelT, bool kRoots>
__global__ void __launch_bounds__(kThreads) k_recolor(const Bufs b, const Lattice lat, LabelT* roots) {
  using R = TileRec<TH>;
  constexpr int kRpw = TH / kWarps;
  __shared__ uint8_t ns[kRoots ? 1 : kTW * TH];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t t = blockIdx.x;
  uint64_t x0, y0;
  int w, h;
  tile_geom(lat, t, TH, x0, y0, w, h);
  const uint64_t L = lat.L;
  LabelT* T = reinterpret_cast<LabelT*>(b.T);
  const uint32_t sweep = (uint32_t)b.ctl[1];
  if (!kRoots) {
    const uint32_t n = b.ocnt[t];
    const uint16_t* ol = b.olist + (uint64_t)t * R::kOpenCap;
    for (uint32_t k = tid; k < n; k += kThreads) {
      const uint32_t l = ol[k];
      const LabelT r = find_global(T, (LabelT)global_index(lat, x0, y0, l), b.err);
      ns[l] = (uint8_t)cluster_state(b.seed, (uint64_t)r, sweep, b.q);
    }
    __syncthreads();
  }
  const int lx0 = 4 * lane;
#pragma unroll
  for (int rr = 0; rr < kRpw; ++rr) {
    const int ly = warp + rr * kWarps;
    if (ly < h && lx0 < w) {
      const uint64_t gi = (y0 + ly) * L + x0 + lx0;
      uint32_t c[4];
      if (lat.vec4) {
        const uint2 v = *reinterpret_cast<const uint2*>(b.code + gi);
        c[0] = v.x & 0xFFFFu; c[1] = v.x >> 16; c[2] = v.y & 0xFFFFu; c[3] = v.y >> 16;
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) c[k] = lx0 + k < w ? b.code[gi + k] : 0u;
      }
      if (kRoots) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (lx0 + k < w) {
            const uint64_t g = global_index(lat, x0, y0, c[k] & kIdx);
            roots[gi + k] = (c[k] & kClosed) ? (LabelT)g : find_global(T, (LabelT)g, b.err);
          }
        }
      } else {
        uint32_t s = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint32_t v = (c[k] & kClosed) ? (c[k] & 0xFFu) : ns[c[k] & kIdx];
          s |= v << (8 * k);
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
__global__ void k_init_spins(uint8_t* s, uint64_t N, uint32_t q, uint64_t seed) {
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

// E_sat and n[s] of a configuration (the configuration no later sweep reads).
// One thread per group of 4 sites of a row; 4-byte loads when rows are
// 4-byte aligned, per-state counts in registers for q <= 8.
__global__ void __launch_bounds__(256) k_measure(const uint8_t* s, Lattice lat, uint32_t q,
                                                 unsigned long long* acc) {
  __shared__ uint32_t hist[257];
  for (int k = threadIdx.x; k < 257; k += blockDim.x) hist[k] = 0;
  __syncthreads();
  const uint64_t L = lat.L;
  const uint64_t groups = (L + 3) >> 2;
  const uint64_t total = groups * L;
  const uint32_t qs = q <= 8 ? q - 1 : 0;
  uint32_t e = 0, cnt[7] = {0, 0, 0, 0, 0, 0, 0}, nsites = 0;
  for (uint64_t it = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; it < total;
       it += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t y = it / groups, x = (it % groups) * 4;
    const uint64_t yd = (y + 1 == L) ? 0 : y + 1;
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
    e += __popc(__vcmpeq4(v, vr) & vm & 0x01010101u) + __popc(__vcmpeq4(v, vd) & vm & 0x01010101u);
    nsites += __popc(vm & 0x01010101u);
    if (qs) {
#pragma unroll
      for (uint32_t st = 0; st < 7; ++st)
        if (st < qs) cnt[st] += __popc(__vcmpeq4(v, st * 0x01010101u) & vm & 0x01010101u);
    } else {
      for (int k = 0; k < 4; ++k)
        if ((vm >> (8 * k)) & 1u) atomicAdd(&hist[1 + ((v >> (8 * k)) & 0xFFu)], 1u);
    }
  }
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

// Sets *bad if any of the N spins is >= q (validation of a new configuration).
__global__ void k_check_spins(const uint8_t* s, uint64_t N, uint32_t q, uint32_t* bad) {
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

// Files the accumulated observables as configuration ctl[0].
__global__ void k_commit(Bufs b) {
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
