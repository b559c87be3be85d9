// sw_label.cuh -- k_label_rows, the tile labeller of the Potts sweep with
// one lane per half tile row.
//
// It labels a 128 x TH tile (Sec. 2 steps (1)-(3), tile-local part, plus the
// measurement of Sec. 4) and writes the records of the boundary pass -- the
// 16-bit site codes, the open slots of the four edge lines, the cross-edge
// bond bits and the open roots' nodes of the global union-find -- that
// k_merge, k_resolve and k_recolor read.  Its work mapping:
//
//   * a lane owns 64 consecutive sites of one tile row (two 32-bit words),
//     so a warp covers 16 rows of a 128-wide tile and a CTA of TH/16 warps
//     the whole 128 x TH tile;
//   * spins are packed into bit planes (q <= 4), so the equal-neighbour
//     tests, the E_sat / n[s] counts and the horizontal runs are word
//     operations on 32 sites at a time; the row below comes from the lane
//     that owns it (one shuffle per word);
//   * run starts are a bit mask, and a site's run start is the highest set
//     bit at or below it: only run starts are union-find nodes, and no
//     per-site parent is ever written;
//   * the union-find entries are 16 bits (tile-local index j = ly*128 + lx),
//     so a 128 x 128 tile needs 32 KB of shared memory; linking a root is a
//     compare-and-swap of the 32-bit word that holds its entry.
//
// Phases of a tile (a barrier after each):
//   A  bonds (Philox, one call per two sites; the XY form's embedded bond
//      rule, or given bonds), observables of the configuration read,
//      cross-edge bond bits, run-start masks;
//   B  vertical unions: each warp first joins its 16 rows top-down with
//      __syncwarp only (a forest whose band-top runs are local roots),
//      pointer jumping joins the bands, and the remaining unions go through
//      per-warp queues (lockstep walks, path splitting, CAS links);
//   C  clusters that touch the tile edge are flagged open at their root;
//      linked roots and the bands' parented starts are pointed at their
//      roots (every start at most two links below its root);
//   D  roots: a closed cluster draws its new state at its root (Sec. 2
//      step (3)), an open root takes a slot in the tile's open list and its
//      node of the global union-find;
//   F  per-site codes (8-site groups, 16-byte stores) and the edge lines;
//   M  (fused merge schedule only) the boundary unions of the edges this
//      tile finished second on.
//
// Entry encoding in P: a plain index (< 0x4000) is a parent (a root names
// itself); phase C adds 0x8000 to open roots; phase D replaces every root's
// entry by its code, 0x8000 | payload (closed: the new state, or the root
// index in the labelling-only form) or 0x4000 | slot (open), so that phase
// F walks from a run start to the first entry with a marker.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sw_kernels.cuh"

namespace swgb {

constexpr uint32_t kIdx16 = 0x3FFFu;    // index bits of a 16-bit entry
constexpr uint32_t kMarkA = 0x8000u;    // open flag of a root; closed code marker
constexpr uint32_t kMarkB = 0x4000u;    // open code marker
constexpr uint32_t kMarks = kMarkA | kMarkB;

// CTA shape: a lane owns kW words (32 sites each) of a row, kLpr lanes a
// row, kRpw rows a warp.
template <int TH>
struct RowCta {
  static constexpr int kW = 2;
  static constexpr int kLpr = 4 / kW;
  static constexpr int kRpw = 32 / kLpr;
  static constexpr int kWarps = TH / kRpw;
  static constexpr int kThreads = 32 * kWarps;
  static constexpr int kMinBlocks = 1024 / kThreads;  // 64 registers a thread
  static_assert(TH % kRpw == 0, "tile height");
  // a warp's work queue in the staging buffer: 512 entries (32 lanes x 16)
  static constexpr int kQCap = (TH + 1) * 128 / 4 / kWarps;
  static_assert(kQCap >= 512, "work queue");
  // while L2 (a bitmap of the roots linked by unions, 4 words a row) is in
  // use behind them, the queues hold kQ8 entries a lane
  static constexpr int kQ8 = 12;
  static_assert(kWarps * 32 * kQ8 + 4 * TH <= (TH + 1) * 128 / 4, "work queue beside L2");
};

// Shared memory of k_label_rows.
template <int TH>
struct RowSmem {
  static constexpr int kP = 0;                                          // u16 [TH*128]
  static constexpr int kSp = align16(kP + 2 * kTW * TH);                 // u8 [(TH+1)*128], swizzled
  static constexpr int kHal = kSp + (TH + 1) * kTW;                      // u8 [TH+1][4] halo column
  static constexpr int kRS = align16(kHal + 4 * (TH + 1));               // u32 [TH][4] run starts
  static constexpr int kRC = kRS + 16 * TH;                              // u8 [TH][4] run start of bit 0
  static constexpr int kNR = align16(kRC + 4 * TH);                      // u32 [TH][4] linked (non-root) starts
  static constexpr int kCb = align16(kNR + 16 * TH);                     // u32 cross bits
  static constexpr int kCnt = align16(kCb + 4 * TileRec<TH>::kBitWords);  // u32 [4]
  static constexpr int kObs = kCnt + 16;                                 // u32 [8], or [257] for q > 4
  static constexpr int kBytesSmallQ = align16(kObs + 4 * 8);
  static constexpr int kBytes = align16(kObs + 4 * 257);
};

// ---------------------------------------------------------------- 16-bit union-find
// Root of x after the unions (entries may carry the open flag).
__device__ __forceinline__ uint32_t root16(const uint16_t* P, uint32_t x, uint32_t& bad) {
  const volatile uint16_t* vp = P;
  for (uint32_t it = 0; it < kLocalCap; ++it) {
    const uint32_t p = vp[x] & kIdx16;
    if (p == x) return x;
    x = p;
  }
  bad = 1;
  return x;
}

// Run start of bit b of a word whose starts are m, columns from cw; c is the
// run start of bit 0 (a run that begins in an earlier word).
__device__ __forceinline__ uint32_t run_start(uint32_t m, int b, uint32_t cw, uint32_t c) {
  const uint32_t mm = m & (0xFFFFFFFFu >> (31 - b));
  return mm ? cw + 31u - (uint32_t)__clz(mm) : c;
}

// Run start of column c0 + x of a lane's 64 columns whose starts are m; c
// is the run start of the lane's first column (a run from an earlier part).
__device__ __forceinline__ uint32_t run_start64(uint64_t m, uint32_t x, uint32_t c0, uint32_t c) {
  const uint64_t mm = m & (0xFFFFFFFFFFFFFFFFull >> (63u - x));
  return mm ? c0 + 63u - (uint32_t)__clzll(mm) : c;
}

// Warp work queue: each lane appends up to kCap of its remaining items (the
// set bits of rem, lowest first, as f(bit)) to Q; returns how many the warp
// queued.  Entries are ordered by lane, each lane's contiguous.
template <uint32_t kCap = 16, typename Fn>
__device__ __forceinline__ uint32_t enqueue16(uint64_t& rem, uint32_t* Q, int lane, Fn f) {
  const uint32_t cnt = min((uint32_t)__popcll(rem), kCap);
  uint32_t inc = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= o) inc += y;
  }
  const uint32_t nq = __shfl_sync(0xFFFFFFFFu, inc, 31);
  uint32_t pos = inc - cnt;
  for (uint32_t k = 0; k < cnt; ++k) {
    const uint32_t x = (uint32_t)(__ffsll(rem) - 1);
    rem &= rem - 1ull;
    Q[pos++] = f(x);
  }
  __syncwarp();
  return nq;
}

// Bit k of the result = bit `pl` of byte k of w (k = 0..3).
__device__ __forceinline__ uint32_t plane4(uint32_t w, int pl) {
  return ((((w >> pl) & 0x01010101u) * 0x01020408u) >> 24) & 0xFu;
}

// Staged spin rows are 128 bytes apart with their eight 16-byte chunks
// permuted by the row (chunk k of row y at position k ^ (y & 7)), so that
// the lanes of a warp, each reading its own row, hit distinct banks.  Byte
// offset of (row y, column col < 128):
__device__ __forceinline__ uint32_t swz(int y, int col) {
  return (uint32_t)(y * kTW + ((((col >> 4) ^ y) & 7) << 4) + (col & 15));
}

// The 32 sites at columns col .. col+31 of staged row y (col a multiple of
// 16) as one word of bit plane 0 and one of bit plane 1.
__device__ __forceinline__ void pack32(const uint8_t* sp, int y, int col, bool two, uint32_t& p0, uint32_t& p1) {
  const uint4 u = *reinterpret_cast<const uint4*>(sp + swz(y, col));
  const uint4 v = *reinterpret_cast<const uint4*>(sp + swz(y, col + 16));
  const uint32_t w[8] = {u.x, u.y, u.z, u.w, v.x, v.y, v.z, v.w};
  uint32_t a = 0, c = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) a |= plane4(w[k], 0) << (4 * k);
  if (two) {
#pragma unroll
    for (int k = 0; k < 8; ++k) c |= plane4(w[k], 1) << (4 * k);
  }
  p0 = a;
  p1 = c;
}

// The same 32 sites as bit planes 0, 1 and 2 (states below 8).
__device__ __forceinline__ void pack32x3(const uint8_t* sp, int y, int col, uint32_t& p0, uint32_t& p1,
                                         uint32_t& p2) {
  const uint4 u = *reinterpret_cast<const uint4*>(sp + swz(y, col));
  const uint4 v = *reinterpret_cast<const uint4*>(sp + swz(y, col + 16));
  const uint32_t w[8] = {u.x, u.y, u.z, u.w, v.x, v.y, v.z, v.w};
  uint32_t a = 0, c = 0, e = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    a |= plane4(w[k], 0) << (4 * k);
    c |= plane4(w[k], 1) << (4 * k);
    e |= plane4(w[k], 2) << (4 * k);
  }
  p0 = a;
  p1 = c;
  p2 = e;
}

// Even / odd bits of a 32-bit word, compacted into 16 bits (bond bytes:
// bit 2k = right bond of site k, bit 2k+1 = down bond).
__device__ __forceinline__ uint32_t even_bits(uint32_t x) {
  x &= 0x55555555u;
  x = (x | (x >> 1)) & 0x33333333u;
  x = (x | (x >> 2)) & 0x0F0F0F0Fu;
  x = (x | (x >> 4)) & 0x00FF00FFu;
  x = (x | (x >> 8)) & 0x0000FFFFu;
  return x;
}

// Stages a tile's spin rows 0..h (row h is the halo row) into buf (the
// swizzled layout of swz) and each row's halo byte (column w) at column w of
// the row when the tile is narrower than 128, else into hal[4*y];
// asynchronous (cp.async) when rows are 4-byte aligned, with 16-byte copies
// when L % 16 == 0.
template <int TH, int kThreads, typename Src>
__device__ __forceinline__ void stage_rows(const Src& src, uint32_t gg, uint8_t* buf, uint8_t* hal, bool async) {
  constexpr int kWarps = kThreads / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t fr = src.rep(gg);
  const Lattice& fl = src.lattice(fr);
  const uint8_t* fspin = src.bufs(fr).spin;
  const uint64_t FL = fl.L;
  uint64_t fx0, fy0;
  int fw, fh;
  tile_geom(fl, gg - src.tile0(fr), TH, fx0, fy0, fw, fh);
  const uint64_t hx = (fx0 + fw == FL) ? 0 : fx0 + fw;
  const uint64_t hy = (fy0 + fh == FL) ? 0 : fy0 + fh;
  if (async && (FL & 15u) == 0 && (reinterpret_cast<uintptr_t>(fspin) & 15u) == 0) {
    const int c16 = (lane & 7) * 16;
    for (int ly = warp * 4 + (lane >> 3); ly <= fh; ly += 4 * kWarps) {
      const uint64_t gy = (ly < fh) ? (fy0 + ly) : hy;
      if (c16 < fw) cp_async16(buf + swz(ly, c16), fspin + gy * FL + fx0 + c16);
    }
    for (int ly = tid; ly <= fh; ly += kThreads) {
      const uint64_t gy = (ly < fh) ? (fy0 + ly) : hy;
      cp_async4(fw < kTW ? buf + swz(ly, fw) : hal + 4 * ly, fspin + gy * FL + hx);
    }
    return;
  }
  const int lx0 = 4 * lane;  // 32 lanes x 4 bytes: the 128 columns
  for (int ly = warp; ly <= fh; ly += kWarps) {
    const uint64_t gy = (ly < fh) ? (fy0 + ly) : hy;
    const uint8_t* row = fspin + gy * FL;
    if (async) {
      if (lx0 < fw) cp_async4(buf + swz(ly, lx0), row + fx0 + lx0);
      if (lane == 31) cp_async4(fw < kTW ? buf + swz(ly, fw) : hal + 4 * ly, row + hx);
    } else {
      uint32_t v = 0;
      if (lx0 < fw) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (lx0 + k < fw) v |= (uint32_t)row[fx0 + lx0 + k] << (8 * k);
      }
      *reinterpret_cast<uint32_t*>(buf + swz(ly, lx0)) = v;
      __syncwarp();
      if (lane == 0) {
        if (fw < kTW) buf[swz(ly, fw)] = row[hx];
        else hal[4 * ly] = row[hx];
      }
    }
  }
}

// ================================================================== k_label_rows
// Persistent: CTA c labels tiles c, c + gridDim.x, ...; the next tile's spins
// are copied into the staging buffer as soon as the bonds of the current
// one are drawn.
//
// kGiven: bonds are read from b.bonds instead of drawn (labelling-only entry).
// kRoots: closed clusters keep their local root in the code (no new state).
// kFuse: the labeller also does the boundary unions (phase M; the fused
// merge schedule).
// kXY: the XY model's embedded-cluster bonds (Sec. 5): a bond is a
// candidate when both sites' projections on the sweep's axis have the same
// (non-zero) sign, and active when its word is below the threshold of the
// two sites' fold indices; clusters draw a coin (q = 2).
template <int TH, typename LabelT, bool kGiven, bool kRoots, typename Src, bool kFuse = false,
          bool kXY = false>
__global__ void __launch_bounds__(RowCta<TH>::kThreads, RowCta<TH>::kMinBlocks)
    k_label_rows(const __grid_constant__ Src src) {
  using C = RowCta<TH>;
  using S = RowSmem<TH>;
  using R = TileRec<TH>;
  constexpr int kW = C::kW, kLpr = C::kLpr, kRpw = C::kRpw, kThreads = C::kThreads, kQCap = C::kQCap;
  constexpr unsigned kFull = 0xFFFFFFFFu;

  extern __shared__ __align__(16) unsigned char smem[];
  uint16_t* P = reinterpret_cast<uint16_t*>(smem + S::kP);
  uint8_t* sp = smem + S::kSp;
  uint8_t* hal = smem + S::kHal;
  uint32_t* RS = reinterpret_cast<uint32_t*>(smem + S::kRS);
  uint8_t* RC = smem + S::kRC;
  uint32_t* NR = reinterpret_cast<uint32_t*>(smem + S::kNR);
  uint32_t* cbits = reinterpret_cast<uint32_t*>(smem + S::kCb);
  uint32_t* wcnt = reinterpret_cast<uint32_t*>(smem + S::kCnt);
  uint32_t* sobs = reinterpret_cast<uint32_t*>(smem + S::kObs);
  // replica batch: the current tile's replica record (buffers, Philox round
  // keys, geometry), two copies by tile parity.  A lattice of its own has
  // these among the kernel parameters, as free constant operands; read from
  // the replica table in global memory they would take registers.
  __shared__ __align__(16) unsigned char srec[Src::kMulti ? 2 * sizeof(Rep) : 16];
  __shared__ __align__(16) uint32_t srk[Src::kMulti ? 2 * 20 : 4];  // its Philox round keys, 16-byte aligned
  // replica batch, 4 < q <= 8: the CTA's bit-plane subset counts of the
  // current replica (|a0|, |a1|, |a2|, |a0 a1|, |a0 a2|, |a1 a2|, |a0 a1 a2|)
  __shared__ uint32_t sc3[Src::kMulti ? 8 : 1];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int part = lane % kLpr;
  const int ly = warp * kRpw + lane / kLpr;  // this lane's row
  const int c0 = part * 32 * kW;             // its first column
  const uint32_t total = src.ntiles();
  uint32_t bad = 0, spin_max = 0;
  const bool big_q = !kGiven && src.bufs(0).q > 4 && !Src::kMulti;  // shared state histogram

  for (int k = tid; k < (Src::kMulti ? 257 : (big_q ? 257 : 8)); k += kThreads) sobs[k] = 0;
  for (int k = tid; k < R::kBitWords; k += kThreads) cbits[k] = 0;
  if (Src::kMulti && tid < 8) sc3[tid] = 0;
  uint32_t e_loc = 0, nsites = 0;
  uint32_t ncnt[3] = {0, 0, 0};

  // observables accumulated so far go to the lattice's accumulator (E_sat,
  // bit-plane counts c1 = n1 + n3, c2 = n2 + n3, c3 = n3 for q <= 4, n[s]
  // in shared memory otherwise; n[0] from the site count).  All threads.
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
        atomicAdd(&sobs[2], ncnt[0] - ncnt[2]);
        if (fq > 2) atomicAdd(&sobs[3], ncnt[1] - ncnt[2]);
        if (fq > 3) atomicAdd(&sobs[4], ncnt[2]);
      }
    }
    __syncthreads();
    if (fregs && tid == 0) {
      uint32_t rest = nsites;
      for (uint32_t st = 1; st < fq; ++st) rest -= sobs[1 + st];
      sobs[1] = rest;
    }
    if constexpr (Src::kMulti) {
      // three bit planes (4 < q <= 8): n[s] = sum over the plane subsets T
      // that contain the set bits of s of (-1)^|T - s| c_T, where c_T counts
      // the sites with every plane of T set (the empty set: every site)
      if (fq > 4 && fq <= 8 && tid == 0) {
        const uint32_t cT[8] = {nsites, sc3[0], sc3[1], sc3[3], sc3[2], sc3[4], sc3[5], sc3[6]};
        for (uint32_t st = 0; st < fq; ++st) {
          uint32_t n = 0;
          for (uint32_t T = st; T < 8; ++T)
            if ((T & st) == st) n += (__popc(T ^ st) & 1u) ? 0u - cT[T] : cT[T];
          sobs[1 + st] = n;
        }
        for (int k = 0; k < 7; ++k) sc3[k] = 0;
      }
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
  // The same for one tile's bit-plane counts (q <= 4), warp by warp: a
  // warp's sites are its rows of the tile, n[0] the rest of them.
  auto warp_flush = [&](const Bufs& fb, uint32_t fq, int fw, int fh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e_loc += __shfl_xor_sync(kFull, e_loc, o);
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ncnt[k] += __shfl_xor_sync(kFull, ncnt[k], o);
    if (lane == 0) {
      const int nr = min(max(fh - warp * kRpw, 0), kRpw);
      const uint32_t n1 = ncnt[0] - ncnt[2];
      const uint32_t n2 = fq > 2 ? ncnt[1] - ncnt[2] : 0u;
      const uint32_t n3 = fq > 3 ? ncnt[2] : 0u;
      atomicAdd(&fb.acc[0], (unsigned long long)e_loc);
      atomicAdd(&fb.acc[1], (unsigned long long)((uint32_t)(nr * fw) - n1 - n2 - n3));
      atomicAdd(&fb.acc[2], (unsigned long long)n1);
      if (fq > 2) atomicAdd(&fb.acc[3], (unsigned long long)n2);
      if (fq > 3) atomicAdd(&fb.acc[4], (unsigned long long)n3);
    }
    e_loc = 0;
    if (tid == 0) nsites = 0;
    ncnt[0] = ncnt[1] = ncnt[2] = 0;
  };

  bool pre = false;
  if (!kGiven && blockIdx.x < total && src.lattice(src.rep(blockIdx.x)).vec4) {
    stage_rows<TH, kThreads>(src, blockIdx.x, sp, hal, true);
    cp_async_commit();
    pre = true;
  }

  uint32_t par = 0;  // tile parity: the shared copy of the replica record in use (batch)
  for (uint32_t g = blockIdx.x; g < total; g += gridDim.x, par ^= 1u) {
    const uint32_t rep = src.rep(g);
    if constexpr (Src::kMulti) {
      // the other copy may still be read by the previous tile's last phase
      const uint32_t* from = reinterpret_cast<const uint32_t*>(src.reps + rep);
      uint32_t* to = reinterpret_cast<uint32_t*>(srec + par * sizeof(Rep));
      for (int k = tid; k < (int)(sizeof(Rep) / 4); k += kThreads) to[k] = __ldg(from + k);
      if (tid < 20) srk[20 * par + tid] = src.reps[rep].b.rk[tid];
    }
    const uint32_t t = g - src.tile0(rep);
    uint64_t x0, y0;
    int w, h;
    tile_geom(src.lattice(rep), t, TH, x0, y0, w, h);
    if (!kGiven) {
      if (pre) cp_async_wait();
      else stage_rows<TH, kThreads>(src, g, sp, hal, false);
    }
    if (tid == 0) nsites += (uint32_t)(w * h);
    if constexpr (kXY) {
      // the projection class of every angle on this sweep's embedding axis
      // (Wolff's embedding), built for the CTA's first tile (one lattice,
      // one sweep): sign of sigma in bits 8-9 (1 negative, 2 positive, 0
      // zero), fold index c of |sigma| = sin(pi c / M) below.  The shared
      // observables area holds it (this form measures nothing).
      if (g == blockIdx.x) {
        const Bufs& xb = src.bufs(rep);
        const uint32_t M = xb.M;
        const uint32_t jx = pick_state(stream4_rk(xb.rk, 0ull, (uint32_t)xb.ctl[0], kDomAxis).x, M);
        uint16_t* xcls = reinterpret_cast<uint16_t*>(sobs);
        for (uint32_t k = tid; k < M; k += kThreads) {
          const uint32_t a = (2 * k >= jx) ? 2 * k - jx : 2 * k + 2 * M - jx;  // (2k - j) mod 2M
          const uint32_t sg = (a == 0 || a == M) ? 0u : (a < M ? 1u : 2u);
          const uint32_t bm = a >= M ? a - M : a;
          xcls[k] = (uint16_t)((sg << 8) | (bm < M - bm ? bm : M - bm));
        }
      }
    }
    __syncthreads();  // staged spins visible; the previous tile is done with every shared array
    const Bufs& b = [&]() -> const Bufs& {
      if constexpr (Src::kMulti) return reinterpret_cast<const Rep*>(srec)[par].b;
      else return src.bufs(rep);
    }();
    const Lattice& lat = [&]() -> const Lattice& {
      if constexpr (Src::kMulti) return reinterpret_cast<const Rep*>(srec)[par].lat;
      else return src.lattice(rep);
    }();
    const uint64_t L = lat.L;
    const uint32_t q_states = b.q;
    const bool measure = !kGiven && b.measure;
    const uint32_t sweep = kGiven ? 0u : (uint32_t)b.ctl[0];
    auto philox = [&](uint64_t idx, uint32_t dom) -> Words4 {
      if constexpr (Src::kMulti)
        return philox4x32_10_k4((uint32_t)idx, (uint32_t)(idx >> 32), sweep, dom,
                                reinterpret_cast<const uint4*>(srk + 20 * par));
      else return stream4_rk(b.rk, idx, sweep, dom);
    };
    const uint32_t thr = b.thr;

    // ================================================= A: bonds, observables, runs
    uint32_t vm[kW], H[kW], V[kW], Sm[kW], Cw[kW];
#pragma unroll
    for (int wi = 0; wi < kW; ++wi) {
      const int nv = w - (c0 + 32 * wi);
      vm[wi] = (ly < h) ? (nv >= 32 ? 0xFFFFFFFFu : (nv > 0 ? (1u << nv) - 1u : 0u)) : 0u;
      H[wi] = V[wi] = 0;
    }
    if constexpr (kXY) {
      // four sites at a time: classes of the sites, their right and lower
      // neighbours; one Philox call per two sites, as for the Potts bonds;
      // thresholds from the lower triangle of the (fold index, fold index)
      // table in global memory (read through L1)
      const uint16_t* xcls = reinterpret_cast<const uint16_t*>(sobs);
      auto thr_of = [&](uint32_t c, uint32_t d) -> uint32_t {
        const uint32_t hi = c > d ? c : d, lo = c > d ? d : c;
        return __ldg(b.tt + ((hi * (hi + 1)) >> 1) + lo);
      };
      const uint64_t rowg = (y0 + ly) * L + x0 + c0;
#pragma unroll
      for (int wi = 0; wi < kW; ++wi) {
        if (vm[wi] == 0) continue;
#pragma unroll 2
        for (int gq = 0; gq < 8; ++gq) {
          const uint32_t sh = 4 * gq;
          const uint32_t m4 = (vm[wi] >> sh) & 0xFu;
          if (!m4) continue;
          const int cc = c0 + 32 * wi + 4 * gq;
          const uint32_t sv = *reinterpret_cast<const uint32_t*>(sp + swz(ly, cc));
          const uint32_t sn = cc + 4 < kTW ? *reinterpret_cast<const uint32_t*>(sp + swz(ly, cc + 4))
                                            : *reinterpret_cast<const uint32_t*>(hal + 4 * ly);
          const uint32_t sd = *reinterpret_cast<const uint32_t*>(sp + swz(ly + 1, cc));
          uint32_t cs[5], cl[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            cs[k] = xcls[(sv >> (8 * k)) & 0xFFu];
            cl[k] = xcls[(sd >> (8 * k)) & 0xFFu];
          }
          cs[4] = xcls[sn & 0xFFu];
          uint32_t er = 0, ed = 0;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint32_t sg = cs[k] >> 8;
            er |= (sg != 0u && sg == (cs[k + 1] >> 8)) ? (1u << k) : 0u;
            ed |= (sg != 0u && sg == (cl[k] >> 8)) ? (1u << k) : 0u;
          }
          er &= m4;
          ed &= m4;
          if (er | ed) {
            const uint64_t i0 = rowg + 32 * wi + sh;
            const uint64_t pa = i0 >> 1;
            const Words4 A = philox(pa, kDomBond);
            const Words4 B = philox(pa + 1, kDomBond);
            uint32_t wr[4], wd[4];
            if ((i0 & 1u) == 0u) {
              wr[0] = A.x; wd[0] = A.y; wr[1] = A.z; wd[1] = A.w;
              wr[2] = B.x; wd[2] = B.y; wr[3] = B.z; wd[3] = B.w;
            } else {
              const Words4 Cc = philox(pa + 2, kDomBond);
              wr[0] = A.z; wd[0] = A.w; wr[1] = B.x; wd[1] = B.y;
              wr[2] = B.z; wd[2] = B.w; wr[3] = Cc.x; wd[3] = Cc.y;
            }
            uint32_t br = 0, bd = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              if ((er >> k) & 1u) br |= (wr[k] < thr_of(cs[k] & 0xFFu, cs[k + 1] & 0xFFu) ? 1u : 0u) << k;
              if ((ed >> k) & 1u) bd |= (wd[k] < thr_of(cs[k] & 0xFFu, cl[k] & 0xFFu) ? 1u : 0u) << k;
            }
            H[wi] |= br << sh;
            V[wi] |= bd << sh;
          }
        }
      }
    } else if constexpr (kGiven) {
      if (ly < h) {
        const uint8_t* brow = b.bonds + (y0 + ly) * lat.bp;
#pragma unroll
        for (int wi = 0; wi < kW; ++wi) {
          if (vm[wi]) {
            const uint64_t byte0 = (x0 + c0 + 32 * wi) >> 2;
            uint32_t lo = 0, hi = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const uint32_t v = (byte0 + k < lat.bp) ? (uint32_t)brow[byte0 + k] : 0u;
              if (k < 4) lo |= v << (8 * k);
              else hi |= v << (8 * (k - 4));
            }
            H[wi] = (even_bits(lo) | (even_bits(hi) << 16)) & vm[wi];
            V[wi] = (even_bits(lo >> 1) | (even_bits(hi >> 1) << 16)) & vm[wi];
          }
        }
      }
    } else {
      // bit planes: one for q = 2, two for q <= 4; a replica batch also
      // keeps q <= 8 in three planes (its state counts go to the shared
      // histogram warp by warp), a lattice of its own takes the byte path
      constexpr bool kP3 = Src::kMulti;
      const uint32_t np = q_states <= 2 ? 1u : (q_states <= 4 ? 2u : ((kP3 && q_states <= 8) ? 3u : 0u));
      uint32_t eqr[kW], eqd[kW];
      if (np) {
        const bool two = np >= 2;
        const bool three = kP3 && np == 3;
        uint32_t a0[kW], a1[kW], a2[kW], d0[kW], d1[kW], d2[kW];
#pragma unroll
        for (int wi = 0; wi < kW; ++wi) a0[wi] = a1[wi] = a2[wi] = 0;
        uint32_t nb = 0;  // the byte right of this lane's range (last part: the halo column)
        if (ly <= h) {
#pragma unroll
          for (int wi = 0; wi < kW; ++wi) {
            if (three) pack32x3(sp, ly, c0 + 32 * wi, a0[wi], a1[wi], a2[wi]);
            else pack32(sp, ly, c0 + 32 * wi, two, a0[wi], a1[wi]);
          }
          if (part == kLpr - 1) nb = hal[4 * ly];  // column 128 (a narrower tile masks it)
          if constexpr (Src::kCheck) {
            if (ly < h) {
#pragma unroll
              for (int k = 0; k < 8 * kW; ++k) {
                const int cc = c0 + 4 * k;
                const int nv = w - cc;
                const uint32_t m4 = nv >= 4 ? 0xFu : (nv > 0 ? (1u << nv) - 1u : 0u);
                spin_max = __vmaxu4(spin_max, *reinterpret_cast<const uint32_t*>(sp + swz(ly, cc)) & byte_mask(m4));
              }
            }
          }
        }
        // right neighbours: bit 0 of the next part of the row, or the halo byte
        const uint32_t n0 = __shfl_down_sync(kFull, a0[0], 1), n1 = __shfl_down_sync(kFull, a1[0], 1);
        const uint32_t nr0 = part == kLpr - 1 ? (nb & 1u) : (n0 & 1u);
        const uint32_t nr1 = part == kLpr - 1 ? ((nb >> 1) & 1u) : (n1 & 1u);
        uint32_t nr2 = 0;
        if (three) {
          const uint32_t n2 = __shfl_down_sync(kFull, a2[0], 1);
          nr2 = part == kLpr - 1 ? ((nb >> 2) & 1u) : (n2 & 1u);
        }
        // the row below: from the lane that owns it, or staged (last row of the warp)
#pragma unroll
        for (int wi = 0; wi < kW; ++wi) {
          d0[wi] = __shfl_down_sync(kFull, a0[wi], kLpr);
          d1[wi] = __shfl_down_sync(kFull, a1[wi], kLpr);
          d2[wi] = three ? __shfl_down_sync(kFull, a2[wi], kLpr) : 0u;
        }
        if (lane / kLpr == kRpw - 1 && ly < h) {
#pragma unroll
          for (int wi = 0; wi < kW; ++wi) {
            if (three) pack32x3(sp, ly + 1, c0 + 32 * wi, d0[wi], d1[wi], d2[wi]);
            else pack32(sp, ly + 1, c0 + 32 * wi, two, d0[wi], d1[wi]);
          }
        }
        // bit-plane subset counts of the three-plane form: |a0|, |a1|, |a2|,
        // |a0 a1|, |a0 a2|, |a1 a2|, |a0 a1 a2|
        uint32_t c3[7] = {0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int wi = 0; wi < kW; ++wi) {
          const uint32_t x0n = wi + 1 < kW ? (a0[wi + 1] & 1u) : nr0;
          const uint32_t x1n = wi + 1 < kW ? (a1[wi + 1] & 1u) : nr1;
          const uint32_t r0 = (a0[wi] >> 1) | (x0n << 31), r1 = (a1[wi] >> 1) | (x1n << 31);
          uint32_t dr = (a0[wi] ^ r0) | (a1[wi] ^ r1), dd = (a0[wi] ^ d0[wi]) | (a1[wi] ^ d1[wi]);
          if (three) {
            const uint32_t x2n = wi + 1 < kW ? (a2[wi + 1] & 1u) : nr2;
            dr |= a2[wi] ^ ((a2[wi] >> 1) | (x2n << 31));
            dd |= a2[wi] ^ d2[wi];
          }
          eqr[wi] = ~dr & vm[wi];
          eqd[wi] = ~dd & vm[wi];
          if (measure) {
            e_loc += __popc(eqr[wi]) + __popc(eqd[wi]);
            if (three) {
              const uint32_t b0 = a0[wi] & vm[wi], b1 = a1[wi] & vm[wi], b2 = a2[wi] & vm[wi];
              const uint32_t b01 = b0 & b1;
              c3[0] += __reduce_add_sync(kFull, __popc(b0));
              c3[1] += __reduce_add_sync(kFull, __popc(b1));
              c3[2] += __reduce_add_sync(kFull, __popc(b2));
              c3[3] += __reduce_add_sync(kFull, __popc(b01));
              c3[4] += __reduce_add_sync(kFull, __popc(b0 & b2));
              c3[5] += __reduce_add_sync(kFull, __popc(b1 & b2));
              c3[6] += __reduce_add_sync(kFull, __popc(b01 & b2));
            } else {
              ncnt[0] += __popc(a0[wi] & vm[wi]);
              if (two) {
                ncnt[1] += __popc(a1[wi] & vm[wi]);
                ncnt[2] += __popc(a0[wi] & a1[wi] & vm[wi]);
              }
            }
          }
        }
        if (three && measure && lane == 0) {
          // the warp's plane-subset counts into the CTA's; the flush turns
          // them into state counts
#pragma unroll
          for (int k = 0; k < 7; ++k)
            if (c3[k]) atomicAdd(&sc3[k], c3[k]);
        }
      } else {
        // q > 4: byte-wise comparisons, state counts in a shared histogram
#pragma unroll
        for (int wi = 0; wi < kW; ++wi) {
          eqr[wi] = eqd[wi] = 0;
          if (ly < h) {
#pragma unroll
            for (int gq = 0; gq < 8; ++gq) {
              const uint32_t sh = 4 * gq;
              const int cc = c0 + 32 * wi + 4 * gq;
              const uint32_t m4 = (vm[wi] >> sh) & 0xFu;
              const uint32_t s = *reinterpret_cast<const uint32_t*>(sp + swz(ly, cc));
              const uint32_t sn = cc + 4 < kTW ? *reinterpret_cast<const uint32_t*>(sp + swz(ly, cc + 4))
                                                : *reinterpret_cast<const uint32_t*>(hal + 4 * ly);
              const uint32_t sd = *reinterpret_cast<const uint32_t*>(sp + swz(ly + 1, cc));
              if constexpr (Src::kCheck) spin_max = __vmaxu4(spin_max, s & byte_mask(m4));
              const uint32_t er = zero_bytes4(s ^ __funnelshift_r(s, sn, 8)) & m4;
              const uint32_t ed = zero_bytes4(s ^ sd) & m4;
              eqr[wi] |= er << sh;
              eqd[wi] |= ed << sh;
              if (measure) {
                e_loc += __popc(er) + __popc(ed);
#pragma unroll
                for (int k = 0; k < 4; ++k)
                  if (m4 & (1u << k)) atomicAdd(&sobs[1 + ((s >> (8 * k)) & 0xFFu)], 1u);
              }
            }
          }
        }
      }
      // bond draws: one Philox call per two sites (right and down words);
      // a replica batch reads the round keys from shared memory, so two
      // groups in flight would not fit in the registers
      const uint64_t rowg = (y0 + ly) * L + x0 + c0;
#pragma unroll
      for (int wi = 0; wi < kW; ++wi) {
#pragma unroll(Src::kMulti ? 1 : 2)
        for (int gq = 0; gq < 8; ++gq) {
          const uint32_t sh = 4 * gq;
          const uint32_t er = (eqr[wi] >> sh) & 0xFu, ed = (eqd[wi] >> sh) & 0xFu;
          uint32_t br = 0, bd = 0;
          if (er | ed) {
            const uint64_t i0 = rowg + 32 * wi + sh;
            const uint64_t pa = i0 >> 1;
            const Words4 A = philox(pa, kDomBond);
            const Words4 B = philox(pa + 1, kDomBond);
            uint32_t wr[4], wd[4];
            if ((i0 & 1u) == 0u) {
              wr[0] = A.x; wd[0] = A.y; wr[1] = A.z; wd[1] = A.w;
              wr[2] = B.x; wd[2] = B.y; wr[3] = B.z; wd[3] = B.w;
            } else {
              const Words4 Cc = philox(pa + 2, kDomBond);
              wr[0] = A.z; wd[0] = A.w; wr[1] = B.x; wd[1] = B.y;
              wr[2] = B.z; wd[2] = B.w; wr[3] = Cc.x; wd[3] = Cc.y;
            }
            br = er & lt_mask4(wr, thr);
            bd = ed & lt_mask4(wd, thr);
            H[wi] |= br << sh;
            V[wi] |= bd << sh;
          }
          if (b.bonds && ((vm[wi] >> sh) & 0xFu)) {
            uint32_t byte = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k)
              byte |= (((br >> k) & 1u) << (2 * k)) | (((bd >> k) & 1u) << (2 * k + 1));
            b.bonds[(y0 + ly) * lat.bp + ((x0 + c0 + 32 * wi + sh) >> 2)] = (uint8_t)byte;
          }
        }
      }
    }
    // bonds that leave the tile: right edge (column w-1) and bottom edge
    if (ly < h) {
      const int e = w - 1 - c0;
#pragma unroll
      for (int wi = 0; wi < kW; ++wi) {
        if (e >= 32 * wi && e < 32 * wi + 32) {
          const uint32_t bit = 1u << (e - 32 * wi);
          if (H[wi] & bit) atomicOr(&cbits[ly >> 5], 1u << (ly & 31));
          H[wi] &= ~bit;
        }
      }
      if (ly == h - 1) {
#pragma unroll
        for (int wi = 0; wi < kW; ++wi) {
          if (c0 + 32 * wi < w) cbits[R::kRightWords + (c0 >> 5) + wi] = V[wi];
          V[wi] = 0;
        }
      }
    }
    // horizontal runs: a site without a bond to its left starts a run
    {
      uint32_t hp = __shfl_up_sync(kFull, H[kW - 1] >> 31, 1);
      if (part == 0) hp = 0;
#pragma unroll
      for (int wi = 0; wi < kW; ++wi) Sm[wi] = ~((H[wi] << 1) | (wi ? H[wi - 1] >> 31 : hp)) & vm[wi];
      int lst = -1;
#pragma unroll
      for (int wi = 0; wi < kW; ++wi)
        if (Sm[wi]) lst = c0 + 32 * wi + 31 - __clz(Sm[wi]);
      int cin = __shfl_up_sync(kFull, lst, 1);
      if (part == 0 || cin < 0) cin = 0;
      Cw[0] = (uint32_t)cin;
#pragma unroll
      for (int wi = 1; wi < kW; ++wi)
        Cw[wi] = Sm[wi - 1] ? (uint32_t)(c0 + 32 * (wi - 1) + 31 - __clz(Sm[wi - 1])) : Cw[wi - 1];
#pragma unroll
      for (int wi = 0; wi < kW; ++wi) {
        RS[ly * 4 + (c0 >> 5) + wi] = Sm[wi];
        RC[ly * 4 + (c0 >> 5) + wi] = (uint8_t)Cw[wi];
        NR[ly * 4 + (c0 >> 5) + wi] = 0u;
      }
    }
    // every entry of the row names itself (only run starts are ever used);
    // the eight 16-byte chunks in a lane-rotated order (no bank conflicts)
    if (ly < h) {
      const uint32_t j0 = (uint32_t)(ly * kTW + c0);
      uint4* dst = reinterpret_cast<uint4*>(P + j0);
#pragma unroll
      for (int k = 0; k < 4 * kW; ++k) {
        const uint32_t ch = (uint32_t)(k + lane) & (4 * kW - 1);
        const uint32_t v = (j0 + 8 * ch) | ((j0 + 8 * ch + 1) << 16);
        dst[ch] = make_uint4(v, v + 0x00020002u, v + 0x00040004u, v + 0x00060006u);
      }
    }
    __syncthreads();  // (1) runs, cross bits and entries of every row

    if (tid < R::kBitWords) b.ebits[(uint64_t)t * R::kBitWords + tid] = cbits[tid];
    // from here to phase F the staging buffer holds the warps' work queues
    // (512 entries each, or 32 * kQ8 while L2 -- the roots linked by unions,
    // a bitmap like NR -- is in use behind them)
    uint32_t* Q = reinterpret_cast<uint32_t*>(sp) + warp * kQCap;
    uint32_t* Q8 = reinterpret_cast<uint32_t*>(sp) + warp * 32 * C::kQ8;
    uint32_t* L2 = reinterpret_cast<uint32_t*>(sp) + C::kWarps * 32 * C::kQ8;

    // ================================================= B: vertical unions
    // Each lane looks at the vertical bonds from its row y to the row below
    // over its 64 columns.  Only the first bond of each stretch along which
    // both rows continue horizontally counts (the others join the same two
    // runs).  The first such bond of each run of row y+1 (FM) gives that
    // run a parent: in a top-down pass over the tile's rows (one thread per
    // column, a barrier per row), its start is pointed at the root of the
    // row-y run it meets, which is one lookup away because row y is already
    // done.  This forest needs no atomics, its trees have depth one, and its
    // roots are the smallest index of their tree.  The remaining bonds (a
    // run of row y+1 meeting a second run above) join two trees: they are
    // queued and taken by the warp's lanes in lockstep, one step of their
    // current task per iteration (both endpoints move up to two levels,
    // path splitting on the way; a pair of roots is linked by a
    // compare-and-swap of the word holding the larger one's entry, the
    // larger under the smaller).  Every start given a parent is marked in
    // NR; a finished task points both run starts at the root.
    {
      uint32_t* FM = reinterpret_cast<uint32_t*>(sp);  // [TH][4] first bonds (staging buffer)
      const bool pv = ly + 1 < h;  // V is zero otherwise (phase A)
      const uint4 sq = pv ? *reinterpret_cast<const uint4*>(RS + (ly + 1) * 4) : make_uint4(0u, 0u, 0u, 0u);
      // the row below over this lane's columns: run starts, the run start of
      // the first column, whether the column after the last continues a run
      const uint64_t S1 = part == 0 ? ((uint64_t)sq.x | ((uint64_t)sq.y << 32))
                                    : ((uint64_t)sq.z | ((uint64_t)sq.w << 32));
      const uint32_t c1 = part == 0 ? 0u : (sq.y ? 63u - (uint32_t)__clz(sq.y) : 31u - (uint32_t)__clz(sq.x));
      const uint64_t nb1 = part == 0 ? (uint64_t)(sq.z & 1u) : 1ull;
      const uint64_t h1 = ~((S1 >> 1) | (nb1 << 63));  // row y+1 continues from column x to x+1
      const uint64_t Sa = (uint64_t)Sm[0] | ((uint64_t)Sm[1] << 32);
      const uint64_t Ha = (uint64_t)H[0] | ((uint64_t)H[1] << 32);
      const uint64_t Va = (uint64_t)V[0] | ((uint64_t)V[1] << 32);
      // carry-lookahead over a lane's 64 columns: the carry into column x of
      // gen + (gen | prop) is set iff a generating column x' < x reaches x
      // through propagating columns.  Tasks: bonds not reached by an earlier
      // bond along columns where both rows continue.
      const uint64_t g = Ha & h1 & 0x7FFFFFFFFFFFFFFFull;
      const uint64_t gen = Va & g;
      const uint64_t tk = Va & ~((gen + (gen | g)) ^ gen ^ (gen | g));
      // first task of each run of row y+1 (the run that continues into the
      // second part of the row carries the answer across)
      const uint64_t gc = tk & h1;
      const uint64_t cov0 = (gc + h1) ^ gc ^ h1;
      uint32_t cin = __shfl_up_sync(kFull, (uint32_t)(((cov0 | tk) & h1) >> 63), 1);
      if (part == 0) cin = 0;
      const uint64_t first = tk & ~((gc + h1 + cin) ^ gc ^ h1);
      uint64_t rem = tk & ~first;
      FM[ly * 4 + (c0 >> 5)] = (uint32_t)first;
      FM[ly * 4 + (c0 >> 5) + 1] = (uint32_t)(first >> 32);
      L2[ly * 4 + (c0 >> 5)] = 0u;
      L2[ly * 4 + (c0 >> 5) + 1] = 0u;
      __syncthreads();
      volatile uint16_t* vp = P;
      // top-down, each warp over its own band of kRpw rows (lane l: columns
      // 4l .. 4l+3): row y+1's first-met runs under the parent of the row-y
      // run, which is its local root once row y is done; a run of the band's
      // top row counts as a local root itself, and its own parent in the row
      // above (where another warp may still be at work) is an ancestor,
      // resolved by the jumps below and the compression of phase C
      {
        const int lx = 4 * lane;
#pragma unroll 1
        for (int k = 0; k < kRpw; ++k) {
          const int y = warp * kRpw - 1 + k;  // the pair (y, y+1), y+1 in the band
          if (y >= 0 && y + 1 < h) {          // warp-uniform
            const int wd = y * 4 + (lx >> 5);
            const uint32_t f4 = (FM[wd] >> (lx & 31)) & 0xFu;
            if (f4) {
              const uint32_t sa = RS[wd], sc = RS[wd + 4];
              const uint32_t ca = RC[wd], cc = RC[wd + 4];
              const uint32_t cw = (uint32_t)(lx & ~31);
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                if ((f4 >> q) & 1u) {
                  const int b = (lx & 31) + q;
                  const uint32_t a = y * kTW + run_start(sa, b, cw, ca);
                  const uint32_t c = (y + 1) * kTW + run_start(sc, b, cw, cc);
                  // a run of the band's top row is the local root of the
                  // band's runs below it (its own parent, from the band above,
                  // may not be final yet)
                  vp[c] = y == warp * kRpw ? (uint16_t)a : vp[a];
                  atomicOr(&NR[c >> 5], 1u << (c & 31u));
                }
              }
            }
          }
          __syncwarp();
        }
      }
      __syncthreads();
      // the bands' top rows: pointer jumping (every band above resolved in
      // log2(bands) + 1 rounds), after which every parented start is at most
      // two links below its root
      {
        constexpr int kBands = TH / kRpw;
        constexpr int kJumps = kBands <= 1 ? 0 : (kBands <= 2 ? 1 : (kBands <= 4 ? 3 : 4));
        const int yt = warp * kRpw;  // this warp's top row
        const int lx = 4 * lane;
#pragma unroll 1
        for (int r = 0; r < kJumps; ++r) {
          if (warp > 0 && yt < h) {
            const int wd = yt * 4 + (lx >> 5);
            const uint32_t m4 = (RS[wd] & NR[wd]) >> (lx & 31) & 0xFu;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              if ((m4 >> q) & 1u) {
                const uint32_t sj = (uint32_t)(yt * kTW + lx + q);
                vp[sj] = vp[vp[sj]];
              }
            }
          }
          __syncthreads();
        }
      }
      // the trees joined again by the remaining bonds
      const uint32_t ja = (uint32_t)(ly * kTW), jc = ja + kTW;
      volatile uint32_t* vP32 = reinterpret_cast<volatile uint32_t*>(P);
      for (;;) {
        const uint32_t nq = enqueue16<C::kQ8>(rem, Q8, lane, [&](uint32_t x) {
          return (ja + run_start64(Sa, x, (uint32_t)c0, Cw[0])) |
                 ((jc + run_start64(S1, x, (uint32_t)c0, c1)) << 16);
        });
        if (nq == 0) break;  // warp-uniform
        uint32_t idx = (uint32_t)lane;
        uint32_t a = 0, c = 0, a0 = 0, c0s = 0;  // idle lanes look at entry 0 (always a valid index)
        bool act = false;
        for (uint32_t it = 0;; ++it) {
          const bool fetch = !act && idx < nq;
          const uint32_t e = fetch ? Q8[idx] : 0u;
          idx += fetch ? 32u : 0u;
          a = fetch ? (e & 0xFFFFu) : a;
          c = fetch ? (e >> 16) : c;
          a0 = fetch ? a : a0;
          c0s = fetch ? c : c0s;
          act = act || fetch;
          if (!__any_sync(kFull, act)) break;
          if (it >= kLocalCap) {  // warp-uniform
            bad = 1;
            break;
          }
          const uint32_t pa = vp[a], pc = vp[c];
          const uint32_t qa = vp[pa], qc = vp[pc];
          const bool ra = (pa == a) || (qa == pa), rc = (pc == c) || (qc == pc);
          if (act && !ra) vp[a] = (uint16_t)qa;
          if (act && !rc) vp[c] = (uint16_t)qc;
          a = (pa == a) ? a : ((qa == pa) ? pa : qa);
          c = (pc == c) ? c : ((qc == pc) ? pc : qc);
          const bool both = act && ra && rc;
          const uint32_t hi = a > c ? a : c, lo = a ^ c ^ hi;
          const uint32_t sh = (hi & 1u) << 4;
          const uint32_t old = vP32[hi >> 1];
          bool done = both && a == c;
          if (both && a != c && ((old >> sh) & 0xFFFFu) == hi) {
            const uint32_t nw = (old & ~(0xFFFFu << sh)) | (lo << sh);
            if (atomicCAS(reinterpret_cast<uint32_t*>(P) + (hi >> 1), old, nw) == old) {
              atomicOr(&NR[hi >> 5], 1u << (hi & 31u));
              atomicOr(&L2[hi >> 5], 1u << (hi & 31u));
              done = true;
            }
          }
          const uint32_t root = lo;
          if (done && a0 != root) vp[a0] = (uint16_t)root;
          if (done && c0s != root) vp[c0s] = (uint16_t)root;
          act = act && !done;
        }
        __syncwarp();  // the queue is refilled next round
      }
    }
    __syncthreads();  // (2) every union done

    // ================================================= C: open flags
    // A cluster that touches the tile edge is open: every edge site flags
    // its root (row edges: only run starts, the rest of a run shares them).
    if (tid < R::kBitWords) cbits[tid] = 0;
    if (tid == 0) wcnt[0] = 0;
    {
      const int nedge = 2 * (w + h);
      for (int e = tid; e < nedge; e += kThreads) {
        int lx, yy;
        bool col;
        if (e < h) { lx = w - 1; yy = e; col = true; }
        else if (e < 2 * h) { lx = 0; yy = e - h; col = true; }
        else if (e < 2 * h + w) { lx = e - 2 * h; yy = 0; col = false; }
        else { lx = e - 2 * h - w; yy = h - 1; col = false; }
        const uint32_t Sw = RS[yy * 4 + (lx >> 5)];
        if (!col && !((Sw >> (lx & 31)) & 1u)) continue;
        const uint32_t st = run_start(Sw, lx & 31, (uint32_t)(lx & ~31), RC[yy * 4 + (lx >> 5)]);
        const uint32_t r = root16(P, (uint32_t)(yy * kTW) + st, bad);
        atomicOr(reinterpret_cast<uint32_t*>(P) + (r >> 1), kMarkA << ((r & 1u) << 4));
      }
    }
    // the roots that unions linked, and the parented starts of the bands'
    // top rows, are pointed straight at their root: any start then is at
    // most two links below its root (its parent in the forest, one of these,
    // and the root), which phase F looks up at once.  The lanes queue these
    // starts of their rows and walk them in lockstep, two links per
    // iteration (path splitting on the way).
    {
      volatile uint16_t* vp = P;
      uint64_t rem = 0;
      if (ly < h) {
        rem = (uint64_t)L2[ly * 4 + (c0 >> 5)] | ((uint64_t)L2[ly * 4 + (c0 >> 5) + 1] << 32);
        if (ly == warp * kRpw && warp > 0)  // a band's top row: its parented starts
          rem |= ((uint64_t)Sm[0] & NR[ly * 4 + (c0 >> 5)]) |
                 (((uint64_t)Sm[1] & NR[ly * 4 + (c0 >> 5) + 1]) << 32);
      }
      const uint32_t jb = (uint32_t)(ly * kTW + c0);
      __syncwarp();
      for (;;) {
        const uint32_t nq = enqueue16<C::kQ8>(rem, Q8, lane, [&](uint32_t x) { return jb + x; });
        if (nq == 0) break;  // warp-uniform
        uint32_t idx = (uint32_t)lane, sj = 0, x = 0;  // idle lanes look at entry 0
        bool act = false;
        for (uint32_t it = 0;; ++it) {
          const bool fetch = !act && idx < nq;
          const uint32_t e = fetch ? Q8[idx] : 0u;
          idx += fetch ? 32u : 0u;
          sj = fetch ? e : sj;
          x = fetch ? e : x;
          act = act || fetch;
          if (!__any_sync(kFull, act)) break;
          if (it >= kLocalCap) {  // warp-uniform
            bad = 1;
            break;
          }
          const uint32_t p1 = vp[x] & kIdx16;
          const uint32_t p2 = vp[p1] & kIdx16;
          const uint32_t p3 = vp[p2] & kIdx16;
          const bool r1 = p2 == p1, r2 = p3 == p2;
          if (act && !r1 && !r2) vp[p1] = (uint16_t)p3;  // splitting (p1 is not a root)
          const bool done = act && (r1 || r2);
          const uint32_t root = r1 ? p1 : p2;
          if (done) vp[sj] = (uint16_t)root;
          x = r1 ? p1 : (r2 ? p2 : p3);
          act = act && !done;
        }
        __syncwarp();
      }
    }
    __syncthreads();  // (3) flags set

    // ================================================= D: roots
    // The roots among a lane's run starts are the starts no link marked
    // (NR).  The lanes queue their roots and take them in lockstep: a
    // closed root draws its cluster's new state (Sec. 2 step (3)), an open
    // root (flagged in phase C) takes a slot in the tile's open list (in
    // whatever order: a slot only names the root to later kernels) and its
    // node of the global union-find.  Other starts keep pointing at their
    // root: phase F looks the code up there.
    {
      volatile uint16_t* vp = P;
      uint64_t rem = 0;
      if (ly < h)
        rem = ((uint64_t)Sm[0] & ~NR[ly * 4 + (c0 >> 5)]) |
              (((uint64_t)Sm[1] & ~NR[ly * 4 + (c0 >> 5) + 1]) << 32);
      const uint32_t jb = (uint32_t)(ly * kTW + c0);
      for (;;) {
        const uint32_t nq = enqueue16(rem, Q, lane, [&](uint32_t x) { return jb + x; });
        if (nq == 0) break;  // warp-uniform
        for (uint32_t k0 = 0; k0 < nq; k0 += 32) {
          const uint32_t k = k0 + (uint32_t)lane;
          const uint32_t r = k < nq ? Q[k] : 0u;
          const uint32_t e = vp[r];
          if (k < nq) {
            if (e & kMarkA) {
              const uint32_t slot = atomicAdd(&wcnt[0], 1u);
              const uint64_t d = (uint64_t)t * R::kOpenCap + slot;
              b.G[d] = gword(lat, d, x0, y0, r, slot);
              vp[r] = (uint16_t)(kMarkB | slot);
            } else {
              uint32_t code;
              if constexpr (kRoots) {
                code = kMarkA | r;
              } else {
                code = kMarkA |
                       pick_state(philox(global_index(lat, x0, y0, r), kDomSpin).x, q_states);
              }
              vp[r] = (uint16_t)code;
            }
          }
        }
        __syncwarp();
      }
    }
    __syncthreads();  // (4) every root coded

    // the next tile's spins into the staging buffer (free again), while
    // this tile's codes are written
    pre = false;
    if (!kGiven) {
      const uint32_t gn = g + gridDim.x;
      if (gn < total && src.lattice(src.rep(gn)).vec4) {
        stage_rows<TH, kThreads>(src, gn, sp, hal, true);
        cp_async_commit();
        pre = true;
      }
    }

    // ================================================= F: site codes, edge lines
    {
      uint16_t* edge = b.edge + (uint64_t)t * R::kEdge;
      const volatile uint16_t* vp = P;
      const int cx = 8 * (tid & 15);
      for (int yy = tid >> 4; yy < h; yy += kThreads / 16) {
        if (cx < w) {
          const uint32_t Sw = RS[yy * 4 + (cx >> 5)];
          const uint32_t s8 = (Sw >> (cx & 31)) & 0xFFu;
          const uint32_t jr = (uint32_t)(yy * kTW), j8 = jr + (uint32_t)cx;
          // the run start of the group's first site
          const uint32_t st0 = (s8 & 1u) ? j8 : jr + run_start(Sw, cx & 31, (uint32_t)(cx & ~31), RC[yy * 4 + (cx >> 5)]);
          // the group's eight entries in one 16-byte load: a start's entry
          // is its code (a root) or a link towards its root
          const uint4 E = *reinterpret_cast<const uint4*>(P + j8);
          const uint32_t ew[4] = {E.x, E.y, E.z, E.w};
          uint32_t cd[8], rt[8];
          // a run start's root is the first entry with a marker on its path:
          // three lookups cover the paths of length two or less, longer
          // ones are walked afterwards
          bool deep = false;
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const uint32_t ek = (ew[k >> 1] >> (16 * (k & 1))) & 0xFFFFu;
            const bool sk = (s8 >> k) & 1u;
            if (k == 0 || sk) {
              uint32_t x = sk ? j8 + k : st0;          // the run start
              uint32_t e = sk ? ek : (uint32_t)vp[x];  // its entry
              if (!(e & kMarks)) {
                x = e;
                e = vp[x];
              }
              if (!(e & kMarks)) {
                x = e;
                e = vp[x];
              }
              deep = deep || !(e & kMarks);
              rt[k] = x;
              cd[k] = e;
            } else {
              rt[k] = rt[k - 1];
              cd[k] = cd[k - 1];
            }
          }
          if (deep) {  // rare: a start more than two links below its root
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              if (k == 0 || ((s8 >> k) & 1u)) {
                uint32_t x = rt[k], e = cd[k];
                for (uint32_t it = 0; !(e & kMarks); ++it) {
                  if (it >= kLocalCap) {
                    bad = 1;
                    break;
                  }
                  x = e;
                  e = vp[x];
                }
                rt[k] = x;
                cd[k] = e;
              } else {
                rt[k] = rt[k - 1];
                cd[k] = cd[k - 1];
              }
            }
          }
          // final codes: a closed cluster's entry (kMarkA | payload, payload
          // below 0x4000) is its code; an open root's (kMarkB | slot) becomes
          // the slot -- both by clearing kMarkB, two codes per operation
          constexpr uint32_t kKeep2 = ~(kMarkB | (kMarkB << 16));
          const uint32_t cp[4] = {(cd[0] | (cd[1] << 16)) & kKeep2, (cd[2] | (cd[3] << 16)) & kKeep2,
                                  (cd[4] | (cd[5] << 16)) & kKeep2, (cd[6] | (cd[7] << 16)) & kKeep2};
          const uint64_t gi = (y0 + yy) * L + x0 + cx;
          if ((L & 7u) == 0 && cx + 8 <= w) {
            *reinterpret_cast<uint4*>(b.code + gi) = make_uint4(cp[0], cp[1], cp[2], cp[3]);
          } else {
#pragma unroll
            for (int k = 0; k < 8; ++k)
              if (cx + k < w) b.code[gi + k] = (uint16_t)(cp[k >> 1] >> (16 * (k & 1)));
          }
          // edge sites belong to open clusters: their codes are open slots
          if (yy == 0 || yy == h - 1) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              if (cx + k < w) {
                const uint16_t c = (uint16_t)(cp[k >> 1] >> (16 * (k & 1)));
                if (yy == h - 1) edge[2 * TH + cx + k] = c;
                if (yy == 0) edge[2 * TH + kTW + cx + k] = c;
              }
            }
          }
          if (cx == 0) edge[TH + yy] = (uint16_t)cp[0];
          if (cx + 8 >= w) {  // the group that holds the row's last site
            const int kl = w - 1 - cx;
            uint32_t v = cp[0];
#pragma unroll
            for (int k = 1; k < 8; ++k)
              if (k == kl) v = cp[k >> 1] >> (16 * (k & 1));
            edge[yy] = (uint16_t)v;
          }
        }
      }
      if (tid == 0) b.ocnt[t] = wcnt[0];
    }

    // ================================================= M: boundary unions (fused merge schedule)
    // Each tile edge is shared by two tiles; the one that finishes second
    // unites the clusters across it, so k_merge is not needed.  A tile
    // makes its records (nodes, edge slots, cross bits) visible to every SM,
    // then counts each of its four edges with an atomicAdd; every sweep adds
    // two to every counter, so the counter's old value is odd for the
    // second tile, which then reads the other tile's records (loads that
    // bypass L1) and does the unions of k_merge for that edge.  Nothing
    // waits for another CTA.
    if constexpr (kFuse && !kGiven) {
      uint32_t tx, ty;
      tile_xy(lat, t, tx, ty);
      const uint32_t tl = ty * lat.ntx + (tx == 0 ? lat.ntx - 1 : tx - 1);  // owner of the left edge
      const uint32_t tt = (ty == 0 ? lat.nty - 1 : ty - 1) * lat.ntx + tx;  // owner of the top edge
      __threadfence();
      __syncthreads();  // every thread's records are out
      if (tid < 4) {
        const uint32_t ce = tid == 0 ? 2 * t : (tid == 1 ? 2 * t + 1 : (tid == 2 ? 2 * tl : 2 * tt + 1));
        const uint32_t old = atomicAdd(b.ecnt + ce, 1u);
        __threadfence();
        reinterpret_cast<volatile uint8_t*>(wcnt + 1)[tid] = (uint8_t)(old & 1u);
      }
      __syncthreads();
      const uint32_t f = wcnt[1];  // byte e: this tile unites across edge e
      const int n0 = (f & 1u) ? h : 0, n1 = ((f >> 8) & 1u) ? w : 0;
      const int n2 = ((f >> 16) & 1u) ? h : 0, n3 = ((f >> 24) & 1u) ? w : 0;
      const int ntot = n0 + n1 + n2 + n3;
      const uint32_t cap = b.walk_cap ? b.walk_cap : kFindCap;
      for (int i0 = 0; i0 < ntot; i0 += kThreads) {  // CTA-uniform
        const int i = i0 + tid;
        uint64_t na = 0, nc = 0;
        uint32_t key = 0xFFFFFFFFu;
        bool act = false;
        if (i < ntot) {
          // edge e: 0 this tile's right, 1 its bottom, 2 the left (tl's
          // right), 3 the top (tt's bottom); k: row or column along it
          const int e = i < n0 ? 0 : (i < n0 + n1 ? 1 : (i < n0 + n1 + n2 ? 2 : 3));
          const int k = i - (e > 0 ? n0 : 0) - (e > 1 ? n1 : 0) - (e > 2 ? n2 : 0);
          const uint32_t owner = e < 2 ? t : (e == 2 ? tl : tt);
          uint32_t sa, sc;
          act = crossing_bond<TH, true>(b, lat, owner, (e & 1) ? TH + k : k, na, nc, sa, sc);
          key = ((uint32_t)e << 18) | (sa << kSlotBits) | sc;
        }
        // one lane per distinct pair of nodes in the warp does the union
        const unsigned same = __match_any_sync(kFull, act ? key : 0xFFFFFFFFu);
        if (act && lane == __ffs(same) - 1) gunite<TH>(b.G, lat, na, nc, b.err, cap);
      }
    }
    // a replica's observables go out when the CTA's next tile belongs to
    // another replica (or there is none); with the bit-plane counts (q <= 4)
    // each warp adds its own share at once, with no barrier
    if (Src::kMulti && measure) {
      if (q_states <= 4) {
        warp_flush(b, q_states, w, h);
      } else {
        const uint32_t gn = g + gridDim.x;
        if (gn >= total || src.rep(gn) != rep) flush(b, q_states);
      }
    }
  }

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

}  // namespace swgb
