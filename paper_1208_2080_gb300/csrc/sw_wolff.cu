// sw_wolff.cu -- C ABI of the Wolff single-cluster update of the 2D q-state
// Potts model (include/sw.h, sw_wolff_*), the comparison workload of the
// paper's related work (Sec. 1: Wolff's single-cluster algorithm, grown on
// a GPU by processing the newly added spins in parallel).
//
// One step: k_wolff_seed picks the seed site and the new state and puts
// the seed in the queue; k_wolff_grow grows the cluster with every warp of a
// persistent grid taking queued sites, testing their four neighbours
// (state, then the bond's Philox word), claiming a joining neighbour with a
// compare-and-swap of its spin (old state -> new state) and appending it;
// k_wolff_finish files the cluster size.  Every bond has one fixed Philox
// word per step, so the cluster is the connected component of the seed
// among the active bonds whatever order the warps visit it in: the result
// is bit-identical to the sequential oracle.
//
// A second mode finds the same cluster by labelling (the route of the
// related work's connected-component Wolff): k_wolff_bonds writes every
// active bond of the step (both ends in the seed's old state, word below the
// threshold), the tile union-find of the SW sweep labels them, and
// k_wolff_flip gives the new state to the sites whose root is the seed's.
// Its cost is that of labelling the lattice, independent of the cluster.
//
// The queue has one slot per site.  Warps reserve slots ahead of the
// producers (atomic head), wait for them to be written, and reset each slot
// they consume so the queue is empty again for the next step.  The growth
// ends when every appended site has been processed (processed == tail,
// both monotone); every wait is bounded and reports SW_ERR_TIMEOUT instead
// of spinning on.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/sw.h"
#include "philox.cuh"
#include "sw_internal.h"
#include "sw_kernels.cuh"
#include "sw_launch.cuh"

using namespace swgb;

namespace {

constexpr uint32_t kEmpty = 0xFFFFFFFFu;  // a free queue slot (site indices are < 2^30)
constexpr uint32_t kDomSeed = 4, kDomWolffBond = 5;
constexpr int kGrowThreads = 256;
constexpr uint32_t kIdleCap = 1u << 22;   // idle polls of one warp before it gives up
constexpr uint32_t kErrWolffTimeout = 1u, kErrWolffCas = 2u;

struct WolffCtl {
  uint32_t head, tail, processed, s_old;
  uint32_t s_new, err, pad0, pad1;
  unsigned long long step;
};

struct WolffArgs {
  uint8_t* spin;
  uint32_t* queue;            // growth mode
  uint8_t* bonds;             // labelling mode: packed bonds of the step
  uint32_t* roots;            // labelling mode: root of every site
  WolffCtl* ctl;
  unsigned long long* sizes;  // ring of cluster sizes
  uint32_t L, q, thr, ring;
  uint64_t N, bp;
  uint32_t rk[20];
  uint32_t idle_cap;          // growth mode: idle polls of one warp before it gives up
};

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t* p) {
  return *reinterpret_cast<const volatile uint32_t*>(p);
}

// grow: also flips the seed and queues it (growth mode); otherwise the
// seed index is kept in pad0 for the flip of the labelling mode.
__global__ void k_wolff_seed(const __grid_constant__ WolffArgs a, int grow) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  WolffCtl* c = a.ctl;
  const uint32_t t = (uint32_t)c->step;
  const Words4 w = stream4_rk(a.rk, 0ull, t, kDomSeed);
  const uint64_t i0 = ((uint64_t)w.x * a.N) >> 32;
  const uint32_t old = a.spin[i0];
  const uint32_t sn = (old + 1u + pick_state(w.y, a.q - 1u)) % a.q;
  if (grow) {
    a.spin[i0] = (uint8_t)sn;
    a.queue[0] = (uint32_t)i0;
  }
  c->head = 0;
  c->tail = grow ? 1 : 0;
  c->processed = 0;
  c->s_old = old;
  c->s_new = sn;
  c->pad0 = (uint32_t)i0;
}

// Labelling mode, bonds of the step: a bond is active iff both ends are in
// the seed's old state and its word is below the threshold.  A thread
// writes the packed byte of 4 sites (bits 2k right, 2k+1 down).  When L is
// a multiple of 4 the four spins, the four below them and the right
// neighbour come in three loads, and the two sites of a pair share their
// Philox call (one call gives the words of sites 2m and 2m+1).
__global__ void __launch_bounds__(256) k_wolff_bonds(const __grid_constant__ WolffArgs a) {
  const uint32_t s_old = a.ctl->s_old;
  const uint32_t t = (uint32_t)a.ctl->step;
  const uint64_t L = a.L, groups = a.bp;
  const bool vec = (L & 3u) == 0;
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < L * groups;
       g += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t y = g / groups, x0 = (g - y * groups) * 4;
    const uint64_t yd = (y + 1 == L) ? 0 : y + 1;
    uint32_t byte = 0;
    if (vec) {
      const uint64_t i0 = y * L + x0;  // a multiple of 4: the pairs are (i0, i0+1), (i0+2, i0+3)
      const uint32_t sw = *reinterpret_cast<const uint32_t*>(a.spin + i0);
      const uint32_t dw = *reinterpret_cast<const uint32_t*>(a.spin + yd * L + x0);
      const uint32_t rn = a.spin[y * L + (x0 + 4 == L ? 0 : x0 + 4)];
      const uint32_t rw = (sw >> 8) | (rn << 24);  // the right neighbours of the four sites
      uint32_t need = 0;                          // per site: bit 0 right, bit 1 down candidate
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t sk = (sw >> (8 * k)) & 0xFFu;
        if (sk != s_old) continue;
        if (((rw >> (8 * k)) & 0xFFu) == s_old) need |= 1u << (2 * k);
        if (((dw >> (8 * k)) & 0xFFu) == s_old) need |= 2u << (2 * k);
      }
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const uint32_t np = (need >> (4 * p)) & 0xFu;
        if (!np) continue;
        const Words4 w = stream4_rk(a.rk, (i0 >> 1) + p, t, kDomWolffBond);
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};  // right, down of the even site; of the odd one
#pragma unroll
        for (int b = 0; b < 4; ++b)
          if (((np >> b) & 1u) && ws[b] < a.thr) byte |= 1u << (4 * p + b);
      }
    } else {
      for (int k = 0; k < 4 && x0 + k < L; ++k) {
        const uint64_t x = x0 + k, i = y * L + x;
        if (a.spin[i] != s_old) continue;
        const uint64_t xr = (x + 1 == L) ? 0 : x + 1;
        const bool er = a.spin[y * L + xr] == s_old, ed = a.spin[yd * L + x] == s_old;
        if (!er && !ed) continue;
        const Words4 w = stream4_rk(a.rk, i >> 1, t, kDomWolffBond);
        const uint32_t wr = (i & 1u) ? w.z : w.x, wd = (i & 1u) ? w.w : w.y;
        if (er && wr < a.thr) byte |= 1u << (2 * k);
        if (ed && wd < a.thr) byte |= 2u << (2 * k);
      }
    }
    a.bonds[y * a.bp + x0 / 4] = (uint8_t)byte;
  }
}

// Labelling mode, the update: sites whose root is the seed's take the new
// state; the cluster size goes to ctl->tail.
__global__ void __launch_bounds__(256) k_wolff_flip(const __grid_constant__ WolffArgs a) {
  const uint32_t r0 = a.roots[a.ctl->pad0];
  const uint32_t s_new = a.ctl->s_new;
  uint32_t n = 0;
  if ((a.N & 3u) == 0) {  // four roots per 16-byte load
    const uint4* r4 = reinterpret_cast<const uint4*>(a.roots);
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < a.N / 4;
         v += (uint64_t)gridDim.x * blockDim.x) {
      const uint4 r = __ldcs(r4 + v);
      const uint32_t rv[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (rv[k] == r0) {
          a.spin[4 * v + k] = (uint8_t)s_new;
          ++n;
        }
      }
    }
  } else {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.N;
         i += (uint64_t)gridDim.x * blockDim.x) {
      if (a.roots[i] == r0) {
        a.spin[i] = (uint8_t)s_new;
        ++n;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xFFFFFFFFu, n, o);
  if ((threadIdx.x & 31) == 0 && n) atomicAdd(&a.ctl->tail, n);
}

// Claims site j for the cluster: its spin byte goes from s_old to s_new in
// one compare-and-swap of the aligned word that holds it.  False if j is not
// (or no longer) in the old state.
__device__ __forceinline__ bool claim(uint8_t* spin, uint64_t j, uint32_t s_old, uint32_t s_new,
                                      uint32_t* err) {
  uint32_t* wp = reinterpret_cast<uint32_t*>(spin + (j & ~3ull));
  const uint32_t sh = 8u * (uint32_t)(j & 3u);
  uint32_t w = ld_volatile(wp);
  for (int it = 0; it < 64; ++it) {
    if (((w >> sh) & 0xFFu) != s_old) return false;
    const uint32_t nw = (w & ~(0xFFu << sh)) | (s_new << sh);
    const uint32_t prev = atomicCAS(wp, w, nw);
    if (prev == w) return true;
    w = prev;  // a neighbouring byte changed (or this one was claimed): retry
  }
  atomicOr(err, kErrWolffCas);
  return false;
}

__global__ void __launch_bounds__(kGrowThreads) k_wolff_grow(const __grid_constant__ WolffArgs a) {
  constexpr unsigned kFull = 0xFFFFFFFFu;
  WolffCtl* c = a.ctl;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t s_old = c->s_old, s_new = c->s_new;
  const uint32_t t = (uint32_t)c->step;
  const uint64_t L = a.L;
  uint64_t slot = ~0ull;  // the queue slot this lane waits on
  uint32_t idle = 0, nap = 32;
  while (true) {
    // lanes without a slot reserve the next ones
    const unsigned need = __ballot_sync(kFull, slot == ~0ull);
    if (need) {
      uint32_t base = 0;
      if (lane == (uint32_t)(__ffs(need) - 1)) base = atomicAdd(&c->head, (uint32_t)__popc(need));
      base = __shfl_sync(kFull, base, __ffs(need) - 1);
      if (slot == ~0ull) slot = base + __popc(need & ((1u << lane) - 1u));
    }
    // take the item of the slot if it has been written
    uint32_t item = kEmpty;
    if (slot < a.N) {
      item = ld_volatile(a.queue + slot);
      if (item != kEmpty) {
        a.queue[slot] = kEmpty;  // consumed: the queue is empty again after the step
        slot = ~0ull;
      }
    }
    const bool have = item != kEmpty;
    const unsigned got = __ballot_sync(kFull, have);
    if (!got) {
      // nothing to do: stop once every appended site has been processed
      uint32_t done = 0;
      if (lane == 0) {
        const uint32_t p = ld_volatile(&c->processed);
        __threadfence();
        const uint32_t tl = ld_volatile(&c->tail);
        done = (p == tl) ? 1u : 0u;
      }
      if (__shfl_sync(kFull, done, 0)) return;
      if (++idle >= a.idle_cap) {
        if (lane == 0) atomicOr(&c->err, kErrWolffTimeout);
        return;
      }
      __nanosleep(nap);
      if (nap < 1024) nap *= 2;
      continue;
    }
    idle = 0;
    nap = 32;
    // grow from the item: four neighbours, the bond that joins each
    uint32_t add[4];
    uint32_t nadd = 0;
    if (have) {
      const uint64_t i = item;
      const uint64_t y = i / L, x = i - y * L;
      const uint64_t xr = (x + 1 == L) ? 0 : x + 1, xl = x ? x - 1 : L - 1;
      const uint64_t yd = (y + 1 == L) ? 0 : y + 1, yu = y ? y - 1 : L - 1;
      const uint64_t nb[4] = {y * L + xr, y * L + xl, yd * L + x, yu * L + x};
      const uint64_t own[4] = {i, y * L + xl, i, yu * L + x};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint64_t j = nb[k];
        if (a.spin[j] != s_old) continue;  // already in the cluster, or another state
        const Words4 w = stream4_rk(a.rk, own[k] >> 1, t, kDomWolffBond);
        const uint32_t word = (own[k] & 1u) ? ((k >= 2) ? w.w : w.z) : ((k >= 2) ? w.y : w.x);
        if (word >= a.thr) continue;
        if (claim(a.spin, j, s_old, s_new, &c->err)) add[nadd++] = (uint32_t)j;
      }
    }
    // append the claimed sites (one atomic per warp), then count the
    // processed items: appends are visible in tail before processed moves
    uint32_t off = nadd;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(kFull, off, o);
      if (lane >= (uint32_t)o) off += v;
    }
    const uint32_t total = __shfl_sync(kFull, off, 31);
    uint32_t pos = 0;
    if (total) {
      if (lane == 31) pos = atomicAdd(&c->tail, total);
      pos = __shfl_sync(kFull, pos, 31);
      const uint32_t mine = pos + off - nadd;
      for (uint32_t k = 0; k < nadd; ++k) {
        if (mine + k < a.N)
          a.queue[mine + k] = add[k];
        else
          atomicOr(&c->err, kErrWolffCas);  // unreachable: every site joins at most once
      }
    }
    __threadfence();
    __syncwarp();
    if (lane == 0) atomicAdd(&c->processed, (uint32_t)__popc(got));
  }
}

__global__ void k_wolff_finish(const __grid_constant__ WolffArgs a) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  WolffCtl* c = a.ctl;
  const unsigned long long t = c->step;
  a.sizes[t % a.ring] = c->tail;
  c->step = t + 1;
}

}  // namespace

// Labelling-mode instantiations of the tile kernels, private to this file
// (their launch set-up is not shared with the other translation units).
struct WolffSrc : SingleSrc {};

struct sw_wolff {
  uint64_t L = 0, N = 0;
  int mode = SW_WOLFF_LABEL;
  uint32_t th = 64;
  Lattice lat{};
  Bufs lb{};  // labelling buffers (labelling mode)
  uint32_t q = 0, ring = 1024;
  double T = 0;
  cudaStream_t stream = nullptr;
  DeviceAllocator alloc{};
  std::vector<std::pair<void*, size_t>> blocks;
  WolffArgs a{};
  uint64_t step = 0;
  uint64_t valid_from = 0;  // first step whose size is held
  int grid = 0;
  int last_err = SW_OK;
};

namespace {

void* wtake(sw_wolff* w, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  void* p = w->alloc.allocate(bytes);
  if (p) w->blocks.emplace_back(p, bytes);
  return p;
}

void wrelease(sw_wolff* w) {
  for (auto& kv : w->blocks) w->alloc.release(kv.first, kv.second);
  w->blocks.clear();
}

int wcuda(sw_wolff* w) {
  cudaGetLastError();
  w->last_err = SW_ERR_CUDA;
  return SW_ERR_CUDA;
}

int wcheck(sw_wolff* w) {
  uint32_t err = 0, lerr = 0;
  cudaError_t e = cudaMemcpyAsync(&err, &w->a.ctl->err, 4, cudaMemcpyDeviceToHost, w->stream);
  if (!e && w->a.roots) e = cudaMemcpyAsync(&lerr, w->lb.err, 4, cudaMemcpyDeviceToHost, w->stream);
  if (!e) e = cudaStreamSynchronize(w->stream);
  if (e) return wcuda(w);
  if ((err & kErrWolffTimeout) || (lerr & (kErrFind | kErrUnion | kErrLocal))) return w->last_err = SW_ERR_TIMEOUT;
  if (err || lerr) return w->last_err = SW_ERR_DEVICE;
  return SW_OK;
}

// k_check_spins of the Potts path, restated for this translation unit: sets
// *bad if a spin is >= q.
__global__ void k_wolff_check(const uint8_t* s, uint64_t N, uint32_t q, uint32_t* bad) {
  uint32_t any = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x)
    any |= s[i] >= q;
  if (__any_sync(0xFFFFFFFFu, any != 0) && (threadIdx.x & 31) == 0) atomicOr(bad, 1u);
}

__global__ void k_wolff_init(uint8_t* s, uint64_t N, uint32_t q, const __grid_constant__ WolffArgs a) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
    const Words4 w = stream4_rk(a.rk, i >> 2, 0u, kDomInit);
    const uint32_t v[4] = {w.x, w.y, w.z, w.w};
    s[i] = (uint8_t)pick_state(v[i & 3], q);
  }
}

int wolff_label_setup(sw_wolff* w);

}  // namespace

extern "C" {

int sw_wolff_create(uint64_t L, uint32_t q, double T, uint64_t seed, uint32_t init, uint32_t ring,
                    sw_wolff** out) {
  if (!out) return SW_ERR_INVAL;
  *out = nullptr;
  if (L < 2 || L > 32768 || q < 2 || q > 255 || !(T > 0.0) || !isfinite(T) || init > SW_INIT_ZERO)
    return SW_ERR_INVAL;
  sw_wolff* w = new (std::nothrow) sw_wolff();
  if (!w) return SW_ERR_NOMEM;
  w->L = L;
  w->N = L * L;
  w->q = q;
  w->T = T;
  w->ring = ring ? ring : 1024u;
  w->th = pick_tile_h(L, 0);
  w->alloc = current_allocator();
  WolffArgs& a = w->a;
  a.spin = (uint8_t*)wtake(w, w->N + 16);
  a.queue = (uint32_t*)wtake(w, w->N * 4);
  a.ctl = (WolffCtl*)wtake(w, sizeof(WolffCtl));
  a.sizes = (unsigned long long*)wtake(w, (size_t)w->ring * 8);
  if (!a.spin || !a.queue || !a.ctl || !a.sizes) {
    wrelease(w);
    delete w;
    return SW_ERR_NOMEM;
  }
  a.L = (uint32_t)L;
  a.N = w->N;
  a.q = q;
  a.thr = bond_threshold(T);
  a.idle_cap = kIdleCap;
  a.ring = w->ring;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    a.rk[2 * r] = k0;
    a.rk[2 * r + 1] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  int per_sm = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_wolff_grow, kGrowThreads, 0);
  if (sms <= 0) sms = 152;
  if (per_sm <= 0) per_sm = 1;
  if (per_sm > 4) per_sm = 4;
  w->grid = sms * per_sm;
  cudaError_t e = cudaMemsetAsync(a.queue, 0xFF, w->N * 4, w->stream);
  if (!e) e = cudaMemsetAsync(a.ctl, 0, sizeof(WolffCtl), w->stream);
  if (!e) e = cudaMemsetAsync(a.sizes, 0, (size_t)w->ring * 8, w->stream);
  if (!e) {
    if (init == SW_INIT_ZERO) {
      e = cudaMemsetAsync(a.spin, 0, w->N, w->stream);
    } else {
      k_wolff_init<<<152 * 8, 256, 0, w->stream>>>(a.spin, w->N, q, a);
      e = cudaGetLastError();
    }
  }
  if (!e) e = cudaStreamSynchronize(w->stream);
  if (e) {
    cudaGetLastError();
    wrelease(w);
    delete w;
    return SW_ERR_CUDA;
  }
  // the labelling mode is the default: its buffers are taken now
  const int rc = wolff_label_setup(w);
  if (rc) {
    wrelease(w);
    delete w;
    return rc;
  }
  *out = w;
  return SW_OK;
}

void sw_wolff_destroy(sw_wolff* w) {
  if (!w) return;
  cudaStreamSynchronize(w->stream);
  wrelease(w);
  delete w;
}

int sw_wolff_bind_stream(sw_wolff* w, void* stream) {
  if (!w) return SW_ERR_INVAL;
  w->stream = (cudaStream_t)stream;
  return SW_OK;
}

}  // extern "C"

namespace {

template <int TH>
cudaError_t wolff_label(sw_wolff* w) {
  WolffSrc src;
  src.b = w->lb;
  src.lat = w->lat;
  cudaError_t e = launch_label_src<TH, uint32_t, true, true>(src, w->lat.ntiles, w->stream);
  if (e) return e;
  e = launch_merge_src<TH, uint32_t>(src, w->lat.ntiles, w->stream);
  if (e) return e;
  return launch_recolor_src<TH, uint32_t, true>(src, w->lat.ntiles, w->a.roots, w->stream);
}

// Allocates the labelling buffers on first use of the labelling mode.
int wolff_label_setup(sw_wolff* w) {
  if (w->a.roots) return SW_OK;
  const uint32_t th = w->th;
  w->lat = make_lattice(w->L, th);
  const uint64_t nt = w->lat.ntiles;
  Bufs& b = w->lb;
  w->a.bp = w->lat.bp;
  w->a.bonds = (uint8_t*)wtake(w, w->L * w->lat.bp + 16);
  w->a.roots = (uint32_t*)wtake(w, w->N * 4);
  b.bonds = w->a.bonds;
  b.code = (uint16_t*)wtake(w, w->N * 2 + 16);
  b.G = (uint64_t*)wtake(w, nt * open_cap(th) * 8);
  b.edge = (uint16_t*)wtake(w, nt * edge_u16(th) * 2);
  b.ebits = (uint32_t*)wtake(w, nt * bit_words(th) * 4);
  b.ocnt = (uint32_t*)wtake(w, nt * 4);
  b.ctl = (unsigned long long*)wtake(w, 64);
  b.err = (uint32_t*)wtake(w, 64);
  b.q = 2;
  b.measure = 0;
  if (!w->a.bonds || !w->a.roots || !b.code || !b.G || !b.edge || !b.ebits || !b.ocnt ||
      !b.ctl || !b.err) {
    w->a.roots = nullptr;  // the blocks taken so far are freed with the handle
    return SW_ERR_NOMEM;
  }
  cudaError_t e = cudaMemsetAsync(b.G, 0, nt * open_cap(th) * 8, w->stream);
  if (!e) e = cudaMemsetAsync(b.ctl, 0, 64, w->stream);
  if (!e) e = cudaMemsetAsync(b.err, 0, 64, w->stream);
  if (!e) e = cudaMemsetAsync(b.ocnt, 0, nt * 4, w->stream);
  if (!e) {
    WolffSrc src;
    src.b = b;
    src.lat = w->lat;
    switch (th) {
      case 16: e = configure_label<16, uint32_t, true, true, WolffSrc>(src, nullptr); break;
      case 32: e = configure_label<32, uint32_t, true, true, WolffSrc>(src, nullptr); break;
      case 64: e = configure_label<64, uint32_t, true, true, WolffSrc>(src, nullptr); break;
      default: e = configure_label<128, uint32_t, true, true, WolffSrc>(src, nullptr); break;
    }
  }
  if (!e) e = cudaStreamSynchronize(w->stream);
  if (e) {
    w->a.roots = nullptr;
    return wcuda(w);
  }
  return SW_OK;
}

cudaError_t wolff_step_label(sw_wolff* w) {
  k_wolff_seed<<<1, 32, 0, w->stream>>>(w->a, 0);
  uint64_t items = w->L * w->a.bp, blocks = (items + 255) / 256;
  if (blocks > 152ull * 16) blocks = 152ull * 16;
  k_wolff_bonds<<<(unsigned)blocks, 256, 0, w->stream>>>(w->a);
  cudaError_t e = cudaGetLastError();
  if (e) return e;
  switch (w->th) {
    case 16: e = wolff_label<16>(w); break;
    case 32: e = wolff_label<32>(w); break;
    case 64: e = wolff_label<64>(w); break;
    default: e = wolff_label<128>(w); break;
  }
  if (e) return e;
  blocks = (w->N + 255) / 256;
  if (blocks > 152ull * 16) blocks = 152ull * 16;
  k_wolff_flip<<<(unsigned)blocks, 256, 0, w->stream>>>(w->a);
  k_wolff_finish<<<1, 32, 0, w->stream>>>(w->a);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

int sw_wolff_set_wait_limit(sw_wolff* w, uint32_t idle_polls) {
  if (!w) return SW_ERR_INVAL;
  w->a.idle_cap = idle_polls ? idle_polls : kIdleCap;
  return SW_OK;
}

int sw_wolff_set_mode(sw_wolff* w, int mode) {
  if (!w || (mode != SW_WOLFF_GROW && mode != SW_WOLFF_LABEL)) return SW_ERR_INVAL;
  if (w->last_err) return w->last_err;
  if (mode == SW_WOLFF_LABEL) {
    int rc = wolff_label_setup(w);
    if (rc) return rc;
  }
  w->mode = mode;
  return SW_OK;
}

int sw_wolff_step(sw_wolff* w, uint64_t n) {
  if (!w) return SW_ERR_INVAL;
  if (w->last_err) return w->last_err;
  for (uint64_t k = 0; k < n; ++k) {
    if (w->mode == SW_WOLFF_LABEL) {
      if (wolff_step_label(w) != cudaSuccess) return wcuda(w);
      continue;
    }
    k_wolff_seed<<<1, 32, 0, w->stream>>>(w->a, 1);
    k_wolff_grow<<<w->grid, kGrowThreads, 0, w->stream>>>(w->a);
    k_wolff_finish<<<1, 32, 0, w->stream>>>(w->a);
    if (cudaGetLastError() != cudaSuccess) return wcuda(w);
  }
  w->step += n;
  return SW_OK;
}

int sw_wolff_sync(sw_wolff* w) {
  if (!w) return SW_ERR_INVAL;
  if (w->last_err) return w->last_err;
  return wcheck(w);
}

int sw_wolff_sizes(sw_wolff* w, uint64_t first, uint64_t count, uint64_t* sizes) {
  if (!w || (count && !sizes)) return SW_ERR_INVAL;
  if (w->last_err) return w->last_err;
  if (count == 0) return SW_OK;
  const uint64_t last = first + count - 1;
  if (last < first || last >= w->step) return SW_ERR_RANGE;
  uint64_t oldest = w->valid_from;
  if (w->step > w->ring && w->step - w->ring > oldest) oldest = w->step - w->ring;
  if (first < oldest) return SW_ERR_RANGE;
  std::vector<unsigned long long> host(w->ring);
  if (cudaMemcpyAsync(host.data(), w->a.sizes, (size_t)w->ring * 8, cudaMemcpyDeviceToHost, w->stream))
    return wcuda(w);
  int rc = wcheck(w);
  if (rc) return rc;
  for (uint64_t k = 0; k < count; ++k) sizes[k] = host[(first + k) % w->ring];
  return SW_OK;
}

int sw_wolff_spins(sw_wolff* w, uint8_t* dst, uint64_t n, int dst_on_device) {
  if (!w || !dst || n != w->N) return SW_ERR_INVAL;
  if (w->last_err) return w->last_err;
  if (cudaMemcpyAsync(dst, w->a.spin, w->N, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                      w->stream))
    return wcuda(w);
  if (!dst_on_device) return wcheck(w);
  return SW_OK;
}

int sw_wolff_set_spins(sw_wolff* w, const uint8_t* src, uint64_t n, int src_on_device) {
  if (!w || !src || n != w->N) return SW_ERR_INVAL;
  if (w->last_err) return w->last_err;
  std::vector<uint8_t> keep;
  cudaError_t e = cudaSuccess;
  // validate in a scratch copy first so a bad configuration leaves the
  // lattice as it was
  uint8_t* tmp = (uint8_t*)w->alloc.allocate(((w->N + 16 + 255) / 256) * 256);
  uint32_t* bad = (uint32_t*)w->alloc.allocate(256);
  if (!tmp || !bad) {
    if (tmp) w->alloc.release(tmp, ((w->N + 16 + 255) / 256) * 256);
    if (bad) w->alloc.release(bad, 256);
    return SW_ERR_NOMEM;
  }
  e = cudaMemcpyAsync(tmp, src, w->N, src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                      w->stream);
  if (!e) e = cudaMemsetAsync(bad, 0, 4, w->stream);
  if (!e) {
    k_wolff_check<<<152 * 8, 256, 0, w->stream>>>(tmp, w->N, w->q, bad);
    e = cudaGetLastError();
  }
  uint32_t hbad = 0;
  if (!e) e = cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, w->stream);
  if (!e) e = cudaStreamSynchronize(w->stream);
  if (!e && !hbad) e = cudaMemcpyAsync(w->a.spin, tmp, w->N, cudaMemcpyDeviceToDevice, w->stream);
  if (!e) e = cudaStreamSynchronize(w->stream);
  w->alloc.release(tmp, ((w->N + 16 + 255) / 256) * 256);
  w->alloc.release(bad, 256);
  if (e) return wcuda(w);
  return hbad ? SW_ERR_INVAL : SW_OK;
}

int sw_wolff_get_step(const sw_wolff* w, uint64_t* step) {
  if (!w || !step) return SW_ERR_INVAL;
  *step = w->step;
  return SW_OK;
}

}  // extern "C"
