// sw_le.cu -- the paper's labeller, for comparison with the tile
// union-find: "label equivalence" after Kalentev et al., as described in
// Sec. 2.  Every site starts with its own index as label; then
//   scanning: a site whose active-bond neighbours carry a smaller label
//             lowers label[label[site]] to that smallest label (atomicMin),
//   analysis: every site follows label[] to its end and adopts it,
// repeated until a scan changes nothing.  Labels only ever decrease towards
// the smallest site index of the cluster, so the fixed point is the same
// smallest-index root the rest of the library uses (bit-identical results).
// The whole label array is re-read on every iteration, which is what the
// tile union-find avoids.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sw.h"
#include "sw_internal.h"

namespace swgb {
namespace le {

constexpr int kThreads = 256;
constexpr uint32_t kChainCap = 1u << 24;

template <typename LabelT>
__global__ void k_le_init(LabelT* label, uint64_t N) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (uint64_t)gridDim.x * blockDim.x)
    label[i] = (LabelT)i;
}

__device__ __forceinline__ uint32_t bond_bits(const uint8_t* bonds, uint64_t bp, uint64_t y, uint64_t x) {
  return (bonds[y * bp + (x >> 2)] >> (2 * (x & 3))) & 3u;
}

__device__ __forceinline__ uint32_t atomic_min_l(uint32_t* p, uint32_t v) { return atomicMin(p, v); }
__device__ __forceinline__ uint64_t atomic_min_l(uint64_t* p, uint64_t v) {
  return (uint64_t)atomicMin(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}

// Scanning: one thread per site; the smallest label among the site and its
// active-bond neighbours is written into the entry its own label points to.
template <typename LabelT>
__global__ void __launch_bounds__(kThreads) k_le_scan(const uint8_t* __restrict__ bonds, LabelT* label,
                                                      uint64_t L, uint64_t bp, uint32_t* changed) {
  bool any = false;
  for (uint64_t y = blockIdx.y; y < L; y += gridDim.y) {
    const uint64_t yu = y ? y - 1 : L - 1, yd = (y + 1 == L) ? 0 : y + 1;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < L;
         x += (uint64_t)gridDim.x * blockDim.x) {
      const uint64_t i = y * L + x;
      const uint64_t xl = x ? x - 1 : L - 1, xr = (x + 1 == L) ? 0 : x + 1;
      const LabelT li = label[i];
      LabelT m = li;
      const uint32_t own = bond_bits(bonds, bp, y, x);
      if (own & 1u) m = min(m, label[y * L + xr]);
      if (own & 2u) m = min(m, label[yd * L + x]);
      if (bond_bits(bonds, bp, y, xl) & 1u) m = min(m, label[y * L + xl]);
      if (bond_bits(bonds, bp, yu, x) & 2u) m = min(m, label[yu * L + x]);
      if (m < li) {
        atomic_min_l(label + li, m);
        any = true;
      }
    }
  }
  if (__any_sync(0xFFFFFFFFu, any) && (threadIdx.x & 31) == 0) atomicOr(changed, 1u);
}

// Analysis: every site follows the chain of labels to its end.
template <typename LabelT>
__global__ void __launch_bounds__(kThreads) k_le_analysis(LabelT* label, uint64_t N, uint32_t* err) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (uint64_t)gridDim.x * blockDim.x) {
    LabelT l = label[i];
    uint32_t it = 0;
    for (; it < kChainCap; ++it) {
      const LabelT n = label[l];
      if (n == l) break;
      l = n;
    }
    if (it == kChainCap) atomicOr(err, 1u);
    label[i] = l;
  }
}

template <typename LabelT>
int run_le(uint64_t L, const uint8_t* bonds, LabelT* roots, uint32_t max_iter, uint32_t* iters,
           cudaStream_t st, uint32_t* flags) {
  const uint64_t N = L * L, bp = (L + 3) / 4;
  uint64_t blocks = (N + kThreads - 1) / kThreads;
  if (blocks > 152ull * 64) blocks = 152ull * 64;
  const uint64_t gx = (L + kThreads - 1) / kThreads;
  const dim3 sgrid((unsigned)(gx < 64 ? gx : 64), (unsigned)(L < 65535 ? L : 65535));
  k_le_init<LabelT><<<(unsigned)blocks, kThreads, 0, st>>>(roots, N);
  uint32_t n = 0;
  for (;;) {
    if (n >= max_iter) return SW_ERR_TIMEOUT;
    uint32_t changed = 0;
    cudaError_t e = cudaMemsetAsync(flags, 0, 4, st);
    if (!e) {
      k_le_scan<LabelT><<<sgrid, kThreads, 0, st>>>(bonds, roots, L, bp, flags);
      k_le_analysis<LabelT><<<(unsigned)blocks, kThreads, 0, st>>>(roots, N, flags + 1);
      e = cudaGetLastError();
    }
    if (!e) e = cudaMemcpyAsync(&changed, flags, 4, cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return SW_ERR_CUDA;
    }
    ++n;
    if (!changed) break;
  }
  uint32_t err = 0;
  if (cudaMemcpy(&err, flags + 1, 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return SW_ERR_CUDA;
  }
  if (iters) *iters = n;
  return err ? SW_ERR_TIMEOUT : SW_OK;
}


// ---------------------------------------------------------------------------
// Two-stage labelling of Sec. 3, emulated on one GPU: the lattice is split
// into (L/S)^2 sub-lattices of S x S sites (the paper's per-GPU
// sub-lattices).  Stage 1 labels every sub-lattice with label equivalence,
// ignoring bonds that leave it.  Stage 2 works only on the boundary layers:
// label_total[r] (r = a stage-1 label of a boundary site) is lowered across
// the bonds that cross sub-lattice boundaries (scanning) and its chains are
// resolved (analysis), until nothing changes.  Finally every site adopts
// label_total of its stage-1 label.  Labels are global site indices and
// always move to the smaller one, so the result is again the smallest site
// index of every cluster.

template <typename LabelT>
__global__ void __launch_bounds__(kThreads) k_2s_scan_local(const uint8_t* __restrict__ bonds, LabelT* label,
                                                            uint64_t L, uint64_t bp, uint64_t S,
                                                            uint32_t* changed) {
  bool any = false;
  for (uint64_t y = blockIdx.y; y < L; y += gridDim.y) {
    const uint64_t yu = y ? y - 1 : L - 1, yd = (y + 1 == L) ? 0 : y + 1;
    const uint32_t ys = (uint32_t)y % (uint32_t)S;  // L, S <= 2^20: 32-bit remainders
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < L;
         x += (uint64_t)gridDim.x * blockDim.x) {
      const uint64_t i = y * L + x;
      const uint32_t xs = (uint32_t)x % (uint32_t)S;
      const uint64_t xl = x ? x - 1 : L - 1, xr = (x + 1 == L) ? 0 : x + 1;
      const LabelT li = label[i];
      LabelT m = li;
      const uint32_t own = bond_bits(bonds, bp, y, x);
      if ((own & 1u) && xs != S - 1) m = min(m, label[y * L + xr]);
      if ((own & 2u) && ys != S - 1) m = min(m, label[yd * L + x]);
      if (xs != 0 && (bond_bits(bonds, bp, y, xl) & 1u)) m = min(m, label[y * L + xl]);
      if (ys != 0 && (bond_bits(bonds, bp, yu, x) & 2u)) m = min(m, label[yu * L + x]);
      if (m < li) {
        atomic_min_l(label + li, m);
        any = true;
      }
    }
  }
  if (__any_sync(0xFFFFFFFFu, any) && (threadIdx.x & 31) == 0) atomicOr(changed, 1u);
}

// Boundary site number e of sub-lattice (sx, sy): its 4S - 4 boundary sites
// enumerated as right column, left column, top row, bottom row (corners twice).
__device__ __forceinline__ bool boundary_site(uint64_t e, uint64_t S, uint64_t& lx, uint64_t& ly) {
  if (e < S) { lx = S - 1; ly = e; return true; }
  e -= S;
  if (e < S) { lx = 0; ly = e; return true; }
  e -= S;
  if (e < S) { lx = e; ly = 0; return true; }
  e -= S;
  if (e < S) { lx = e; ly = S - 1; return true; }
  return false;
}

template <typename LabelT>
__global__ void k_2s_total_init(const LabelT* label, LabelT* total, uint64_t L, uint64_t S, uint64_t G) {
  const uint64_t items = G * G * 4 * S;
  for (uint64_t it = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; it < items;
       it += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t sub = it / (4 * S), e = it % (4 * S);
    uint64_t lx, ly;
    boundary_site(e, S, lx, ly);
    const uint64_t i = ((sub / G) * S + ly) * L + (sub % G) * S + lx;
    const LabelT r = label[i];
    total[r] = r;
  }
}

// Inter-sub-lattice scanning over the bonds that cross a boundary: the right
// bonds of each sub-lattice's last column and the down bonds of its last row.
template <typename LabelT>
__global__ void k_2s_scan_boundary(const uint8_t* __restrict__ bonds, const LabelT* label, LabelT* total,
                                   uint64_t L, uint64_t bp, uint64_t S, uint64_t G, uint32_t* changed) {
  const uint64_t items = G * G * 2 * S;
  bool any = false;
  for (uint64_t it = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; it < items;
       it += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t sub = it / (2 * S), e = it % (2 * S);
    const uint64_t X0 = (sub % G) * S, Y0 = (sub / G) * S;
    uint64_t a, c;
    bool on;
    if (e < S) {  // right bond of (X0+S-1, Y0+e)
      const uint64_t y = Y0 + e, x = X0 + S - 1;
      on = bond_bits(bonds, bp, y, x) & 1u;
      a = y * L + x;
      c = y * L + ((x + 1 == L) ? 0 : x + 1);
    } else {  // down bond of (X0+e-S, Y0+S-1)
      const uint64_t y = Y0 + S - 1, x = X0 + e - S;
      on = (bond_bits(bonds, bp, y, x) >> 1) & 1u;
      a = y * L + x;
      c = ((y + 1 == L) ? 0 : y + 1) * L + x;
    }
    if (on) {
      const LabelT ra = label[a], rc = label[c];
      const LabelT ta = total[ra], tc = total[rc];
      if (tc < ta) {
        atomic_min_l(total + ta, tc);
        any = true;
      } else if (ta < tc) {
        atomic_min_l(total + tc, ta);
        any = true;
      }
    }
  }
  if (__any_sync(0xFFFFFFFFu, any) && (threadIdx.x & 31) == 0) atomicOr(changed, 1u);
}

// Inter-sub-lattice analysis on the boundary entries of label_total.
template <typename LabelT>
__global__ void k_2s_analysis_boundary(const LabelT* label, LabelT* total, uint64_t L, uint64_t S, uint64_t G,
                                       uint32_t* err) {
  const uint64_t items = G * G * 4 * S;
  for (uint64_t it = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; it < items;
       it += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t sub = it / (4 * S), e = it % (4 * S);
    uint64_t lx, ly;
    boundary_site(e, S, lx, ly);
    const LabelT r = label[((sub / G) * S + ly) * L + (sub % G) * S + lx];
    LabelT t = total[r];
    uint32_t k = 0;
    for (; k < kChainCap; ++k) {
      const LabelT n = total[t];
      if (n == t) break;
      t = n;
    }
    if (k == kChainCap) atomicOr(err, 1u);
    total[r] = t;
  }
}

// Every site adopts label_total of its stage-1 label (entries never set for
// clusters that stay inside one sub-lattice hold the all-ones sentinel).
template <typename LabelT>
__global__ void k_2s_final(LabelT* label, const LabelT* total, uint64_t N) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const LabelT r = label[i];
    const LabelT t = total[r];
    label[i] = (t == (LabelT)~(LabelT)0) ? r : t;
  }
}

template <typename LabelT>
int run_2s(uint64_t L, uint64_t S, const uint8_t* bonds, LabelT* roots, LabelT* total, uint32_t* it1,
           uint32_t* it2, cudaStream_t st, uint32_t* flags, cudaEvent_t* ev) {
  const uint64_t N = L * L, bp = (L + 3) / 4, G = L / S;
  uint64_t blocks = (N + kThreads - 1) / kThreads;
  if (blocks > 152ull * 64) blocks = 152ull * 64;
  const uint64_t gx = (L + kThreads - 1) / kThreads;
  const dim3 sgrid((unsigned)(gx < 64 ? gx : 64), (unsigned)(L < 65535 ? L : 65535));
  uint64_t bb = (G * G * 4 * S + kThreads - 1) / kThreads;
  if (bb > 152ull * 64) bb = 152ull * 64;
  cudaEventRecord(ev[0], st);
  k_le_init<LabelT><<<(unsigned)blocks, kThreads, 0, st>>>(roots, N);
  // stage 1: label equivalence inside every sub-lattice
  uint32_t n = 0, changed = 1;
  while (changed) {
    if (n >= (1u << 20)) return SW_ERR_TIMEOUT;
    cudaError_t e = cudaMemsetAsync(flags, 0, 4, st);
    if (!e) {
      k_2s_scan_local<LabelT><<<sgrid, kThreads, 0, st>>>(bonds, roots, L, bp, S, flags);
      k_le_analysis<LabelT><<<(unsigned)blocks, kThreads, 0, st>>>(roots, N, flags + 1);
      e = cudaGetLastError();
    }
    if (!e) e = cudaMemcpyAsync(&changed, flags, 4, cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return SW_ERR_CUDA;
    }
    ++n;
  }
  *it1 = n;
  // stage 2: boundary layers only
  cudaEventRecord(ev[1], st);
  cudaError_t e = cudaMemsetAsync(total, 0xFF, N * sizeof(LabelT), st);
  if (!e) {
    k_2s_total_init<LabelT><<<(unsigned)bb, kThreads, 0, st>>>(roots, total, L, S, G);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SW_ERR_CUDA;
  }
  n = 0;
  changed = 1;
  while (changed) {
    if (n >= (1u << 20)) return SW_ERR_TIMEOUT;
    e = cudaMemsetAsync(flags, 0, 4, st);
    if (!e) {
      k_2s_scan_boundary<LabelT><<<(unsigned)bb, kThreads, 0, st>>>(bonds, roots, total, L, bp, S, G, flags);
      k_2s_analysis_boundary<LabelT><<<(unsigned)bb, kThreads, 0, st>>>(roots, total, L, S, G, flags + 1);
      e = cudaGetLastError();
    }
    if (!e) e = cudaMemcpyAsync(&changed, flags, 4, cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return SW_ERR_CUDA;
    }
    ++n;
  }
  *it2 = n;
  cudaEventRecord(ev[2], st);
  k_2s_final<LabelT><<<(unsigned)blocks, kThreads, 0, st>>>(roots, total, N);
  cudaEventRecord(ev[3], st);
  uint32_t err = 0;
  e = cudaGetLastError();
  if (!e) e = cudaMemcpyAsync(&err, flags + 1, 4, cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SW_ERR_CUDA;
  }
  return err ? SW_ERR_TIMEOUT : SW_OK;
}

}  // namespace le
}  // namespace swgb

extern "C" int sw_label_bonds_le(uint64_t L, const uint8_t* bonds, void* roots, uint32_t label_bits,
                                 uint32_t max_iter, uint32_t* iterations, void* stream) {
  using namespace swgb;
  if (L < 2 || L > (1ull << 20) || !bonds || !roots) return SW_ERR_INVAL;
  if (label_bits != 32 && label_bits != 64) return SW_ERR_INVAL;
  if (label_bits == 32 && L * L > (1ull << 32)) return SW_ERR_INVAL;
  if (max_iter == 0) max_iter = 1u << 20;
  const DeviceAllocator al = current_allocator();
  void* flags = al.allocate(256);
  if (!flags) return SW_ERR_NOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(flags, 0, 256, st);
  int rc = e == cudaSuccess ? SW_OK : SW_ERR_CUDA;
  if (!rc)
    rc = label_bits == 64
             ? le::run_le<uint64_t>(L, bonds, (uint64_t*)roots, max_iter, iterations, st, (uint32_t*)flags)
             : le::run_le<uint32_t>(L, bonds, (uint32_t*)roots, max_iter, iterations, st, (uint32_t*)flags);
  cudaStreamSynchronize(st);
  al.release(flags, 256);
  return rc;
}

extern "C" int sw_label_bonds_2stage(uint64_t L, uint64_t sub, const uint8_t* bonds, void* roots,
                                     uint32_t label_bits, uint32_t* iterations, float* stage_ms,
                                     void* stream) {
  using namespace swgb;
  if (L < 2 || L > (1ull << 20) || !bonds || !roots || sub < 2 || sub > L || L % sub) return SW_ERR_INVAL;
  if (label_bits != 32 && label_bits != 64) return SW_ERR_INVAL;
  if (label_bits == 32 && L * L > (1ull << 32)) return SW_ERR_INVAL;
  const DeviceAllocator al = current_allocator();
  const uint64_t N = L * L;
  const size_t tb = (size_t)N * (label_bits / 8);
  void* flags = al.allocate(256);
  void* total = al.allocate(tb);
  if (!flags || !total) {
    if (flags) al.release(flags, 256);
    if (total) al.release(total, tb);
    return SW_ERR_NOMEM;
  }
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t it1 = 0, it2 = 0;
  cudaEvent_t ev[4] = {};
  int rc = SW_OK;
  for (int k = 0; k < 4 && !rc; ++k)
    if (cudaEventCreate(&ev[k]) != cudaSuccess) rc = SW_ERR_CUDA;
  if (!rc && cudaMemsetAsync(flags, 0, 256, st) != cudaSuccess) rc = SW_ERR_CUDA;
  if (!rc)
    rc = label_bits == 64 ? le::run_2s<uint64_t>(L, sub, bonds, (uint64_t*)roots, (uint64_t*)total, &it1, &it2,
                                                 st, (uint32_t*)flags, ev)
                          : le::run_2s<uint32_t>(L, sub, bonds, (uint32_t*)roots, (uint32_t*)total, &it1, &it2,
                                                 st, (uint32_t*)flags, ev);
  cudaStreamSynchronize(st);
  if (!rc && stage_ms) {
    for (int k = 0; k < 3; ++k)
      if (cudaEventElapsedTime(&stage_ms[k], ev[k], ev[k + 1]) != cudaSuccess) rc = SW_ERR_CUDA;
  }
  for (int k = 0; k < 4; ++k)
    if (ev[k]) cudaEventDestroy(ev[k]);
  cudaGetLastError();
  al.release(flags, 256);
  al.release(total, tb);
  if (iterations) {
    iterations[0] = it1;
    iterations[1] = it2;
  }
  return rc;
}
