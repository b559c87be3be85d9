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
