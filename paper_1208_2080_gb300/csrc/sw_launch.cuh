// sw_launch.cuh -- host-side launchers of the sweep kernels for any tile
// source (one lattice or a batch of replicas).  Included by the library's
// translation units; not part of the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sw_kernels.cuh"

namespace swgb {

// Sets the kernel's shared-memory attributes and returns how many tile CTAs
// fit on the GPU at once (done once per instantiation; call it before any
// stream capture).
template <int TH, typename LabelT, bool kGiven, bool kRoots, typename Src, bool kXY = false>
cudaError_t configure_label(int* resident_out) {
  auto kern = k_label_tile<TH, LabelT, kGiven, kRoots, Src, kXY>;
  const int smem = kXY ? LabelSmem<TH>::kXYBytes : LabelSmem<TH>::kBytes;
  static int resident = 0;
  if (!resident) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TileCta<TH>::kThreads, smem);
    if (sms <= 0) sms = 152;
    if (per_sm <= 0) per_sm = 1;
    resident = sms * per_sm;
  }
  if (resident_out) *resident_out = resident;
  return cudaSuccess;
}

template <int TH, typename LabelT, bool kGiven, bool kRoots, typename Src, bool kXY = false>
cudaError_t launch_label_src(const Src& src, uint32_t ntiles, cudaStream_t st) {
  auto kern = k_label_tile<TH, LabelT, kGiven, kRoots, Src, kXY>;
  const int smem = kXY ? LabelSmem<TH>::kXYBytes : LabelSmem<TH>::kBytes;
  int resident = 0;
  cudaError_t e = configure_label<TH, LabelT, kGiven, kRoots, Src, kXY>(&resident);
  if (e != cudaSuccess) return e;
  const uint32_t grid = ntiles < (uint32_t)resident ? ntiles : (uint32_t)resident;
  kern<<<grid, TileCta<TH>::kThreads, smem, st>>>(src);
  return cudaGetLastError();
}

template <int TH, typename LabelT, typename Src>
cudaError_t launch_merge_src(const Src& src, uint32_t ntiles, cudaStream_t st) {
  const uint64_t items = (uint64_t)ntiles * (TH + kTW);
  const uint64_t blocks = (items + kMergeThreads - 1) / kMergeThreads;
  k_merge<TH, LabelT, Src><<<(unsigned)blocks, kMergeThreads, 0, st>>>(src);
  return cudaGetLastError();
}

template <int TH, typename LabelT, typename Src>
cudaError_t launch_resolve_src(const Src& src, uint32_t ntiles, cudaStream_t st) {
  const uint64_t items = (uint64_t)ntiles * 32;  // a warp per tile
  const uint64_t blocks = (items + kMergeThreads - 1) / kMergeThreads;
  k_resolve<TH, LabelT, Src><<<(unsigned)blocks, kMergeThreads, 0, st>>>(src);
  return cudaGetLastError();
}

template <int TH, typename LabelT, bool kRoots, typename Src, bool kXY = false>
cudaError_t launch_recolor_src(const Src& src, uint32_t ntiles, LabelT* roots, cudaStream_t st) {
  k_recolor<TH, LabelT, kRoots, Src, kXY><<<ntiles, kThreads, 0, st>>>(src, roots);
  return cudaGetLastError();
}

// One full sweep (four launches) of every lattice the source names; `ev`
// (four events or null) is recorded before, between and after the phases.
// kXY: the embedded-cluster sweep of the XY model (Potts kernels with the
// XY bond rule and reflections).
template <int TH, typename LabelT, typename Src, bool kXY = false>
cudaError_t sweep_src(const Src& src, uint32_t ntiles, cudaStream_t st, cudaEvent_t* ev) {
  cudaError_t e;
  if (ev && (e = cudaEventRecord(ev[0], st))) return e;
  if ((e = launch_label_src<TH, LabelT, false, false, Src, kXY>(src, ntiles, st))) return e;
  if (ev && (e = cudaEventRecord(ev[1], st))) return e;
  if ((e = launch_merge_src<TH, LabelT>(src, ntiles, st))) return e;
  if ((e = launch_resolve_src<TH, LabelT>(src, ntiles, st))) return e;
  if (ev && (e = cudaEventRecord(ev[2], st))) return e;
  if ((e = launch_recolor_src<TH, LabelT, false, Src, kXY>(src, ntiles, (LabelT*)nullptr, st))) return e;
  if (ev) return cudaEventRecord(ev[3], st);
  return cudaSuccess;
}

// Dispatch on the tile height.
template <typename LabelT, typename Src, bool kXY = false>
cudaError_t sweep_th(uint32_t th, const Src& src, uint32_t ntiles, cudaStream_t st, cudaEvent_t* ev) {
  switch (th) {
    case 16: return sweep_src<16, LabelT, Src, kXY>(src, ntiles, st, ev);
    case 32: return sweep_src<32, LabelT, Src, kXY>(src, ntiles, st, ev);
    case 64: return sweep_src<64, LabelT, Src, kXY>(src, ntiles, st, ev);
    default: return cudaErrorInvalidValue;
  }
}

template <typename LabelT, typename Src>
cudaError_t configure_th(uint32_t th) {
  switch (th) {
    case 16: return configure_label<16, LabelT, false, false, Src>(nullptr);
    case 32: return configure_label<32, LabelT, false, false, Src>(nullptr);
    case 64: return configure_label<64, LabelT, false, false, Src>(nullptr);
    default: return cudaErrorInvalidValue;
  }
}

// Host helpers shared by the translation units (defined in sw_api.cu).
Lattice make_lattice(uint64_t L, uint32_t th);
size_t edge_u16(uint32_t th);
size_t bit_words(uint32_t th);
size_t open_cap(uint32_t th);
cudaError_t launch_measure(const uint8_t* spin, const Lattice& lat, uint32_t q, const Bufs& b,
                           cudaStream_t st);
cudaError_t launch_init(uint8_t* spin, uint64_t N, uint32_t q, uint64_t seed, uint32_t mode,
                        cudaStream_t st);

}  // namespace swgb
