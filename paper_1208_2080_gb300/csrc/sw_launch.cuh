// sw_launch.cuh -- host-side launchers of the sweep kernels for any tile
// source (one lattice or a batch of replicas).  Included by the library's
// translation units; not part of the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "sw_kernels.cuh"
#include "sw_label.cuh"

namespace swgb {

constexpr int kMaxDevices = 64;

// Sets a labelling kernel's shared-memory attributes on the current device
// and returns how many of its CTAs fit on that device at once.  Function
// attributes belong to a device, so this is done once per device (and per
// shared-memory size) and the count is kept per device; call it before any
// stream capture.
template <typename Kern>
cudaError_t configure_on_device(Kern kern, int threads, int smem, int smem_max, std::atomic<int>* resident,
                                int* resident_out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  int r = resident[dev].load(std::memory_order_acquire);
  if (!r) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    cudaGetLastError();
    if (sms <= 0) sms = 152;
    if (per_sm <= 0) per_sm = 1;
    r = sms * per_sm;
    resident[dev].store(r, std::memory_order_release);
  }
  if (resident_out) *resident_out = r;
  return cudaSuccess;
}

// Shared memory of the labeller for a source: the per-state histogram
// (q > 4, or any replica batch) and the XY form's class table need the
// larger layout.
template <int TH, bool kGiven, typename Src, bool kXY = false>
int rows_smem(const Src& src) {
  if constexpr (kXY) {
    (void)src;
    return RowSmem<TH>::kBytes;
  } else if constexpr (kGiven) {
    (void)src;
    return RowSmem<TH>::kBytesSmallQ;
  } else if constexpr (Src::kMulti) {
    (void)src;
    return RowSmem<TH>::kBytes;
  } else {
    return src.b.q > 4 ? RowSmem<TH>::kBytes : RowSmem<TH>::kBytesSmallQ;
  }
}

// The labeller (k_label_rows): attributes and resident CTAs on this device.
template <int TH, typename LabelT, bool kGiven, bool kRoots, typename Src, bool kFuse, bool kXY>
cudaError_t configure_rows(int smem, int* resident_out) {
  static std::atomic<int> resident[2][kMaxDevices];
  const int big = smem > RowSmem<TH>::kBytesSmallQ ? 1 : 0;
  return configure_on_device(k_label_rows<TH, LabelT, kGiven, kRoots, Src, kFuse, kXY>, RowCta<TH>::kThreads,
                             smem, RowSmem<TH>::kBytes, resident[big], resident_out);
}

template <int TH, typename LabelT, bool kGiven, bool kRoots, typename Src, bool kXY = false, bool kFuse = false>
cudaError_t configure_label(const Src& src, int* resident_out) {
  return configure_rows<TH, LabelT, kGiven, kRoots, Src, kFuse, kXY>(rows_smem<TH, kGiven, Src, kXY>(src),
                                                                      resident_out);
}

// One labelling launch: a persistent grid of as many tile CTAs as fit.
template <int TH, typename LabelT, bool kGiven, bool kRoots, typename Src, bool kXY = false, bool kFuse = false>
cudaError_t launch_label_src(const Src& src, uint32_t ntiles, cudaStream_t st) {
  int resident = 0;
  cudaError_t e = configure_label<TH, LabelT, kGiven, kRoots, Src, kXY, kFuse>(src, &resident);
  if (e != cudaSuccess) return e;
  const uint32_t grid = ntiles < (uint32_t)resident ? ntiles : (uint32_t)resident;
  if (grid == 0) return cudaSuccess;
  k_label_rows<TH, LabelT, kGiven, kRoots, Src, kFuse, kXY>
      <<<grid, RowCta<TH>::kThreads, rows_smem<TH, kGiven, Src, kXY>(src), st>>>(src);
  return cudaGetLastError();
}

template <int TH, typename LabelT, typename Src>
cudaError_t launch_merge_src(const Src& src, uint32_t ntiles, cudaStream_t st) {
  const uint64_t items = (uint64_t)ntiles * (TH + kTW);
  const uint64_t blocks = (items + kMergeThreads - 1) / kMergeThreads;
  k_merge<TH, LabelT, Src><<<(unsigned)blocks, kMergeThreads, 0, st>>>(src);
  return cudaGetLastError();
}

// The sweep's filing after a labelling that did the boundary unions itself.
template <typename Src>
cudaError_t launch_file_src(const Src& src, uint32_t nreps, cudaStream_t st) {
  k_file<Src><<<(nreps + 127) / 128, 128, 0, st>>>(src);
  return cudaGetLastError();
}

template <int TH, typename LabelT, typename Src>
cudaError_t launch_resolve_src(const Src& src, uint32_t ntiles, cudaStream_t st) {
  if (ntiles == 0) return cudaSuccess;
  k_resolve<TH, LabelT, Src><<<ntiles, kResolveThreads, 0, st>>>(src);
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
// XY bond rule and reflections).  fused: the labeller does the boundary
// unions (its lattices' Bufs::fuse set, edge counters allocated), and a
// one-block filing kernel replaces k_merge.
template <int TH, typename LabelT, typename Src, bool kXY = false>
cudaError_t sweep_src(const Src& src, uint32_t ntiles, uint32_t nreps, bool fused, cudaStream_t st,
                      cudaEvent_t* ev) {
  cudaError_t e;
  if (ev && (e = cudaEventRecord(ev[0], st))) return e;
  if (fused && !kXY) e = launch_label_src<TH, LabelT, false, false, Src, false, true>(src, ntiles, st);
  else e = launch_label_src<TH, LabelT, false, false, Src, kXY>(src, ntiles, st);
  if (e) return e;
  if (ev && (e = cudaEventRecord(ev[1], st))) return e;
  if (fused && !kXY) {
    if ((e = launch_file_src(src, nreps, st))) return e;
  } else {
    if ((e = launch_merge_src<TH, LabelT>(src, ntiles, st))) return e;
  }
  if ((e = launch_resolve_src<TH, LabelT>(src, ntiles, st))) return e;
  if (ev && (e = cudaEventRecord(ev[2], st))) return e;
  if ((e = launch_recolor_src<TH, LabelT, false, Src, kXY>(src, ntiles, (LabelT*)nullptr, st))) return e;
  if (ev) return cudaEventRecord(ev[3], st);
  return cudaSuccess;
}

// Dispatch on the tile height.
template <typename LabelT, typename Src, bool kXY = false>
cudaError_t sweep_th(uint32_t th, const Src& src, uint32_t ntiles, cudaStream_t st, cudaEvent_t* ev,
                     uint32_t nreps = 1, bool fused = false) {
  switch (th) {
    case 16: return sweep_src<16, LabelT, Src, kXY>(src, ntiles, nreps, fused, st, ev);
    case 32: return sweep_src<32, LabelT, Src, kXY>(src, ntiles, nreps, fused, st, ev);
    case 64: return sweep_src<64, LabelT, Src, kXY>(src, ntiles, nreps, fused, st, ev);
    case 128: return sweep_src<128, LabelT, Src, kXY>(src, ntiles, nreps, fused, st, ev);
    default: return cudaErrorInvalidValue;
  }
}

template <typename LabelT, typename Src>
cudaError_t configure_th(uint32_t th, const Src& src, bool fused = false) {
  switch (th) {
#define SWGB_CONF(THV)                                                                           \
  case THV:                                                                                      \
    return fused ? configure_label<THV, LabelT, false, false, Src, false, true>(src, nullptr)    \
                 : configure_label<THV, LabelT, false, false, Src>(src, nullptr);
    SWGB_CONF(16)
    SWGB_CONF(32)
    SWGB_CONF(64)
    SWGB_CONF(128)
#undef SWGB_CONF
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
