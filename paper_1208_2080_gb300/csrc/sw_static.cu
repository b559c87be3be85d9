// sw_static.cu -- labelling of a given bond lattice without any device
// allocation, for callers that cannot allocate device memory themselves: a
// host program whose GPU memory is owned by a framework with its own pool
// (and no hook to lend it), an embedding that forbids cudaMalloc/cudaFree
// after start-up because they synchronise the device, or code that runs
// where an allocation could fail at a bad moment.  The entry point computes
// exactly what sw_label_bonds computes (uint32 labels), with all working
// memory in one file-scope __device__ array of fixed size.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/sw.h"
#include "sw_internal.h"
#include "sw_launch.cuh"

using namespace swgb;

namespace {

// Working memory of every call, on every device that loads the library,
// held until the process exits.  Sized for L <= SW_LABEL_STATIC_MAX_L with
// any tile height: per-site codes (2 B/site), the global union-find (8 B
// per possible open root of a tile), the per-tile edge records and control
// words (under 4 MiB at L = 1024 with the smallest tiles).
constexpr size_t kScratchBytes = 8u << 20;
static __device__ __align__(256) unsigned char g_label_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned char* g_scratch_dev[kMaxDevices];  // device address of g_label_scratch, per device

// In host code g_label_scratch names a host-side stand-in, not device
// memory; the device address is looked up once per device, with that device
// current, and reused.
int scratch_on_current_device(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return SW_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return SW_ERR_INVAL;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_label_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return SW_ERR_CUDA;
    }
    g_scratch_dev[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_dev[dev];
  return SW_OK;
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// A tile source of its own type, so that the kernels this file launches are
// instantiated here only (their launch set-up is not shared with the
// instantiations of the other translation units).
struct StaticSrc : SingleSrc {};

template <int TH>
cudaError_t label_static(const Bufs& b, const Lattice& lat, uint32_t* roots, cudaStream_t st) {
  StaticSrc src;
  src.b = b;
  src.lat = lat;
  cudaError_t e = launch_label_src<TH, uint32_t, true, true>(src, lat.ntiles, st);
  if (e != cudaSuccess) return e;
  e = launch_merge_src<TH, uint32_t>(src, lat.ntiles, st);
  if (e != cudaSuccess) return e;
  return launch_recolor_src<TH, uint32_t, true>(src, lat.ntiles, roots, st);
}

}  // namespace

extern "C" int sw_label_bonds_static(uint64_t L, const uint8_t* bonds, uint32_t* roots,
                                     uint32_t tile_h, void* stream) {
  if (L > SW_LABEL_STATIC_MAX_L) return SW_ERR_INVAL;  // beyond the fixed working memory
  if (L < 2 || !bonds || !roots) return SW_ERR_INVAL;
  const uint32_t th = pick_tile_h(L, tile_h);
  if (th != 16 && th != 32 && th != 64) return SW_ERR_INVAL;
  const Lattice lat = make_lattice(L, th);
  const uint64_t N = L * L, nt = lat.ntiles;

  // layout of the working memory
  const size_t o_code = 0;
  const size_t o_G = o_code + up256(2 * N + 16);
  const size_t o_edge = o_G + up256(nt * open_cap(th) * 8);
  const size_t o_ebits = o_edge + up256(nt * edge_u16(th) * 2);
  const size_t o_ocnt = o_ebits + up256(nt * bit_words(th) * 4);
  const size_t o_ctl = o_ocnt + up256(nt * 4);
  const size_t o_err = o_ctl + 256;
  if (o_err + 256 > kScratchBytes) return SW_ERR_INVAL;

  unsigned char* base = nullptr;
  int rc = scratch_on_current_device(&base);
  if (rc) return rc;

  Bufs b{};
  b.bonds = const_cast<uint8_t*>(bonds);
  b.code = reinterpret_cast<uint16_t*>(base + o_code);
  b.G = reinterpret_cast<uint64_t*>(base + o_G);
  b.edge = reinterpret_cast<uint16_t*>(base + o_edge);
  b.ebits = reinterpret_cast<uint32_t*>(base + o_ebits);
  b.ocnt = reinterpret_cast<uint32_t*>(base + o_ocnt);
  b.ctl = reinterpret_cast<unsigned long long*>(base + o_ctl);
  b.err = reinterpret_cast<uint32_t*>(base + o_err);
  b.q = 2;
  b.measure = 0;

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents: clear what must start at zero
  cudaError_t e = cudaMemsetAsync(b.ctl, 0, 256, st);
  if (!e) e = cudaMemsetAsync(b.err, 0, 256, st);
  if (!e) {
    switch (th) {
      case 16: e = label_static<16>(b, lat, roots, st); break;
      case 32: e = label_static<32>(b, lat, roots, st); break;
      default: e = label_static<64>(b, lat, roots, st); break;
    }
  }
  uint32_t err = 0;
  if (!e) e = cudaMemcpyAsync(&err, b.err, sizeof(err), cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SW_ERR_CUDA;
  }
  if (err & (kErrFind | kErrUnion | kErrLocal)) return SW_ERR_TIMEOUT;
  if (err) return SW_ERR_DEVICE;
  return SW_OK;
}
