// sw_api.cu -- C ABI of the single-lattice Swendsen-Wang library (include/sw.h).
//
// Host side only: argument checks, device memory layout, launches of the
// kernels in sw_kernels.cuh on the handle's stream, observable bookkeeping.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/sw.h"
#include "sw_internal.h"
#include "sw_kernels.cuh"
#include "sw_launch.cuh"

using namespace swgb;

// ------------------------------------------------------------------ allocator
namespace swgb {
static sw_alloc_fn g_alloc = nullptr;
static sw_free_fn g_free = nullptr;
static void* g_alloc_ctx = nullptr;

DeviceAllocator current_allocator() { return DeviceAllocator{g_alloc, g_free, g_alloc_ctx}; }

void* DeviceAllocator::allocate(size_t bytes) const {
  if (bytes == 0) bytes = 256;
  if (alloc) return alloc(bytes, ctx);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void DeviceAllocator::release(void* p, size_t bytes) const {
  if (!p) return;
  if (bytes == 0) bytes = 256;
  if (free_fn)
    free_fn(p, bytes, ctx);
  else
    cudaFree(p);
}

uint32_t bond_threshold(double T) {
  // p = 1 - exp(-J/T), J = 1: the SW bond probability for H = -J sum delta
  const double p = -expm1(-1.0 / T);
  const double t = floor(p * 4294967296.0);
  if (!(t > 0.0)) return 0u;
  if (t >= 4294967295.0) return 0xFFFFFFFFu;
  return (uint32_t)t;
}

uint32_t pick_tile_h(uint64_t L, uint32_t requested) {
  if (requested) return requested;
  if (L <= 32) return 16;
  if (L <= 256) return 32;
  if (L <= 1024) return 64;
  return 128;
}

Lattice make_lattice(uint64_t L, uint32_t th) {
  Lattice lat;
  lat.L = L;
  lat.ntx = (uint32_t)((L + kTW - 1) / kTW);
  lat.nty = (uint32_t)((L + th - 1) / th);
  lat.bp = (L + 3) / 4;
  lat.vec4 = (L % 4 == 0) ? 1u : 0u;
  lat.ntiles = lat.ntx * lat.nty;
  lat.ntx_m = lat.ntx == 1 ? 0xFFFFFFFFu : (uint32_t)((1ull << 32) / lat.ntx);
  lat.xb = 0;
  while ((1ull << lat.xb) < L) ++lat.xb;
  // node words carry the node index when key and node fit in 64 bits
  const uint64_t nodes = (uint64_t)lat.ntiles * open_cap(th);
  lat.db = 1;
  while ((1ull << lat.db) < nodes) ++lat.db;
  if (2 * lat.xb + lat.db > 64) lat.db = 0;
  return lat;
}

size_t edge_u16(uint32_t th) { return 2 * (size_t)th + 2 * kTW; }
size_t bit_words(uint32_t th) { return (th + 31) / 32 + kTW / 32; }
size_t open_cap(uint32_t th) { return 2 * (size_t)th + 2 * kTW; }

template <int TH, typename LabelT, bool kGiven, bool kRoots>
static cudaError_t launch_label_t(const Bufs& b, const Lattice& lat, cudaStream_t st) {
  return launch_label_src<TH, LabelT, kGiven, kRoots>(SingleSrc{b, lat}, lat.ntiles, st);
}

template <int TH, typename LabelT>
static cudaError_t launch_merge_t(const Bufs& b, const Lattice& lat, cudaStream_t st) {
  return launch_merge_src<TH, LabelT>(SingleSrc{b, lat}, lat.ntiles, st);
}

template <int TH, typename LabelT, bool kRoots>
static cudaError_t launch_recolor_t(const Bufs& b, const Lattice& lat, LabelT* roots, cudaStream_t st) {
  return launch_recolor_src<TH, LabelT, kRoots>(SingleSrc{b, lat}, lat.ntiles, roots, st);
}

cudaError_t launch_sweep_events(uint32_t label_bits, uint32_t th, const Bufs& b, const Lattice& lat,
                                cudaStream_t st, cudaEvent_t* ev) {
  const SingleSrc src{b, lat};
  return label_bits == 64 ? sweep_th<uint64_t>(th, src, lat.ntiles, st, ev, 1, b.fuse != 0)
                          : sweep_th<uint32_t>(th, src, lat.ntiles, st, ev, 1, b.fuse != 0);
}

cudaError_t launch_sweep(uint32_t label_bits, uint32_t th, const Bufs& b, const Lattice& lat,
                         cudaStream_t st) {
  return launch_sweep_events(label_bits, th, b, lat, st, nullptr);
}

template <typename LabelT>
static cudaError_t label_given_t(uint32_t th, const Bufs& b, const Lattice& lat, LabelT* roots,
                                 cudaStream_t st) {
  cudaError_t e;
  switch (th) {
#define SWGB_CASE(THV)                                                      \
  case THV:                                                                 \
    if ((e = launch_label_t<THV, LabelT, true, true>(b, lat, st))) return e; \
    if ((e = launch_merge_t<THV, LabelT>(b, lat, st))) return e;            \
    return launch_recolor_t<THV, LabelT, true>(b, lat, roots, st);
    SWGB_CASE(16)
    SWGB_CASE(32)
    SWGB_CASE(64)
    SWGB_CASE(128)
#undef SWGB_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_measure(const uint8_t* spin, const Lattice& lat, uint32_t q,
                           const Bufs& b, cudaStream_t st) {
  if ((lat.L & 15u) == 0) {
    // column strips of 256 16-site groups x row strips of kMeasRows rows
    const dim3 grid((unsigned)((lat.L / 16 + 255) / 256), (unsigned)((lat.L + kMeasRows - 1) / kMeasRows));
    if (q == 2) k_measure16<1><<<grid, 256, 0, st>>>(spin, lat.L, q, b.acc);
    else if (q <= 4) k_measure16<2><<<grid, 256, 0, st>>>(spin, lat.L, q, b.acc);
    else if (q <= 8) k_measure16<3><<<grid, 256, 0, st>>>(spin, lat.L, q, b.acc);
    else k_measure16<0><<<grid, 256, 0, st>>>(spin, lat.L, q, b.acc);
  } else {
    uint64_t blocks = lat.L;  // one block per row, at most 16 per SM
    if (blocks > 152ull * 16) blocks = 152ull * 16;
    k_measure<<<(unsigned)blocks, 256, 0, st>>>(spin, lat, q, b.acc);
  }
  cudaError_t e = cudaGetLastError();
  if (e) return e;
  k_commit<<<1, 32, 0, st>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_init(uint8_t* spin, uint64_t N, uint32_t q, uint64_t seed, uint32_t mode,
                        cudaStream_t st) {
  if (mode == SW_INIT_ZERO) return cudaMemsetAsync(spin, 0, N, st);
  const uint64_t nq = (N + 3) / 4;
  uint64_t blocks = (nq + 255) / 256;
  if (blocks > 152ull * 32) blocks = 152ull * 32;
  if (blocks == 0) blocks = 1;
  k_init_spins<<<(unsigned)blocks, 256, 0, st>>>(spin, N, q, seed);
  return cudaGetLastError();
}

}  // namespace swgb

// ------------------------------------------------------------------ handle
constexpr uint32_t kUploadBands = 16;  // sw_sweep_host: bands of tile rows

struct sw_sim {
  sw_params p;
  uint64_t L = 0, N = 0;
  uint32_t q = 0, thr = 0, label_bits = 32, th = 64, ring = 1024;
  Lattice lat{};
  cudaStream_t stream = nullptr;
  DeviceAllocator alloc{};
  std::vector<std::pair<void*, size_t>> blocks;
  uint64_t dev_bytes = 0;
  Bufs b{};
  uint64_t sweep = 0;          // host mirror of ctl[0]
  uint64_t measured_from = 0;  // oldest configuration whose observables are valid
  bool pending = true;         // current configuration not measured yet
  bool measure_on = true;
  int last_err = SW_OK;
  int device = 0;
  bool spins_invalid = false;  // last sw_set_spins was rejected
  // per-phase event timing (sw_profile)
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;   // free events
  std::vector<cudaEvent_t> ev_used;   // 4 per profiled sweep, in order
  double prof_ms[3] = {0, 0, 0};
  // sw_sweep_host: upload stream and one event per band (created on first use)
  cudaStream_t up = nullptr;
  cudaEvent_t up_ev[kUploadBands + 1] = {};
  uint64_t prof_launches[3] = {0, 0, 0};
};

namespace {

int fail(sw_sim* s, int code) {
  if (s && (code == SW_ERR_CUDA || code == SW_ERR_DEVICE || code == SW_ERR_TIMEOUT)) s->last_err = code;
  return code;
}

int cuda_fail(sw_sim* s, cudaError_t e) {
  (void)e;
  cudaGetLastError();
  return fail(s, SW_ERR_CUDA);
}

void* take(sw_sim* s, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  void* p = s->alloc.allocate(bytes);
  if (p) {
    s->blocks.emplace_back(p, bytes);
    s->dev_bytes += bytes;
  }
  return p;
}

cudaEvent_t get_event(sw_sim* s) {
  if (!s->ev_pool.empty()) {
    cudaEvent_t e = s->ev_pool.back();
    s->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Folds recorded event quads into the per-phase totals (after a sync).
int drain_events(sw_sim* s) {
  for (size_t k = 0; k + 3 < s->ev_used.size(); k += 4) {
    for (int ph = 0; ph < 3; ++ph) {
      float ms = 0.f;
      cudaError_t e = cudaEventElapsedTime(&ms, s->ev_used[k + ph], s->ev_used[k + ph + 1]);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return SW_ERR_CUDA;
      }
      s->prof_ms[ph] += ms;
      s->prof_launches[ph] += 1;
    }
  }
  for (cudaEvent_t e : s->ev_used) s->ev_pool.push_back(e);
  s->ev_used.clear();
  return SW_OK;
}

void release_all(sw_sim* s) {
  for (cudaEvent_t& e : s->up_ev)
    if (e) cudaEventDestroy(e), e = nullptr;
  if (s->up) cudaStreamDestroy(s->up);
  s->up = nullptr;
  for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
  for (cudaEvent_t e : s->ev_used) cudaEventDestroy(e);
  s->ev_pool.clear();
  s->ev_used.clear();
  for (auto& kv : s->blocks) s->alloc.release(kv.first, kv.second);
  s->blocks.clear();
  s->dev_bytes = 0;
}

bool sticky(const sw_sim* s) { return s->last_err != SW_OK; }

// Reads the device error word; maps it onto an error code.
int check_device(sw_sim* s) {
  uint32_t err = 0;
  cudaError_t e = cudaMemcpyAsync(&err, s->b.err, sizeof(err), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e);
  if (err & (kErrFind | kErrUnion | kErrLocal)) return fail(s, SW_ERR_TIMEOUT);
  if (err) return fail(s, SW_ERR_DEVICE);
  return SW_OK;
}

int measure_current(sw_sim* s) {
  if (!s->pending) return SW_OK;
  cudaError_t e = launch_measure(s->b.spin, s->lat, s->q, s->b, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e);
  s->pending = false;
  return SW_OK;
}

// sw_sweep_host's bands of tile rows: band k is tile rows r[k] .. r[k+1]-1.
// They start at one tile row and double up to an eighth of the lattice, so
// that the labelling starts as soon as the first few rows have arrived and
// the next band's copy (faster than its labelling) keeps ahead of it; the
// last band takes what is left once kUploadBands bands are planned, or when
// less than half a band would be left after it.
uint32_t plan_bands(uint32_t nty, uint32_t* r) {
  const uint32_t cap = (nty + 7) / 8;
  uint32_t nb = 0, r0 = 0, sz = 1;
  while (r0 < nty) {
    r[nb] = r0;
    r0 = (nb == kUploadBands - 1 || nty - r0 <= sz + sz / 2) ? nty : r0 + sz;
    ++nb;
    sz = 2 * sz < cap ? 2 * sz : cap;
  }
  r[nb] = nty;
  return nb;
}

// One sweep whose labelling runs band by band: band k starts as soon as the
// copy of its rows and of its halo row (the first row of band k+1, copied
// with band k; the last band's halo is row 0, in the first copy) has landed,
// i.e. on event ev[k] of the upload stream, whose copies complete in order.
// The labelling of a band also checks every spin it reads (BandSrc).
template <int TH, typename LabelT>
cudaError_t sweep_banded(sw_sim* s, const uint32_t* r, uint32_t nb) {
  const Lattice& lat = s->lat;
  cudaError_t e;
  for (uint32_t bnd = 0; bnd < nb; ++bnd) {
    if ((e = cudaStreamWaitEvent(s->stream, s->up_ev[bnd], 0))) return e;
    const BandSrc src{s->b, lat, r[bnd] * lat.ntx, (r[bnd + 1] - r[bnd]) * lat.ntx};
    const uint32_t n = (r[bnd + 1] - r[bnd]) * lat.ntx;
    e = s->b.fuse ? launch_label_src<TH, LabelT, false, false, BandSrc, false, true>(src, n, s->stream)
                  : launch_label_src<TH, LabelT, false, false>(src, n, s->stream);
    if (e) return e;
  }
  const SingleSrc full{s->b, lat};
  if (s->b.fuse) {
    if ((e = launch_file_src(full, 1, s->stream))) return e;
  } else {
    if ((e = launch_merge_src<TH, LabelT>(full, lat.ntiles, s->stream))) return e;
  }
  if ((e = launch_resolve_src<TH, LabelT>(full, lat.ntiles, s->stream))) return e;
  return launch_recolor_src<TH, LabelT, false>(full, lat.ntiles, (LabelT*)nullptr, s->stream);
}

template <typename LabelT>
cudaError_t sweep_banded_th(sw_sim* s, const uint32_t* r, uint32_t nb) {
  switch (s->th) {
    case 16: return sweep_banded<16, LabelT>(s, r, nb);
    case 32: return sweep_banded<32, LabelT>(s, r, nb);
    case 64: return sweep_banded<64, LabelT>(s, r, nb);
    case 128: return sweep_banded<128, LabelT>(s, r, nb);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

extern "C" {

int sw_set_allocator(sw_alloc_fn alloc, sw_free_fn free_fn, void* ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr)) return SW_ERR_INVAL;
  swgb::g_alloc = alloc;
  swgb::g_free = free_fn;
  swgb::g_alloc_ctx = ctx;
  return SW_OK;
}

int sw_threshold(double T, uint32_t* thr) {
  if (!thr || !(T > 0.0) || !isfinite(T)) return SW_ERR_INVAL;
  *thr = bond_threshold(T);
  return SW_OK;
}

int sw_create(uint64_t L, uint32_t q, double T, uint64_t seed, sw_sim** out) {
  sw_params p;
  memset(&p, 0, sizeof(p));
  p.L = L;
  p.q = q;
  p.T = T;
  p.seed = seed;
  return sw_create_ex(&p, out);
}

int sw_create_ex(const sw_params* prm, sw_sim** out) {
  if (!prm || !out) return SW_ERR_INVAL;
  *out = nullptr;
  const uint64_t L = prm->L;
  if (L < 2 || L > (1ull << 20) || prm->q < 2 || prm->q > 255 || !(prm->T > 0.0) ||
      !isfinite(prm->T) || prm->init > SW_INIT_ZERO || prm->store_bonds > 1 || prm->measure > 2 ||
      prm->merge > SW_MERGE_FUSED)
    return SW_ERR_INVAL;
  uint32_t lb = prm->label_bits ? prm->label_bits : (L <= 32768 ? 32u : 64u);
  if (lb != 32 && lb != 64) return SW_ERR_INVAL;
  if (lb == 32 && L * L > (1ull << 32)) return SW_ERR_INVAL;
  const uint32_t th = pick_tile_h(L, prm->tile_h);
  if (th != 16 && th != 32 && th != 64 && th != 128) return SW_ERR_INVAL;
  const uint32_t ring = prm->ring ? prm->ring : 1024u;

  sw_sim* s = new (std::nothrow) sw_sim();
  if (!s) return SW_ERR_NOMEM;
  s->p = *prm;
  s->L = L;
  s->N = L * L;
  s->q = prm->q;
  s->thr = bond_threshold(prm->T);
  s->label_bits = lb;
  s->th = th;
  s->ring = ring;
  s->lat = make_lattice(L, th);
  s->alloc = current_allocator();
  s->measure_on = prm->measure != 2;
  cudaGetDevice(&s->device);

  const uint64_t nt = s->lat.ntiles;
  Bufs& b = s->b;
  b.spin = (uint8_t*)take(s, s->N + 16);
  b.code = (uint16_t*)take(s, s->N * 2 + 16);
  b.bonds = prm->store_bonds ? (uint8_t*)take(s, L * s->lat.bp + 16) : nullptr;
  b.G = (uint64_t*)take(s, nt * open_cap(th) * 8);
  b.edge = (uint16_t*)take(s, nt * edge_u16(th) * 2);
  b.ebits = (uint32_t*)take(s, nt * bit_words(th) * 4);
  b.ocnt = (uint32_t*)take(s, nt * 4);
  b.nso = (uint8_t*)take(s, nt * open_cap(th));
  b.fuse = prm->merge == SW_MERGE_FUSED ? 1u : 0u;
  b.ecnt = b.fuse ? (uint32_t*)take(s, nt * 2 * 4) : nullptr;
  b.acc = (unsigned long long*)take(s, 8 * 260);
  b.ring = (unsigned long long*)take(s, (size_t)ring * (2 + s->q) * 8);
  b.ctl = (unsigned long long*)take(s, 64);
  b.err = (uint32_t*)take(s, 64);
  if (!b.spin || !b.code || (prm->store_bonds && !b.bonds) || !b.G || !b.edge || !b.ebits ||
      !b.ocnt || !b.nso || (b.fuse && !b.ecnt) || !b.acc || !b.ring || !b.ctl || !b.err) {
    release_all(s);
    delete s;
    return SW_ERR_NOMEM;
  }
  b.seed = prm->seed;
  set_round_keys(b);
  b.thr = s->thr;
  b.q = s->q;
  b.ring_cap = ring;
  b.measure = s->measure_on ? 1u : 0u;
  b.walk_cap = prm->walk_cap;

  cudaError_t e = cudaSuccess;
  if (!e) e = cudaMemsetAsync(b.G, 0, nt * open_cap(th) * 8, s->stream);
  if (!e) e = cudaMemsetAsync(b.acc, 0, 8 * 260, s->stream);
  if (!e) e = cudaMemsetAsync(b.ring, 0xFF, (size_t)ring * (2 + s->q) * 8, s->stream);
  if (!e) e = cudaMemsetAsync(b.ctl, 0, 64, s->stream);
  if (!e) e = cudaMemsetAsync(b.err, 0, 64, s->stream);
  if (!e) e = cudaMemsetAsync(b.ocnt, 0, nt * 4, s->stream);
  if (!e && b.fuse) e = cudaMemsetAsync(b.ecnt, 0, nt * 2 * 4, s->stream);  // every counter even
  if (!e) e = launch_init(b.spin, s->N, s->q, prm->seed, prm->init, s->stream);
  if (!e) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    release_all(s);
    delete s;
    return SW_ERR_CUDA;
  }
  s->sweep = 0;
  s->measured_from = 0;
  s->pending = true;
  *out = s;
  return SW_OK;
}

void sw_destroy(sw_sim* s) {
  if (!s) return;
  cudaStreamSynchronize(s->stream);
  release_all(s);
  delete s;
}

int sw_bind_stream(sw_sim* s, void* stream) {
  if (!s) return SW_ERR_INVAL;
  s->stream = (cudaStream_t)stream;
  return SW_OK;
}

int sw_sweep(sw_sim* s, uint64_t n) {
  if (!s) return SW_ERR_INVAL;
  if (sticky(s)) return s->last_err;
  if (s->spins_invalid) return SW_ERR_STATE;
  for (uint64_t k = 0; k < n; ++k) {
    cudaError_t e;
    if (s->profiling) {
      cudaEvent_t ev[4];
      for (int j = 0; j < 4; ++j) {
        ev[j] = get_event(s);
        if (!ev[j]) return fail(s, SW_ERR_CUDA);
        s->ev_used.push_back(ev[j]);
      }
      e = launch_sweep_events(s->label_bits, s->th, s->b, s->lat, s->stream, ev);
    } else {
      e = launch_sweep(s->label_bits, s->th, s->b, s->lat, s->stream);
    }
    if (e != cudaSuccess) return cuda_fail(s, e);
  }
  if (n) {
    s->sweep += n;
    s->pending = true;
  }
  return SW_OK;
}

int sw_sync(sw_sim* s) {
  if (!s) return SW_ERR_INVAL;
  if (sticky(s)) return s->last_err;
  return check_device(s);
}

int sw_series(sw_sim* s, uint64_t first, uint64_t count, uint64_t* E, uint64_t* n) {
  if (!s) return SW_ERR_INVAL;
  if (sticky(s)) return s->last_err;
  if (count == 0) return SW_OK;
  const uint64_t cur = s->sweep;
  const uint64_t last = first + count - 1;
  if (last < first || last > cur) return SW_ERR_RANGE;
  uint64_t oldest = s->measured_from;
  if (cur + 1 > s->ring && cur + 1 - s->ring > oldest) oldest = cur + 1 - s->ring;
  if (first < oldest) return SW_ERR_RANGE;
  if (!s->measure_on && !(first == cur && count == 1)) return SW_ERR_RANGE;
  if (last == cur) {
    int rc = measure_current(s);
    if (rc) return rc;
  }
  const size_t rec = 2 + s->q;
  std::vector<unsigned long long> host(count * rec);
  // copy the ring window (at most two contiguous pieces)
  uint64_t done = 0;
  while (done < count) {
    const uint64_t c = first + done;
    const uint64_t slot = c % s->ring;
    uint64_t run = s->ring - slot;
    if (run > count - done) run = count - done;
    cudaError_t e = cudaMemcpyAsync(host.data() + done * rec, s->b.ring + slot * rec,
                                    run * rec * 8, cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e);
    done += run;
  }
  int rc = check_device(s);
  if (rc) return rc;
  for (uint64_t k = 0; k < count; ++k) {
    const unsigned long long* r = host.data() + k * rec;
    if (r[0] != first + k) return SW_ERR_RANGE;
    if (E) E[k] = r[1];
    if (n)
      for (uint32_t j = 0; j < s->q; ++j) n[k * s->q + j] = r[2 + j];
  }
  return SW_OK;
}

int sw_measure(sw_sim* s, sw_obs* out) {
  if (!s || !out) return SW_ERR_INVAL;
  memset(out, 0, sizeof(*out));
  uint64_t E = 0;
  std::vector<uint64_t> n(s->q);
  const uint64_t cur = s->sweep;
  // sw_series would refuse when measurement is off; measure directly then
  if (!s->measure_on) {
    if (sticky(s)) return s->last_err;
    s->pending = true;
    int rc = measure_current(s);
    if (rc) return rc;
    const size_t rec = 2 + s->q;
    std::vector<unsigned long long> host(rec);
    cudaError_t e = cudaMemcpyAsync(host.data(), s->b.ring + (cur % s->ring) * rec, rec * 8,
                                    cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e);
    rc = check_device(s);
    if (rc) return rc;
    if (host[0] != cur) return fail(s, SW_ERR_DEVICE);
    E = host[1];
    for (uint32_t j = 0; j < s->q; ++j) n[j] = host[2 + j];
  } else {
    int rc = sw_series(s, cur, 1, &E, n.data());
    if (rc) return rc;
  }
  out->config = cur;
  out->E_sat = E;
  out->q = s->q;
  for (uint32_t j = 0; j < s->q; ++j) out->n[j] = n[j];
  return SW_OK;
}

int sw_spins(sw_sim* s, uint8_t* dst, uint64_t n, int dst_on_device) {
  if (!s || !dst || n != s->N) return SW_ERR_INVAL;
  if (sticky(s)) return s->last_err;
  cudaError_t e = cudaMemcpyAsync(dst, s->b.spin, s->N,
                                  dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e);
  if (!dst_on_device) return check_device(s);
  return SW_OK;
}

int sw_set_spins(sw_sim* s, const uint8_t* src, uint64_t n, int src_on_device) {
  if (!s || !src || n != s->N) return SW_ERR_INVAL;
  if (sticky(s)) return s->last_err;
  // validate on the device: flag word ctl[3]
  uint32_t* bad = reinterpret_cast<uint32_t*>(s->b.ctl + 3);
  cudaError_t e = cudaMemsetAsync(bad, 0, 4, s->stream);
  // page-locked host memory with a device mapping: one kernel reads it,
  // writes the lattice and validates (no separate copy and check passes)
  const void* mapped = nullptr;
  if (!src_on_device && ((uintptr_t)src & 15u) == 0) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, src) == cudaSuccess && at.type == cudaMemoryTypeHost &&
        at.devicePointer != nullptr)
      mapped = at.devicePointer;
    cudaGetLastError();
  }
  if (!e && mapped) {
    k_copy_check_spins<<<152 * 8, 256, 0, s->stream>>>((const uint8_t*)mapped, s->b.spin, s->N, s->q, bad);
    e = cudaGetLastError();
  } else if (!e) {
    e = cudaMemcpyAsync(s->b.spin, src, s->N,
                        src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->stream);
    if (!e) {
      uint64_t blocks = (s->N / 4 + 255) / 256;
      if (blocks > 152ull * 8) blocks = 152ull * 8;
      if (blocks == 0) blocks = 1;
      k_check_spins<<<(unsigned)blocks, 256, 0, s->stream>>>(s->b.spin, s->N, s->q, bad);
      e = cudaGetLastError();
    }
  }
  uint32_t hbad = 0;
  if (!e) e = cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, s->stream);
  if (!e) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e);
  s->pending = true;
  s->measured_from = s->sweep;
  if (hbad) {
    s->spins_invalid = true;
    return SW_ERR_INVAL;
  }
  s->spins_invalid = false;
  return SW_OK;
}

int sw_sweep_host(sw_sim* s, const uint8_t* src, uint64_t n, uint64_t nsweeps, sw_obs* out) {
  if (!s || !src || n != s->N || nsweeps == 0) return SW_ERR_INVAL;
  if (sticky(s)) return s->last_err;
  cudaError_t e = cudaSuccess;
  if (!s->up) {
    e = cudaStreamCreateWithFlags(&s->up, cudaStreamNonBlocking);
    for (uint32_t k = 0; !e && k <= kUploadBands; ++k)
      e = cudaEventCreateWithFlags(&s->up_ev[k], cudaEventDisableTiming);
    if (e) return cuda_fail(s, e);
  }
  uint32_t r[kUploadBands + 1];
  const uint32_t nb = plan_bands(s->lat.nty, r);
  // the upload may only overwrite the spins once earlier work on them is done
  e = cudaEventRecord(s->up_ev[kUploadBands], s->stream);
  if (!e) e = cudaStreamWaitEvent(s->up, s->up_ev[kUploadBands], 0);
  // copy k: from the end of copy k-1 through band k's halo row
  uint64_t y0 = 0;
  for (uint32_t bnd = 0; !e && bnd < nb; ++bnd) {
    uint64_t y1 = bnd + 1 < nb ? (uint64_t)r[bnd + 1] * s->th + 1 : s->L;
    if (y1 > s->L) y1 = s->L;
    if (y1 > y0)
      e = cudaMemcpyAsync(s->b.spin + y0 * s->L, src + y0 * s->L, (y1 - y0) * s->L, cudaMemcpyHostToDevice,
                          s->up);
    if (!e) e = cudaEventRecord(s->up_ev[bnd], s->up);
    y0 = y1;
  }
  if (!e)
    e = s->label_bits == 64 ? sweep_banded_th<uint64_t>(s, r, nb)
                            : sweep_banded_th<uint32_t>(s, r, nb);
  if (e) return cuda_fail(s, e);
  // the uploaded configuration is configuration `sweep`, measured by the
  // labelling of its first sweep
  s->measured_from = s->sweep;
  s->spins_invalid = false;
  s->sweep += 1;
  s->pending = true;
  if (nsweeps > 1) {
    int rc = sw_sweep(s, nsweeps - 1);
    if (rc) return rc;
  }
  // a spin >= q read by the banded labelling: the configuration was invalid
  uint32_t err = 0;
  e = cudaMemcpyAsync(&err, s->b.err, 4, cudaMemcpyDeviceToHost, s->stream);
  if (!e) e = cudaStreamSynchronize(s->stream);
  if (e) return cuda_fail(s, e);
  if (err & kErrSpin) {
    const uint32_t rest = err & ~kErrSpin;
    e = cudaMemcpyAsync(s->b.err, &rest, 4, cudaMemcpyHostToDevice, s->stream);
    if (!e) e = cudaStreamSynchronize(s->stream);
    if (e) return cuda_fail(s, e);
    s->spins_invalid = true;
    return SW_ERR_INVAL;
  }
  if (out) return sw_measure(s, out);
  return check_device(s);
}

int sw_profile(sw_sim* s, int enable) {
  if (!s) return SW_ERR_INVAL;
  if (enable) {
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e);
    for (cudaEvent_t ev : s->ev_used) s->ev_pool.push_back(ev);
    s->ev_used.clear();
    for (int k = 0; k < 3; ++k) {
      s->prof_ms[k] = 0;
      s->prof_launches[k] = 0;
    }
  }
  s->profiling = enable != 0;
  return SW_OK;
}

int sw_profile_read(sw_sim* s, double* ms, uint64_t* launches, int nphase) {
  if (!s || nphase < 0 || nphase > 3) return SW_ERR_INVAL;
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e);
  int rc = drain_events(s);
  if (rc) return fail(s, rc);
  for (int k = 0; k < nphase; ++k) {
    if (ms) ms[k] = s->prof_ms[k];
    if (launches) launches[k] = s->prof_launches[k];
  }
  return SW_OK;
}

int sw_bonds(sw_sim* s, uint8_t* dst, uint64_t nbytes, int dst_on_device) {
  if (!s || !dst) return SW_ERR_INVAL;
  if (!s->b.bonds) return SW_ERR_STATE;
  if (nbytes != s->L * s->lat.bp) return SW_ERR_INVAL;
  if (sticky(s)) return s->last_err;
  cudaError_t e = cudaMemcpyAsync(dst, s->b.bonds, nbytes,
                                  dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e);
  if (!dst_on_device) return check_device(s);
  return SW_OK;
}

int sw_get_sweep(const sw_sim* s, uint64_t* sweep) {
  if (!s || !sweep) return SW_ERR_INVAL;
  *sweep = s->sweep;
  return SW_OK;
}

int sw_set_sweep(sw_sim* s, uint64_t sweep) {
  if (!s) return SW_ERR_INVAL;
  if (sticky(s)) return s->last_err;
  unsigned long long v = sweep;
  cudaError_t e = cudaMemcpyAsync(s->b.ctl, &v, sizeof(v), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e);
  s->sweep = sweep;
  s->measured_from = sweep;
  s->pending = true;
  return SW_OK;
}

int sw_info(const sw_sim* s, sw_info_t* out) {
  if (!s || !out) return SW_ERR_INVAL;
  out->L = s->L;
  out->q = s->q;
  out->thr = s->thr;
  out->label_bits = s->label_bits;
  out->tile_w = kTW;
  out->tile_h = s->th;
  out->ring = s->ring;
  out->device_bytes = s->dev_bytes;
  out->tiles = s->lat.ntiles;
  out->merge = s->b.fuse ? SW_MERGE_FUSED : SW_MERGE_KERNEL;
  out->pad_ = 0;
  return SW_OK;
}

int sw_last_error(const sw_sim* s) { return s ? s->last_err : SW_ERR_INVAL; }

const char* sw_strerror(int code) {
  switch (code) {
    case SW_OK: return "ok";
    case SW_ERR_INVAL: return "invalid argument";
    case SW_ERR_NOMEM: return "out of memory";
    case SW_ERR_CUDA: return "CUDA runtime error";
    case SW_ERR_TIMEOUT: return "bounded device loop hit its iteration cap";
    case SW_ERR_STATE: return "call not valid in this state";
    case SW_ERR_DEVICE: return "device-side consistency check failed";
    case SW_ERR_RANGE: return "observables not held for the requested configurations";
    default: return "unknown error";
  }
}

int sw_label_bonds(uint64_t L, const uint8_t* bonds, void* roots, uint32_t label_bits,
                   uint32_t tile_h, void* stream) {
  if (L < 2 || L > (1ull << 20) || !bonds || !roots) return SW_ERR_INVAL;
  if (label_bits != 32 && label_bits != 64) return SW_ERR_INVAL;
  if (label_bits == 32 && L * L > (1ull << 32)) return SW_ERR_INVAL;
  const uint32_t th = pick_tile_h(L, tile_h);
  if (th != 16 && th != 32 && th != 64 && th != 128) return SW_ERR_INVAL;
  const Lattice lat = make_lattice(L, th);
  const DeviceAllocator al = current_allocator();
  const uint64_t N = L * L, nt = lat.ntiles;
  struct Blk { void* p; size_t n; };
  std::vector<Blk> blk;
  auto get = [&](size_t n) -> void* {
    n = (n + 255) & ~(size_t)255;
    void* p = al.allocate(n);
    if (p) blk.push_back({p, n});
    return p;
  };
  Bufs b{};
  b.bonds = const_cast<uint8_t*>(bonds);
  b.code = (uint16_t*)get(N * 2 + 16);
  b.G = (uint64_t*)get(nt * open_cap(th) * 8);
  b.edge = (uint16_t*)get(nt * edge_u16(th) * 2);
  b.ebits = (uint32_t*)get(nt * bit_words(th) * 4);
  b.ocnt = (uint32_t*)get(nt * 4);
  b.ctl = (unsigned long long*)get(64);
  b.err = (uint32_t*)get(64);
  b.q = 2;
  b.measure = 0;
  int rc = SW_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (!b.code || !b.G || !b.edge || !b.ebits || !b.ocnt || !b.ctl || !b.err) {
    rc = SW_ERR_NOMEM;
  } else {
    cudaError_t e = cudaMemsetAsync(b.ctl, 0, 64, st);
    if (!e) e = cudaMemsetAsync(b.err, 0, 64, st);
    if (!e) e = cudaMemsetAsync(b.G, 0, nt * open_cap(th) * 8, st);
    if (!e)
      e = label_bits == 64 ? label_given_t<uint64_t>(th, b, lat, (uint64_t*)roots, st)
                           : label_given_t<uint32_t>(th, b, lat, (uint32_t*)roots, st);
    uint32_t err = 0;
    if (!e) e = cudaMemcpyAsync(&err, b.err, 4, cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      rc = SW_ERR_CUDA;
    } else if (err & (kErrFind | kErrUnion | kErrLocal)) {
      rc = SW_ERR_TIMEOUT;
    } else if (err) {
      rc = SW_ERR_DEVICE;
    }
  }
  cudaStreamSynchronize(st);
  for (auto& x : blk) al.release(x.p, x.n);
  return rc;
}

}  // extern "C"
