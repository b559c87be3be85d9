// sw_batch.cu -- C ABI of the batched replica runner (include/sw.h,
// sw_batch_*): R independent lattices of uneven L, q, T advanced together by
// the same kernels as the single-lattice path, over one concatenated tile
// list.  A batch sweep is one persistent labelling launch plus three short
// launches, captured once into a CUDA graph and replayed.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/sw.h"
#include "sw_internal.h"
#include "sw_launch.cuh"

using namespace swgb;

struct sw_batch {
  uint32_t R = 0, th = 64, ring = 64, label_bits = 32;
  bool measure_on = true, want_graph = true;
  bool fuse = false;  // the labeller does the boundary unions (SW_MERGE_FUSED)
  DeviceAllocator alloc{};
  void* arena = nullptr;
  size_t arena_bytes = 0;
  std::vector<Rep> reps;            // host copy of the replica table
  Rep* d_reps = nullptr;            // device replica table
  uint32_t* d_tile_rep = nullptr;   // replica of each global tile
  uint32_t total = 0;               // tiles of all replicas
  uint64_t sites = 0;
  uint32_t* err = nullptr;          // device error word shared by all replicas
  uint32_t* bad = nullptr;          // sw_batch_set_spins validation flag
  cudaStream_t stream = nullptr;    // work stream (bound by the caller)
  cudaStream_t cap_stream = nullptr;  // private stream used only to capture the graph
  cudaGraphExec_t exec = nullptr;
  uint64_t sweep = 0;
  std::vector<uint8_t> pending;     // current configuration not measured yet
  std::vector<uint64_t> measured_from;
  bool spins_invalid = false;
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool, ev_used;
  double prof_ms[3] = {0, 0, 0};
  uint64_t prof_launches[3] = {0, 0, 0};
  int last_err = SW_OK;
};

namespace {

int bfail(sw_batch* b, int code) {
  if (b && (code == SW_ERR_CUDA || code == SW_ERR_DEVICE || code == SW_ERR_TIMEOUT)) b->last_err = code;
  return code;
}

int bcuda(sw_batch* b, cudaError_t e) {
  (void)e;
  cudaGetLastError();
  return bfail(b, SW_ERR_CUDA);
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

void release(sw_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  b->cap_stream = nullptr;
  for (cudaEvent_t e : b->ev_pool) cudaEventDestroy(e);
  for (cudaEvent_t e : b->ev_used) cudaEventDestroy(e);
  b->ev_pool.clear();
  b->ev_used.clear();
  if (b->arena) b->alloc.release(b->arena, b->arena_bytes);
  b->arena = nullptr;
}

int check_err(sw_batch* b) {
  uint32_t err = 0;
  cudaError_t e = cudaMemcpyAsync(&err, b->err, sizeof(err), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(b, e);
  if (err & (kErrFind | kErrUnion | kErrLocal)) return bfail(b, SW_ERR_TIMEOUT);
  if (err) return bfail(b, SW_ERR_DEVICE);
  return SW_OK;
}

cudaError_t batch_sweep_once(sw_batch* b, cudaStream_t st, cudaEvent_t* ev) {
  const BatchSrc src{b->d_reps, b->d_tile_rep, b->total, b->R};
  return b->label_bits == 64 ? sweep_th<uint64_t>(b->th, src, b->total, st, ev, b->R, b->fuse)
                             : sweep_th<uint32_t>(b->th, src, b->total, st, ev, b->R, b->fuse);
}

// Captures one batch sweep into a graph (on a private stream; the graph
// reads the sweep counters from device memory, so one graph serves every
// sweep).
int build_graph(sw_batch* b) {
  const BatchSrc src{b->d_reps, b->d_tile_rep, b->total, b->R};
  cudaError_t e = b->label_bits == 64 ? configure_th<uint64_t, BatchSrc>(b->th, src, b->fuse)
                                      : configure_th<uint32_t, BatchSrc>(b->th, src, b->fuse);
  if (e != cudaSuccess) return bcuda(b, e);
  if (!b->cap_stream) {
    e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bcuda(b, e);
  }
  cudaGraph_t g = nullptr;
  e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return bcuda(b, e);
  cudaError_t le = batch_sweep_once(b, b->cap_stream, nullptr);
  e = cudaStreamEndCapture(b->cap_stream, &g);
  if (le != cudaSuccess || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return bcuda(b, le != cudaSuccess ? le : e);
  }
  e = cudaGraphInstantiate(&b->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    b->exec = nullptr;
    return bcuda(b, e);
  }
  return SW_OK;
}

cudaEvent_t bget_event(sw_batch* b) {
  if (!b->ev_pool.empty()) {
    cudaEvent_t e = b->ev_pool.back();
    b->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

}  // namespace

extern "C" {

int sw_batch_create(uint32_t R, const uint64_t* L, const uint32_t* q, const double* T,
                    const uint64_t* seed, sw_batch** out) {
  sw_batch_params p;
  memset(&p, 0, sizeof(p));
  p.R = R;
  p.L = L;
  p.q = q;
  p.T = T;
  p.seed = seed;
  return sw_batch_create_ex(&p, out);
}

int sw_batch_create_ex(const sw_batch_params* p, sw_batch** out) {
  if (!p || !out || p->R == 0 || !p->L || !p->q || !p->T || !p->seed) return SW_ERR_INVAL;
  *out = nullptr;
  const uint32_t th = p->tile_h ? p->tile_h : 64u;
  if (th != 16 && th != 32 && th != 64 && th != 128) return SW_ERR_INVAL;
  if (p->init > SW_INIT_ZERO || p->measure > 2 || p->graph > 2 || p->merge > SW_MERGE_FUSED) return SW_ERR_INVAL;
  uint32_t lb = 32;
  for (uint32_t r = 0; r < p->R; ++r) {
    if (p->L[r] < 2 || p->L[r] > (1ull << 20) || p->q[r] < 2 || p->q[r] > 255 ||
        !(p->T[r] > 0.0) || !isfinite(p->T[r]))
      return SW_ERR_INVAL;
    if (p->L[r] > 32768) lb = 64;
  }
  sw_batch* b = new (std::nothrow) sw_batch();
  if (!b) return SW_ERR_NOMEM;
  b->R = p->R;
  b->th = th;
  b->ring = p->ring ? p->ring : 64u;
  b->label_bits = lb;
  b->measure_on = p->measure != 2;
  b->want_graph = p->graph != 2;
  b->fuse = p->merge == SW_MERGE_FUSED;
  b->alloc = current_allocator();
  b->reps.resize(p->R);
  b->pending.assign(p->R, 1);
  b->measured_from.assign(p->R, 0);

  // ---- one arena: per-replica buffers, then the shared words and tables
  std::vector<size_t> off(p->R);
  size_t bytes = 0;
  uint64_t total = 0;
  for (uint32_t r = 0; r < p->R; ++r) {
    const uint64_t L = p->L[r], N = L * L;
    const Lattice lat = make_lattice(L, th);
    const uint64_t nt = lat.ntiles;
    off[r] = bytes;
    bytes += up256(N + 16) + up256(2 * N + 16) + up256(nt * open_cap(th) * 8) + up256(nt * edge_u16(th) * 2) +
             up256(nt * bit_words(th) * 4) + up256(nt * 4) +
             up256(nt * open_cap(th)) + up256(nt * 2 * 4) + up256(8 * 260) + up256((size_t)b->ring * (2 + p->q[r]) * 8) +
             up256(64);
    total += nt;
    b->sites += N;
  }
  if (total > 0xFFFFFFFFull) {
    delete b;
    return SW_ERR_INVAL;
  }
  b->total = (uint32_t)total;
  const size_t shared_off = bytes;
  bytes += up256(64) + up256(64) + up256(sizeof(Rep) * p->R) + up256(4 * total);
  b->arena_bytes = bytes;
  b->arena = b->alloc.allocate(bytes);
  if (!b->arena) {
    delete b;
    return SW_ERR_NOMEM;
  }
  uint8_t* base = (uint8_t*)b->arena;
  b->err = (uint32_t*)(base + shared_off);
  b->bad = (uint32_t*)(base + shared_off + 256);
  b->d_reps = (Rep*)(base + shared_off + 512);
  b->d_tile_rep = (uint32_t*)(base + shared_off + 512 + up256(sizeof(Rep) * p->R));

  std::vector<uint32_t> tile_rep(total);
  uint32_t tile0 = 0;
  for (uint32_t r = 0; r < p->R; ++r) {
    const uint64_t L = p->L[r], N = L * L;
    const Lattice lat = make_lattice(L, th);
    const uint64_t nt = lat.ntiles;
    uint8_t* c = base + off[r];
    Bufs& bb = b->reps[r].b;
    memset(&bb, 0, sizeof(bb));
    bb.spin = c; c += up256(N + 16);
    bb.code = (uint16_t*)c; c += up256(2 * N + 16);
    bb.G = (uint64_t*)c; c += up256(nt * open_cap(th) * 8);
    bb.edge = (uint16_t*)c; c += up256(nt * edge_u16(th) * 2);
    bb.ebits = (uint32_t*)c; c += up256(nt * bit_words(th) * 4);
    bb.ocnt = (uint32_t*)c; c += up256(nt * 4);
    bb.nso = c; c += up256(nt * open_cap(th));
    bb.ecnt = (uint32_t*)c; c += up256(nt * 2 * 4);
    bb.fuse = b->fuse ? 1u : 0u;
    bb.acc = (unsigned long long*)c; c += up256(8 * 260);
    bb.ring = (unsigned long long*)c; c += up256((size_t)b->ring * (2 + p->q[r]) * 8);
    bb.ctl = (unsigned long long*)c;
    bb.bonds = nullptr;
    bb.err = b->err;
    bb.seed = p->seed[r];
    set_round_keys(bb);
    bb.thr = bond_threshold(p->T[r]);
    bb.q = p->q[r];
    bb.ring_cap = b->ring;
    bb.measure = b->measure_on ? 1u : 0u;
    b->reps[r].lat = lat;
    b->reps[r].tile0 = tile0;
    b->reps[r].pad_ = 0;
    for (uint64_t k = 0; k < nt; ++k) tile_rep[tile0 + k] = r;
    tile0 += (uint32_t)nt;
  }

  cudaError_t e = cudaMemsetAsync(b->arena, 0, bytes, b->stream);
  for (uint32_t r = 0; r < p->R && !e; ++r)
    e = cudaMemsetAsync(b->reps[r].b.ring, 0xFF, (size_t)b->ring * (2 + p->q[r]) * 8, b->stream);
  if (!e) e = cudaMemcpyAsync(b->d_reps, b->reps.data(), sizeof(Rep) * p->R, cudaMemcpyHostToDevice, b->stream);
  if (!e) e = cudaMemcpyAsync(b->d_tile_rep, tile_rep.data(), 4 * total, cudaMemcpyHostToDevice, b->stream);
  for (uint32_t r = 0; r < p->R && !e; ++r)
    e = launch_init(b->reps[r].b.spin, p->L[r] * p->L[r], p->q[r], p->seed[r], p->init, b->stream);
  if (!e) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    release(b);
    delete b;
    return SW_ERR_CUDA;
  }
  *out = b;
  return SW_OK;
}

void sw_batch_destroy(sw_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  release(b);
  delete b;
}

int sw_batch_bind_stream(sw_batch* b, void* stream) {
  if (!b) return SW_ERR_INVAL;
  b->stream = (cudaStream_t)stream;
  return SW_OK;
}

int sw_batch_sweep(sw_batch* b, uint64_t n) {
  if (!b) return SW_ERR_INVAL;
  if (b->last_err) return b->last_err;
  if (b->spins_invalid) return SW_ERR_STATE;
  for (uint64_t k = 0; k < n; ++k) {
    cudaError_t e;
    if (b->profiling) {
      cudaEvent_t ev[4];
      for (int j = 0; j < 4; ++j) {
        ev[j] = bget_event(b);
        if (!ev[j]) return bfail(b, SW_ERR_CUDA);
        b->ev_used.push_back(ev[j]);
      }
      e = batch_sweep_once(b, b->stream, ev);
    } else if (b->want_graph) {
      if (!b->exec) {
        int rc = build_graph(b);
        if (rc) return rc;
      }
      e = cudaGraphLaunch(b->exec, b->stream);
    } else {
      e = batch_sweep_once(b, b->stream, nullptr);
    }
    if (e != cudaSuccess) return bcuda(b, e);
  }
  if (n) {
    b->sweep += n;
    for (auto& x : b->pending) x = 1;
  }
  return SW_OK;
}

int sw_batch_sync(sw_batch* b) {
  if (!b) return SW_ERR_INVAL;
  if (b->last_err) return b->last_err;
  return check_err(b);
}

int sw_batch_series(sw_batch* b, uint32_t r, uint64_t first, uint64_t count, uint64_t* E, uint64_t* n) {
  if (!b || r >= b->R) return SW_ERR_INVAL;
  if (b->last_err) return b->last_err;
  if (count == 0) return SW_OK;
  const Rep& rp = b->reps[r];
  const uint32_t q = rp.b.q;
  const uint64_t cur = b->sweep, last = first + count - 1;
  if (last < first || last > cur) return SW_ERR_RANGE;
  uint64_t oldest = b->measured_from[r];
  if (cur + 1 > b->ring && cur + 1 - b->ring > oldest) oldest = cur + 1 - b->ring;
  if (first < oldest) return SW_ERR_RANGE;
  if (!b->measure_on && !(first == cur && count == 1)) return SW_ERR_RANGE;
  if (last == cur && b->pending[r]) {
    cudaError_t e = launch_measure(rp.b.spin, rp.lat, q, rp.b, b->stream);
    if (e != cudaSuccess) return bcuda(b, e);
    b->pending[r] = 0;
  }
  const size_t rec = 2 + q;
  std::vector<unsigned long long> host(count * rec);
  uint64_t done = 0;
  while (done < count) {
    const uint64_t c = first + done, slot = c % b->ring;
    uint64_t run = b->ring - slot;
    if (run > count - done) run = count - done;
    cudaError_t e = cudaMemcpyAsync(host.data() + done * rec, rp.b.ring + slot * rec, run * rec * 8,
                                    cudaMemcpyDeviceToHost, b->stream);
    if (e != cudaSuccess) return bcuda(b, e);
    done += run;
  }
  int rc = check_err(b);
  if (rc) return rc;
  for (uint64_t k = 0; k < count; ++k) {
    const unsigned long long* x = host.data() + k * rec;
    if (x[0] != first + k) return SW_ERR_RANGE;
    if (E) E[k] = x[1];
    if (n)
      for (uint32_t j = 0; j < q; ++j) n[k * q + j] = x[2 + j];
  }
  return SW_OK;
}

int sw_batch_measure(sw_batch* b, uint32_t r, sw_obs* out) {
  if (!b || !out || r >= b->R) return SW_ERR_INVAL;
  memset(out, 0, sizeof(*out));
  const uint32_t q = b->reps[r].b.q;
  std::vector<uint64_t> n(q);
  uint64_t E = 0;
  if (!b->measure_on) b->pending[r] = 1;  // the ring holds only what this call files
  int rc = sw_batch_series(b, r, b->sweep, 1, &E, n.data());
  if (rc) return rc;
  out->config = b->sweep;
  out->E_sat = E;
  out->q = q;
  for (uint32_t j = 0; j < q; ++j) out->n[j] = n[j];
  return SW_OK;
}

int sw_batch_spins(sw_batch* b, uint32_t r, uint8_t* dst, uint64_t n, int dst_on_device) {
  if (!b || !dst || r >= b->R) return SW_ERR_INVAL;
  const uint64_t L = b->reps[r].lat.L;
  if (n != L * L) return SW_ERR_INVAL;
  if (b->last_err) return b->last_err;
  cudaError_t e = cudaMemcpyAsync(dst, b->reps[r].b.spin, n,
                                  dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  b->stream);
  if (e != cudaSuccess) return bcuda(b, e);
  if (!dst_on_device) return check_err(b);
  return SW_OK;
}

int sw_batch_set_spins(sw_batch* b, uint32_t r, const uint8_t* src, uint64_t n, int src_on_device) {
  if (!b || !src || r >= b->R) return SW_ERR_INVAL;
  const uint64_t L = b->reps[r].lat.L;
  if (n != L * L) return SW_ERR_INVAL;
  if (b->last_err) return b->last_err;
  uint8_t* spin = b->reps[r].b.spin;
  cudaError_t e = cudaMemcpyAsync(spin, src, n,
                                  src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  b->stream);
  if (!e) e = cudaMemsetAsync(b->bad, 0, 4, b->stream);
  if (!e) {
    uint64_t blocks = (n / 4 + 255) / 256;
    if (blocks > 152ull * 8) blocks = 152ull * 8;
    if (blocks == 0) blocks = 1;
    k_check_spins<<<(unsigned)blocks, 256, 0, b->stream>>>(spin, n, b->reps[r].b.q, b->bad);
    e = cudaGetLastError();
  }
  uint32_t hbad = 0;
  if (!e) e = cudaMemcpyAsync(&hbad, b->bad, 4, cudaMemcpyDeviceToHost, b->stream);
  if (!e) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(b, e);
  b->pending[r] = 1;
  b->measured_from[r] = b->sweep;
  b->spins_invalid = hbad != 0;
  return hbad ? SW_ERR_INVAL : SW_OK;
}

int sw_batch_get_sweep(const sw_batch* b, uint64_t* sweep) {
  if (!b || !sweep) return SW_ERR_INVAL;
  *sweep = b->sweep;
  return SW_OK;
}

int sw_batch_info(const sw_batch* b, sw_batch_info_t* out) {
  if (!b || !out) return SW_ERR_INVAL;
  out->R = b->R;
  out->tile_h = b->th;
  out->tiles = b->total;
  out->sites = b->sites;
  out->device_bytes = b->arena_bytes;
  out->label_bits = b->label_bits;
  out->graph = b->want_graph ? 1u : 0u;
  out->merge = b->fuse ? SW_MERGE_FUSED : SW_MERGE_KERNEL;
  out->pad_ = 0;
  return SW_OK;
}

int sw_batch_profile(sw_batch* b, int enable) {
  if (!b) return SW_ERR_INVAL;
  if (enable) {
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e);
    for (cudaEvent_t ev : b->ev_used) b->ev_pool.push_back(ev);
    b->ev_used.clear();
    for (int k = 0; k < 3; ++k) {
      b->prof_ms[k] = 0;
      b->prof_launches[k] = 0;
    }
  }
  b->profiling = enable != 0;
  return SW_OK;
}

int sw_batch_profile_read(sw_batch* b, double* ms, uint64_t* launches, int nphase) {
  if (!b || nphase < 0 || nphase > 3) return SW_ERR_INVAL;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(b, e);
  for (size_t k = 0; k + 3 < b->ev_used.size(); k += 4) {
    for (int ph = 0; ph < 3; ++ph) {
      float m = 0.f;
      e = cudaEventElapsedTime(&m, b->ev_used[k + ph], b->ev_used[k + ph + 1]);
      if (e != cudaSuccess) return bcuda(b, e);
      b->prof_ms[ph] += m;
      b->prof_launches[ph] += 1;
    }
  }
  for (cudaEvent_t ev : b->ev_used) b->ev_pool.push_back(ev);
  b->ev_used.clear();
  for (int k = 0; k < nphase; ++k) {
    if (ms) ms[k] = b->prof_ms[k];
    if (launches) launches[k] = b->prof_launches[k];
  }
  return SW_OK;
}

int sw_batch_last_error(const sw_batch* b) { return b ? b->last_err : SW_ERR_INVAL; }

}  // extern "C"
