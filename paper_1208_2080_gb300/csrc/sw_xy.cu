// sw_xy.cu -- C ABI of the embedded-cluster Swendsen-Wang sweep of the 2D XY
// model with M equally spaced angles (include/sw.h, sw_xy_*).
//
// Sec. 5 of the paper names the extension of the multi-cluster sweep to the
// classical XY model through Wolff's embedded clusters.  A sweep draws an
// embedding axis, activates bonds between spins whose projections on it
// have the same sign (probability 1 - exp(-2 sigma_i sigma_j / T)), labels
// the clusters with the Potts machinery and reflects each cluster with
// probability 1/2.  The GPU path is the Potts sweep's four kernels in their
// XY form (sw_kernels.cuh, kXY) plus the measurement below; the conventions
// (axis on the half-grid, fold index of |sigma|, coins from the Potts state
// stream with q = 2) are the ones the oracle states.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/sw.h"
#include "sw_internal.h"
#include "sw_kernels.cuh"
#include "sw_launch.cuh"

using namespace swgb;

namespace {

constexpr double kPi = 3.141592653589793;  // the double nearest pi
constexpr uint32_t kMaxAcc = 129 + 256;    // D[0..128] + n[0..255]

// Bond thresholds by fold index: the embedded Ising coupling of two spins is
// |sigma_i| |sigma_j| with |sigma| = sin(pi c / M), and a satisfied embedded
// bond is active with probability 1 - exp(-2 |sigma_i| |sigma_j| / T).
void xy_table(uint32_t M, double T, uint32_t* tt) {
  const uint32_t H = M / 2;
  for (uint32_t c = 0; c <= H; ++c) {
    for (uint32_t d = 0; d <= H; ++d) {
      const double sc = sin(kPi * (double)c / (double)M);
      const double sd = sin(kPi * (double)d / (double)M);
      const double p = -expm1(-2.0 * sc * sd / T);
      const double t = floor(p * 4294967296.0);
      uint32_t v = 0u;
      if (t >= 4294967295.0)
        v = 0xFFFFFFFFu;
      else if (t > 0.0)
        v = (uint32_t)t;
      tt[c * (H + 1) + d] = v;
    }
  }
}

// D[0..M/2] (bonds by folded angle difference) and n[0..M-1] (sites by
// angle) of a configuration, accumulated into acc[0..M/2] and acc[M/2+1..].
// Blocks over rows; each warp counts into its own shared histogram (the
// counts are shared-memory atomics, so warps do not contend with each
// other); 16-site groups with 16-byte loads when L % 16 == 0, else 4-site
// groups.
constexpr int kMeasThreads = 256;
__global__ void __launch_bounds__(kMeasThreads) k_xy_measure(const uint8_t* s, Lattice lat, uint32_t M,
                                                             unsigned long long* acc) {
  constexpr int kW = kMeasThreads / 32;
  __shared__ uint32_t hist[kW][kMaxAcc];
  const uint32_t H = M >> 1, nacc = H + 1 + M;
  for (uint32_t k = threadIdx.x; k < kW * kMaxAcc; k += blockDim.x) (&hist[0][0])[k] = 0;
  __syncthreads();
  uint32_t* h = hist[threadIdx.x >> 5];
  const uint64_t L = lat.L;
  auto fold = [&](uint32_t a, uint32_t b) -> uint32_t {
    const uint32_t t = a >= b ? a - b : a + M - b;
    return t < M - t ? t : M - t;
  };
  auto count4 = [&](uint32_t v, uint32_t vr, uint32_t vd, int nv) {
    for (int k = 0; k < nv; ++k) {
      const uint32_t a = (v >> (8 * k)) & 0xFFu;
      atomicAdd(&h[H + 1 + a], 1u);
      atomicAdd(&h[fold(a, (vr >> (8 * k)) & 0xFFu)], 1u);
      atomicAdd(&h[fold(a, (vd >> (8 * k)) & 0xFFu)], 1u);
    }
  };
  if ((L & 15u) == 0) {
    const uint64_t g16 = L >> 4;
    for (uint64_t y = blockIdx.x; y < L; y += gridDim.x) {
      const uint64_t yd = (y + 1 == L) ? 0 : y + 1;
      for (uint64_t gx = threadIdx.x; gx < g16; gx += blockDim.x) {
        const uint64_t x = gx * 16;
        const uint4 v = __ldcs(reinterpret_cast<const uint4*>(s + y * L + x));
        const uint4 d = *reinterpret_cast<const uint4*>(s + yd * L + x);
        const uint32_t nx = *reinterpret_cast<const uint32_t*>(s + y * L + ((x + 16 == L) ? 0 : x + 16));
        const uint32_t w4[5] = {v.x, v.y, v.z, v.w, nx};
        const uint32_t d4[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) count4(w4[k], __funnelshift_r(w4[k], w4[k + 1], 8), d4[k], 4);
      }
    }
  } else {
    const uint64_t groups = (L + 3) >> 2;
    for (uint64_t y = blockIdx.x; y < L; y += gridDim.x) {
      const uint64_t yd = (y + 1 == L) ? 0 : y + 1;
      for (uint64_t gx = threadIdx.x; gx < groups; gx += blockDim.x) {
        const uint64_t x = gx * 4;
        uint32_t v = 0, vr = 0, vd = 0;
        int nv = 4;
        if (lat.vec4) {
          v = *reinterpret_cast<const uint32_t*>(s + y * L + x);
          const uint64_t xn = (x + 4 == L) ? 0 : x + 4;
          vr = __funnelshift_r(v, *reinterpret_cast<const uint32_t*>(s + y * L + xn), 8);
          vd = *reinterpret_cast<const uint32_t*>(s + yd * L + x);
        } else {
          nv = (int)((L - x) < 4 ? (L - x) : 4);
          for (int k = 0; k < nv; ++k) {
            const uint64_t xk = x + k, xr = (xk + 1 == L) ? 0 : xk + 1;
            v |= (uint32_t)s[y * L + xk] << (8 * k);
            vr |= (uint32_t)s[y * L + xr] << (8 * k);
            vd |= (uint32_t)s[yd * L + xk] << (8 * k);
          }
        }
        count4(v, vr, vd, nv);
      }
    }
  }
  __syncthreads();
  for (uint32_t k = threadIdx.x; k < nacc; k += blockDim.x) {
    uint32_t t = 0;
#pragma unroll
    for (int w = 0; w < kW; ++w) t += hist[w][k];
    if (t) atomicAdd(&acc[k], (unsigned long long)t);
  }
}

// Files the accumulated observables as configuration ctl[0] and clears them.
__global__ void k_xy_commit(Bufs b, uint32_t nacc) {
  const unsigned long long s = b.ctl[0];
  unsigned long long* rec = b.ring + (s % b.ring_cap) * (1ull + nacc);
  if (threadIdx.x == 0) rec[0] = s;
  for (uint32_t k = threadIdx.x; k < nacc; k += blockDim.x) {
    rec[1 + k] = b.acc[k];
    b.acc[k] = 0ull;
  }
}

}  // namespace

struct sw_xy {
  sw_xy_params p;
  uint64_t L = 0, N = 0;
  uint32_t M = 0, H = 0, nacc = 0, label_bits = 32, th = 64, ring = 1024;
  Lattice lat{};
  cudaStream_t stream = nullptr;
  DeviceAllocator alloc{};
  std::vector<std::pair<void*, size_t>> blocks;
  uint64_t dev_bytes = 0;
  Bufs b{};
  uint64_t sweep = 0;
  uint64_t measured_from = 0;
  bool pending = true;
  bool measure_on = true;
  bool spins_invalid = false;
  int last_err = SW_OK;
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool, ev_used;  // 5 per profiled sweep
  double prof_ms[4] = {0, 0, 0, 0};
  uint64_t prof_launches[4] = {0, 0, 0, 0};
};

namespace {

int xfail(sw_xy* s, int code) {
  if (s && (code == SW_ERR_CUDA || code == SW_ERR_DEVICE || code == SW_ERR_TIMEOUT)) s->last_err = code;
  return code;
}

int xcuda(sw_xy* s) {
  cudaGetLastError();
  return xfail(s, SW_ERR_CUDA);
}

void* xtake(sw_xy* s, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  void* p = s->alloc.allocate(bytes);
  if (p) {
    s->blocks.emplace_back(p, bytes);
    s->dev_bytes += bytes;
  }
  return p;
}

void xrelease(sw_xy* s) {
  for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
  for (cudaEvent_t e : s->ev_used) cudaEventDestroy(e);
  s->ev_pool.clear();
  s->ev_used.clear();
  for (auto& kv : s->blocks) s->alloc.release(kv.first, kv.second);
  s->blocks.clear();
  s->dev_bytes = 0;
}

cudaEvent_t xevent(sw_xy* s) {
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

int xcheck(sw_xy* s) {
  uint32_t err = 0;
  cudaError_t e = cudaMemcpyAsync(&err, s->b.err, sizeof(err), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return xcuda(s);
  if (err & (kErrFind | kErrUnion | kErrLocal)) return xfail(s, SW_ERR_TIMEOUT);
  if (err) return xfail(s, SW_ERR_DEVICE);
  return SW_OK;
}

cudaError_t xlaunch_measure(sw_xy* s) {
  uint64_t blocks = s->L;  // one block per row, at most 16 per SM
  if (blocks > 152ull * 16) blocks = 152ull * 16;
  k_xy_measure<<<(unsigned)blocks, kMeasThreads, 0, s->stream>>>(s->b.spin, s->lat, s->M, s->b.acc);
  cudaError_t e = cudaGetLastError();
  if (e) return e;
  k_xy_commit<<<1, 128, 0, s->stream>>>(s->b, s->nacc);
  return cudaGetLastError();
}

int xmeasure_current(sw_xy* s) {
  if (!s->pending) return SW_OK;
  if (xlaunch_measure(s) != cudaSuccess) return xcuda(s);
  s->pending = false;
  return SW_OK;
}

cudaError_t xsweep_once(sw_xy* s, cudaEvent_t* ev) {
  const SingleSrc src{s->b, s->lat};
  cudaError_t e = s->label_bits == 64
                      ? sweep_th<uint64_t, SingleSrc, true>(s->th, src, s->lat.ntiles, s->stream, ev)
                      : sweep_th<uint32_t, SingleSrc, true>(s->th, src, s->lat.ntiles, s->stream, ev);
  if (e) return e;
  if (s->measure_on && (e = xlaunch_measure(s))) return e;
  if (ev) return cudaEventRecord(ev[4], s->stream);
  return cudaSuccess;
}

}  // namespace

extern "C" {

int sw_xy_thresholds(uint32_t M, double T, uint32_t* tt) {
  if (!tt || M < 2 || M > 256 || !(T > 0.0) || !isfinite(T)) return SW_ERR_INVAL;
  xy_table(M, T, tt);
  return SW_OK;
}

int sw_xy_create(const sw_xy_params* prm, sw_xy** out) {
  if (!prm || !out) return SW_ERR_INVAL;
  *out = nullptr;
  const uint64_t L = prm->L;
  if (L < 2 || L > (1ull << 20) || prm->M < 2 || prm->M > 256 || !(prm->T > 0.0) ||
      !isfinite(prm->T) || prm->init > SW_INIT_ZERO || prm->measure > 2)
    return SW_ERR_INVAL;
  const uint32_t lb = prm->label_bits ? prm->label_bits : (L <= 32768 ? 32u : 64u);
  if (lb != 32 && lb != 64) return SW_ERR_INVAL;
  if (lb == 32 && L * L > (1ull << 32)) return SW_ERR_INVAL;
  // the XY form of the labeller takes tiles of at most 64 rows
  const uint32_t th = pick_tile_h(L, prm->tile_h);
  if (th != 16 && th != 32 && th != 64 && th != 128) return SW_ERR_INVAL;

  sw_xy* s = new (std::nothrow) sw_xy();
  if (!s) return SW_ERR_NOMEM;
  s->p = *prm;
  s->L = L;
  s->N = L * L;
  s->M = prm->M;
  s->H = prm->M / 2;
  s->nacc = s->H + 1 + s->M;
  s->label_bits = lb;
  s->th = th;
  s->ring = prm->ring ? prm->ring : 1024u;
  s->lat = make_lattice(L, th);
  s->alloc = current_allocator();
  s->measure_on = prm->measure != 2;

  const uint64_t nt = s->lat.ntiles;
  const size_t ntt = (size_t)(s->H + 1) * (s->H + 1);
  const size_t ntri = (size_t)(s->H + 1) * (s->H + 2) / 2;  // lower triangle on the device
  const size_t rec = 1 + (size_t)s->nacc;
  Bufs& b = s->b;
  b.spin = (uint8_t*)xtake(s, s->N + 16);
  b.code = (uint16_t*)xtake(s, s->N * 2 + 16);
  b.bonds = nullptr;
  b.G = (uint64_t*)xtake(s, nt * open_cap(th) * 8);
  b.edge = (uint16_t*)xtake(s, nt * edge_u16(th) * 2);
  b.ebits = (uint32_t*)xtake(s, nt * bit_words(th) * 4);
  b.ocnt = (uint32_t*)xtake(s, nt * 4);
  b.nso = (uint8_t*)xtake(s, nt * open_cap(th));
  b.acc = (unsigned long long*)xtake(s, 8 * kMaxAcc);
  b.ring = (unsigned long long*)xtake(s, (size_t)s->ring * rec * 8);
  b.ctl = (unsigned long long*)xtake(s, 64);
  b.err = (uint32_t*)xtake(s, 64);
  uint32_t* tt = (uint32_t*)xtake(s, ntri * 4);
  if (!b.spin || !b.code || !b.G || !b.edge || !b.ebits || !b.ocnt || !b.nso || !b.acc ||
      !b.ring || !b.ctl || !b.err || !tt) {
    xrelease(s);
    delete s;
    return SW_ERR_NOMEM;
  }
  b.seed = prm->seed;
  set_round_keys(b);
  b.thr = 0;
  b.q = 2;  // a cluster's "state" is its reflection coin
  b.ring_cap = s->ring;
  b.measure = 0;  // the XY measurement runs after the reflections
  b.M = s->M;
  b.tt = tt;

  std::vector<uint32_t> host_tt(ntt), host_tri(ntri);
  xy_table(s->M, prm->T, host_tt.data());
  for (uint32_t c = 0; c <= s->H; ++c)
    for (uint32_t d = 0; d <= c; ++d) host_tri[c * (c + 1) / 2 + d] = host_tt[c * (s->H + 1) + d];
  cudaError_t e = cudaMemcpyAsync(tt, host_tri.data(), ntri * 4, cudaMemcpyHostToDevice, s->stream);
  if (!e) e = cudaStreamSynchronize(s->stream);  // host_tri is a stack-lifetime buffer
  if (!e) e = cudaMemsetAsync(b.G, 0, nt * open_cap(th) * 8, s->stream);
  if (!e) e = cudaMemsetAsync(b.acc, 0, 8 * kMaxAcc, s->stream);
  if (!e) e = cudaMemsetAsync(b.ring, 0xFF, (size_t)s->ring * rec * 8, s->stream);
  if (!e) e = cudaMemsetAsync(b.ctl, 0, 64, s->stream);
  if (!e) e = cudaMemsetAsync(b.err, 0, 64, s->stream);
  if (!e) e = cudaMemsetAsync(b.ocnt, 0, nt * 4, s->stream);
  if (!e) e = launch_init(b.spin, s->N, s->M, prm->seed, prm->init, s->stream);
  s->pending = true;
  if (!e && s->measure_on) {
    e = xlaunch_measure(s);
    s->pending = false;
  }
  if (!e) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    xrelease(s);
    delete s;
    return SW_ERR_CUDA;
  }
  *out = s;
  return SW_OK;
}

void sw_xy_destroy(sw_xy* s) {
  if (!s) return;
  cudaStreamSynchronize(s->stream);
  xrelease(s);
  delete s;
}

int sw_xy_bind_stream(sw_xy* s, void* stream) {
  if (!s) return SW_ERR_INVAL;
  s->stream = (cudaStream_t)stream;
  return SW_OK;
}

int sw_xy_sweep(sw_xy* s, uint64_t n) {
  if (!s) return SW_ERR_INVAL;
  if (s->last_err) return s->last_err;
  if (s->spins_invalid) return SW_ERR_STATE;
  for (uint64_t k = 0; k < n; ++k) {
    cudaEvent_t ev[5];
    cudaEvent_t* evp = nullptr;
    if (s->profiling) {
      for (int j = 0; j < 5; ++j) {
        ev[j] = xevent(s);
        if (!ev[j]) return xfail(s, SW_ERR_CUDA);
        s->ev_used.push_back(ev[j]);
      }
      evp = ev;
    }
    if (xsweep_once(s, evp) != cudaSuccess) return xcuda(s);
  }
  if (n) {
    s->sweep += n;
    s->pending = !s->measure_on;
  }
  return SW_OK;
}

int sw_xy_sync(sw_xy* s) {
  if (!s) return SW_ERR_INVAL;
  if (s->last_err) return s->last_err;
  return xcheck(s);
}

int sw_xy_series(sw_xy* s, uint64_t first, uint64_t count, uint64_t* D, uint64_t* n) {
  if (!s) return SW_ERR_INVAL;
  if (s->last_err) return s->last_err;
  if (count == 0) return SW_OK;
  const uint64_t cur = s->sweep;
  const uint64_t last = first + count - 1;
  if (last < first || last > cur) return SW_ERR_RANGE;
  uint64_t oldest = s->measured_from;
  if (cur + 1 > s->ring && cur + 1 - s->ring > oldest) oldest = cur + 1 - s->ring;
  if (first < oldest) return SW_ERR_RANGE;
  if (!s->measure_on && !(first == cur && count == 1)) return SW_ERR_RANGE;
  if (last == cur) {
    int rc = xmeasure_current(s);
    if (rc) return rc;
  }
  const size_t rec = 1 + (size_t)s->nacc;
  std::vector<unsigned long long> host(count * rec);
  uint64_t done = 0;
  while (done < count) {
    const uint64_t slot = (first + done) % s->ring;
    uint64_t run = s->ring - slot;
    if (run > count - done) run = count - done;
    if (cudaMemcpyAsync(host.data() + done * rec, s->b.ring + slot * rec, run * rec * 8,
                        cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
      return xcuda(s);
    done += run;
  }
  int rc = xcheck(s);
  if (rc) return rc;
  for (uint64_t k = 0; k < count; ++k) {
    const unsigned long long* r = host.data() + k * rec;
    if (r[0] != first + k) return SW_ERR_RANGE;
    if (D)
      for (uint32_t d = 0; d <= s->H; ++d) D[k * (s->H + 1) + d] = r[1 + d];
    if (n)
      for (uint32_t j = 0; j < s->M; ++j) n[k * s->M + j] = r[2 + s->H + j];
  }
  return SW_OK;
}

int sw_xy_spins(sw_xy* s, uint8_t* dst, uint64_t n, int dst_on_device) {
  if (!s || !dst || n != s->N) return SW_ERR_INVAL;
  if (s->last_err) return s->last_err;
  if (cudaMemcpyAsync(dst, s->b.spin, s->N, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                      s->stream) != cudaSuccess)
    return xcuda(s);
  if (!dst_on_device) return xcheck(s);
  return SW_OK;
}

int sw_xy_set_spins(sw_xy* s, const uint8_t* src, uint64_t n, int src_on_device) {
  if (!s || !src || n != s->N) return SW_ERR_INVAL;
  if (s->last_err) return s->last_err;
  cudaError_t e = cudaMemcpyAsync(s->b.spin, src, s->N,
                                  src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->stream);
  uint32_t* bad = reinterpret_cast<uint32_t*>(s->b.ctl + 3);
  if (!e) e = cudaMemsetAsync(bad, 0, 4, s->stream);
  if (!e) {
    uint64_t blocks = (s->N / 4 + 255) / 256;
    if (blocks > 152ull * 8) blocks = 152ull * 8;
    if (blocks == 0) blocks = 1;
    k_check_spins<<<(unsigned)blocks, 256, 0, s->stream>>>(s->b.spin, s->N, s->M, bad);
    e = cudaGetLastError();
  }
  uint32_t hbad = 0;
  if (!e) e = cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, s->stream);
  if (!e) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return xcuda(s);
  s->measured_from = s->sweep;
  s->pending = true;
  if (hbad) {
    s->spins_invalid = true;
    return SW_ERR_INVAL;
  }
  s->spins_invalid = false;
  if (s->measure_on) return xmeasure_current(s);
  return SW_OK;
}

int sw_xy_get_sweep(const sw_xy* s, uint64_t* sweep) {
  if (!s || !sweep) return SW_ERR_INVAL;
  *sweep = s->sweep;
  return SW_OK;
}

int sw_xy_profile(sw_xy* s, int enable) {
  if (!s) return SW_ERR_INVAL;
  if (enable) {
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return xcuda(s);
    for (cudaEvent_t ev : s->ev_used) s->ev_pool.push_back(ev);
    s->ev_used.clear();
    for (int k = 0; k < 4; ++k) {
      s->prof_ms[k] = 0;
      s->prof_launches[k] = 0;
    }
  }
  s->profiling = enable != 0;
  return SW_OK;
}

int sw_xy_profile_read(sw_xy* s, double* ms, uint64_t* launches, int nphase) {
  if (!s || nphase < 0 || nphase > 4) return SW_ERR_INVAL;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return xcuda(s);
  for (size_t k = 0; k + 4 < s->ev_used.size(); k += 5) {
    for (int ph = 0; ph < 4; ++ph) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, s->ev_used[k + ph], s->ev_used[k + ph + 1]) != cudaSuccess)
        return xcuda(s);
      s->prof_ms[ph] += t;
      s->prof_launches[ph] += 1;
    }
  }
  for (cudaEvent_t e : s->ev_used) s->ev_pool.push_back(e);
  s->ev_used.clear();
  for (int k = 0; k < nphase; ++k) {
    if (ms) ms[k] = s->prof_ms[k];
    if (launches) launches[k] = s->prof_launches[k];
  }
  return SW_OK;
}

int sw_xy_last_error(const sw_xy* s) { return s ? s->last_err : SW_ERR_INVAL; }

}  // extern "C"
