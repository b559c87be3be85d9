// sw_mlp.cu -- the surrogate network's kernels and C ABI (include/sw.h,
// sw_mlp_*): a 3 -> 64 -> 64 -> 64 -> 4 tanh MLP with bfloat16 weights and
// fp32 accumulation, trained on the GPU by its own forward, loss, backward
// and Adam kernels.  It maps (q, log2 L, T/T_c) to standardised (energy,
// |M|, log chi, U4) and only ever places temperatures; it never touches the
// Markov chain.  Not part of the paper.
//
// Parameter layout (flat, 8836 values): W1[64][3], b1[64], W2[64][64], b2[64],
// W3[64][64], b3[64], W4[4][64], b4[4].  Every parameter and every layer
// input is rounded to bfloat16 before use; products are accumulated in fp32.
// The network is tiny (4.5 MFLOP per 512-row forward), so these are CUDA-core
// kernels with the weights broadcast from shared memory: one thread per row
// for the forward and the row-wise backward, one thread per parameter for
// the weight gradients (a sum over rows) and the update.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>

#include "../../include/sw.h"
#include "sw_internal.h"

namespace swgb {
namespace mlp {

constexpr int kH = 64, kIn = 3, kOut = 4;
constexpr int kW1 = 0, kB1 = kW1 + kH * kIn, kW2 = kB1 + kH, kB2 = kW2 + kH * kH, kW3 = kB2 + kH,
              kB3 = kW3 + kH * kH, kW4 = kB3 + kH, kB4 = kW4 + kOut * kH, kNP = kB4 + kOut;
static_assert(kNP == 8836, "parameter count");
constexpr int kRowThreads = 128;
constexpr int kAct = 3 * kH;  // saved activations per row: a1, a2, a3

__device__ __forceinline__ float rbf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ void load_weights(float* w, const __nv_bfloat16* P) {
  for (int i = threadIdx.x; i < kNP; i += blockDim.x) w[i] = __bfloat162float(P[i]);
}

// Forward pass, one thread per row.  A (optional) receives a1, a2, a3.
__global__ void __launch_bounds__(kRowThreads) k_mlp_forward(const __nv_bfloat16* __restrict__ P,
                                                             const float* __restrict__ X, uint32_t B,
                                                             float* __restrict__ A, float* __restrict__ Y) {
  extern __shared__ float w[];
  load_weights(w, P);
  __syncthreads();
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  float in[kH], out[kH];
  const float x0 = rbf(X[3 * b]), x1 = rbf(X[3 * b + 1]), x2 = rbf(X[3 * b + 2]);
#pragma unroll
  for (int i = 0; i < kH; ++i) {
    float z = w[kW1 + 3 * i] * x0;
    z = fmaf(w[kW1 + 3 * i + 1], x1, z);
    z = fmaf(w[kW1 + 3 * i + 2], x2, z);
    out[i] = tanhf(z + w[kB1 + i]);
  }
  if (A)
#pragma unroll
    for (int i = 0; i < kH; ++i) A[(size_t)b * kAct + i] = out[i];
#pragma unroll
  for (int i = 0; i < kH; ++i) in[i] = rbf(out[i]);
#pragma unroll 4
  for (int i = 0; i < kH; ++i) {
    float z = 0.f;
#pragma unroll
    for (int j = 0; j < kH; ++j) z = fmaf(w[kW2 + kH * i + j], in[j], z);
    out[i] = tanhf(z + w[kB2 + i]);
  }
  if (A)
#pragma unroll
    for (int i = 0; i < kH; ++i) A[(size_t)b * kAct + kH + i] = out[i];
#pragma unroll
  for (int i = 0; i < kH; ++i) in[i] = rbf(out[i]);
#pragma unroll 4
  for (int i = 0; i < kH; ++i) {
    float z = 0.f;
#pragma unroll
    for (int j = 0; j < kH; ++j) z = fmaf(w[kW3 + kH * i + j], in[j], z);
    out[i] = tanhf(z + w[kB3 + i]);
  }
  if (A)
#pragma unroll
    for (int i = 0; i < kH; ++i) A[(size_t)b * kAct + 2 * kH + i] = out[i];
#pragma unroll
  for (int i = 0; i < kH; ++i) in[i] = rbf(out[i]);
#pragma unroll
  for (int k = 0; k < kOut; ++k) {
    float z = 0.f;
#pragma unroll
    for (int j = 0; j < kH; ++j) z = fmaf(w[kW4 + kH * k + j], in[j], z);
    Y[4 * b + k] = z + w[kB4 + k];
  }
}

// Masked mean-squared error and its gradient with respect to the outputs.
__global__ void __launch_bounds__(256) k_mlp_loss(const float* __restrict__ Y, const float* __restrict__ Tg,
                                                  const float* __restrict__ mask, uint32_t B,
                                                  float* __restrict__ dY, float* __restrict__ loss) {
  __shared__ float part[8];
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (b < B) {
    const float scale = 2.f / (4.f * (float)B);
#pragma unroll
    for (int k = 0; k < kOut; ++k) {
      const float m = mask ? mask[4 * b + k] : 1.f;
      const float d = Y[4 * b + k] - Tg[4 * b + k];
      l = fmaf(m * d, d, l);
      dY[4 * b + k] = scale * m * d;
    }
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xFFFFFFFFu, l, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = l;
  __syncthreads();
  if (threadIdx.x == 0 && loss) {
    float s = 0.f;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += part[k];
    atomicAdd(loss, s / (4.f * (float)B));
  }
}

// Row-wise backward: D receives dz1, dz2, dz3 of every row.
__global__ void __launch_bounds__(kRowThreads) k_mlp_backward(const __nv_bfloat16* __restrict__ P,
                                                              const float* __restrict__ A,
                                                              const float* __restrict__ dY, uint32_t B,
                                                              float* __restrict__ D) {
  extern __shared__ float w[];
  load_weights(w, P);
  __syncthreads();
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const float* a = A + (size_t)b * kAct;
  float* d = D + (size_t)b * kAct;
  float cur[kH], nxt[kH];
  const float g0 = dY[4 * b], g1 = dY[4 * b + 1], g2 = dY[4 * b + 2], g3 = dY[4 * b + 3];
#pragma unroll
  for (int i = 0; i < kH; ++i) {
    float s = w[kW4 + i] * g0;
    s = fmaf(w[kW4 + kH + i], g1, s);
    s = fmaf(w[kW4 + 2 * kH + i], g2, s);
    s = fmaf(w[kW4 + 3 * kH + i], g3, s);
    const float a3 = a[2 * kH + i];
    cur[i] = s * (1.f - a3 * a3);  // dz3
    d[2 * kH + i] = cur[i];
  }
#pragma unroll 4
  for (int i = 0; i < kH; ++i) {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kH; ++j) s = fmaf(w[kW3 + kH * j + i], cur[j], s);
    const float a2 = a[kH + i];
    nxt[i] = s * (1.f - a2 * a2);  // dz2
  }
#pragma unroll
  for (int i = 0; i < kH; ++i) {
    d[kH + i] = nxt[i];
    cur[i] = nxt[i];
  }
#pragma unroll 4
  for (int i = 0; i < kH; ++i) {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kH; ++j) s = fmaf(w[kW2 + kH * j + i], cur[j], s);
    const float a1 = a[i];
    d[i] = s * (1.f - a1 * a1);  // dz1
  }
}

// Weight gradients: one thread per parameter, summing over the rows.
__global__ void __launch_bounds__(256) k_mlp_wgrad(const float* __restrict__ X, const float* __restrict__ A,
                                                   const float* __restrict__ D, const float* __restrict__ dY,
                                                   uint32_t B, float* __restrict__ G) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kNP) return;
  float s = 0.f;
  if (p < kB1) {  // W1[i][j] = sum dz1[i] r(x[j])
    const int i = p / kIn, j = p % kIn;
    for (uint32_t b = 0; b < B; ++b) s = fmaf(D[(size_t)b * kAct + i], rbf(X[3 * b + j]), s);
  } else if (p < kW2) {
    const int i = p - kB1;
    for (uint32_t b = 0; b < B; ++b) s += D[(size_t)b * kAct + i];
  } else if (p < kB2) {  // W2[i][j] = sum dz2[i] r(a1[j])
    const int i = (p - kW2) / kH, j = (p - kW2) % kH;
    for (uint32_t b = 0; b < B; ++b) s = fmaf(D[(size_t)b * kAct + kH + i], rbf(A[(size_t)b * kAct + j]), s);
  } else if (p < kW3) {
    const int i = p - kB2;
    for (uint32_t b = 0; b < B; ++b) s += D[(size_t)b * kAct + kH + i];
  } else if (p < kB3) {  // W3[i][j] = sum dz3[i] r(a2[j])
    const int i = (p - kW3) / kH, j = (p - kW3) % kH;
    for (uint32_t b = 0; b < B; ++b)
      s = fmaf(D[(size_t)b * kAct + 2 * kH + i], rbf(A[(size_t)b * kAct + kH + j]), s);
  } else if (p < kW4) {
    const int i = p - kB3;
    for (uint32_t b = 0; b < B; ++b) s += D[(size_t)b * kAct + 2 * kH + i];
  } else if (p < kB4) {  // W4[k][j] = sum dy[k] r(a3[j])
    const int k = (p - kW4) / kH, j = (p - kW4) % kH;
    for (uint32_t b = 0; b < B; ++b) s = fmaf(dY[4 * b + k], rbf(A[(size_t)b * kAct + 2 * kH + j]), s);
  } else {
    const int k = p - kB4;
    for (uint32_t b = 0; b < B; ++b) s += dY[4 * b + k];
  }
  G[p] = s;
}

// Adam with bias correction on the fp32 master weights; refreshes the
// bfloat16 copy the other kernels read.
__global__ void __launch_bounds__(256) k_mlp_adam(float* __restrict__ master, const float* __restrict__ G,
                                                  float* __restrict__ m, float* __restrict__ v,
                                                  __nv_bfloat16* __restrict__ P, float lr, float c1, float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kNP) return;
  constexpr float kB1c = 0.9f, kB2c = 0.999f, kEps = 1e-8f;
  const float g = G[p];
  const float mm = kB1c * m[p] + (1.f - kB1c) * g;
  const float vv = kB2c * v[p] + (1.f - kB2c) * g * g;
  m[p] = mm;
  v[p] = vv;
  const float upd = lr * (mm / c1) / (sqrtf(vv / c2) + kEps);
  const float w = master[p] - upd;
  master[p] = w;
  P[p] = __float2bfloat16_rn(w);
}

__global__ void k_mlp_to_bf16(const float* __restrict__ master, __nv_bfloat16* __restrict__ P) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kNP) P[p] = __float2bfloat16_rn(master[p]);
}

}  // namespace mlp
}  // namespace swgb

using namespace swgb;
using namespace swgb::mlp;

struct sw_mlp {
  DeviceAllocator alloc{};
  cudaStream_t stream = nullptr;
  float* master = nullptr;   // fp32 master weights
  float* m = nullptr;        // Adam moments
  float* v = nullptr;
  __nv_bfloat16* P = nullptr;  // bfloat16 copy used by the kernels
  float* G = nullptr;        // gradient
  float* scratch = nullptr;  // per-row activations, deltas, outputs
  uint32_t cap = 0;          // rows the scratch holds
  size_t scratch_bytes = 0;
  uint64_t step = 0;
  void* block = nullptr;
  size_t block_bytes = 0;
};

namespace {

constexpr size_t kFixed = 4 * sizeof(float) * kNP + sizeof(__nv_bfloat16) * kNP + 1024;

int ensure_rows(sw_mlp* h, uint32_t B) {
  if (B <= h->cap) return SW_OK;
  const size_t per_row = (2 * kAct + 2 * kOut) * sizeof(float);
  const size_t bytes = per_row * (size_t)B + 256;
  void* p = h->alloc.allocate(bytes);
  if (!p) return SW_ERR_NOMEM;
  if (h->scratch) {
    cudaStreamSynchronize(h->stream);
    h->alloc.release(h->scratch, h->scratch_bytes);
  }
  h->scratch = (float*)p;
  h->scratch_bytes = bytes;
  h->cap = B;
  return SW_OK;
}

int run_forward(sw_mlp* h, const float* X, uint32_t B, float* A, float* Y) {
  const size_t smem = sizeof(float) * kNP;
  static bool configured = false;
  if (!configured) {
    if (cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ||
        cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) {
      cudaGetLastError();
      return SW_ERR_CUDA;
    }
    configured = true;
  }
  const uint32_t blocks = (B + kRowThreads - 1) / kRowThreads;
  k_mlp_forward<<<blocks, kRowThreads, smem, h->stream>>>(h->P, X, B, A, Y);
  return cudaGetLastError() == cudaSuccess ? SW_OK : SW_ERR_CUDA;
}

// Forward with saved activations, loss, backward, weight gradients into h->G.
int run_gradients(sw_mlp* h, const float* X, const float* Tg, const float* mask, uint32_t B, float* loss) {
  int rc = ensure_rows(h, B);
  if (rc) return rc;
  float* A = h->scratch;
  float* D = A + (size_t)h->cap * kAct;
  float* Y = D + (size_t)h->cap * kAct;
  float* dY = Y + (size_t)h->cap * kOut;
  rc = run_forward(h, X, B, A, Y);
  if (rc) return rc;
  if (loss && cudaMemsetAsync(loss, 0, sizeof(float), h->stream)) return SW_ERR_CUDA;
  k_mlp_loss<<<(B + 255) / 256, 256, 0, h->stream>>>(Y, Tg, mask, B, dY, loss);
  k_mlp_backward<<<(B + kRowThreads - 1) / kRowThreads, kRowThreads, sizeof(float) * kNP, h->stream>>>(
      h->P, A, dY, B, D);
  k_mlp_wgrad<<<(kNP + 255) / 256, 256, 0, h->stream>>>(X, A, D, dY, B, h->G);
  return cudaGetLastError() == cudaSuccess ? SW_OK : SW_ERR_CUDA;
}

}  // namespace

extern "C" {

int sw_mlp_create(const float* init, sw_mlp** out) {
  if (!init || !out) return SW_ERR_INVAL;
  *out = nullptr;
  sw_mlp* h = new (std::nothrow) sw_mlp();
  if (!h) return SW_ERR_NOMEM;
  h->alloc = current_allocator();
  h->block_bytes = kFixed;
  h->block = h->alloc.allocate(kFixed);
  if (!h->block) {
    delete h;
    return SW_ERR_NOMEM;
  }
  float* f = (float*)h->block;
  h->master = f;
  h->m = f + kNP;
  h->v = f + 2 * kNP;
  h->G = f + 3 * kNP;
  h->P = (__nv_bfloat16*)(f + 4 * kNP);
  cudaError_t e = cudaMemcpyAsync(h->master, init, sizeof(float) * kNP, cudaMemcpyHostToDevice, h->stream);
  if (!e) e = cudaMemsetAsync(h->m, 0, 2 * sizeof(float) * kNP, h->stream);
  if (!e) {
    k_mlp_to_bf16<<<(kNP + 255) / 256, 256, 0, h->stream>>>(h->master, h->P);
    e = cudaGetLastError();
  }
  if (!e) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    h->alloc.release(h->block, h->block_bytes);
    delete h;
    return SW_ERR_CUDA;
  }
  *out = h;
  return SW_OK;
}

void sw_mlp_destroy(sw_mlp* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  if (h->scratch) h->alloc.release(h->scratch, h->scratch_bytes);
  h->alloc.release(h->block, h->block_bytes);
  delete h;
}

int sw_mlp_bind_stream(sw_mlp* h, void* stream) {
  if (!h) return SW_ERR_INVAL;
  h->stream = (cudaStream_t)stream;
  return SW_OK;
}

int sw_mlp_forward(sw_mlp* h, const float* X, uint32_t B, float* Y) {
  if (!h || !X || !Y || B == 0) return SW_ERR_INVAL;
  return run_forward(h, X, B, nullptr, Y);
}

int sw_mlp_predict(sw_mlp* h, const float* X, uint32_t B, float* Y) { return sw_mlp_forward(h, X, B, Y); }

int sw_mlp_gradients(sw_mlp* h, const float* X, const float* Tg, const float* mask, uint32_t B,
                     float* grad, float* loss) {
  if (!h || !X || !Tg || !grad || B == 0) return SW_ERR_INVAL;
  int rc = run_gradients(h, X, Tg, mask, B, loss);
  if (rc) return rc;
  return cudaMemcpyAsync(grad, h->G, sizeof(float) * kNP, cudaMemcpyDeviceToDevice, h->stream) == cudaSuccess
             ? SW_OK
             : SW_ERR_CUDA;
}

int sw_mlp_train_step(sw_mlp* h, const float* X, const float* Tg, const float* mask, uint32_t B, float lr,
                      float* loss) {
  if (!h || !X || !Tg || B == 0 || !(lr >= 0.f)) return SW_ERR_INVAL;
  int rc = run_gradients(h, X, Tg, mask, B, loss);
  if (rc) return rc;
  h->step += 1;
  const float c1 = 1.f - powf(0.9f, (float)h->step), c2 = 1.f - powf(0.999f, (float)h->step);
  k_mlp_adam<<<(kNP + 255) / 256, 256, 0, h->stream>>>(h->master, h->G, h->m, h->v, h->P, lr, c1, c2);
  return cudaGetLastError() == cudaSuccess ? SW_OK : SW_ERR_CUDA;
}

int sw_mlp_get_params(sw_mlp* h, float* master, uint16_t* bf16) {
  if (!h) return SW_ERR_INVAL;
  cudaError_t e = cudaSuccess;
  if (master) e = cudaMemcpyAsync(master, h->master, sizeof(float) * kNP, cudaMemcpyDeviceToHost, h->stream);
  if (!e && bf16) e = cudaMemcpyAsync(bf16, h->P, 2 * kNP, cudaMemcpyDeviceToHost, h->stream);
  if (!e) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? SW_OK : SW_ERR_CUDA;
}

int sw_mlp_set_params(sw_mlp* h, const float* master) {
  if (!h || !master) return SW_ERR_INVAL;
  cudaError_t e = cudaMemcpyAsync(h->master, master, sizeof(float) * kNP, cudaMemcpyHostToDevice, h->stream);
  if (!e) e = cudaMemsetAsync(h->m, 0, 2 * sizeof(float) * kNP, h->stream);
  if (!e) {
    k_mlp_to_bf16<<<(kNP + 255) / 256, 256, 0, h->stream>>>(h->master, h->P);
    e = cudaGetLastError();
  }
  if (!e) e = cudaStreamSynchronize(h->stream);
  h->step = 0;
  return e == cudaSuccess ? SW_OK : SW_ERR_CUDA;
}

}  // extern "C"
