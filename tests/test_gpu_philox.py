"""The library's device Philox4x32-10 (csrc/philox.cuh, both the keyed form
and the precomputed-round-key form) against cuRAND's device Philox4x32-10
routine, called in a test kernel compiled here, and against the CPU oracle:
an independent implementation of the published generator on each side."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_1208_2080_gb300", "csrc")

KERNEL = r'''
#include <cuda_runtime.h>
#include <curand_kernel.h>
#include <stdint.h>
#include "philox.cuh"
using namespace swgb;
__global__ void k(const uint32_t* in, uint32_t* ours, uint32_t* ours_rk, uint32_t* lib, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t* a = in + 6 * i;
  Words4 w = philox4x32_10(a[0], a[1], a[2], a[3], a[4], a[5]);
  uint32_t rk[20];
  uint32_t k0 = a[4], k1 = a[5];
  for (int r = 0; r < 10; ++r) { rk[2 * r] = k0; rk[2 * r + 1] = k1; k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
  Words4 v = philox4x32_10_rk(a[0], a[1], a[2], a[3], rk);
  uint4 c = curand_Philox4x32_10(make_uint4(a[0], a[1], a[2], a[3]), make_uint2(a[4], a[5]));
  ours[4 * i] = w.x; ours[4 * i + 1] = w.y; ours[4 * i + 2] = w.z; ours[4 * i + 3] = w.w;
  ours_rk[4 * i] = v.x; ours_rk[4 * i + 1] = v.y; ours_rk[4 * i + 2] = v.z; ours_rk[4 * i + 3] = v.w;
  lib[4 * i] = c.x; lib[4 * i + 1] = c.y; lib[4 * i + 2] = c.z; lib[4 * i + 3] = c.w;
}
// Counter and key of test i, spread over all 32-bit words by a 64-bit mixer
// (SplitMix64's finaliser) of i and i + 2^40.
__device__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
// Mismatches of both device forms against cuRAND over tests 0 .. n-1.
__global__ void kcount(unsigned long long n, unsigned long long* bad) {
  const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t a = mix64(i), b = mix64(i + (1ull << 40)), c = mix64(i + (2ull << 40));
  const uint32_t c0 = (uint32_t)a, c1 = (uint32_t)(a >> 32), c2 = (uint32_t)b, c3 = (uint32_t)(b >> 32);
  const uint32_t k0 = (uint32_t)c, k1 = (uint32_t)(c >> 32);
  Words4 w = philox4x32_10(c0, c1, c2, c3, k0, k1);
  uint32_t rk[20];
  uint32_t q0 = k0, q1 = k1;
  for (int r = 0; r < 10; ++r) { rk[2 * r] = q0; rk[2 * r + 1] = q1; q0 += 0x9E3779B9u; q1 += 0xBB67AE85u; }
  Words4 v = philox4x32_10_rk(c0, c1, c2, c3, rk);
  uint4 e = curand_Philox4x32_10(make_uint4(c0, c1, c2, c3), make_uint2(k0, k1));
  if (w.x != e.x || w.y != e.y || w.z != e.z || w.w != e.w ||
      v.x != e.x || v.y != e.y || v.z != e.z || v.w != e.w)
    atomicAdd(bad, 1ull);
}
extern "C" int count(unsigned long long n, unsigned long long* bad) {
  kcount<<<(unsigned)((n + 255) / 256), 256>>>(n, bad);
  return (int)cudaDeviceSynchronize();
}
extern "C" int run(const uint32_t* in, uint32_t* ours, uint32_t* ours_rk, uint32_t* lib, int n) {
  k<<<(n + 255) / 256, 256>>>(in, ours, ours_rk, lib, n);
  return (int)cudaDeviceSynchronize();
}
'''


def test_device_philox_matches_curand_and_the_oracle(tmp_path):
    import torch
    src = tmp_path / "philox_check.cu"
    src.write_text(KERNEL)
    so = tmp_path / "philox_check.so"
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                    "-shared", "-Xcompiler", "-fPIC", "-I", CSRC, "-o", str(so), str(src)],
                   check=True)
    lib = ctypes.CDLL(str(so))
    rng = np.random.default_rng(2024)
    n = 1 << 20
    inp = rng.integers(0, 2 ** 32, size=(n, 6), dtype=np.uint64).astype(np.uint32)
    inp[:16] = 0
    inp[16:32, :4] = 0xFFFFFFFF
    d_in = torch.from_numpy(inp.view(np.int32).reshape(-1).copy()).cuda()
    outs = [torch.empty(4 * n, dtype=torch.int32, device="cuda") for _ in range(3)]
    rc = lib.run(ctypes.c_void_p(d_in.data_ptr()), *[ctypes.c_void_p(o.data_ptr()) for o in outs],
                 ctypes.c_int(n))
    assert rc == 0
    ours, ours_rk, ref = [o.cpu().numpy().view(np.uint32).reshape(n, 4) for o in outs]
    assert np.array_equal(ours, ref)
    assert np.array_equal(ours_rk, ref)
    # the CPU oracle's independent copy on every one of the 2^20 inputs
    assert np.array_equal(oracle.philox_many(inp), ref)
    # 10^8 further (counter, key) pairs, derived and compared on the device
    bad = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert lib.count(ctypes.c_ulonglong(10 ** 8), ctypes.c_void_p(bad.data_ptr())) == 0
    assert int(bad.item()) == 0
