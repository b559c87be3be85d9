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
    for i in range(0, n, n // 4096):
        assert list(oracle.philox(inp[i, :4], inp[i, 4:])) == list(ref[i])
