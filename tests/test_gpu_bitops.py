"""Unit tests of the device bit tricks of the labellers against their plain
definitions, in a test kernel compiled here: the bond-threshold mask (PTX
carry chains) at the edge words (w == thr, thr - 1, thr + 1, 0, 2^32 - 1),
the zero-byte mask, the run-start lookups of 32- and 64-site masks, and the
even-bit compaction of packed bond bytes."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_1208_2080_gb300", "csrc")

KERNEL = r'''
#include <cuda_runtime.h>
#include <stdint.h>
#include "sw_label.cuh"
using namespace swgb;
// lt: per test i, words w[4i..4i+3] against thr[i]
__global__ void klt(const uint32_t* w, const uint32_t* thr, uint32_t* out, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t v[4] = {w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]};
  out[i] = lt_mask4(v, thr[i]);
}
__global__ void kzb(const uint32_t* x, uint32_t* out, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = zero_bytes4(x[i]);
}
// run starts: test i = (mask, bit, column base, carry)
__global__ void krs(const uint32_t* a, uint32_t* out, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = run_start(a[4 * i], (int)a[4 * i + 1], a[4 * i + 2], a[4 * i + 3]);
}
__global__ void krs64(const uint32_t* a, uint32_t* out, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const uint64_t m = (uint64_t)a[5 * i] | ((uint64_t)a[5 * i + 1] << 32);
    out[i] = run_start64(m, a[5 * i + 2], a[5 * i + 3], a[5 * i + 4]);
  }
}
__global__ void keb(const uint32_t* x, uint32_t* out, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = even_bits(x[i]);
}
extern "C" int run_lt(const uint32_t* w, const uint32_t* t, uint32_t* o, int n) {
  klt<<<(n + 255) / 256, 256>>>(w, t, o, n); return (int)cudaDeviceSynchronize(); }
extern "C" int run_zb(const uint32_t* x, uint32_t* o, int n) {
  kzb<<<(n + 255) / 256, 256>>>(x, o, n); return (int)cudaDeviceSynchronize(); }
extern "C" int run_rs(const uint32_t* a, uint32_t* o, int n) {
  krs<<<(n + 255) / 256, 256>>>(a, o, n); return (int)cudaDeviceSynchronize(); }
extern "C" int run_rs64(const uint32_t* a, uint32_t* o, int n) {
  krs64<<<(n + 255) / 256, 256>>>(a, o, n); return (int)cudaDeviceSynchronize(); }
extern "C" int run_eb(const uint32_t* x, uint32_t* o, int n) {
  keb<<<(n + 255) / 256, 256>>>(x, o, n); return (int)cudaDeviceSynchronize(); }
'''


@pytest.fixture(scope="module")
def dev(tmp_path_factory):
    import torch
    d = tmp_path_factory.mktemp("bitops")
    src = d / "bitops.cu"
    src.write_text(KERNEL)
    so = d / "bitops.so"
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                    "--expt-relaxed-constexpr", "-shared", "-Xcompiler", "-fPIC", "-I", CSRC,
                    "-o", str(so), str(src)], check=True)
    lib = ctypes.CDLL(str(so))

    def call(name, arrays, n_out):
        ins = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()
               for a in arrays]
        out = torch.zeros(n_out, dtype=torch.int32, device="cuda")
        args = [ctypes.c_void_p(t.data_ptr()) for t in ins] + [ctypes.c_void_p(out.data_ptr())]
        assert getattr(lib, name)(*args, ctypes.c_int(n_out)) == 0
        return out.cpu().numpy().view(np.uint32)
    return call


EDGE = np.array([0, 1, 2, 0x7FFFFFFF, 0x80000000, 0x80000001, 0xFFFFFFFE, 0xFFFFFFFF],
                dtype=np.uint64)


def test_threshold_mask_at_edge_words(dev):
    rng = np.random.default_rng(5)
    thrs = np.concatenate([EDGE, rng.integers(0, 2**32, 56, dtype=np.uint64)])
    ws, ts = [], []
    for t in thrs:
        t = int(t)
        cand = np.concatenate([EDGE, np.array([t, (t - 1) % 2**32, (t + 1) % 2**32], dtype=np.uint64),
                               rng.integers(0, 2**32, 5, dtype=np.uint64)])
        # every ordered 4-tuple of the candidate set would be too many: all
        # 4-windows of a shuffled, repeated list of them cover each word in
        # every position
        seq = np.concatenate([rng.permutation(cand) for _ in range(8)])
        for k in range(0, len(seq) - 3):
            ws.append(seq[k:k + 4])
            ts.append(t)
    w = np.array(ws, dtype=np.uint64).reshape(-1)
    t = np.array(ts, dtype=np.uint64)
    got = dev("run_lt", [w.astype(np.uint32), t.astype(np.uint32)], len(t))
    ref = ((w.reshape(-1, 4) < t[:, None]) * (1 << np.arange(4))).sum(axis=1)
    assert np.array_equal(got, ref.astype(np.uint32))


def test_zero_byte_mask(dev):
    rng = np.random.default_rng(6)
    byts = rng.integers(0, 256, (4096, 4))
    byts[rng.random((4096, 4)) < 0.4] = 0
    byts[:16] = [[0, 0, 0, 0], [255, 255, 255, 255], [0, 128, 0, 128], [128, 0, 128, 0],
                 [1, 0, 0, 0], [0, 0, 0, 1], [127, 0, 255, 0], [0, 0, 0, 0x80]] * 2
    x = (byts[:, 0] | (byts[:, 1] << 8) | (byts[:, 2] << 16) | (byts[:, 3] << 24)).astype(np.uint32)
    got = dev("run_zb", [x], len(x))
    ref = ((byts == 0) * (1 << np.arange(4))).sum(axis=1)
    assert np.array_equal(got, ref.astype(np.uint32))


def _run_start_ref(mask, b, cw, carry, nbits):
    below = [k for k in range(b + 1) if (mask >> k) & 1]
    return cw + below[-1] if below else carry


def test_run_start_lookups(dev):
    rng = np.random.default_rng(7)
    rows, ref = [], []
    for i in range(3000):
        m = int(rng.integers(0, 2**32)) & int(rng.integers(0, 2**32))
        if i % 7 == 0:
            m = 0
        b, cw, carry = int(rng.integers(0, 32)), int(rng.integers(0, 4)) * 32, int(rng.integers(0, 128))
        rows.append([m, b, cw, carry])
        ref.append(_run_start_ref(m, b, cw, carry, 32))
    got = dev("run_rs", [np.array(rows, dtype=np.uint64).reshape(-1).astype(np.uint32)], len(rows))
    assert np.array_equal(got, np.array(ref, dtype=np.uint32))
    rows, ref = [], []
    for i in range(3000):
        m = int(rng.integers(0, 2**63)) & int(rng.integers(0, 2**63)) & int(rng.integers(0, 2**63))
        if i % 5 == 0:
            m &= (1 << 63) - (1 << int(rng.integers(0, 63)))  # no start below some bit
        x, c0, carry = int(rng.integers(0, 64)), int(rng.integers(0, 2)) * 64, int(rng.integers(0, 128))
        rows.append([m & 0xFFFFFFFF, m >> 32, x, c0, carry])
        ref.append(_run_start_ref(m, x, c0, carry, 64))
    got = dev("run_rs64", [np.array(rows, dtype=np.uint64).reshape(-1).astype(np.uint32)], len(rows))
    assert np.array_equal(got, np.array(ref, dtype=np.uint32))


def test_even_bit_compaction(dev):
    rng = np.random.default_rng(8)
    x = np.concatenate([[0, 0xFFFFFFFF, 0x55555555, 0xAAAAAAAA, 1, 0x80000000],
                        rng.integers(0, 2**32, 4000)]).astype(np.uint64)
    got = dev("run_eb", [x.astype(np.uint32)], len(x))
    ref = np.zeros(len(x), dtype=np.uint64)
    for k in range(16):
        ref |= ((x >> (2 * k)) & 1) << k
    assert np.array_equal(got, ref.astype(np.uint32))
