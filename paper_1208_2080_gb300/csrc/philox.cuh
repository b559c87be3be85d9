// philox.cuh -- device Philox4x32-10 counter-based generator.
//
// Written from the published algorithm (Salmon, Moraes, Dror, Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11, Sec. 5): ten rounds
// of two 32x32->64 multiplications whose high halves are xored into the other
// two counter words together with the round key, the key advancing by two
// Weyl constants between rounds.  The Swendsen-Wang streams built on it
// (bonds, new cluster states, initial spins) are the counter layouts of
// include/sw.h; the same streams are reimplemented independently by the CPU
// oracle, and tested against cuRAND's device Philox at run time.
#pragma once
#include <stdint.h>

namespace swgb {

struct Words4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ Words4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                uint32_t c3, uint32_t k0, uint32_t k1) {
  constexpr uint32_t kMul0 = 0xD2511F53u, kMul1 = 0xCD9E8D57u;
  constexpr uint32_t kWeyl0 = 0x9E3779B9u, kWeyl1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    // one 32x32->64 product per word pair (a single wide multiply-add)
    const uint64_t p0 = (uint64_t)kMul0 * c0, p1 = (uint64_t)kMul1 * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += kWeyl0;
    k1 += kWeyl1;
  }
  return Words4{c0, c1, c2, c3};
}

// Same function with the ten round keys given (rk[2r], rk[2r+1] = key of
// round r); when rk lives in the kernel's parameter space the keys are
// instruction operands and the per-round key additions disappear.
__device__ __forceinline__ Words4 philox4x32_10_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                   const uint32_t (&rk)[20]) {
  constexpr uint32_t kMul0 = 0xD2511F53u, kMul1 = 0xCD9E8D57u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)kMul0 * c0, p1 = (uint64_t)kMul1 * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c1 ^ rk[2 * r];
    const uint32_t n2 = hi0 ^ c3 ^ rk[2 * r + 1];
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return Words4{c0, c1, c2, c3};
}

// Same function with the round keys in shared memory, two rounds' keys per
// 16-byte load (k4[i] = keys of rounds 2i and 2i+1).
__device__ __forceinline__ Words4 philox4x32_10_k4(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                   const uint4* k4) {
  constexpr uint32_t kMul0 = 0xD2511F53u, kMul1 = 0xCD9E8D57u;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const uint4 k = k4[i];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint64_t p0 = (uint64_t)kMul0 * c0, p1 = (uint64_t)kMul1 * c2;
      const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
      const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
      const uint32_t n0 = hi1 ^ c1 ^ (h ? k.z : k.x);
      const uint32_t n2 = hi0 ^ c3 ^ (h ? k.w : k.y);
      c0 = n0;
      c1 = lo1;
      c2 = n2;
      c3 = lo0;
    }
  }
  return Words4{c0, c1, c2, c3};
}

// Stream domains (fourth counter word).
enum : uint32_t { kDomBond = 0, kDomSpin = 1, kDomInit = 2, kDomAxis = 3 };

__device__ __forceinline__ Words4 stream4(uint64_t seed, uint64_t idx, uint32_t sweep,
                                          uint32_t dom) {
  return philox4x32_10((uint32_t)idx, (uint32_t)(idx >> 32), sweep, dom, (uint32_t)seed,
                       (uint32_t)(seed >> 32));
}

__device__ __forceinline__ Words4 stream4_rk(const uint32_t (&rk)[20], uint64_t idx, uint32_t sweep,
                                             uint32_t dom) {
  return philox4x32_10_rk((uint32_t)idx, (uint32_t)(idx >> 32), sweep, dom, rk);
}

// floor(w * q / 2^32): the state a 32-bit word picks.
__device__ __forceinline__ uint32_t pick_state(uint32_t w, uint32_t q) { return __umulhi(w, q); }

// New state of the cluster whose root (smallest site index) is r.
__device__ __forceinline__ uint32_t cluster_state(uint64_t seed, uint64_t r, uint32_t sweep,
                                                  uint32_t q) {
  return pick_state(stream4(seed, r, sweep, kDomSpin).x, q);
}

}  // namespace swgb
