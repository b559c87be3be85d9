// sw_internal.h -- host-side helpers shared by the translation units of
// libswgb (single lattice, batched replicas).  Not part of the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/sw.h"

namespace swgb {

struct Lattice;
struct Bufs;

// Device allocator captured by a handle at creation.
struct DeviceAllocator {
  sw_alloc_fn alloc;
  sw_free_fn free_fn;
  void* ctx;
  void* allocate(size_t bytes) const;
  void release(void* p, size_t bytes) const;
};
DeviceAllocator current_allocator();

uint32_t bond_threshold(double T);
uint32_t pick_tile_h(uint64_t L, uint32_t requested);

}  // namespace swgb
