// Bulk L2 prefetch (the TMA unit's cp.async.bulk.prefetch): one instruction moves a contiguous
// range of global memory into L2 ahead of the loads that will read it, without registers, shared
// memory or a completion to wait for. Rules the callers keep: source 16-byte aligned, size a
// positive multiple of 16 bytes, range inside its allocation.
#pragma once

#include <cstdint>

namespace helm {

__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

}  // namespace helm
