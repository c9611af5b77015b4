// Tensor-memory-accelerator (TMA) plane loads for the 3D kernels that stage planes of
// a tile in shared memory: one cp.async.bulk.tensor per plane tile, completion counted
// on an mbarrier, so the load engine rather than the threads moves the data and no
// registers hold the next plane.
//
// Requirements checked on the host (tma_plane_map): the array's base address 16-byte
// aligned and its row pitch even (row and plane strides multiples of 16 bytes).  The
// box starts at an even x (x * 8 bytes a multiple of 16), any y and z; coordinates
// outside the array read as zero.  Waits are bounded: a wait that exceeds its limit
// reports failure to the caller, which records an error and leaves the kernel.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace stencil {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make mbarrier initialisations visible before the barriers are used by other threads
// and by the TMA unit.
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Make generic-proxy shared-memory accesses (and mbarrier inits) visible to the TMA
// (async proxy) before it writes the same memory.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// One thread: expect `bytes` on the barrier and start the 3D tile load into dst.
__device__ __forceinline__ void tma_load_plane(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar,
                                               unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(smem_u32(dst)),
      "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// Wait for the barrier phase `parity` to complete; false if `limit` polls ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, unsigned limit) {
  for (unsigned it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (it > 64) __nanosleep(64);
  }
  return false;
}

// Host: a 3D tensor map over a vertex array of geometry q (x fastest, pitch, plane)
// with a box of box_w x box_h x 1 doubles.  Returns false (no map) when the array
// does not meet TMA's alignment rules or the driver has no encoder.
bool tma_plane_map(const Geo &q, const void *base, int box_w, int box_h, CUtensorMap *map);

// The same for elements of elem_bytes bytes (8: FP64 or int64, 4: FP32, 2: bf16); the row pitch
// in bytes must be a multiple of 16 and the box must start at an x whose byte offset
// is a multiple of 16.
bool tma_plane_map_elem(const Geo &q, const void *base, int elem_bytes, int box_w, int box_h, CUtensorMap *map);

}  // namespace stencil
