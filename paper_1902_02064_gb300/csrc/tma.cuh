// TMA (cp.async.bulk.tensor) and mbarrier helpers for sm_103a kernels.
//
// Every wait on an mbarrier is bounded: after kWaitLimit polls it gives up,
// records an error code in a device word and returns false, so a kernel
// never spins forever.
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "internal.h"

namespace trbl {

constexpr uint32_t kWaitLimit = 1u << 26;  // polls before a wait gives up
constexpr int kErrTmaTimeout = 1;

// Host: 2-D FP32 tensor map over a row-major array of `rows` rows, `cols`
// used columns and leading dimension `ld` (elements), box of box_cols x
// box_rows, 128-byte swizzle, out-of-range elements read as zero.
int make_tmap_2d_f32(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows, uint64_t ld,
                     uint32_t box_cols, uint32_t box_rows);
// The same without swizzle: a box lands in shared memory as box_rows rows of
// box_cols * 4 contiguous bytes.
int make_tmap_2d_f32_rows(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows, uint64_t ld,
                          uint32_t box_cols, uint32_t box_rows);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Plain arrival (release) on a barrier.
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Wait until the barrier's phase with the given parity has completed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t i = 0; i < kWaitLimit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  if (err) atomicExch(err, kErrTmaTimeout);
  return false;
}

// 2-D tiled TMA load of the box at (x = column, y = row) into shared memory;
// completion is signalled on `bar` (complete_tx by the box's bytes).
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

}  // namespace trbl
