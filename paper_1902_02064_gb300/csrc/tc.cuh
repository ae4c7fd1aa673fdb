// tcgen05 (fifth-generation tensor core) helpers for sm_103a kernels:
// tensor-memory allocation, TF32 MMA issue with shared-memory operand
// descriptors, completion through mbarriers, and tensor-memory loads.
//
// Operand tiles are K-major with 128-byte swizzle: a row of the tile holds
// 32 consecutive K values (128 bytes), 16-byte chunk c of row r sits at
// chunk position c ^ (r & 7), and 8-row groups are 1024 bytes apart.  That
// is the layout a TMA box of 32 FP32 columns x R rows with 128-byte swizzle
// produces, so TMA-loaded K-major tiles feed the MMA directly.
#pragma once

#include "tma.cuh"

namespace trbl {

// Shared-memory matrix descriptor of a K-major, 128-byte-swizzled tile that
// starts at p (1024-byte aligned; +32 bytes per K step of 8 TF32 values).
// Fields: start address >> 4 (bits 0-13), leading byte offset >> 4 (16-29,
// unused for this layout), stride byte offset >> 4 (32-45: 1024 bytes
// between 8-row groups), descriptor version 1 (46-47), swizzle mode 2 =
// 128-byte (61-63).
__device__ __forceinline__ uint64_t sdesc_k128(const void* p) {
  const uint64_t a = smem_u32(p);
  return ((a >> 4) & 0x3FFFull) | (1ull << 16) | (uint64_t(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

// Instruction descriptor of a dense MMA with FP32 accumulator, TF32 A and B,
// both K-major, tile M x N: D format (bits 4-5) = 1, A and B formats (7-9,
// 10-12) = 2, N >> 3 (17-22), M >> 4 (24-28).
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

// Whole warp: allocate ncols (power of two >= 32) tensor-memory columns; the
// base address is written to *slot in shared memory.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// One thread: D[tmem] (+)= A * B^T for the descriptors' tiles.
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

// One thread: arrive once on bar when all MMAs this thread issued so far
// have completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Makes this thread's ordinary shared-memory stores visible to the tensor
// core and TMA (async proxy).
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Whole warp: 16 consecutive 32-bit columns starting at taddr of the warp's
// 32 tensor-memory lanes (lane = thread), waited for.
// 16 columns of this thread's tensor-memory lane into registers, without
// waiting: the values may be used only after tmem_wait_ld().
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Round an FP32 value to the nearest TF32 value (10 explicit mantissa bits;
// ties away from zero) on the bit pattern: add half of the dropped 13-bit
// unit to the sign-magnitude pattern and clear the dropped bits.  Not for
// NaN: the addition carries a high payload into the sign bit (the all-ones
// payload of CUDA arithmetic becomes -0).
__device__ __forceinline__ float tf32_round_bits(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// NaN-safe rounding for occasional values.
__device__ __forceinline__ float tf32_round(float x) { return x != x ? x : tf32_round_bits(x); }

// x = hi + lo with hi, lo TF32: |x - hi - lo| <= 2^-22 |x|.  A NaN x gives
// a NaN hi, which carries it into every product; lo is then immaterial, so
// only hi pays for the NaN test (testing both parts cost 24 % of the
// projection's time, testing hi 3 %; the hardware conversion
// cvt.rna.tf32.f32 for hi measured 5 %).
__device__ __forceinline__ void tf32_split(float x, float& hi, float& lo) {
  hi = x != x ? x : tf32_round_bits(x);
  lo = tf32_round_bits(x - hi);
}

}  // namespace trbl
