// tcgen05 (kind::tf32) primitives of the 3xTF32 Schur-complement updates:
// tile and chunk geometry, the TF32 rounding used by the hi/lo split, the
// shared-memory matrix descriptor of the canonical K-major no-swizzle layout
// (core matrices of 8 rows x 16 bytes), the instruction descriptor, mbarrier
// set-up, one MMA and its commit.  The kernels are in tc_pipe.cuh.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace viv {
namespace tc {

constexpr int BM = 128, BN = 128, KC = 32;        // tile and K chunk
constexpr int CORE_BYTES = 128;                   // 8 rows x 16 bytes
constexpr int KCORE_STRIDE = (BM / 8) * CORE_BYTES;   // bytes between K-adjacent core matrices (LBO)
constexpr int OPERAND_BYTES = BM * KC * 4;        // one 128 x 32 TF32 operand chunk (16 KB)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// shared-memory matrix descriptor: start, LBO (K direction), SBO (M/N
// direction), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor of kind::tf32: D f32, A and B tf32, both K-major
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

}  // namespace tc
}  // namespace viv
