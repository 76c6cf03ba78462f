// Standalone tensor-core Schur update (one launch, one 128 x 128 tile per CTA);
// the device code is in tc_mma.cuh.
#include <cuda_runtime.h>

#include <mutex>

#include "tc_mma.cuh"
#include "viv_internal.h"

namespace viv {
namespace tc {

__global__ void __launch_bounds__(THREADS, 3) gemm_standalone_kernel(const float* A, int lda, const float* B, int ldb,
                                                                   float* C, int ldc, int M, int N, int K, int* err) {
  extern __shared__ __align__(1024) unsigned char raw[];
  Smem& sm = *reinterpret_cast<Smem*>(raw);
  const int tiles_m = (M + BM - 1) / BM;
  const int rb = (blockIdx.x % tiles_m) * BM, cb = (blockIdx.x / tiles_m) * BN;
  tile_update(sm, A, lda, B, ldb, C, ldc, M, N, K, rb, cb, err);
}

}  // namespace tc

size_t tc_smem_bytes() { return sizeof(tc::Smem) + 1024; }

void tc_gemm_update(const float* A, int lda, const float* B, int ldb, float* C, int ldc, int M, int N, int K,
                    int* err, cudaStream_t s) {
  constexpr int MAX_DEV = 64;
  static std::once_flag once[MAX_DEV];   // per device; callers may be concurrent threads
  const int smem = (int)tc_smem_bytes();
  int dev = 0;
  VIV_CUDA(cudaGetDevice(&dev));
  VIV_CHECK(dev >= 0 && dev < MAX_DEV, VIV_ERR_ARG, "device index out of range");
  std::call_once(once[dev], [&] {
    VIV_CUDA(cudaFuncSetAttribute(tc::gemm_standalone_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  });
  const int tiles = ((M + tc::BM - 1) / tc::BM) * ((N + tc::BN - 1) / tc::BN);
  if (tiles == 0 || K <= 0) return;
  Launched L(K_TCGEMM, s);
  tc::gemm_standalone_kernel<<<tiles, tc::THREADS, smem, s>>>(A, lda, B, ldb, C, ldc, M, N, K, err);
  VIV_CUDA(cudaGetLastError());
}

}  // namespace viv
