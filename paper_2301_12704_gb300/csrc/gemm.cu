// Stand-alone entry to the tensor-core FP64 product tile used by the
// factorisation's Schur update (no counterpart in the paper; exported so its
// accuracy can be checked against an FP64 product).
#include <cuda_runtime.h>

#include "../../include/aifmm_kernels.h"
#include "ozaki.cuh"
#include "tc05.cuh"

namespace aifmm {
namespace {

template <bool KB, int S>
__global__ void __launch_bounds__(256) k_gemm_oz(const double* A, int64_t lda, const double* B, int64_t ldb,
                                                 double* C, int64_t ldc, int m, int n, int k, double alpha) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  tile_gemm_64_oz<false, KB, S>(A + i0, (int)lda, B + (size_t)j0 * ldb, (int)ldb, C + i0 + (size_t)j0 * ldc, (int)ldc,
                  min(64, m - i0), min(64, n - j0), k, alpha, smem);
}

__global__ void __launch_bounds__(256) k_gemm_tc05(const double* A, int64_t lda, const double* B, int64_t ldb,
                                                   double* C, int64_t ldc, int m, int n, int k, double alpha,
                                                   int* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  tile_gemm_64_tc(A + i0, (int)lda, B + (size_t)j0 * ldb, (int)ldb, C + i0 + (size_t)j0 * ldc, (int)ldc,
                  min(64, m - i0), min(64, n - j0), k, alpha, smem, err);
}

}  // namespace
}  // namespace aifmm

extern "C" int aifmm_dgemm_tc05(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
                                int m, int n, int k, double alpha, void* stream) {
  if (!A || !B || !C || m < 0 || n < 0 || k < 0 || lda < m || ldb < k || ldc < m || lda > INT32_MAX ||
      ldb > INT32_MAX || ldc > INT32_MAX)
    return 1;
  if (m == 0 || n == 0) return 0;
  static int* err = nullptr;
  if (!err) {
    if (cudaFuncSetAttribute(aifmm::k_gemm_tc05, cudaFuncAttributeMaxDynamicSharedMemorySize, aifmm::TC_SMEM) !=
        cudaSuccess)
      return 6;
    if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) return 2;
  }
  if (cudaMemsetAsync(err, 0, sizeof(int), (cudaStream_t)stream) != cudaSuccess) return 6;
  dim3 grid((n + 63) / 64, (m + 63) / 64);
  aifmm::k_gemm_tc05<<<grid, 256, aifmm::TC_SMEM, (cudaStream_t)stream>>>(A, lda, B, ldb, C, ldc, m, n, k, alpha,
                                                                          err);
  if (cudaGetLastError() != cudaSuccess) return 6;
  int h = 0;
  if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream) != cudaSuccess) return 6;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return 6;
  return h ? 7 : 0;
}

namespace aifmm {
namespace {

template <bool KB, int S>
int dgemm_tc(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc, int m, int n, int k,
             double alpha, void* stream) {
  if (!A || !B || !C || m < 0 || n < 0 || k < 0 || lda < m || ldb < k || ldc < m || lda > INT32_MAX ||
      ldb > INT32_MAX || ldc > INT32_MAX)
    return 1;
  if (m == 0 || n == 0) return 0;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_gemm_oz<KB, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, oz_smem(S)) !=
        cudaSuccess)
      return 6;
    attr = true;
  }
  dim3 grid((n + 63) / 64, (m + 63) / 64);
  k_gemm_oz<KB, S><<<grid, 256, oz_smem(S), (cudaStream_t)stream>>>(A, lda, B, ldb, C, ldc, m, n, k, alpha);
  if (cudaGetLastError() != cudaSuccess) return 6;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return 6;
  return 0;
}

}  // namespace
}  // namespace aifmm

extern "C" int aifmm_dgemm_tc(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
                              int m, int n, int k, double alpha, void* stream) {
  return aifmm::dgemm_tc<false, aifmm::OZ_S>(A, lda, B, ldb, C, ldc, m, n, k, alpha, stream);
}

extern "C" int aifmm_dgemm_tc8(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
                               int m, int n, int k, double alpha, void* stream) {
  return aifmm::dgemm_tc<true, aifmm::OZ_S8>(A, lda, B, ldb, C, ldc, m, n, k, alpha, stream);
}
