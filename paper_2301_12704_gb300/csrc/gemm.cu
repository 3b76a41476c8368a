// Stand-alone entry to the tensor-core FP64 product tile used by the
// factorisation's Schur update (no counterpart in the paper; exported so its
// accuracy can be checked against an FP64 product).
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "../../include/aifmm_kernels.h"
#include "dense.cuh"
#include "ozaki.cuh"
#include "tc05.cuh"

namespace aifmm {
namespace {

template <bool KB, int S>
__global__ void __launch_bounds__(256, 2) k_gemm_oz(const double* A, int64_t lda, const double* B, int64_t ldb,
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

// the kernels' shared-memory limits, raised once per device and kernel;
// callers may come from several threads
std::mutex g_attr_mu;

bool raise_smem_once(const void* fn, int bytes, int slot) {
  static bool done[64][4] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
  std::lock_guard<std::mutex> g(g_attr_mu);
  if (!done[dev][slot]) {
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) return false;
    done[dev][slot] = true;
  }
  return true;
}

}  // namespace
}  // namespace aifmm

extern "C" int aifmm_dgemm_tc05(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
                                int m, int n, int k, double alpha, void* stream) {
  if (!A || !B || !C || m < 0 || n < 0 || k < 0 || lda < m || ldb < k || ldc < m || lda > INT32_MAX ||
      ldb > INT32_MAX || ldc > INT32_MAX)
    return 1;
  if (m == 0 || n == 0) return 0;
  if (!aifmm::raise_smem_once((const void*)aifmm::k_gemm_tc05, aifmm::TC_SMEM, 0)) return 6;
  // the error word of this call only (stream-ordered, on the current device),
  // so concurrent calls from several threads or devices do not share it
  cudaStream_t st = (cudaStream_t)stream;
  int* err = nullptr;
  if (cudaMallocAsync((void**)&err, sizeof(int), st) != cudaSuccess) {
    cudaGetLastError();
    return 2;
  }
  int rc = 0;
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) rc = 6;
  dim3 grid((n + 63) / 64, (m + 63) / 64);
  if (!rc) {
    aifmm::k_gemm_tc05<<<grid, 256, aifmm::TC_SMEM, st>>>(A, lda, B, ldb, C, ldc, m, n, k, alpha, err);
    if (cudaGetLastError() != cudaSuccess) rc = 6;
  }
  int h = 0;
  if (!rc && cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) rc = 6;
  cudaFreeAsync(err, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) rc = 6;
  return rc ? rc : h ? 7 : 0;
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
  if (!raise_smem_once((const void*)k_gemm_oz<KB, S>, oz_smem(S, KB), KB ? 2 : 1)) return 6;
  dim3 grid((n + 63) / 64, (m + 63) / 64);
  k_gemm_oz<KB, S><<<grid, 256, oz_smem(S, KB), (cudaStream_t)stream>>>(A, lda, B, ldb, C, ldc, m, n, k, alpha);
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

// ---------------------------------------------------------------------------
// FMA throughput probe: the roofline peak of the FP64 (and FP32) arithmetic
// pipes of the GPU it runs on, measured rather than taken from a data sheet.
// Every thread runs 8 independent FMA chains (enough to cover the pipe's
// latency), 8 CTAs of 256 threads per SM; the result is the
// best of several timed launches (CUDA events on the given stream).
namespace aifmm {
namespace {

template <class T>
__global__ void __launch_bounds__(256) k_fma_probe(T* out, int iters, T a, T c) {
  T x[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) x[u] = (T)(threadIdx.x + u) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = fma(x[u], a, c);
  }
  T s = 0;
#pragma unroll
  for (int u = 0; u < 8; ++u) s += x[u];
  if (s == (T)-1.2345) out[0] = s;   // keeps the chains live; never true for these inputs
}

template <class T>
int fma_rate(void* stream, double* tflops) {
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess)
    return 6;
  T* out = nullptr;
  if (cudaMallocAsync((void**)&out, sizeof(T), st) != cudaSuccess) {
    cudaGetLastError();
    return 2;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int iters = 1 << 14, blocks = nsm * 8, threads = 256;
  double best = 0.0;
  int rc = 0;
  for (int rep = 0; rep < 6 && !rc; ++rep) {
    cudaEventRecord(e0, st);
    k_fma_probe<T><<<blocks, threads, 0, st>>>(out, iters, (T)0.999999, (T)1e-7);
    cudaEventRecord(e1, st);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      rc = 6;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double flops = 2.0 * 8.0 * iters * (double)blocks * threads;
    if (rep > 0 && ms > 0.f) best = std::max(best, flops / (ms * 1e-3) / 1e12);   // rep 0 warms up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(out, st);
  if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = 6;
  *tflops = best;
  return rc;
}

}  // namespace
}  // namespace aifmm

extern "C" int aifmm_fma_rate(int fp32, void* stream, double* tflops) {
  if (!tflops) return 1;
  *tflops = 0.0;
  return fp32 ? aifmm::fma_rate<float>(stream, tflops) : aifmm::fma_rate<double>(stream, tflops);
}

// ---------------------------------------------------------------------------
// The TF32 tensor-core tile of the preconditioner mode, on its own.
namespace aifmm {
namespace {

template <bool TA>
__global__ void __launch_bounds__(256) k_gemm_tf32(const double* A, int64_t lda, const double* B, int64_t ldb,
                                                   double* C, int64_t ldc, int m, int n, int k, double alpha) {
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  const double* Ab = TA ? A + (size_t)i0 * lda : A + i0;
  tile_gemm_64_tf32<TA>(Ab, (int)lda, B + (size_t)j0 * ldb, (int)ldb, C + i0 + (size_t)j0 * ldc, (int)ldc,
                        min(64, m - i0), min(64, n - j0), k, alpha);
}

}  // namespace
}  // namespace aifmm

extern "C" int aifmm_gemm_tf32(int trans_a, const double* A, int64_t lda, const double* B, int64_t ldb, double* C,
                               int64_t ldc, int m, int n, int k, double alpha, void* stream) {
  if (!A || !B || !C || m < 0 || n < 0 || k < 0 || lda < (trans_a ? k : m) || ldb < k || ldc < m ||
      lda > INT32_MAX || ldb > INT32_MAX || ldc > INT32_MAX)
    return 1;
  if (m == 0 || n == 0) return 0;
  dim3 grid((n + 63) / 64, (m + 63) / 64);
  cudaStream_t st = (cudaStream_t)stream;
  if (trans_a)
    aifmm::k_gemm_tf32<true><<<grid, 256, 0, st>>>(A, lda, B, ldb, C, ldc, m, n, k, alpha);
  else
    aifmm::k_gemm_tf32<false><<<grid, 256, 0, st>>>(A, lda, B, ldb, C, ldc, m, n, k, alpha);
  if (cudaGetLastError() != cudaSuccess) return 6;
  if (cudaStreamSynchronize(st) != cudaSuccess) return 6;
  return 0;
}
