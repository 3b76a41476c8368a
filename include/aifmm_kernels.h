/*
 * aifmm_kernels.h -- building blocks of the AIFMM library exported for
 * checking on their own.  No counterpart in the paper.
 */
#ifndef AIFMM_KERNELS_H
#define AIFMM_KERNELS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* C += alpha * A * B in FP64 precision on the BF16 tensor cores: each
 * operand row (A) / column (B) of every 64-deep chunk is cut into seven
 * 7-bit integer digits below its largest binary exponent, digit pairs are
 * multiplied exactly by warp MMAs with FP32 accumulation and recombined in
 * FP64 (the product tile of the factorisation's Schur update).  Entries
 * below 2^-49 of their row's (column's) largest magnitude in a chunk are
 * rounded at that level; subnormal inputs are flushed to zero.
 *   A  m x k, B  k x n, C  m x n: DEVICE pointers, column-major, leading
 *      dimensions lda >= m, ldb >= k, ldc >= m (each < 2^31).
 *   stream  cudaStream_t (NULL: the legacy default stream); the call
 *      synchronises the stream before returning.
 * Returns 0 (AIFMM_OK), 1 (invalid argument) or 6 (CUDA error). */
int aifmm_dgemm_tc(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc, int m, int n,
                   int k, double alpha, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* AIFMM_KERNELS_H */
