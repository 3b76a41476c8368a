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

/* The same product with eight 7-bit digits per entry (56-bit slices: an
 * entry 2^-d below its row's / column's largest keeps 56 - d bits, those
 * within 3 binades are exact; 49 digit-pair MMAs per 16-deep step) and a
 * balanced contraction: in every 64-deep chunk, A's column k and B's row k
 * are first rescaled by 2^d_k and 2^-d_k, 2^d_k the binade of row k of B
 * over the 64 columns of the output tile, so rows of B of very different
 * magnitudes keep their digits (the tile of the factorisation's blocked
 * Z = Piv^-1 B solve).  Arguments and returns as aifmm_dgemm_tc. */
int aifmm_dgemm_tc8(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc, int m, int n,
                    int k, double alpha, void* stream);

/* The same product on the 5th-generation tensor cores: tcgen05.mma with
 * BF16 digit operands in shared memory and FP32 accumulators in tensor
 * memory (two digits of A stacked per 128-row MMA), the exact digit-pair
 * sums combined in 64-bit integer fixed point across K and converted to
 * FP64 once per output.  Same digits and rounding rules as aifmm_dgemm_tc;
 * k <= 8192.  Arguments as aifmm_dgemm_tc; additionally returns 7
 * (AIFMM_ERR_TIMEOUT) if a bounded wait for the tensor cores ran out (C is
 * then left unchanged for the tiles concerned). */
int aifmm_dgemm_tc05(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc, int m, int n,
                     int k, double alpha, void* stream);

/* C += alpha * op(A) * B on the tensor cores in TF32 with FP32 accumulation
 * (the tile of the factorisation's precision = 2 mode): op(A) = A (m x k,
 * trans_a = 0) or A^T (A k x m, trans_a != 0); operands rounded FP64 ->
 * FP32 -> TF32 (10-bit mantissa, round to nearest), products summed in FP32,
 * added to C in FP64; error about 2^-10 |op(A)| |B|.  DEVICE pointers,
 * column-major, lda >= (trans_a ? k : m), ldb >= k, ldc >= m (each < 2^31);
 * the call synchronises `stream`.  Returns 0, 1 (invalid argument) or 6. */
int aifmm_gemm_tf32(int trans_a, const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
                    int m, int n, int k, double alpha, void* stream);

/* Measured FMA throughput of the current device, for roofline peaks: every
 * thread of 8 x (SM count) CTAs of 256 threads runs 8 independent FMA chains
 * of 16,384 steps; *tflops receives 2 x FMAs / time in TFLOP/s, the best of
 * five timed launches after one warm-up (CUDA events on `stream`, NULL: the
 * legacy default stream).  fp32 = 0: FP64 FMAs (DFMA), else FP32 FMAs.
 * Returns 0, 1 (tflops NULL), 2 (allocation failed) or 6 (CUDA error). */
int aifmm_fma_rate(int fp32, void* stream, double* tflops);

#ifdef __cplusplus
}
#endif
#endif /* AIFMM_KERNELS_H */
