// Batched dense FP64 building blocks used by the factorisation, the top
// solve and the sweeps: blocked right-looking LU with partial pivoting
// (panel / TRSM / trailing GEMM launches), multi-RHS LU solve, and a 64x64
// register-tiled GEMM tile.
#pragma once
#include "common.cuh"
#include "ozaki.cuh"

namespace aifmm {

struct LuItem {
  double* a;       // column-major n x n, leading dimension ld
  int* ipiv;       // n row interchanges (LAPACK convention, 0-based)
  const double* colmax;  // n column maxima of the original matrix (singularity test)
  int n, ld;
  // right-hand columns factored along with A (the augmented matrix [A | B]):
  // the row interchanges, the panels' triangular solves and the trailing
  // updates are applied to B too, which ends as L^-1 P B.  nb = 0: none.
  double* b;       // column-major n x nb, leading dimension ldb
  int ldb, nb;
};

// column c of the augmented matrix [A | B]
__device__ inline double* lu_col(const LuItem& it, int c) {
  return c < it.n ? it.a + (size_t)c * it.ld : it.b + (size_t)(c - it.n) * it.ldb;
}

constexpr int LU_NB = 32;

// U12 = L11^-1 A12 for the columns right of the panel: one warp per column,
// lane i holding row k0 + i, x_j broadcast with a shuffle (lane-dense FP64;
// see k_lus_diag_w).  grid (column groups of 4, items), 128 threads
// (columns of B included: grid columns cover n + nb)
static __global__ void __launch_bounds__(128) k_lu_trsm(const LuItem* items, int k0) {
  __shared__ double L[LU_NB][LU_NB + 1];
  LuItem it = items[blockIdx.y];
  int n = it.n;
  if (k0 >= n) return;
  int kend = min(n, k0 + LU_NB), nb = kend - k0;
  double* A = it.a;
  const int ld = it.ld;
  for (int e = threadIdx.x; e < LU_NB * LU_NB; e += blockDim.x) {
    int i = e % LU_NB, j = e / LU_NB;
    L[i][j] = (i < nb && j < nb) ? A[(k0 + i) + (size_t)(k0 + j) * ld] : 0.0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  int c = kend + blockIdx.x * 4 + (threadIdx.x >> 5);
  if (c >= n + it.nb) return;
  double* X = lu_col(it, c) + k0;
  double x = lane < nb ? X[lane] : 0.0;
  for (int j = 0; j < nb; ++j) {
    double xj = __shfl_sync(0xffffffffu, x, j);
    if (lane > j) x -= L[lane][j] * xj;
  }
  if (lane < nb) X[lane] = x;
}

// The same U12 = L11^-1 A12 with one thread per column, its 32 entries in
// registers and L broadcast from shared memory.  Every FP64 lane does useful
// work (496 warp FMAs per 32 columns against 1024 lane slots per column in
// the warp form, half of them masked), at the price of a longer chain per
// thread; each entry sees the same FMAs in the same order as in the warp
// form, so the results are equal bit for bit.  grid (column groups of
// blockDim.x, items), 32 to 128 threads.
static __global__ void __launch_bounds__(128) k_lu_trsm_t(const LuItem* items, int k0) {
  __shared__ double L[LU_NB][LU_NB + 1];
  LuItem it = items[blockIdx.y];
  int n = it.n;
  if (k0 >= n) return;
  int kend = min(n, k0 + LU_NB), nb = kend - k0;
  const double* A = it.a;
  const int ld = it.ld;
  for (int e = threadIdx.x; e < LU_NB * LU_NB; e += blockDim.x) {
    int i = e % LU_NB, j = e / LU_NB;
    L[i][j] = (i < nb && j < nb) ? A[(k0 + i) + (size_t)(k0 + j) * ld] : 0.0;
  }
  __syncthreads();
  int c = kend + blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n + it.nb) return;
  double* X = lu_col(it, c) + k0;
  double x[LU_NB];
#pragma unroll
  for (int i = 0; i < LU_NB; ++i) x[i] = i < nb ? X[i] : 0.0;
#pragma unroll
  for (int j = 0; j < LU_NB; ++j)
#pragma unroll
    for (int i = j + 1; i < LU_NB; ++i) x[i] -= L[i][j] * x[j];
#pragma unroll
  for (int i = 0; i < LU_NB; ++i)
    if (i < nb) X[i] = x[i];
}

// Threads per CTA of the thread-per-column trsm for `cols` columns in one
// launch (at capacity), or 0 for the warp form.  The thread form issues half
// the FP64 warp instructions but runs 496 dependent-ish FMAs per warp, and an
// FP64 warp instruction holds its SM sub-partition's pipe for many clocks, so
// it pays only with several warps per sub-partition: measured at 65,536
// points, 22% faster on the leaf level (over a hundred boxes per launch, about
// 1,000 columns each at capacity) and slower on the levels above (at most 28
// boxes per launch).
inline int lu_trsm_threads(long long cols) { return cols < 98304 ? 0 : 128; }

// narrow right operand (nc <= 8 columns, e.g. a single right-hand side):
// 64 rows x 4 slices of K, one thread per (row, slice), every column of B
// in registers; the slices are summed through shared memory
// CT: the arithmetic type of the products and sums (double, or float for
// the FP32 factorisation used as a preconditioner); operands and results
// stay FP64 in memory.
constexpr int THIN_NC = 8;
template <typename CT = double>
__device__ inline void tile_gemm_64_thin(const double* A, int lda, const double* B, int ldb, double* C, int ldc,
                                         int mr, int nc, int K, double alpha) {
  __shared__ CT red[4][THIN_NC][64 + 1];
  const int i = threadIdx.x & 63, sl = threadIdx.x >> 6;   // 256 threads
  CT acc[THIN_NC];
#pragma unroll
  for (int c = 0; c < THIN_NC; ++c) acc[c] = CT(0);
  const int kq = (K + 3) / 4, ka = sl * kq, kb = min(K, ka + kq);
  if (i < mr)
    for (int k = ka; k < kb; ++k) {
      CT a = (CT)A[i + (size_t)k * lda];
#pragma unroll
      for (int c = 0; c < THIN_NC; ++c)
        if (c < nc) acc[c] = fma(a, (CT)B[k + (size_t)c * ldb], acc[c]);
    }
#pragma unroll
  for (int c = 0; c < THIN_NC; ++c) red[sl][c][i] = acc[c];
  __syncthreads();
  for (int e = threadIdx.x; e < 64 * nc; e += blockDim.x) {
    int r = e & 63, c = e >> 6;
    if (r < mr) C[r + (size_t)c * ldc] += alpha * (double)(((red[0][c][r] + red[1][c][r]) + red[2][c][r]) + red[3][c][r]);
  }
  __syncthreads();
}

// 64x64 FP64 tile: C[i0.., j0..] += alpha * A[i0.., 0..K) * B[0..K, j0..]
// (A column-major lda, B column-major ldb, C column-major ldc), bounds
// rows < mr, cols < nc.  256 threads, 4x4 outputs each (the thin form above
// when nc <= THIN_NC).
template <typename CT = double>
__device__ inline void tile_gemm_64(const double* A, int lda, const double* B, int ldb, double* C, int ldc,
                                    int mr, int nc, int K, double alpha) {
  if (nc <= THIN_NC) {
    tile_gemm_64_thin<CT>(A, lda, B, ldb, C, ldc, mr, nc, K, alpha);
    return;
  }
  __shared__ CT As[16][64 + 1];
  __shared__ CT Bs[16][64 + 1];
  int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  CT acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = CT(0);
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      int kk = e >> 6, ii = e & 63;
      As[kk][ii] = (ii < mr && k0 + kk < K) ? (CT)A[ii + (size_t)(k0 + kk) * lda] : CT(0);
      int jj = e >> 4, k2 = e & 15;
      Bs[k2][jj] = (jj < nc && k0 + k2 < K) ? (CT)B[(k0 + k2) + (size_t)jj * ldb] : CT(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      CT av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int i = ty + 16 * a, j = tx + 16 * b;
      if (i < mr && j < nc) C[i + (size_t)j * ldc] += alpha * (double)acc[a][b];
    }
}

// 64x64 tile on the tensor cores in TF32 with FP32 accumulation (the
// preconditioner's low-precision products, aifmm_options.precision = 2):
// C[0..mr, 0..nc] += alpha * op(A) B, op(A) = A (column-major, lda) or, with
// TA, A^T for A column-major K x mr.  K in chunks of 32: the chunk's
// operands are rounded FP64 -> FP32 -> TF32 (round to nearest, ties away)
// into shared memory; 8 warps, each a 32 x 16 sub-tile of 2 x 2
// mma.sync m16n8k8 tf32 products per 8 of K, FP32 accumulators; the
// result is added to C in FP64.  Products of TF32 values are exact in the
// FP32 accumulator, so the error is the operands' rounding (2^-11 relative)
// plus the FP32 sums.  256 threads; 18 KB of static shared memory.
constexpr int TF_KC = 32;
constexpr int TF_LD = TF_KC + 4;            // padded rows: conflict-free fragment loads

__device__ inline uint32_t tf32_bits(double x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"((float)x));
  return u;
}

__device__ inline void tf32_mma(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <bool TA = false>
__device__ inline void tile_gemm_64_tf32(const double* A, int lda, const double* B, int ldb, double* C, int ldc,
                                         int mr, int nc, int K, double alpha) {
  __shared__ uint32_t As[64][TF_LD];   // (row of op(A), k)
  __shared__ uint32_t Bs[64][TF_LD];   // (column of B, k)
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int g = lane >> 2, tq = lane & 3;
  const int r0 = 32 * (w & 1), c0 = 16 * (w >> 1);
  float acc[2][2][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[a][b][q] = 0.f;
  for (int k0 = 0; k0 < K; k0 += TF_KC) {
    const int kc = min(TF_KC, K - k0);
    for (int e = threadIdx.x; e < 64 * TF_KC; e += blockDim.x) {
      int i, k;
      if (TA) {
        k = e & (TF_KC - 1);
        i = e / TF_KC;
      } else {
        i = e & 63;
        k = e >> 6;
      }
      double a = 0.0;
      if (i < mr && k < kc) a = TA ? A[(k0 + k) + (size_t)i * lda] : A[i + (size_t)(k0 + k) * lda];
      As[i][k] = tf32_bits(a);
      const int kb = e & (TF_KC - 1), j = e / TF_KC;
      const double bv = (j < nc && kb < kc) ? B[(k0 + kb) + (size_t)j * ldb] : 0.0;
      Bs[j][kb] = tf32_bits(bv);
    }
    __syncthreads();
#pragma unroll
    for (int k8 = 0; k8 < TF_KC; k8 += 8) {
      uint32_t af[2][4], bf[2][2];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        const int r = r0 + 16 * mi + g;
        af[mi][0] = As[r][k8 + tq];
        af[mi][1] = As[r + 8][k8 + tq];
        af[mi][2] = As[r][k8 + tq + 4];
        af[mi][3] = As[r + 8][k8 + tq + 4];
      }
#pragma unroll
      for (int ni = 0; ni < 2; ++ni) {
        const int c = c0 + 8 * ni + g;
        bf[ni][0] = Bs[c][k8 + tq];
        bf[ni][1] = Bs[c][k8 + tq + 4];
      }
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 2; ++ni) tf32_mma(acc[mi][ni], af[mi], bf[ni]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 2; ++ni)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = r0 + 16 * mi + g + 8 * (q >> 1), j = c0 + 8 * ni + 2 * tq + (q & 1);
        if (i < mr && j < nc) C[i + (size_t)j * ldc] += alpha * (double)acc[mi][ni][q];
      }
}

// Product modes of the tile kernels: PM_FMA FP64 FMAs; PM_OZ FP64 precision
// on the BF16 warp MMAs (ozaki.cuh, for more than THIN_NC columns; kernels
// instantiated with it are launched with OZ_SMEM bytes of dynamic shared
// memory); PM_TC05 the same digits on tcgen05 (tc05.cuh, the Schur update
// only, TC_SMEM bytes); PM_F32 FP32 products and sums of FP64 operands (the
// factorisation used as a preconditioner).
// PM_OZ8: the warp-MMA tile with 8 digits (56-bit slices) and the balanced
// contraction (the Z = Piv^-1 B solve and the pivot LU's trailing updates,
// whose operands mix entries of very different sizes; oz_smem(OZ_S8) bytes).
// PM_TF32: TF32 tensor-core products with FP32 sums (tile_gemm_64_tf32) for
// more than THIN_NC columns, FP32 FMAs for fewer (the preconditioner's
// low-precision mode, aifmm_options.precision = 2).
enum { PM_FMA = 0, PM_OZ = 1, PM_TC05 = 2, PM_F32 = 3, PM_OZ8 = 4, PM_TF32 = 5 };

// C += alpha A B, 64 x 64 tile (A column-major lda, B column-major ldb)
template <int PM>
__device__ inline void tile_gemm(const double* A, int lda, const double* B, int ldb, double* C, int ldc, int mr,
                                 int nc, int K, double alpha) {
  if (PM == PM_OZ && nc > THIN_NC) {
    extern __shared__ __align__(16) unsigned char oz_dyn[];
    tile_gemm_64_oz<false>(A, lda, B, ldb, C, ldc, mr, nc, K, alpha, oz_dyn);
  } else if (PM == PM_OZ8 && nc > THIN_NC) {
    extern __shared__ __align__(16) unsigned char oz_dyn[];
    tile_gemm_64_oz<false, true, OZ_S8>(A, lda, B, ldb, C, ldc, mr, nc, K, alpha, oz_dyn);
  } else if (PM == PM_TF32 && nc > THIN_NC) {
    tile_gemm_64_tf32<false>(A, lda, B, ldb, C, ldc, mr, nc, K, alpha);
  } else if (PM == PM_F32 || PM == PM_TF32) {
    tile_gemm_64<float>(A, lda, B, ldb, C, ldc, mr, nc, K, alpha);
  } else {
    tile_gemm_64(A, lda, B, ldb, C, ldc, mr, nc, K, alpha);
  }
}

// A22 -= L21 U12, and B2 -= L21 B1 for the right-hand columns; grid
// (coltiles of A22 then of B, rowtiles, items); PM_FMA, PM_OZ8 or PM_F32
template <int PM = PM_FMA>
static __global__ void __launch_bounds__(256, 2) k_lu_gemm(const LuItem* items, int k0) {
  LuItem it = items[blockIdx.z];
  int n = it.n;
  int kend = min(n, k0 + LU_NB);
  int i0 = kend + blockIdx.y * 64;
  if (k0 >= n || i0 >= n) return;
  double* A = it.a;
  const int ld = it.ld;
  const int ta = (n - kend + 63) / 64;          // column tiles of A22
  if ((int)blockIdx.x < ta) {
    const int j0 = kend + blockIdx.x * 64;
    tile_gemm<PM>(A + i0 + (size_t)k0 * ld, ld, A + k0 + (size_t)j0 * ld, ld, A + i0 + (size_t)j0 * ld, ld,
                  n - i0, n - j0, kend - k0, -1.0);
    return;
  }
  const int jb = ((int)blockIdx.x - ta) * 64;
  if (jb >= it.nb) return;
  double* B = it.b;
  tile_gemm<PM>(A + i0 + (size_t)k0 * ld, ld, B + k0 + (size_t)jb * it.ldb, it.ldb, B + i0 + (size_t)jb * it.ldb,
                it.ldb, n - i0, it.nb - jb, kend - k0, -1.0);
}

// X := A^-1 X for an LU-factored A (ipiv interchanges, unit L, U), per item;
// X column-major with leading dimension ldx, ncols columns.
struct SolveItem {
  const double* a;
  const int* ipiv;
  int n, ld;
  double* x;
  int ldx, ncols;
  const int* perm;   // net row permutation of ipiv (solve sweeps only), or null
};

// column maxima of |A| (n x n), one block per item, one warp per column
// (lanes over the rows, coalesced; fmax ignores NaNs and is order-free, so
// the result is that of a sequential scan)
static __global__ void k_colmax(const LuItem* items, double* out, int stride) {
  LuItem it = items[blockIdx.x];
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int c = threadIdx.x >> 5; c < it.n; c += nw) {
    const double* col = it.a + (size_t)c * it.ld;
    double mx = 0.0;
    for (int i = lane; i < it.n; i += 32) mx = fmax(mx, fabs(col[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) out[(size_t)blockIdx.x * stride + c] = mx;
  }
}

}  // namespace aifmm

namespace aifmm {

// ---- blocked multi-RHS LU solve:  X := U^-1 L^-1 P X  -------------------------
// Row interchanges of every right-hand-side column (one thread per column).
static __global__ void __launch_bounds__(128) k_lus_swap(const SolveItem* items) {
  SolveItem it = items[blockIdx.y];
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= it.ncols || it.n == 0) return;
  double* X = it.x + (size_t)c * it.ldx;
  for (int k = 0; k < it.n; ++k) {
    int p = it.ipiv[k];
    if (p != k) {
      double t = X[k];
      X[k] = X[p];
      X[p] = t;
    }
  }
}

constexpr int TB = 64;   // diagonal block of the blocked triangular solves

// Divisions by a pivot or a diagonal entry of U are multiplications by its
// reciprocal, taken once (an FP64 division is a multi-instruction sequence
// on the narrow FP64 pipe, and in the triangular solves it sat on the
// dependency chain); one more rounding than a division, as in LAPACK's
// unblocked LU.  The LU panels reject pivots below the smallest normal
// number as singular, so every reciprocal is finite.
constexpr double LU_PIV_MIN = 2.2250738585072014e-308;

// diagonal block k0..k0+TB of the unit-lower (lower=1) or upper (lower=0)
// factor applied to every column; the block sits in shared memory, one
// thread per column keeps its TB entries in registers.
template <int LOWER>
static __global__ void __launch_bounds__(128) k_lus_diag(const SolveItem* items, int k0) {
  __shared__ double T[TB][TB + 1];
  __shared__ double Rd[TB];              // upper: reciprocals of the diagonal
  SolveItem it = items[blockIdx.y];
  int n = it.n;
  if (k0 >= n) return;
  int nb = min(TB, n - k0);
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
    int i = e % TB, j = e / TB;
    T[i][j] = (i < nb && j < nb) ? it.a[(k0 + i) + (size_t)(k0 + j) * it.ld] : 0.0;
  }
  __syncthreads();
  if (!LOWER) {
    if (threadIdx.x < TB) Rd[threadIdx.x] = threadIdx.x < nb ? 1.0 / T[threadIdx.x][threadIdx.x] : 0.0;
    __syncthreads();
  }
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= it.ncols) return;
  double* X = it.x + (size_t)c * it.ldx + k0;
  double x[TB];
#pragma unroll
  for (int i = 0; i < TB; ++i) x[i] = i < nb ? X[i] : 0.0;
  if (LOWER) {
#pragma unroll
    for (int j = 0; j < TB; ++j)
#pragma unroll
      for (int i = j + 1; i < TB; ++i) x[i] -= T[i][j] * x[j];
  } else {
#pragma unroll
    for (int j = TB - 1; j >= 0; --j) {
      if (j < nb) x[j] *= Rd[j];
#pragma unroll
      for (int i = 0; i < j; ++i) x[i] -= T[i][j] * x[j];
    }
  }
#pragma unroll
  for (int i = 0; i < TB; ++i)
    if (i < nb) X[i] = x[i];
}

// The same diagonal-block solve for a few columns: one warp per column, the
// 64 rows spread over the lanes (two each), x_j broadcast with a shuffle.  On
// a part whose FP64 pipe retires a warp instruction at a fraction of the FP32
// rate, thread-per-column with one live column would issue 2080 warp-wide FMAs
// per column; lane-parallel rows need 128.  grid ((ncols + 3) / 4, items), 128 threads.
template <int LOWER>
static __global__ void __launch_bounds__(128) k_lus_diag_w(const SolveItem* items, int k0) {
  __shared__ double T[TB][TB + 1];
  __shared__ double Rd[TB];              // upper: reciprocals of the diagonal
  SolveItem it = items[blockIdx.y];
  int n = it.n;
  if (k0 >= n) return;
  int nb = min(TB, n - k0);
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
    int i = e % TB, j = e / TB;
    T[i][j] = (i < nb && j < nb) ? it.a[(k0 + i) + (size_t)(k0 + j) * it.ld] : 0.0;
  }
  __syncthreads();
  if (!LOWER) {
    if (threadIdx.x < TB) Rd[threadIdx.x] = threadIdx.x < nb ? 1.0 / T[threadIdx.x][threadIdx.x] : 0.0;
    __syncthreads();
  }
  const int lane = threadIdx.x & 31, c = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (c >= it.ncols) return;
  double* X = it.x + (size_t)c * it.ldx + k0;
  double x0 = lane < nb ? X[lane] : 0.0, x1 = lane + 32 < nb ? X[lane + 32] : 0.0;
  if (LOWER) {
    for (int j = 0; j < nb; ++j) {
      double xj = __shfl_sync(0xffffffffu, j < 32 ? x0 : x1, j & 31);
      if (lane > j) x0 -= T[lane][j] * xj;
      if (lane + 32 > j) x1 -= T[lane + 32][j] * xj;
    }
  } else {
    for (int j = nb - 1; j >= 0; --j) {
      if (j < 32) {
        if (lane == j) x0 *= Rd[j];
      } else if (lane == j - 32) {
        x1 *= Rd[j];
      }
      double xj = __shfl_sync(0xffffffffu, j < 32 ? x0 : x1, j & 31);
      if (lane < j) x0 -= T[lane][j] * xj;
      if (lane + 32 < j) x1 -= T[lane + 32][j] * xj;
    }
  }
  if (lane < nb) X[lane] = x0;
  if (lane + 32 < nb) X[lane + 32] = x1;
}

// Which diagonal-block form to launch for `cols` columns in total: one
// thread per column issues 2080 FP64 warp instructions per 32 columns, one
// warp per column 128 per column; with at most one warp per SM sub-partition
// (152 x 4) each form takes max(1, cols / (32 * 608)) resp. cols / 608 rounds,
// so the warp form wins below 608 * 2080 / 128 = 9880 columns.
inline bool lus_warp_diag(int items, int ncols) { return (long long)items * ncols < 9880; }

// row interchanges as one gather: X[i] := X[perm[i]] with perm the net
// permutation of the LU's sequential interchanges; a column at a time
// through shared memory (n doubles).  grid (column groups of 8, items)
static __global__ void __launch_bounds__(256) k_lus_gather(const SolveItem* items) {
  extern __shared__ double tmp[];
  SolveItem it = items[blockIdx.y];
  const int n = it.n;
  if (n == 0) return;
  const int c0 = blockIdx.x * 8, c1 = min(it.ncols, c0 + 8);
  for (int c = c0; c < c1; ++c) {
    double* X = it.x + (size_t)c * it.ldx;
    for (int i = threadIdx.x; i < n; i += blockDim.x) tmp[i] = X[it.perm[i]];
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) X[i] = tmp[i];
    __syncthreads();
  }
}

// X := A^-1 X for an LU-factored A and a few right-hand sides (NC columns
// at most), one CTA of 256 threads per item, everything in one launch: the
// rows of X are gathered into shared memory by the net permutation (gather
// = 1) or taken as they are (0); then the unit-lower and the upper
// triangular solves run in 32-row blocks: warp 0 solves the diagonal block
// with its 32 rows in registers (x_j broadcast by a shuffle), and all
// threads update the rows below (above) with the block's 32 new entries,
// one barrier per block.  For the solve sweeps with one to NC columns,
// where the blocked multi-launch solve pays ~4 dependent launches per
// 64 rows for a few thousand flops.  dynamic shared memory: n_cap * NC doubles.
template <int NC>
static __global__ void __launch_bounds__(256) k_lus_small(const SolveItem* items, int gather) {
  extern __shared__ double xs[];          // [NC][n] column-major, ld n
  const SolveItem it = items[blockIdx.x];
  const int n = it.n, nc = min(NC, it.ncols);
  if (n == 0) return;
  const double* A = it.a;
  const int ld = it.ld;
  for (int e = threadIdx.x; e < n * NC; e += blockDim.x) {
    const int i = e % n, c = e / n;
    const int src = gather ? it.perm[i] : i;
    xs[e] = c < nc ? it.x[src + (size_t)c * it.ldx] : 0.0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // ---- unit lower, forward
  for (int k0 = 0; k0 < n; k0 += 32) {
    const int kb = min(32, n - k0);
    if (w == 0) {
      double x[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) x[c] = lane < kb ? xs[k0 + lane + c * n] : 0.0;
      // the lane's row of the block's strictly lower part, loaded before the
      // chain (independent loads, one memory latency instead of one per step)
      double lr[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) lr[j] = lane > j && lane < kb ? A[(k0 + lane) + (size_t)(k0 + j) * ld] : 0.0;
#pragma unroll
      for (int j = 0; j < 31; ++j)
        if (j < kb - 1)
#pragma unroll
          for (int c = 0; c < NC; ++c) x[c] -= lr[j] * __shfl_sync(0xffffffffu, x[c], j);
      if (lane < kb)
#pragma unroll
        for (int c = 0; c < NC; ++c) xs[k0 + lane + c * n] = x[c];
    }
    __syncthreads();
    for (int i = k0 + kb + threadIdx.x; i < n; i += blockDim.x) {
      double acc[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[c] = 0.0;
      if (kb == 32) {   // full block: the 32 loads of the row issued together
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const double l = A[i + (size_t)(k0 + j) * ld];
#pragma unroll
          for (int c = 0; c < NC; ++c) acc[c] = fma(l, xs[k0 + j + c * n], acc[c]);
        }
      } else {
        for (int j = 0; j < kb; ++j) {
          const double l = A[i + (size_t)(k0 + j) * ld];
#pragma unroll
          for (int c = 0; c < NC; ++c) acc[c] = fma(l, xs[k0 + j + c * n], acc[c]);
        }
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) xs[i + c * n] -= acc[c];
    }
    __syncthreads();
  }
  // ---- upper, backward
  for (int k0 = ((n - 1) / 32) * 32; k0 >= 0; k0 -= 32) {
    const int kb = min(32, n - k0);
    if (w == 0) {
      double x[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) x[c] = lane < kb ? xs[k0 + lane + c * n] : 0.0;
      // reciprocals of the block's diagonal, one per lane, and the lane's
      // row of the block's strictly upper part, loaded before the chain
      const double rdl = lane < kb ? 1.0 / A[(k0 + lane) + (size_t)(k0 + lane) * ld] : 0.0;
      double ur[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) ur[j] = lane < j && j < kb ? A[(k0 + lane) + (size_t)(k0 + j) * ld] : 0.0;
#pragma unroll
      for (int j = 31; j >= 0; --j) {
        if (j < kb) {
          const double rd = __shfl_sync(0xffffffffu, rdl, j);
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            const double xj = __shfl_sync(0xffffffffu, x[c], j) * rd;
            if (lane == j) x[c] = xj;
            x[c] -= ur[j] * xj;
          }
        }
      }
      if (lane < kb)
#pragma unroll
        for (int c = 0; c < NC; ++c) xs[k0 + lane + c * n] = x[c];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < k0; i += blockDim.x) {
      double acc[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[c] = 0.0;
      if (kb == 32) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const double u = A[i + (size_t)(k0 + j) * ld];
#pragma unroll
          for (int c = 0; c < NC; ++c) acc[c] = fma(u, xs[k0 + j + c * n], acc[c]);
        }
      } else {
        for (int j = 0; j < kb; ++j) {
          const double u = A[i + (size_t)(k0 + j) * ld];
#pragma unroll
          for (int c = 0; c < NC; ++c) acc[c] = fma(u, xs[k0 + j + c * n], acc[c]);
        }
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) xs[i + c * n] -= acc[c];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * nc; e += blockDim.x) {
    const int i = e % n, c = e / n;
    it.x[i + (size_t)c * it.ldx] = xs[e];
  }
}

// net permutation of the sequential interchanges ipiv[0..n): perm[i] is the
// original row that ends in row i (one thread; n integer swaps)
__device__ inline void ipiv_to_perm(const int* ipiv, int n, int* perm) {
  for (int i = 0; i < n; ++i) perm[i] = i;
  for (int k = 0; k < n; ++k) {
    int q = ipiv[k];
    if (q != k) {
      int x = perm[k];
      perm[k] = perm[q];
      perm[q] = x;
    }
  }
}

// the same in shared memory (n <= 4096): the interchanges are read in one
// coalesced pass, the sequential composition runs on shared memory in one
// thread, and the permutation is written back in one pass; one CTA
__device__ inline void ipiv_to_perm_sm(const int* ipiv, int n, int* perm, int* sp, int* sq) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    sp[i] = i;
    sq[i] = ipiv[i];
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int k = 0; k < n; ++k) {
      const int q = sq[k];
      if (q != k) {
        const int x = sp[k];
        sp[k] = sp[q];
        sp[q] = x;
      }
    }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) perm[i] = sp[i];
}

// dynamic shared memory 2 n ints (n <= 4096); the global form beyond
static __global__ void k_ipiv_perm(const int* ipiv, int n, int* perm) {
  extern __shared__ int ipsm[];
  if (n > 4096) {
    if (threadIdx.x == 0) ipiv_to_perm(ipiv, n, perm);
    return;
  }
  ipiv_to_perm_sm(ipiv, n, perm, ipsm, ipsm + n);
}

// trailing update after diagonal block k0: lower -> rows below, upper -> rows
// above:  X[rows] -= A[rows, k0:k0+TB] X[k0:k0+TB];  grid (coltiles, rowtiles, items)
template <int LOWER, int PM = PM_FMA>
static __global__ void __launch_bounds__(256, 2) k_lus_update(const SolveItem* items, int k0) {
  SolveItem it = items[blockIdx.z];
  int n = it.n;
  if (k0 >= n) return;
  int nb = min(TB, n - k0);
  int r0, r1;
  if (LOWER) {
    r0 = k0 + nb;
    r1 = n;
  } else {
    r0 = 0;
    r1 = k0;
  }
  int i0 = r0 + blockIdx.y * 64, j0 = blockIdx.x * 64;
  if (i0 >= r1 || j0 >= it.ncols) return;
  tile_gemm<PM>(it.a + i0 + (size_t)k0 * it.ld, it.ld, it.x + k0 + (size_t)j0 * it.ldx, it.ldx,
                it.x + i0 + (size_t)j0 * it.ldx, it.ldx, r1 - i0, it.ncols - j0, nb, -1.0);
}

}  // namespace aifmm

namespace aifmm {

// 64x64 FP64 tile with a transposed left operand:
// C[0..mr, 0..nc] += alpha * A^T B, A column-major K x mr (lda), B K x nc (ldb)
template <typename CT = double>
__device__ inline void tile_gemm_64_tn(const double* A, int lda, const double* B, int ldb, double* C, int ldc,
                                       int mr, int nc, int K, double alpha) {
  __shared__ CT As[16][64 + 1];
  __shared__ CT Bs[16][64 + 1];
  int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  CT acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = CT(0);
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      int k2 = e & 15, ii = e >> 4;
      As[k2][ii] = (ii < mr && k0 + k2 < K) ? (CT)A[(k0 + k2) + (size_t)ii * lda] : CT(0);
      Bs[k2][ii] = (ii < nc && k0 + k2 < K) ? (CT)B[(k0 + k2) + (size_t)ii * ldb] : CT(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      CT av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int i = ty + 16 * a, j = tx + 16 * b;
      if (i < mr && j < nc) C[i + (size_t)j * ldc] += alpha * (double)acc[a][b];
    }
}

// C += alpha A^T B, 64 x 64 tile (A column-major K x mr, lda)
template <int PM>
__device__ inline void tile_gemm_tn(const double* A, int lda, const double* B, int ldb, double* C, int ldc, int mr,
                                    int nc, int K, double alpha) {
  if (PM == PM_OZ && nc > THIN_NC) {
    extern __shared__ __align__(16) unsigned char oz_dyn[];
    tile_gemm_64_oz<true>(A, lda, B, ldb, C, ldc, min(64, mr), min(64, nc), K, alpha, oz_dyn);
  } else if (PM == PM_TF32 && nc > THIN_NC) {
    tile_gemm_64_tf32<true>(A, lda, B, ldb, C, ldc, min(64, mr), min(64, nc), K, alpha);
  } else if (PM == PM_F32 || PM == PM_TF32) {
    tile_gemm_64_tn<float>(A, lda, B, ldb, C, ldc, mr, nc, K, alpha);
  } else {
    tile_gemm_64_tn(A, lda, B, ldb, C, ldc, mr, nc, K, alpha);
  }
}


}  // namespace aifmm

namespace aifmm {

// panel k0..k0+LU_NB of a batched LU factored in shared memory (rows k0..n,
// column-major with ld h = n - k0).  Warp 0 searches the pivot and swaps the
// two panel rows; then every thread scales and updates the rows it owns.
// Interchanges outside the panel are applied afterwards by k_lu_laswp.
// Any block size that is a multiple of 32 (lu_panel_threads: more threads
// for taller panels, whose rank-1 updates sit on the critical path of every
// column step).  dynamic shared memory: (maxh * LU_NB) doubles; items with
// n - k0 > maxh are skipped here (they take the global-memory panel path).
static __global__ void __launch_bounds__(1024) k_lu_panel_sm(const LuItem* items, int k0, int maxh, int* err) {
  extern __shared__ double Ps[];
  __shared__ int sing;
  LuItem it = items[blockIdx.x];
  const int n = it.n;
  if (k0 >= n) return;
  const int h = n - k0;
  if (h > maxh) return;
  const int nbw = min(LU_NB, h);
  double* A = it.a;
  const int ld = it.ld;
  for (int e = threadIdx.x; e < h * nbw; e += blockDim.x) {
    int i = e % h, j = e / h;
    Ps[i + (size_t)j * h] = A[(k0 + i) + (size_t)(k0 + j) * ld];
  }
  if (threadIdx.x == 0) sing = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (int jj = 0; jj < nbw; ++jj) {
    if (threadIdx.x < 32) {
      double bv = -1.0;
      int bi = -1;
      for (int i = jj + lane; i < h; i += 32) {
        double x = fabs(Ps[i + (size_t)jj * h]);
        if (x > bv) {
          bv = x;
          bi = i;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi >= 0 && (bi < 0 || oi < bi))) {
          bv = ov;
          bi = oi;
        }
      }
      double cm = it.colmax ? it.colmax[k0 + jj] : 0.0;
      if (!(bv > 1e-14 * cm) || !(bv >= LU_PIV_MIN)) {
        if (lane == 0) sing = 1;
      } else {
        if (lane == 0) it.ipiv[k0 + jj] = k0 + bi;
        if (bi != jj && lane < nbw) {
          double x = Ps[jj + (size_t)lane * h];
          Ps[jj + (size_t)lane * h] = Ps[bi + (size_t)lane * h];
          Ps[bi + (size_t)lane * h] = x;
        }
      }
    }
    __syncthreads();
    if (sing) {
      // the interchanges of the columns not reached stay the identity, so
      // the kernels that follow in this step read valid rows
      for (int q = jj + threadIdx.x; q < nbw; q += blockDim.x) it.ipiv[k0 + q] = k0 + q;
      if (threadIdx.x == 0) set_err(err, DERR_SINGULAR);
      return;
    }
    const double rpiv = 1.0 / Ps[jj + (size_t)jj * h];
    for (int i = jj + 1 + threadIdx.x; i < h; i += blockDim.x) {
      double l = Ps[i + (size_t)jj * h] * rpiv;
      Ps[i + (size_t)jj * h] = l;
      for (int cc = jj + 1; cc < nbw; ++cc) Ps[i + (size_t)cc * h] -= l * Ps[jj + (size_t)cc * h];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < h * nbw; e += blockDim.x) {
    int i = e % h, j = e / h;
    A[(k0 + i) + (size_t)(k0 + j) * ld] = Ps[i + (size_t)j * h];
  }
}

// The same panel with every row in one thread's registers, for panels of at
// most LU_RG_MAXH rows (one thread per row).  Rows never move: a thread
// tracks the position of its row under the LAPACK interchanges (the pivot
// row takes position jj, the row at jj takes the pivot's) and writes the
// row to its final position at the end.  Per column one barrier: each warp
// finds its best candidate (largest |a|, then the smallest position; the
// bit patterns of non-negative doubles order as their values, so the
// search is integer work) and its winning lane publishes the row and the
// pivot's reciprocal in a double-buffered shared slot; after the barrier
// every thread picks the block's winner from the warps' slots and updates
// its row.  The multipliers and updates are the same operations as in
// k_lu_panel_sm, and the interchanges the same, so the results are equal
// bit for bit.  Singularity test as there, on bit patterns.  grid items,
// blockDim a multiple of 32 covering n - k0 rows (at most LU_RG_MAXH).
constexpr int LU_RG_MAXH = 512;
static __global__ void __launch_bounds__(LU_RG_MAXH) k_lu_panel_rg(const LuItem* items, int k0, int* err) {
  __shared__ long long ck[2][LU_RG_MAXH / 32];            // warp candidates: key
  __shared__ int cp[2][LU_RG_MAXH / 32];                  // and position
  __shared__ double crow[2][LU_RG_MAXH / 32][LU_NB + 1];  // their rows; [LU_NB]: 1 / pivot
  __shared__ long long thr[LU_NB];                        // bits of 1e-14 x column maximum
  const LuItem it = items[blockIdx.x];
  const int n = it.n;
  if (k0 >= n) return;
  const int h = n - k0;
  const int nbw = min(LU_NB, h);
  const int t = threadIdx.x, lane = t & 31, w = t >> 5, nw = blockDim.x >> 5;
  double* A = it.a;
  const int ld = it.ld;
  double a[LU_NB];
#pragma unroll
  for (int j = 0; j < LU_NB; ++j) a[j] = (t < h && j < nbw) ? A[(k0 + t) + (size_t)(k0 + j) * ld] : 0.0;
  if (t < LU_NB) thr[t] = __double_as_longlong(1e-14 * ((it.colmax && t < nbw) ? it.colmax[k0 + t] : 0.0));
  int pos = t;
  bool live = t < h;   // not yet a pivot row
  __syncthreads();
#pragma unroll
  for (int jj = 0; jj < LU_NB; ++jj) {
    if (jj < nbw) {
      const int par = jj & 1;
      long long key = -1;   // -1: no candidate (pivot rows, padding, NaN)
      if (live) {
        const long long kb = __double_as_longlong(fabs(a[jj]));
        key = kb > 0x7ff0000000000000LL ? -1 : kb;
      }
      long long wk = key;
      int wp = pos;
      for (int o = 16; o > 0; o >>= 1) {
        const long long ok = __shfl_xor_sync(0xffffffffu, wk, o);
        const int op = __shfl_xor_sync(0xffffffffu, wp, o);
        if (ok > wk || (ok == wk && op < wp)) {
          wk = ok;
          wp = op;
        }
      }
      if (wk >= 0 && pos == wp) {   // the warp's winning lane
        double* cr = crow[par][w];
#pragma unroll
        for (int cc = 0; cc < LU_NB; ++cc)
          if (cc >= jj) cr[cc] = a[cc];
        cr[LU_NB] = 1.0 / a[jj];
      }
      if (lane == 0) {
        ck[par][w] = wk;
        cp[par][w] = wp;
      }
      __syncthreads();
      long long bk = ck[par][0];
      int bp = cp[par][0], bw = 0;
      for (int u = 1; u < nw; ++u) {
        const long long k2 = ck[par][u];
        const int p2 = cp[par][u];
        if (k2 > bk || (k2 == bk && p2 < bp)) {
          bk = k2;
          bp = p2;
          bw = u;
        }
      }
      // bk > thr: |pivot| > 1e-14 x column maximum; bk >= 2^52: a normal number
      if (!(bk > thr[jj]) || !(bk >= 0x0010000000000000LL)) {
        for (int q = jj + t; q < nbw; q += blockDim.x) it.ipiv[k0 + q] = k0 + q;
        if (t == 0) set_err(err, DERR_SINGULAR);
        return;
      }
      const double* pr = crow[par][bw];
      if (live && pos == bp) {
        it.ipiv[k0 + jj] = k0 + bp;
        live = false;
        pos = jj;
      } else if (pos == jj) {
        pos = bp;
      }
      if (live) {
        const double l = a[jj] * pr[LU_NB];
        a[jj] = l;
#pragma unroll
        for (int cc = 0; cc < LU_NB; ++cc)
          if (cc > jj && cc < nbw) a[cc] -= l * pr[cc];
      }
    }
  }
  if (t < h)
#pragma unroll
    for (int j = 0; j < LU_NB; ++j)
      if (j < nbw) A[(k0 + pos) + (size_t)(k0 + j) * ld] = a[j];
}

// the panel's interchanges applied to every column outside the panel
// (left: the L factor, right: the part still to be factored, then B);
// grid (colchunks over n + nb, items)
static __global__ void __launch_bounds__(128) k_lu_laswp(const LuItem* items, int k0, int maxh) {
  LuItem it = items[blockIdx.y];
  const int n = it.n;
  if (k0 >= n || n - k0 > maxh) return;
  const int nbw = min(LU_NB, n - k0);
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n + it.nb || (c >= k0 && c < k0 + nbw)) return;
  double* col = lu_col(it, c);
  for (int jj = 0; jj < nbw; ++jj) {
    int p = it.ipiv[k0 + jj];
    if (p != k0 + jj) {
      double x = col[k0 + jj];
      col[k0 + jj] = col[p];
      col[p] = x;
    }
  }
}

// threads of k_lu_panel_sm for panels of up to h rows
inline int lu_panel_threads(int h) { return h > 512 ? 1024 : h > 256 ? 512 : 256; }

// global-memory panel for items too tall for shared memory
static __global__ void __launch_bounds__(256) k_lu_panel_big(const LuItem* items, int k0, int maxh, int* err) {
  LuItem it = items[blockIdx.x];
  if (k0 >= it.n || it.n - k0 <= maxh) return;
  // the panel algorithm of k_lu_panel_sm in global memory, full-row
  // interchanges (through the columns of B too)
  __shared__ double shv[32];
  __shared__ int shi[32];
  int n = it.n;
  double* A = it.a;
  const int ld = it.ld;
  int kend = min(n, k0 + LU_NB);
  for (int j = k0; j < kend; ++j) {
    ArgMax best;
    best.v = -1.0;
    best.i = -1;
    for (int i = j + threadIdx.x; i < n; i += blockDim.x) {
      ArgMax c;
      c.v = fabs(A[i + (size_t)j * ld]);
      c.i = i;
      best = amax_pick(best, c);
    }
    best = block_amax(best, shv, shi);
    int p = best.i;
    double cm = it.colmax ? it.colmax[j] : 0.0;
    if (!(best.v > 1e-14 * cm) || !(best.v >= LU_PIV_MIN)) {
      for (int q = j + threadIdx.x; q < kend; q += blockDim.x) it.ipiv[q] = q;
      if (threadIdx.x == 0) set_err(err, DERR_SINGULAR);
      return;
    }
    if (threadIdx.x == 0) it.ipiv[j] = p;
    if (p != j)
      for (int c = threadIdx.x; c < n + it.nb; c += blockDim.x) {
        double* col = lu_col(it, c);
        double t = col[j];
        col[j] = col[p];
        col[p] = t;
      }
    __syncthreads();
    const double rpiv = 1.0 / A[j + (size_t)j * ld];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[i + (size_t)j * ld] *= rpiv;
    __syncthreads();
    int w = kend - j - 1, hh = n - j - 1;
    for (int e = threadIdx.x; e < w * hh; e += blockDim.x) {
      int i = j + 1 + e % hh, c = j + 1 + e / hh;
      A[i + (size_t)c * ld] -= A[i + (size_t)j * ld] * A[j + (size_t)c * ld];
    }
    __syncthreads();
  }
}

}  // namespace aifmm
