// Device view of one level of the extended system (see FacLevel).
#pragma once
#include "common.cuh"

namespace aifmm {

struct LV {
  int l, d, n, nb, M, R, P, Rp, ns5, ns6;
  int* m;
  int* r;
  double* XX;
  double* XY;
  double* LX;
  double* LY;
  double* U;
  double* V;
  double* Ud;
  double* Vd;
  double* LU;
  int* ipiv;
  int* pperm;     // net row permutation of each pivot LU (ipiv applied in order)
  unsigned* flag;

  __host__ __device__ double* xx(int p, int s) const { return XX + ((size_t)p * ns5 + s) * M * M; }  // ld M
  __host__ __device__ double* xy(int p, int s) const { return XY + ((size_t)p * ns5 + s) * M * R; }  // ld M
  __host__ __device__ double* lx(int p, int s) const { return LX + ((size_t)p * ns5 + s) * R * M; }  // ld R
  __host__ __device__ double* ly(int p, int s) const { return LY + ((size_t)p * ns6 + s) * R * R; }  // ld R
  __host__ __device__ double* u(int p) const { return U + (size_t)p * M * R; }                       // ld M
  __host__ __device__ double* v(int p) const { return V + (size_t)p * M * R; }                       // ld M
  __host__ __device__ double* ud(int p) const { return Ud + (size_t)p * R * Rp; }                    // ld R
  __host__ __device__ double* vd(int p) const { return Vd + (size_t)p * R * Rp; }                    // ld R
  __host__ __device__ double* lu(int p) const { return LU + (size_t)p * P * P; }                     // ld P
  __host__ __device__ int* piv(int p) const { return ipiv + (size_t)p * P; }
  __host__ __device__ int* pp(int p) const { return pperm + (size_t)p * P; }
  __host__ __device__ int centre5() const { return d == 2 ? 12 : 62; }
};

// coupled row / column descriptors of the box being eliminated
struct Coupled {
  int box;      // partner box (Morton), or the eliminated box itself for the special entry
  int type;     // rows: 0 = X_p, 1 = Lc_p, 2 = Lc_b (special); cols: 0 = x_q, 1 = y_q, 2 = y_b
  int size;     // rows or columns
  int off;      // offset in the stacked rows / columns
};

constexpr int MAXC = 28;  // 3^d + 1 for d <= 3

}  // namespace aifmm
