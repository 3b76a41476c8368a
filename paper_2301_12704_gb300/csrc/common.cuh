// Shared device helpers: kernel evaluation, box index arithmetic on the
// uniform 2^d tree, stencil slots, colours, reductions, error reporting.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace aifmm {

// ---- error word (device -> host) ------------------------------------------
enum DevErr : int {
  DERR_NONE = 0,
  DERR_SINGULAR = 1,
  DERR_CAPACITY = 2,
  DERR_DUPLICATE = 3,
  DERR_NUMERIC = 4,
};

__device__ inline void set_err(int* err, int code) {
  if (err) atomicCAS(err, 0, code);
}

// ---- interaction kernels (Sec. 4) -----------------------------------------
struct KParams {
  int kind;        // 0 log2d, 1 invr3d, 2 invr2d, 3 gauss
  int dim;
  double diag;
  double inv_len2; // 1 / length^2
};

// Points are stored SoA in tree order: x[N], y[N], z[N] (z unused in 2D).
struct Pts {
  const double* x;
  const double* y;
  const double* z;
};

// A_ij for tree positions i, j.  The squared distance is formed with
// explicit round-to-nearest operations (no contraction) so that it is the
// same IEEE value as the oracle's.
__device__ inline double keval(const KParams& k, const Pts& p, int i, int j) {
  if (i == j) return k.diag;
  double dx = __dsub_rn(p.x[i], p.x[j]);
  double dy = __dsub_rn(p.y[i], p.y[j]);
  double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
  if (k.dim == 3) {
    double dz = __dsub_rn(p.z[i], p.z[j]);
    r2 = __dadd_rn(r2, __dmul_rn(dz, dz));
  }
  switch (k.kind) {
    case 0: return 0.5 * log(r2);
    case 1:
    case 2: return 1.0 / sqrt(r2);
    default: return exp(-r2 * k.inv_len2);
  }
}

// ---- uniform tree index arithmetic ----------------------------------------
// Boxes of level l are numbered in Morton (Z) order, x the lowest bit.
__host__ __device__ inline int morton_key(const int* c, int d, int l) {
  int key = 0;
  for (int b = 0; b < l; ++b)
    for (int k = 0; k < d; ++k) key |= ((c[k] >> b) & 1) << (b * d + k);
  return key;
}

__host__ __device__ inline void morton_coords(int key, int d, int l, int* c) {
  for (int k = 0; k < 3; ++k) c[k] = 0;
  for (int b = 0; b < l; ++b)
    for (int k = 0; k < d; ++k) c[k] |= ((key >> (b * d + k)) & 1) << b;
}

__host__ __device__ inline int ipow(int a, int e) {
  int r = 1;
  for (int i = 0; i < e; ++i) r *= a;
  return r;
}

// slot of q in the 5^d stencil around p (offsets -2..2), -1 if outside
__host__ __device__ inline int slot5(const int* p, const int* q, int d) {
  int s = 0, m = 1;
  for (int k = 0; k < d; ++k) {
    int o = q[k] - p[k];
    if (o < -2 || o > 2) return -1;
    s += (o + 2) * m;
    m *= 5;
  }
  return s;
}

// coordinates of stencil-5 slot s around p (may fall outside the grid)
__host__ __device__ inline void slot5_coords(const int* p, int s, int d, int* q) {
  for (int k = 0; k < 3; ++k) q[k] = 0;
  for (int k = 0; k < d; ++k) {
    q[k] = p[k] + (s % 5) - 2;
    s /= 5;
  }
}

// origin of the 6^d window of p: the children of N(parent(p)) (IL + N)
__host__ __device__ inline int win6_origin(int pk) { return 2 * ((pk >> 1) - 1); }

__host__ __device__ inline int slot6(const int* p, const int* q, int d) {
  int s = 0, m = 1;
  for (int k = 0; k < d; ++k) {
    int o = q[k] - win6_origin(p[k]);
    if (o < 0 || o >= 6) return -1;
    s += o * m;
    m *= 6;
  }
  return s;
}

__host__ __device__ inline void slot6_coords(const int* p, int s, int d, int* q) {
  for (int k = 0; k < 3; ++k) q[k] = 0;
  for (int k = 0; k < d; ++k) {
    q[k] = win6_origin(p[k]) + (s % 6);
    s /= 6;
  }
}

__host__ __device__ inline bool in_grid(const int* q, int d, int n) {
  for (int k = 0; k < d; ++k)
    if (q[k] < 0 || q[k] >= n) return false;
  return true;
}

__host__ __device__ inline int cheb(const int* p, const int* q, int d) {
  int m = 0;
  for (int k = 0; k < d; ++k) {
    int o = q[k] - p[k];
    o = o < 0 ? -o : o;
    m = o > m ? o : m;
  }
  return m;
}

// distance-2 colour: sum_k (c_k mod 3) 3^k
__host__ __device__ inline int colour_of(const int* c, int d) {
  int s = 0, m = 1;
  for (int k = 0; k < d; ++k) {
    s += (c[k] % 3) * m;
    m *= 3;
  }
  return s;
}

// number of boxes of colour col on an n^d grid
__host__ __device__ inline int colour_count(int col, int d, int n) {
  int cnt = 1;
  for (int k = 0; k < d; ++k) {
    int ck = col % 3;
    col /= 3;
    cnt *= (ck < n) ? (n - ck + 2) / 3 : 0;
  }
  return cnt;
}

// t-th box (Morton index) of colour col, t in [0, colour_count)
__host__ __device__ inline int colour_box(int col, int t, int d, int l) {
  int n = 1 << l;
  int c[3] = {0, 0, 0};
  for (int k = 0; k < d; ++k) {
    int ck = col % 3;
    col /= 3;
    int cntk = (n - ck + 2) / 3;
    c[k] = ck + 3 * (t % cntk);
    t /= cntk;
  }
  return morton_key(c, d, l);
}

// index of the box with coordinates c among the boxes of its colour on an
// n^d grid (the inverse of colour_box)
__host__ __device__ inline int colour_index(const int* c, int d, int n) {
  int t = 0, stride = 1;
  for (int k = 0; k < d; ++k) {
    const int ck = c[k] % 3;
    t += (c[k] / 3) * stride;
    stride *= (n - ck + 2) / 3;
  }
  return t;
}

// ---- reductions -------------------------------------------------------------
__device__ inline double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// four warp sums at once, the result in every lane: a transposing butterfly
// (the first two steps halve the values a lane keeps, so lane groups of 8
// finish one sum each), 6 FP64 additions instead of 20, then a broadcast
__device__ inline void warp_sum4(double (&v)[4]) {
  const int lane = threadIdx.x & 31;
  const bool h16 = lane & 16, h8 = lane & 8;
  double k0 = h16 ? v[2] : v[0], k1 = h16 ? v[3] : v[1];
  k0 += __shfl_xor_sync(0xffffffffu, h16 ? v[0] : v[2], 16);
  k1 += __shfl_xor_sync(0xffffffffu, h16 ? v[1] : v[3], 16);
  double s = h8 ? k1 : k0;                         // sum number 2 h16 + h8
  s += __shfl_xor_sync(0xffffffffu, h8 ? k0 : k1, 8);
  s += __shfl_xor_sync(0xffffffffu, s, 4);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  s += __shfl_xor_sync(0xffffffffu, s, 1);
#pragma unroll
  for (int u = 0; u < 4; ++u) v[u] = __shfl_sync(0xffffffffu, s, 8 * u);
}

// argmax of |v| with the lowest index on ties; returns (value, index)
struct ArgMax {
  double v;
  int i;
};

__device__ inline ArgMax amax_pick(ArgMax a, ArgMax b) {
  if (b.v > a.v || (b.v == a.v && b.i >= 0 && (a.i < 0 || b.i < a.i))) return b;
  return a;
}

__device__ inline ArgMax warp_amax(ArgMax a) {
  for (int o = 16; o > 0; o >>= 1) {
    ArgMax b;
    b.v = __shfl_xor_sync(0xffffffffu, a.v, o);
    b.i = __shfl_xor_sync(0xffffffffu, a.i, o);
    a = amax_pick(a, b);
  }
  return a;
}

// block-wide argmax; every thread gets the result.  `sh` needs 2*32 slots.
__device__ inline ArgMax block_amax(ArgMax a, double* shv, int* shi) {
  a = warp_amax(a);
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) {
    shv[w] = a.v;
    shi[w] = a.i;
  }
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  if (w == 0) {
    ArgMax b;
    b.v = lane < nw ? shv[lane] : -1.0;
    b.i = lane < nw ? shi[lane] : -1;
    b = warp_amax(b);
    if (lane == 0) {
      shv[0] = b.v;
      shi[0] = b.i;
    }
  }
  __syncthreads();
  ArgMax r;
  r.v = shv[0];
  r.i = shi[0];
  __syncthreads();
  return r;
}

__device__ inline double block_sum(double v, double* sh) {
  v = warp_sum(v);
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  if (w == 0) {
    double s = lane < nw ? sh[lane] : 0.0;
    s = warp_sum(s);
    if (lane == 0) sh[0] = s;
  }
  __syncthreads();
  double r = sh[0];
  __syncthreads();
  return r;
}

}  // namespace aifmm
