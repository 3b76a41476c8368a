// Solve phase on the GPU (Sec. 3.6, Algorithm 3 and the Remark after it):
// the right-hand-side Schur operations replayed in elimination order
// (forward sweep, part of T_As), the dense level-1 solve for the level-2
// multipoles, and back substitution level 2..L in reverse colour order.
// Also the NNCA H^2 product (upward P2M/M2M, M2L, downward L2L/L2P, P2P) and
// the exact direct-sum product used to measure true residuals.
#include <algorithm>
#include <mutex>

#include "dense.cuh"
#include "internal.h"
#include "level.cuh"

namespace aifmm {

namespace {

LV view(Handle& h, FacLevel& F) {
  LV v;
  v.l = F.l;
  v.d = h.d;
  v.n = F.n;
  v.nb = F.nb;
  v.M = F.M;
  v.R = F.R;
  v.P = F.P;
  v.Rp = F.Rp;
  v.ns5 = F.ns5;
  v.ns6 = F.ns6;
  v.m = F.m;
  v.r = F.r;
  v.XX = F.XX;
  v.XY = F.XY;
  v.LX = F.LX;
  v.LY = F.LY;
  v.U = F.U;
  v.V = F.V;
  v.Ud = F.Ud;
  v.Vd = F.Vd;
  v.LU = F.LU;
  v.ipiv = F.ipiv;
  v.pperm = F.pperm;
  v.flag = F.flag;
  return v;
}

// per-level solve vectors: X rows (m), Lc rows (r), solution x (m); each box
// holds an (M x nrhs) / (R x nrhs) column-major block.
struct SV {
  double* bX;
  double* bL;
  double* xX;
  double* w;      // per-box workspace (P x nrhs)
  int nrhs;
};

__device__ inline double* bx(const LV& v, const SV& s, int b) { return s.bX + (size_t)b * v.M * s.nrhs; }
__device__ inline double* bl(const LV& v, const SV& s, int b) { return s.bL + (size_t)b * v.R * s.nrhs; }
__device__ inline double* xx_(const LV& v, const SV& s, int b) { return s.xX + (size_t)b * v.M * s.nrhs; }
__device__ inline double* ws(const LV& v, const SV& s, int b) { return s.w + (size_t)b * v.P * s.nrhs; }

// original-order rhs -> leaf X rows (tree order)
__global__ void k_leaf_in(LV v, SV s, const int* __restrict__ start, const int* __restrict__ perm,
                          const double* __restrict__ rhs, int64_t ld) {
  int b = blockIdx.x;
  int st = start[b], m = start[b + 1] - st;
  for (int e = threadIdx.x; e < m * s.nrhs; e += blockDim.x) {
    int i = e % m, k = e / m;
    bx(v, s, b)[i + (size_t)k * v.M] = rhs[perm[st + i] + (size_t)k * ld];
  }
}

__global__ void k_leaf_out(LV v, SV s, const int* __restrict__ start, const int* __restrict__ perm,
                           double* __restrict__ x, int64_t ld) {
  int b = blockIdx.x;
  int st = start[b], m = start[b + 1] - st;
  for (int e = threadIdx.x; e < m * s.nrhs; e += blockDim.x) {
    int i = e % m, k = e / m;
    x[perm[st + i] + (size_t)k * ld] = xx_(v, s, b)[i + (size_t)k * v.M];
  }
}

// Each box's Piv^-1 is applied with the batched blocked LU solve of the
// factorisation (row interchanges, unit-lower and upper 64-row diagonal
// blocks, tiled GEMM trailing updates) over the boxes of one colour; the
// coupling products are 64x64 register-tiled GEMMs.

// forward sweep, step 1: w = P^T [beta; 0] and the solve item of each box
__global__ void k_fwd_prep(LV v, SV s, int col, SolveItem* items) {
  int t = blockIdx.x;
  int b = colour_box(col, t, v.d, v.l);
  const int m = v.m[b], r = v.r[b], n = m + r;
  double* w = ws(v, s, b);
  if (threadIdx.x == 0) {
    SolveItem it;
    it.a = v.lu(b);
    it.ipiv = v.piv(b);
    it.n = m ? n : 0;
    it.ld = v.P;
    it.x = w;
    it.ldx = v.P;
    it.ncols = s.nrhs;
    it.perm = v.pp(b);
    items[t] = it;
  }
  if (m == 0) return;
  // the LU's row interchanges are applied here, as a gather
  const double* beta = bx(v, s, b);
  const int* pr = v.pp(b);
  for (int e = threadIdx.x; e < n * s.nrhs; e += blockDim.x) {
    int i = e % n, k = e / n;
    int src = pr[i];
    w[i + (size_t)k * v.P] = src < m ? beta[src + (size_t)k * v.M] : 0.0;
  }
}

// forward sweep, step 2: right-hand-side Schur operations on the coupled
// rows: X_p -= K_pb w_x (p not yet eliminated), Lc_p -= P2L_pb w_x
// (p eliminated), Lc_b += w_z.  grid (3^d * rt, column tiles, cnt), 64-row
// tiles of the target block.  PM: the products' mode (PM_FMA, or the
// 8-digit balanced tensor-core tile for many right-hand sides)
template <int PM>
__global__ void __launch_bounds__(256) k_fwd_upd(LV v, SV s, int col, int rt) {
  int t = blockIdx.z, o = blockIdx.x / rt, ti = blockIdx.x % rt;
  int b = colour_box(col, t, v.d, v.l);
  const int m = v.m[b], r = v.r[b];
  if (m == 0) return;
  int i0 = ti * 64, j0 = blockIdx.y * 64;
  if (j0 >= s.nrhs) return;
  int bc[3], q[3];
  morton_coords(b, v.d, v.l, bc);
  int oo = o;
  for (int k = 0; k < 3; ++k) q[k] = bc[k];
  for (int k = 0; k < v.d; ++k) {
    q[k] = bc[k] + (oo % 3) - 1;
    oo /= 3;
  }
  if (!in_grid(q, v.d, v.n)) return;
  int p = morton_key(q, v.d, v.l);
  const double* w = ws(v, s, b);
  const int nc = min(64, s.nrhs - j0);
  if (p == b) {
    if (i0 >= r) return;
    double* tb = bl(v, s, b);
    int mr = min(64, r - i0);
    for (int e = threadIdx.x; e < mr * nc; e += blockDim.x) {
      int i = i0 + e % mr, k = j0 + e / mr;
      tb[i + (size_t)k * v.R] += w[m + i + (size_t)k * v.P];
    }
    return;
  }
  bool elim = colour_of(q, v.d) < col;
  int sp = slot5(q, bc, v.d);
  const double* A;
  int lda, rows, ldt;
  double* tp;
  if (elim) {
    A = v.lx(p, sp);
    lda = v.R;
    rows = v.r[p];
    tp = bl(v, s, p);
    ldt = v.R;
  } else {
    A = v.xx(p, sp);
    lda = v.M;
    rows = v.m[p];
    tp = bx(v, s, p);
    ldt = v.M;
  }
  if (i0 >= rows) return;
  tile_gemm<PM>(A + i0, lda, w + (size_t)j0 * v.P, v.P, tp + i0 + (size_t)j0 * ldt, ldt, min(64, rows - i0), nc, m,
               -1.0);
}

// level transition of the right-hand side: X rows of parent P are the Lc
// rows of its children
__global__ void k_rhs_up(LV vc, SV sc, LV vp, SV sp, const int* __restrict__ cxoff) {
  int P = blockIdx.x;
  int nch = 1 << vc.d;
  for (int a = 0; a < nch; ++a) {
    int c = (P << vc.d) + a;
    int r = vc.r[c], o = cxoff[c];
    const double* src = bl(vc, sc, c);
    double* dst = bx(vp, sp, P);
    for (int e = threadIdx.x; e < r * sc.nrhs; e += blockDim.x) {
      int i = e % r, k = e / r;
      dst[o + i + (size_t)k * vp.M] = src[i + (size_t)k * vc.R];
    }
  }
}

// level-2 multipole right-hand sides into the dense top vector; block 0 also
// writes the top system's solve item
__global__ void k_top_in(LV v, SV s, const int* __restrict__ toff, double* __restrict__ y, int ntop,
                         const double* top, const int* top_ipiv, const int* top_perm, SolveItem* item) {
  int b = blockIdx.x;
  if (b == 0 && threadIdx.x == 0) {
    SolveItem it;
    it.a = top;
    it.ipiv = top_ipiv;
    it.n = ntop;
    it.ld = ntop;
    it.x = y;
    it.ldx = ntop;
    it.ncols = s.nrhs;
    it.perm = top_perm;
    *item = it;
  }
  int r = v.r[b], o = toff[b];
  for (int e = threadIdx.x; e < r * s.nrhs; e += blockDim.x) {
    int i = e % r, k = e / r;
    y[o + i + (size_t)k * ntop] = bl(v, s, b)[i + (size_t)k * v.R];
  }
}

// multipoles y_q of level l: from the level-1 solution (l = 2) or from the
// parent's particles (l >= 3)
struct YSrc {
  const double* top;
  int ntop;
  const int* toff;
  const double* px;    // parent level x
  int pM;
  const int* xoff;
  int d;
};

// y_q as a column-major block: first entry and leading dimension
__device__ inline const double* ybase(const YSrc& y, int l, int q, int nrhs, int& ld) {
  if (l == 2) {
    ld = y.ntop;
    return y.top + y.toff[q];
  }
  ld = y.pM;
  return y.px + (size_t)(q >> y.d) * y.pM * nrhs + y.xoff[q];
}

// back substitution, step 1: w = [beta_b; y_b] and the solve item
__global__ void k_bwd_prep(LV v, SV s, int col, YSrc y, SolveItem* items) {
  int t = blockIdx.x;
  int b = colour_box(col, t, v.d, v.l);
  const int m = v.m[b], r = v.r[b], n = m + r;
  double* w = ws(v, s, b);
  if (threadIdx.x == 0) {
    SolveItem it;
    it.a = v.lu(b);
    it.ipiv = v.piv(b);
    it.n = m ? n : 0;
    it.ld = v.P;
    it.x = w;
    it.ldx = v.P;
    it.ncols = s.nrhs;
    it.perm = v.pp(b);
    items[t] = it;
  }
  if (m == 0) return;
  int ldy;
  const double* yb = ybase(y, v.l, b, s.nrhs, ldy);
  const double* beta = bx(v, s, b);
  for (int e = threadIdx.x; e < n * s.nrhs; e += blockDim.x) {
    int i = e % n, k = e / n;
    w[i + (size_t)k * v.P] = i < m ? beta[i + (size_t)k * v.M] : yb[(i - m) + (size_t)k * ldy];
  }
}

// neighbour o of box b for the backward products: its Morton index and
// stencil slot, the block A (rows of b) and the right operand B (x_q, or
// the multipoles y_q of an eliminated q); false if there is none
__device__ inline bool bwd_term(const LV& v, const SV& s, int col, const YSrc& y, int b, int o, const double*& A,
                                const double*& B, int& ldb, int& cols) {
  int bc[3], q[3];
  morton_coords(b, v.d, v.l, bc);
  int oo = o;
  for (int k = 0; k < 3; ++k) q[k] = bc[k];
  for (int k = 0; k < v.d; ++k) {
    q[k] = bc[k] + (oo % 3) - 1;
    oo /= 3;
  }
  if (!in_grid(q, v.d, v.n)) return false;
  int p = morton_key(q, v.d, v.l);
  if (p == b) return false;
  int sq = slot5(bc, q, v.d);
  bool elim = colour_of(q, v.d) < col;
  cols = elim ? v.r[p] : v.m[p];
  if (cols == 0) return false;
  A = elim ? v.xy(b, sq) : v.xx(b, sq);
  if (elim) {
    B = ybase(y, v.l, p, s.nrhs, ldb);
  } else {
    B = xx_(v, s, p);
    ldb = v.M;
  }
  return true;
}

// back substitution, step 2: w_x -= sum_q K_bq x_q + sum_r M2P_br y_r over
// the neighbours, in two launches: k_bwd_part computes every neighbour's
// product P_o = K_bq x_q (or M2P_bq y_q) into its own zeroed block of Pb,
// one CTA per (row tile, neighbour), so the neighbours' products run side by
// side; k_bwd_sum then takes w_x += (-1) P_o over the neighbours in order
// and clears Pb for the next colour.
// Pb: [cnt][3^d][M x nrhs], ld M.  grid (row tiles * 3^d, column tiles, cnt)
template <int PM>
__global__ void __launch_bounds__(256) k_bwd_part(LV v, SV s, int col, YSrc y, int mt, double* __restrict__ Pb) {
  int t = blockIdx.z;
  int b = colour_box(col, t, v.d, v.l);
  const int m = v.m[b], o = blockIdx.x / mt;
  int i0 = (blockIdx.x % mt) * 64, j0 = blockIdx.y * 64;
  if (i0 >= m || j0 >= s.nrhs) return;
  const double* A;
  const double* B;
  int ldb, cols;
  if (!bwd_term(v, s, col, y, b, o, A, B, ldb, cols)) return;
  const int n3 = ipow(3, v.d);
  double* P = Pb + ((size_t)t * n3 + o) * v.M * s.nrhs;
  tile_gemm<PM>(A + i0, v.M, B + (size_t)j0 * ldb, ldb, P + i0 + (size_t)j0 * v.M, v.M, min(64, m - i0),
               min(64, s.nrhs - j0), cols, 1.0);
}

// grid (row tiles, column tiles, cnt)
__global__ void __launch_bounds__(256) k_bwd_sum(LV v, SV s, int col, YSrc y, double* __restrict__ Pb) {
  int t = blockIdx.z;
  int b = colour_box(col, t, v.d, v.l);
  const int m = v.m[b];
  int i0 = blockIdx.x * 64, j0 = blockIdx.y * 64;
  if (i0 >= m || j0 >= s.nrhs) return;
  const int mr = min(64, m - i0), nc = min(64, s.nrhs - j0);
  const int n3 = ipow(3, v.d);
  __shared__ unsigned live;
  if (threadIdx.x == 0) {
    unsigned f = 0;
    for (int o = 0; o < n3 && o < 32; ++o) {
      const double* A;
      const double* B;
      int ldb, cols;
      if (bwd_term(v, s, col, y, b, o, A, B, ldb, cols)) f |= 1u << o;
    }
    live = f;
  }
  __syncthreads();
  const unsigned f = live;
  double* w = ws(v, s, b);
  double* P = Pb + (size_t)t * n3 * v.M * s.nrhs;
  for (int e = threadIdx.x; e < mr * nc; e += blockDim.x) {
    const int i = i0 + e % mr, c = j0 + e / mr;
    double acc = w[i + (size_t)c * v.P];
    for (int o = 0; o < n3; ++o) {
      if (!(f >> o & 1u)) continue;
      double* po = P + (size_t)o * v.M * s.nrhs + i + (size_t)c * v.M;
      acc += -1.0 * *po;
      *po = 0.0;
    }
    w[i + (size_t)c * v.P] = acc;
  }
}

// back substitution, step 3: x_b = w_x
__global__ void k_bwd_out(LV v, SV s, int col) {
  int b = colour_box(col, blockIdx.x, v.d, v.l);
  const int m = v.m[b];
  const double* w = ws(v, s, b);
  double* xo = xx_(v, s, b);
  for (int e = threadIdx.x; e < m * s.nrhs; e += blockDim.x) {
    int i = e % m, k = e / m;
    xo[i + (size_t)k * v.M] = w[i + (size_t)k * v.P];
  }
}

// ---------------------------------------------------------------- H^2 product
// upward: q_b = U_b^T x_b (leaf) or U_b^T [q_children] ; one block per box
__global__ void k_h2_up(const int* __restrict__ m, const int* __restrict__ rank, const double* __restrict__ U,
                        int M, int R, const double* __restrict__ xin, int ldin, const int* __restrict__ inoff,
                        double* __restrict__ qout, int nrhs, int d, int leaf, const int* __restrict__ start,
                        const int* __restrict__ crank) {
  int b = blockIdx.x;
  int mb = m[b], rb = rank[b];
  const double* Ub = U + (size_t)b * M * R;
  for (int e = threadIdx.x; e < rb * nrhs; e += blockDim.x) {
    int j = e % rb, k = e / rb;
    double acc = 0.0;
    if (leaf) {
      int s0 = start[b];
      for (int i = 0; i < mb; ++i) acc += Ub[i + (size_t)j * M] * xin[s0 + i + (size_t)k * ldin];
    } else {
      // children multipoles, stacked in child order (rank R_c slots each)
      int i = 0;
      for (int c = b << d; c < (b + 1) << d; ++c) {
        int rc = crank[c];
        for (int a = 0; a < rc; ++a, ++i) acc += Ub[i + (size_t)j * M] * xin[(size_t)c * ldin * nrhs + a + (size_t)k * ldin];
      }
    }
    qout[(size_t)b * R * nrhs + j + (size_t)k * R] = acc;
  }
}

// M2L: z_b = sum_{d in IL(b)} A(t^{b,i}, t^{d,i}) q_d ; one block per box
__global__ void k_h2_m2l(int l, int d, const int* __restrict__ rank, const int* __restrict__ piv, int R,
                         const double* __restrict__ q, double* __restrict__ z, int nrhs, KParams kp, Pts P) {
  int b = blockIdx.x;
  int n = 1 << l;
  int bc[3], qc[3];
  morton_coords(b, d, l, bc);
  int rb = rank[b];
  int ns6 = ipow(6, d);
  for (int e = threadIdx.x; e < rb * nrhs; e += blockDim.x) {
    int i = e % rb, k = e / rb;
    double acc = 0.0;
    for (int s = 0; s < ns6; ++s) {
      slot6_coords(bc, s, d, qc);
      if (!in_grid(qc, d, n) || cheb(bc, qc, d) <= 1) continue;
      int db = morton_key(qc, d, l);
      int rd = rank[db];
      for (int j = 0; j < rd; ++j)
        acc += keval(kp, P, piv[(size_t)b * R + i], piv[(size_t)db * R + j]) * q[(size_t)db * R * nrhs + j + (size_t)k * R];
    }
    z[(size_t)b * R * nrhs + i + (size_t)k * R] = acc;
  }
}

// downward: z_c += U^dag_c z_P = U_P[rows of c] z_P ; one block per child
__global__ void k_h2_down(int d, const int* __restrict__ crank, int cR, double* __restrict__ zc,
                          const int* __restrict__ prank, const double* __restrict__ pU, int pM, int pR,
                          const double* __restrict__ zp, int nrhs) {
  int c = blockIdx.x;
  int P = c >> d;
  int off = 0;
  for (int s = P << d; s < c; ++s) off += crank[s];
  int rc = crank[c], rp = prank[P];
  const double* UP = pU + (size_t)P * pM * pR;
  for (int e = threadIdx.x; e < rc * nrhs; e += blockDim.x) {
    int i = e % rc, k = e / rc;
    double acc = 0.0;
    for (int j = 0; j < rp; ++j) acc += UP[off + i + (size_t)j * pM] * zp[(size_t)P * pR * nrhs + j + (size_t)k * pR];
    zc[(size_t)c * cR * nrhs + i + (size_t)k * cR] += acc;
  }
}

// leaf: y_b = U_b z_b + sum_{q in N(b)} K_bq x_q (tree order vectors)
__global__ void k_h2_leaf(int L, int d, const int* __restrict__ start, const int* __restrict__ rank,
                          const double* __restrict__ U, int M, int R, const double* __restrict__ z,
                          const double* __restrict__ x, double* __restrict__ y, int N, int nrhs, KParams kp, Pts P) {
  int b = blockIdx.x;
  int n = 1 << L;
  int bc[3], qc[3];
  morton_coords(b, d, L, bc);
  int s0 = start[b], mb = start[b + 1] - s0, rb = rank[b];
  const double* Ub = U + (size_t)b * M * R;
  int n3 = ipow(3, d);
  for (int e = threadIdx.x; e < mb * nrhs; e += blockDim.x) {
    int i = e % mb, k = e / mb;
    double acc = 0.0;
    for (int j = 0; j < rb; ++j) acc += Ub[i + (size_t)j * M] * z[(size_t)b * R * nrhs + j + (size_t)k * R];
    for (int o = 0; o < n3; ++o) {
      int oo = o;
      for (int kk = 0; kk < 3; ++kk) qc[kk] = bc[kk];
      for (int kk = 0; kk < d; ++kk) {
        qc[kk] = bc[kk] + (oo % 3) - 1;
        oo /= 3;
      }
      if (!in_grid(qc, d, n)) continue;
      int qb = morton_key(qc, d, L);
      int t0 = start[qb], t1 = start[qb + 1];
      for (int j = t0; j < t1; ++j) acc += keval(kp, P, s0 + i, j) * x[j + (size_t)k * N];
    }
    y[s0 + i + (size_t)k * N] = acc;
  }
}

__global__ void k_permute_in(const int* __restrict__ perm, int N, const double* __restrict__ src, int64_t ld,
                             double* __restrict__ dst, int nrhs) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N * nrhs; e += gridDim.x * blockDim.x) {
    int t = e % N, k = e / N;
    dst[t + (size_t)k * N] = src[perm[t] + (size_t)k * ld];
  }
}

__global__ void k_permute_out(const int* __restrict__ perm, int N, const double* __restrict__ src,
                              double* __restrict__ dst, int64_t ld, int nrhs) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N * nrhs; e += gridDim.x * blockDim.x) {
    int t = e % N, k = e / N;
    dst[perm[t] + (size_t)k * ld] = src[t + (size_t)k * N];
  }
}

// exact direct sum y = A x in tree order; one thread per row, points staged
// through shared memory
__global__ void __launch_bounds__(256) k_direct(const double* __restrict__ x, double* __restrict__ y, int N, int nrhs,
                                                KParams kp, Pts P) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int k = blockIdx.y;
  double acc = 0.0;
  for (int j = 0; j < N; ++j)
    if (i < N) acc += keval(kp, P, i, j) * x[j + (size_t)k * N];
  if (i < N) y[i + (size_t)k * N] = acc;
}

}  // namespace

// Piv^-1 on the solve items of one colour (or the single top item): the
// blocked LU solve sequence of the factorisation
// swap: 0 = interchanges already applied, 1 = gather through shared memory
// (columns of up to MAX_GATHER rows), 2 = sequential interchanges
constexpr int MAX_GATHER = 27 * 1024;   // rows; 216 KB of shared memory
// pivot blocks of up to LS_MAXN rows with up to 4 right-hand sides take the
// one-launch solve (k_lus_small); larger ones the blocked multi-launch solve
constexpr int LS_MAXN = 1024;

// products of the solve sweeps: the 8-digit balanced tensor-core tile for
// more right-hand sides than the narrow FP64 form takes, in the default
// (FP64-precision tensor-core) product mode; FP64 FMAs otherwise
static bool solve_tc(const Handle& h, int ncols) { return !h.tf32 && !h.fp32 && !h.fma_gemm && ncols > THIN_NC; }

static void lus_apply(Handle& h, const SolveItem* items, int cnt, int P, int ncols, int swap, cudaStream_t st) {
  if (P <= LS_MAXN && ncols <= 4 && swap != 2) {
    const int nc = ncols <= 1 ? 1 : ncols <= 2 ? 2 : 4;
    const size_t sm = sizeof(double) * (size_t)P * nc;
    if (nc == 1) k_lus_small<1><<<cnt, 256, sm, st>>>(items, swap);
    else if (nc == 2) k_lus_small<2><<<cnt, 256, sm, st>>>(items, swap);
    else k_lus_small<4><<<cnt, 256, sm, st>>>(items, swap);
    ++h.nlaunch;
    return;
  }
  const int ctiles = (ncols + 63) / 64, cstr = (ncols + 127) / 128, wstr = (ncols + 3) / 4;
  const bool narrow = lus_warp_diag(cnt, ncols);
  if (swap == 1 && P > MAX_GATHER) swap = 2;
  if (swap == 1) {
    k_lus_gather<<<dim3((ncols + 7) / 8, cnt), 256, sizeof(double) * (size_t)P, st>>>(items); ++h.nlaunch;
  } else if (swap == 2) {
    k_lus_swap<<<dim3(cstr, cnt), 128, 0, st>>>(items); ++h.nlaunch;
  }
  for (int k0 = 0; k0 < P; k0 += TB) {
    if (narrow) {
      k_lus_diag_w<1><<<dim3(wstr, cnt), 128, 0, st>>>(items, k0);
    } else {
      k_lus_diag<1><<<dim3(cstr, cnt), 128, 0, st>>>(items, k0);
    }
    ++h.nlaunch;
    if (k0 + TB < P) {
      const dim3 g(ctiles, (P - k0 - TB + 63) / 64, cnt);
      if (solve_tc(h, ncols))
        k_lus_update<1, PM_OZ8><<<g, 256, OZ_SMEM8, st>>>(items, k0);
      else
        k_lus_update<1><<<g, 256, 0, st>>>(items, k0);
      ++h.nlaunch;
    }
  }
  for (int k0 = ((P - 1) / TB) * TB; k0 >= 0; k0 -= TB) {
    if (narrow) {
      k_lus_diag_w<0><<<dim3(wstr, cnt), 128, 0, st>>>(items, k0);
    } else {
      k_lus_diag<0><<<dim3(cstr, cnt), 128, 0, st>>>(items, k0);
    }
    ++h.nlaunch;
    if (k0 > 0) {
      const dim3 g(ctiles, (k0 + 63) / 64, cnt);
      if (solve_tc(h, ncols))
        k_lus_update<0, PM_OZ8><<<g, 256, OZ_SMEM8, st>>>(items, k0);
      else
        k_lus_update<0><<<g, 256, 0, st>>>(items, k0);
      ++h.nlaunch;
    }
  }
}

// the solve vectors of one call (device memory owned by the caller)
struct SolveBufs {
  SV sv[32];
  double* ytop;
  int* toff;
  SolveItem* items;   // max boxes of a colour + 1
  double* part;       // backward products per neighbour, zero between colour steps (part_doubles)
};

// doubles of SolveBufs::part: the largest colour of any level x 3^d
// neighbour blocks of M x nrhs
static size_t part_doubles(const Handle& h, int nrhs) {
  size_t mx = 0;
  const int ncol = ipow(3, h.d);
  for (int l = 2; l <= h.L; ++l) {
    const FacLevel& F = h.fac[l];
    int cmax = 0;
    for (int col = 0; col < ncol; ++col) cmax = std::max(cmax, colour_count(col, h.d, F.n));
    mx = std::max(mx, (size_t)cmax * ncol * F.M * nrhs);
  }
  return std::max(mx, (size_t)1);
}

// number of solve items needed: the largest colour of any level, plus the top
static size_t solve_items(const Handle& h) {
  size_t mx = 1;
  for (int l = 2; l <= h.L; ++l) mx = std::max(mx, (size_t)h.fac[l].nb);
  return mx + 1;
}

// forward sweep (RHS Schur operations in elimination order), top solve,
// back substitution in reverse order; b in original order, in place
static int sweeps(Handle& h, SolveBufs& B, double* b, int nrhs, int64_t ld) {
  const int L = h.L, d = h.d;
  cudaStream_t st = h.stream;
  SV* sv = B.sv;
  const int ncol = ipow(3, d), ct = (nrhs + 63) / 64;
  {
    LV v = view(h, h.fac[L]);
    k_leaf_in<<<v.nb, 256, 0, st>>>(v, sv[L], h.start + h.soff[L], h.perm, b, ld); ++h.nlaunch;
  }
  for (int l = L; l >= 2; --l) {
    FacLevel& F = h.fac[l];
    LV v = view(h, F);
    const int rt = (std::max(F.M, F.R) + 63) / 64;
    for (int col = 0; col < ncol; ++col) {
      int cnt = colour_count(col, d, F.n);
      if (!cnt) continue;
      k_fwd_prep<<<cnt, 256, 0, st>>>(v, sv[l], col, B.items); ++h.nlaunch;
      lus_apply(h, B.items, cnt, F.P, nrhs, 0, st);
      if (solve_tc(h, nrhs))
        k_fwd_upd<PM_OZ8><<<dim3(ncol * rt, ct, cnt), 256, OZ_SMEM8, st>>>(v, sv[l], col, rt);
      else
        k_fwd_upd<PM_FMA><<<dim3(ncol * rt, ct, cnt), 256, 0, st>>>(v, sv[l], col, rt);
      ++h.nlaunch;
    }
    if (l > 2) {
      FacLevel& Fp = h.fac[l - 1];
      LV vp = view(h, Fp);
      k_rhs_up<<<Fp.nb, 256, 0, st>>>(v, sv[l], vp, sv[l - 1], F.xoff); ++h.nlaunch;
    }
  }
  // ---- top
  AIFMM_CUDA_TRY(h, cudaMemcpyAsync(B.toff, h.top_off.data(), sizeof(int) * h.top_off.size(), cudaMemcpyHostToDevice,
                                    st));
  {
    LV v2 = view(h, h.fac[2]);
    SolveItem* top = B.items + (solve_items(h) - 1);
    k_top_in<<<v2.nb, 256, 0, st>>>(v2, sv[2], B.toff, B.ytop, h.ntop, h.top, h.top_ipiv, h.top_perm, top);
    ++h.nlaunch;
    if (h.ntop > 0) lus_apply(h, top, 1, h.ntop, nrhs, 1, st);
  }
  // ---- back substitution, levels 2..L, colours in reverse
  for (int l = 2; l <= L; ++l) {
    FacLevel& F = h.fac[l];
    LV v = view(h, F);
    YSrc y;
    y.top = B.ytop;
    y.ntop = h.ntop;
    y.toff = B.toff;
    y.d = d;
    y.px = l > 2 ? sv[l - 1].xX : nullptr;
    y.pM = l > 2 ? h.fac[l - 1].M : 0;
    y.xoff = F.xoff;
    const int mt = (F.M + 63) / 64;
    for (int col = ncol - 1; col >= 0; --col) {
      int cnt = colour_count(col, d, F.n);
      if (!cnt) continue;
      k_bwd_prep<<<cnt, 256, 0, st>>>(v, sv[l], col, y, B.items); ++h.nlaunch;
      if (solve_tc(h, nrhs))
        k_bwd_part<PM_OZ8><<<dim3(mt * ncol, ct, cnt), 256, OZ_SMEM8, st>>>(v, sv[l], col, y, mt, B.part);
      else
        k_bwd_part<PM_FMA><<<dim3(mt * ncol, ct, cnt), 256, 0, st>>>(v, sv[l], col, y, mt, B.part);
      ++h.nlaunch;
      k_bwd_sum<<<dim3(mt, ct, cnt), 256, 0, st>>>(v, sv[l], col, y, B.part); ++h.nlaunch;
      lus_apply(h, B.items, cnt, F.P, nrhs, 1, st);
      k_bwd_out<<<cnt, 256, 0, st>>>(v, sv[l], col); ++h.nlaunch;
    }
  }
  {
    LV v = view(h, h.fac[L]);
    k_leaf_out<<<v.nb, 256, 0, st>>>(v, sv[L], h.start + h.soff[L], h.perm, b, ld); ++h.nlaunch;
  }
  AIFMM_CUDA_TRY(h, cudaGetLastError());
  return HOK;
}

// the gather's shared-memory limit, raised once per device; handles are
// driven from several host threads (many problems, the serving loop), so the
// per-device flags are guarded
static std::mutex g_attr_mu;

static int solve_attrs(Handle& h) {
  static bool done[64] = {};
  const int dv = (h.device >= 0 && h.device < 64) ? h.device : 0;
  std::lock_guard<std::mutex> g(g_attr_mu);
  if (!done[dv]) {
    AIFMM_CUDA_TRY(h, cudaFuncSetAttribute(k_lus_gather, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(sizeof(double) * MAX_GATHER)));
    AIFMM_CUDA_TRY(h, cudaFuncSetAttribute(k_lus_small<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(sizeof(double) * LS_MAXN * 4)));
    AIFMM_CUDA_TRY(h, cudaFuncSetAttribute(k_lus_update<1, PM_OZ8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           OZ_SMEM8));
    AIFMM_CUDA_TRY(h, cudaFuncSetAttribute(k_lus_update<0, PM_OZ8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           OZ_SMEM8));
    AIFMM_CUDA_TRY(h, cudaFuncSetAttribute(k_fwd_upd<PM_OZ8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           OZ_SMEM8));
    AIFMM_CUDA_TRY(h, cudaFuncSetAttribute(k_bwd_part<PM_OZ8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           OZ_SMEM8));
    done[dv] = true;
  }
  return HOK;
}

int run_solve(Handle& h, double* b, int nrhs, int64_t ld) {
  const int L = h.L;
  cudaStream_t st = h.stream;
  if (int e = solve_attrs(h)) return e;
  if (L + 1 > 32) return HCAPACITY;
  SolveBufs B;
  for (int l = L; l >= 2; --l) {
    FacLevel& F = h.fac[l];
    size_t nb = F.nb;
    B.sv[l].nrhs = nrhs;
    B.sv[l].bX = (double*)hscratch(h, 100 + 4 * l, sizeof(double) * nb * F.M * nrhs);
    B.sv[l].bL = (double*)hscratch(h, 101 + 4 * l, sizeof(double) * nb * F.R * nrhs);
    B.sv[l].xX = (double*)hscratch(h, 102 + 4 * l, sizeof(double) * nb * F.M * nrhs);
    B.sv[l].w = (double*)hscratch(h, 103 + 4 * l, sizeof(double) * nb * F.P * nrhs);
    if (!B.sv[l].bX || !B.sv[l].bL || !B.sv[l].xX || !B.sv[l].w) return HOOM;
    AIFMM_CUDA_TRY(h, cudaMemsetAsync(B.sv[l].bL, 0, sizeof(double) * nb * F.R * nrhs, st));
  }
  const int nt = std::max(1, h.ntop);
  B.ytop = (double*)hscratch(h, 99, sizeof(double) * (size_t)nt * nrhs);
  B.toff = (int*)hscratch(h, 98, sizeof(int) * (h.top_off.size()));
  B.items = (SolveItem*)hscratch(h, 97, sizeof(SolveItem) * solve_items(h));
  const size_t npart = part_doubles(h, nrhs);
  B.part = (double*)hscratch(h, 96, sizeof(double) * npart);
  if (!B.ytop || !B.toff || !B.items || !B.part) return HOOM;
  AIFMM_CUDA_TRY(h, cudaMemsetAsync(B.part, 0, sizeof(double) * npart, st));
  return sweeps(h, B, b, nrhs, ld);
}

int run_h2_matvec(Handle& h, const double* x, double* y, int nrhs, int64_t ld) {
  const int L = h.L, d = h.d, N = (int)h.N;
  cudaStream_t st = h.stream;
  double* xt = (double*)hscratch(h, 200, sizeof(double) * (size_t)N * nrhs);
  double* yt = (double*)hscratch(h, 201, sizeof(double) * (size_t)N * nrhs);
  if (!xt || !yt) return HOOM;
  k_permute_in<<<512, 256, 0, st>>>(h.perm, N, x, ld, xt, nrhs); ++h.nlaunch;
  std::vector<double*> q(L + 1), z(L + 1);
  for (int l = 2; l <= L; ++l) {
    NnLevel& Nl = h.nn[l];
    q[l] = (double*)hscratch(h, 202 + 2 * l, sizeof(double) * (size_t)Nl.nb * Nl.R * nrhs);
    z[l] = (double*)hscratch(h, 203 + 2 * l, sizeof(double) * (size_t)Nl.nb * Nl.R * nrhs);
    if (!q[l] || !z[l]) return HOOM;
  }
  for (int l = L; l >= 2; --l) {
    NnLevel& Nl = h.nn[l];
    if (l == L) {
      k_h2_up<<<Nl.nb, 128, 0, st>>>(Nl.m, Nl.rank, Nl.U, Nl.M, Nl.R, xt, N, nullptr, q[l], nrhs, d, 1,
                                     h.start + h.soff[L], nullptr); ++h.nlaunch;
    } else {
      k_h2_up<<<Nl.nb, 128, 0, st>>>(Nl.m, Nl.rank, Nl.U, Nl.M, Nl.R, q[l + 1], h.nn[l + 1].R, nullptr, q[l], nrhs,
                                     d, 0, nullptr, h.nn[l + 1].rank); ++h.nlaunch;
    }
  }
  for (int l = 2; l <= L; ++l) {
    NnLevel& Nl = h.nn[l];
    k_h2_m2l<<<Nl.nb, 128, 0, st>>>(l, d, Nl.rank, Nl.pivpos, Nl.R, q[l], z[l], nrhs, h.kp, h.P()); ++h.nlaunch;
    if (l > 2) {
      NnLevel& Np = h.nn[l - 1];
      k_h2_down<<<Nl.nb, 128, 0, st>>>(d, Nl.rank, Nl.R, z[l], Np.rank, Np.U, Np.M, Np.R, z[l - 1], nrhs); ++h.nlaunch;
    }
  }
  NnLevel& NL = h.nn[L];
  k_h2_leaf<<<NL.nb, 128, 0, st>>>(L, d, h.start + h.soff[L], NL.rank, NL.U, NL.M, NL.R, z[L], xt, yt, N, nrhs,
                                   h.kp, h.P()); ++h.nlaunch;
  k_permute_out<<<512, 256, 0, st>>>(h.perm, N, yt, y, ld, nrhs); ++h.nlaunch;
  AIFMM_CUDA_TRY(h, cudaGetLastError());
  return HOK;
}

int run_direct_matvec(Handle& h, const double* x, double* y, int nrhs, int64_t ld) {
  const int N = (int)h.N;
  cudaStream_t st = h.stream;
  double* xt = (double*)hscratch(h, 200, sizeof(double) * (size_t)N * nrhs);
  double* yt = (double*)hscratch(h, 201, sizeof(double) * (size_t)N * nrhs);
  if (!xt || !yt) return HOOM;
  k_permute_in<<<512, 256, 0, st>>>(h.perm, N, x, ld, xt, nrhs); ++h.nlaunch;
  k_direct<<<dim3((N + 255) / 256, nrhs), 256, 0, st>>>(xt, yt, N, nrhs, h.kp, h.P()); ++h.nlaunch;
  k_permute_out<<<512, 256, 0, st>>>(h.perm, N, yt, y, ld, nrhs); ++h.nlaunch;
  AIFMM_CUDA_TRY(h, cudaGetLastError());
  return HOK;
}

}  // namespace aifmm

// ---------------------------------------------------------------------------
// Allocation-free solve.  Same kernels and order as run_solve, but every
// temporary vector lives in one file-scope device array instead of memory
// obtained from cudaMalloc, for callers that must not allocate once their
// factorisation is resident.  The array is shared by every call on a device
// and keeps the previous call's contents; the parts that must start at zero
// are cleared here.  Calls whose work overlaps on the GPU race on it.
namespace aifmm {

constexpr size_t NOALLOC_SCRATCH_DOUBLES = (size_t)8 << 20;   // 64 MiB per device
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH_DOUBLES];

namespace {
constexpr int kMaxDevices = 64;
double* g_noalloc_addr[kMaxDevices] = {nullptr};
std::mutex g_noalloc_mu;   // first calls on a device may come from several threads
}  // namespace

size_t noalloc_scratch_bytes() { return NOALLOC_SCRATCH_DOUBLES * sizeof(double); }

// device address of the array on the handle's device (host code cannot use
// the symbol itself); looked up once per device, with that device current
// (cudaGetSymbolAddress answers for the current device only)
static int noalloc_scratch(Handle& h, double** out) {
  if (h.device < 0 || h.device >= kMaxDevices) {
    h.err = "aifmm_solve_noalloc: device index out of range";
    return HINVALID;
  }
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != h.device) {
    cudaGetLastError();
    h.err = "aifmm_solve_noalloc: the handle's device is not the current device";
    return HINVALID;
  }
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  if (!g_noalloc_addr[h.device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      h.err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return HCUDA;
    }
    g_noalloc_addr[h.device] = static_cast<double*>(p);
  }
  *out = g_noalloc_addr[h.device];
  return HOK;
}

int run_solve_noalloc(Handle& h, double* b, int nrhs, int64_t ld) {
  const int L = h.L;
  cudaStream_t st = h.stream;
  if (int e = solve_attrs(h)) return e;
  double* base = nullptr;
  int e = noalloc_scratch(h, &base);
  if (e) return e;
  // carve the per-level vectors (256-byte aligned pieces)
  auto round = [](size_t n) { return (n + 31) & ~(size_t)31; };
  const int nt = std::max(1, h.ntop);
  const size_t nitem = round((solve_items(h) * sizeof(SolveItem) + sizeof(double) - 1) / sizeof(double));
  size_t need = 0;
  for (int l = L; l >= 2; --l) {
    FacLevel& F = h.fac[l];
    size_t nb = F.nb;
    need += round(nb * F.M * nrhs) * 2 + round(nb * F.R * nrhs) + round(nb * F.P * nrhs);
  }
  const size_t npart = part_doubles(h, nrhs);
  need += round((size_t)nt * nrhs) + round(h.top_off.size()) + nitem + round(npart);
  if (need > NOALLOC_SCRATCH_DOUBLES) {
    h.err = "aifmm_solve_noalloc: this problem needs " + std::to_string(need * sizeof(double)) +
            " bytes of solve vectors for nrhs=" + std::to_string(nrhs) + "; the static scratch holds " +
            std::to_string(NOALLOC_SCRATCH_DOUBLES * sizeof(double)) + " bytes";
    return HCAPACITY;
  }
  if (L + 1 > 32) {
    h.err = "aifmm_solve_noalloc: tree deeper than 31 levels";
    return HCAPACITY;
  }
  SolveBufs B;
  size_t off = 0;
  for (int l = L; l >= 2; --l) {
    FacLevel& F = h.fac[l];
    size_t nb = F.nb;
    B.sv[l].nrhs = nrhs;
    B.sv[l].bX = base + off;
    off += round(nb * F.M * nrhs);
    B.sv[l].bL = base + off;
    off += round(nb * F.R * nrhs);
    B.sv[l].xX = base + off;
    off += round(nb * F.M * nrhs);
    B.sv[l].w = base + off;
    off += round(nb * F.P * nrhs);
    AIFMM_CUDA_TRY(h, cudaMemsetAsync(B.sv[l].bL, 0, sizeof(double) * nb * F.R * nrhs, st));
  }
  B.ytop = base + off;
  off += round((size_t)nt * nrhs);
  B.toff = reinterpret_cast<int*>(base + off);
  off += round(h.top_off.size());
  B.items = reinterpret_cast<SolveItem*>(base + off);
  off += nitem;
  B.part = base + off;   // must start at zero: the array keeps the previous call's contents
  AIFMM_CUDA_TRY(h, cudaMemsetAsync(B.part, 0, sizeof(double) * npart, st));
  return sweeps(h, B, b, nrhs, ld);
}

}  // namespace aifmm
