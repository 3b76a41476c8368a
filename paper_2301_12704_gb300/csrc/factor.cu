// AIFMM elimination on the GPU (Sec. 3.2-3.5, Algorithm 2).
//
// Level l (L down to 2) holds, per box b, the particle equations X_b, the
// multipole equation Y_b and the locals equation Lc_b (Sec. 3.1).  The boxes
// of a level are eliminated in distance-2 colour order: boxes of one colour
// have disjoint neighbourhoods, so each colour is one batch.  Per colour:
//   1. compress and redirect every pending well-separated fill-in of each box
//      (Sec. 3.2.1-3.2.3; Algorithm 2 compresses a fill-in once, just before
//      one of its boxes is eliminated): RRQR of [U_b | row fill-ins] and
//      [V_b | column fill-ins^T] with the existing basis taken first, ranks
//      made equal, the locals row of b multiplied by L_b = U~^T U_b (other
//      M2L and L2L updates), the multipole column of b by R_b^T = (V~^T V_b)^T
//      (other M2L and M2M updates), M2P/P2L fill-ins added to the M2L, P2P
//      fill-ins turned into P2L / M2P fill-ins of the partner;
//   2. LU (partial pivoting) of the pivot block [[K_bb, U_b], [V_b^T, 0]];
//   3. Z = Piv^-1 [coupled columns]; Schur update of every coupled block
//      (P2P, M2P, P2L, M2L fill-ins, Table Notations), flagging blocks between
//      well-separated boxes as pending.
// Then the level transition builds level l-1 from the locals rows and the
// multipole columns (eqs. particleAtNonLeafLevel, EqXl2), and after level 2
// the dense level-1 system is factored.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <string>

#include <cooperative_groups.h>

#include "dense.cuh"
#include "internal.h"
#include "level.cuh"
#include "ozaki.cuh"
#include "tc05.cuh"

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

// ============================ level setup ====================================

// The kernels are symmetric, K(x, y) = K(y, x), and keval gives bitwise
// equal values for (i, j) and (j, i) (x_i - x_j is exactly -(x_j - x_i));
// the near-field and interaction-list relations between boxes are
// symmetric too.  So the set-up evaluates each pair of boxes once (the
// block of the box with the smaller Morton index) and fills the partner's
// block as its transpose (k_setup_*_mirror), with the same values.

// dst (rows x cols, ld ldd) := src^T, src (cols x rows, ld lds), through a
// 32 x 33 shared tile (both sides coalesced); every thread of the CTA calls it
__device__ inline void copy_transposed(const double* __restrict__ src, int lds, double* __restrict__ dst, int ldd,
                                       int rows, int cols) {
  __shared__ double tile[32][33];
  for (int i0 = 0; i0 < rows; i0 += 32)
    for (int j0 = 0; j0 < cols; j0 += 32) {
      for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
        const int a = e & 31, b = e >> 5;
        if (j0 + a < cols && i0 + b < rows) tile[b][a] = src[(j0 + a) + (size_t)(i0 + b) * lds];
      }
      __syncthreads();
      for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
        const int a = e & 31, b = e >> 5;
        if (i0 + a < rows && j0 + b < cols) dst[(i0 + a) + (size_t)(j0 + b) * ldd] = tile[a][b];
      }
      __syncthreads();
    }
}

// leaf near field K_bq for q in N(b) with b <= q (the rest: k_setup_leaf_K_mirror);
// grid (nb, 3^d)
__global__ void k_setup_leaf_K(LV v, const int* __restrict__ start, KParams kp, Pts P) {
  int b = blockIdx.x;
  int c[3], q[3];
  morton_coords(b, v.d, v.l, c);
  int o = blockIdx.y;
  for (int k = 0; k < 3; ++k) q[k] = c[k];
  int oo = o;
  for (int k = 0; k < v.d; ++k) {
    q[k] = c[k] + (oo % 3) - 1;
    oo /= 3;
  }
  if (!in_grid(q, v.d, v.n)) return;
  int qb = morton_key(q, v.d, v.l);
  if (qb < b) return;
  int s = slot5(c, q, v.d);
  int sb = start[b], mb = start[b + 1] - sb;
  int sq = start[qb], mq = start[qb + 1] - sq;
  double* K = v.xx(b, s);
  for (int e = threadIdx.x; e < mb * mq; e += blockDim.x) {
    int i = e % mb, j = e / mb;
    K[i + (size_t)j * v.M] = keval(kp, P, sb + i, sq + j);
  }
}

// K_bq = K_qb^T for the neighbours q < b; grid (nb, 3^d)
__global__ void k_setup_leaf_K_mirror(LV v, const int* __restrict__ start) {
  int b = blockIdx.x;
  int c[3], q[3];
  morton_coords(b, v.d, v.l, c);
  int o = blockIdx.y;
  for (int k = 0; k < 3; ++k) q[k] = c[k];
  int oo = o;
  for (int k = 0; k < v.d; ++k) {
    q[k] = c[k] + (oo % 3) - 1;
    oo /= 3;
  }
  if (!in_grid(q, v.d, v.n)) return;
  int qb = morton_key(q, v.d, v.l);
  if (qb >= b) return;
  const int mb = start[b + 1] - start[b], mq = start[qb + 1] - start[qb];
  copy_transposed(v.xx(qb, slot5(q, c, v.d)), v.M, v.xx(b, slot5(c, q, v.d)), v.M, mb, mq);
}

// M2L blocks A_bd = A(t^{b,i}, t^{d,i}) for d in IL(b) with b < d (the rest:
// k_setup_m2l_mirror); grid (nb, ns6)
__global__ void k_setup_m2l(LV v, const int* __restrict__ pivpos, int nR, KParams kp, Pts P) {
  int b = blockIdx.x, s = blockIdx.y;
  int c[3], q[3];
  morton_coords(b, v.d, v.l, c);
  slot6_coords(c, s, v.d, q);
  if (!in_grid(q, v.d, v.n) || cheb(c, q, v.d) <= 1) return;
  int qb = morton_key(q, v.d, v.l);
  if (qb < b) return;
  int rb = v.r[b], rq = v.r[qb];
  double* A = v.ly(b, s);
  const int* tb = pivpos + (size_t)b * nR;
  const int* tq = pivpos + (size_t)qb * nR;
  for (int e = threadIdx.x; e < rb * rq; e += blockDim.x) {
    int i = e % rb, j = e / rb;
    A[i + (size_t)j * v.R] = keval(kp, P, tb[i], tq[j]);
  }
}

// A_bd = A_db^T for d in IL(b), d < b; grid (nb, ns6)
__global__ void k_setup_m2l_mirror(LV v) {
  int b = blockIdx.x, s = blockIdx.y;
  int c[3], q[3];
  morton_coords(b, v.d, v.l, c);
  slot6_coords(c, s, v.d, q);
  if (!in_grid(q, v.d, v.n) || cheb(c, q, v.d) <= 1) return;
  int qb = morton_key(q, v.d, v.l);
  if (qb >= b) return;
  copy_transposed(v.ly(qb, slot6(q, c, v.d)), v.R, v.ly(b, s), v.R, v.r[b], v.r[qb]);
}

// U^dag_b / V^dag_b (level l >= 3): rows of the parent's NNCA basis that belong
// to child b; grid nb
__global__ void k_setup_udag(LV v, const double* __restrict__ pU, int pM, int pR, const int* __restrict__ prank,
                             const int* __restrict__ crank0) {
  int b = blockIdx.x;
  int Pb = b >> v.d;
  int off = 0;
  for (int c = Pb << v.d; c < b; ++c) off += crank0[c];
  int rb = crank0[b], rp = prank[Pb];
  const double* src = pU + (size_t)Pb * pM * pR;
  double* Ud = v.ud(b);
  double* Vd = v.vd(b);
  for (int e = threadIdx.x; e < rb * rp; e += blockDim.x) {
    int i = e % rb, j = e / rb;
    double x = src[(off + i) + (size_t)j * pM];
    Ud[i + (size_t)j * v.R] = x;
    Vd[i + (size_t)j * v.R] = x;
  }
}

// non-leaf: K^{(l)}_{PQ} from the level-(l+1) locals/multipole blocks, and
// U_P, V_P stacked from the children's U^dag, V^dag; grid (nb, 3^d)
__global__ void k_setup_parent(LV v, LV c, const int* __restrict__ cxoff) {
  int Pb = blockIdx.x;
  int pc[3], qc[3];
  morton_coords(Pb, v.d, v.l, pc);
  int o = blockIdx.y;
  for (int k = 0; k < 3; ++k) qc[k] = pc[k];
  int oo = o;
  for (int k = 0; k < v.d; ++k) {
    qc[k] = pc[k] + (oo % 3) - 1;
    oo /= 3;
  }
  if (!in_grid(qc, v.d, v.n)) return;
  int Qb = morton_key(qc, v.d, v.l);
  int s = slot5(pc, qc, v.d);
  double* K = v.xx(Pb, s);
  int nch = 1 << v.d;
  for (int a = 0; a < nch; ++a) {
    int ca = (Pb << v.d) + a;
    int ra = c.r[ca], oa = cxoff[ca];
    int cca[3];
    morton_coords(ca, v.d, c.l, cca);
    for (int bq = 0; bq < nch; ++bq) {
      int cb = (Qb << v.d) + bq;
      int rbq = c.r[cb], ob = cxoff[cb];
      int ccb[3];
      morton_coords(cb, v.d, c.l, ccb);
      int s6 = slot6(cca, ccb, v.d);
      const double* src = c.ly(ca, s6);
      for (int e = threadIdx.x; e < ra * rbq; e += blockDim.x) {
        int i = e % ra, j = e / ra;
        K[(oa + i) + (size_t)(ob + j) * v.M] = src[i + (size_t)j * c.R];
      }
    }
  }
  if (o == (ipow(3, v.d) - 1) / 2) {  // centre: stack U^dag and V^dag
    int rp = v.r[Pb];
    for (int a = 0; a < nch; ++a) {
      int ca = (Pb << v.d) + a;
      int ra = c.r[ca], oa = cxoff[ca];
      const double* su = c.ud(ca);
      const double* sv = c.vd(ca);
      for (int e = threadIdx.x; e < ra * rp; e += blockDim.x) {
        int i = e % ra, j = e / ra;
        v.u(Pb)[(oa + i) + (size_t)j * v.M] = su[i + (size_t)j * c.R];
        v.v(Pb)[(oa + i) + (size_t)j * v.M] = sv[i + (size_t)j * c.R];
      }
    }
  }
}

__global__ void k_copy_basis(LV v, const double* __restrict__ nU, int nM, int nR) {
  int b = blockIdx.x;
  int mb = v.m[b], rb = v.r[b];
  const double* src = nU + (size_t)b * nM * nR;
  for (int e = threadIdx.x; e < mb * rb; e += blockDim.x) {
    int i = e % mb, j = e / mb;
    double x = src[i + (size_t)j * nM];
    v.u(b)[i + (size_t)j * v.M] = x;
    v.v(b)[i + (size_t)j * v.M] = x;
  }
}

// ============================ compress and redirect ===========================

struct Cmp {
  int col, cnt;        // colour, boxes in the colour
  int WC;              // column capacity of the gather workspaces
  double* W;           // [cnt][2][M*WC] gather + Householder workspace
  double* Q;           // [cnt][2][M*M]  bases U~ (side 0) and V~ (side 1)
  double* cn;          // [cnt][2][WC]   residual column norms^2
  int* nc;             // [cnt][2] gathered columns
  int* boff;           // [cnt][2][ns5] column offset in W of each pending block, -1: none
  int* rk;             // [cnt][2] own ranks
  int* rn;             // [cnt] equalised rank
  int* rold;           // [cnt] rank before compression
  int* skip;           // [cnt] 1 if nothing is pending
  double* Lm;          // [cnt][2][R*R] L_b (side 0), R_b (side 1), ld R
  double* T;           // [cnt][2][R*WC] Q0^T X of the projections, ld R
  double* tau;         // [cnt][2] max_j ||[U_b | F]_j||^2 over the basis and fill-in columns
                       // (bit pattern, atomicMax); the RRQR threshold is eps * sqrt of it
  int phase;           // k_cmp_qrcp: 1 = QR of the basis columns, 2 = QRCP of the projected fill-ins
  int ccap;            // k_cmp_qrcp: column capacity of the phase (shared-memory norms)
  double eps;
  double* flops;       // device accumulator of algorithmic flops (compress group)
  double* qflops;      // the same for the QR steps (k_cmp_qrcp and the basis QR)
  int* err;
  int all;             // 1: t runs over every box of the level (Morton order), not one colour
  const double* QB;    // [nb][2][M*M] Q0 of every box's basis, factored when the level starts
                       // (k_cmp_qrcp phase 1 over all boxes); k_cmp_gather copies it into Q
  int sym;             // 1: A = A^T, side 1 is never gathered or factored and
                       // V~_b = U~_b (the column fill-ins are the transposed row
                       // fill-ins, so both RRQRs would see the same matrix)
};

// basis of one side; with sym both sides read the side-0 basis
__device__ inline double* qbase(const Cmp& c, int t, int side, int M) {
  return c.Q + ((size_t)t * 2 + (c.sym ? 0 : side)) * M * M;
}

// fill-in flags are read with a load that bypasses the non-coherent cache
// path; they are only ever modified with atomics
__device__ inline unsigned ldflag(const unsigned* p) { return __ldcg(p); }

__device__ inline int cbox(const Cmp& c, const LV& v, int t) { return c.all ? t : colour_box(c.col, t, v.d, v.l); }

// pending well-separated fill-in of box b at stencil slot s, for one side:
// side 0 -> the block in row X_b (P2P_bq in XX if q is not yet eliminated,
// M2P_bq in XY if it is); side 1 -> the block in column x_b of the partner's
// row (P2P_qb in XX, or P2L_qb in LX), gathered transposed.
struct WsBlk {
  const double* src;
  int ld, rows, cols, ok;
};

__device__ __noinline__ WsBlk ws_block(const LV v, int b, int s, int side, int col) {
  WsBlk w;
  w.src = nullptr;
  w.ld = w.rows = w.cols = w.ok = 0;
  int bc[3], q[3];
  morton_coords(b, v.d, v.l, bc);
  slot5_coords(bc, s, v.d, q);
  if (!in_grid(q, v.d, v.n) || cheb(bc, q, v.d) != 2) return w;
  int qb = morton_key(q, v.d, v.l);
  bool elim = colour_of(q, v.d) < col;
  if (side == 0) {
    if (!(ldflag(v.flag + (size_t)b * v.ns5 + s) & 1u)) return w;
    w.src = elim ? v.xy(b, s) : v.xx(b, s);
    w.ld = v.M;
    w.rows = v.m[b];
    w.cols = elim ? v.r[qb] : v.m[qb];
  } else {
    int sq = slot5(q, bc, v.d);
    unsigned f = ldflag(v.flag + (size_t)qb * v.ns5 + sq);
    if (elim) {
      if (!(f & 2u)) return w;
      w.src = v.lx(qb, sq);
      w.ld = v.R;
      w.rows = v.r[qb];
    } else {
      if (!(f & 1u)) return w;
      w.src = v.xx(qb, sq);
      w.ld = v.M;
      w.rows = v.m[qb];
    }
    w.cols = v.m[b];
  }
  w.ok = 1;
  return w;
}

// the pending blocks of each box side and their column offsets in W after
// the basis (stencil-slot order), the gathered column count and r_b; the
// threshold accumulator cleared.  One warp per (box, side).
__global__ void k_cmp_list(LV v, Cmp c, int nsides) {
  // one warp per (box, side), a lane per stencil slot, offsets by a warp
  // prefix sum (in stencil-slot order, as a sequential walk would give)
  const int x = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (x >= c.cnt * nsides) return;   // the whole warp
  const int t = x / nsides, side = x % nsides;
  const int b = cbox(c, v, t);
  const int rb = v.r[b];
  int* off = c.boff + ((size_t)t * 2 + side) * v.ns5;
  int o = rb;
  for (int s0 = 0; s0 < v.ns5; s0 += 32) {
    const int sl = s0 + lane;
    int w = 0;
    bool ok = false;
    if (sl < v.ns5) {
      const WsBlk blk = ws_block(v, b, sl, side, c.col);
      ok = blk.ok != 0;
      w = ok ? (side == 0 ? blk.cols : blk.rows) : 0;
    }
    int incl = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += y;
    }
    if (sl < v.ns5) off[sl] = ok ? o + incl - w : -1;
    o += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) {
    c.nc[t * 2 + side] = o;
    if (side == 0) c.rold[t] = rb;
    c.tau[t * 2 + side] = 0.0;
  }
}

// gather [U_b | row fill-ins] (side 0) and [V_b | column fill-ins^T] (side 1)
// into W; blockIdx.y = 0 copies the basis, blockIdx.y = 1 + s the pending
// block of stencil slot s; each takes the largest squared norm of its
// columns into the threshold accumulator (non-negative doubles order as
// their bit patterns): the RRQR's residual is relative to the augmented
// matrix [U_b | F] (Sec. 3.2.1), basis columns included.
// grid (cnt * sides, ns5 + 1)
__global__ void k_cmp_gather(LV v, Cmp c, int nsides) {
  __shared__ WsBlk sw;
  __shared__ double shm[8];
  const int t = blockIdx.x / nsides, side = blockIdx.x % nsides;
  const int b = cbox(c, v, t);
  const int mb = v.m[b], rb = c.rold[t];
  double* W = c.W + ((size_t)t * 2 + side) * v.M * c.WC;
  int off, ncol;
  const double* nsrc;   // the copied columns, for their norms (ld M)
  if (blockIdx.y == 0) {
    // the basis: its Householder Q0 was factored when the level started
    // (the basis of a box changes only at its own compression); W keeps
    // no copy of U_b, whose norms enter the threshold
    const double* base = side == 0 ? v.u(b) : v.v(b);
    const double* q0 = c.QB + ((size_t)b * 2 + side) * v.M * v.M;
    double* Q = c.Q + ((size_t)t * 2 + side) * v.M * v.M;
    for (int e = threadIdx.x; e < mb * rb; e += blockDim.x) {
      int i = e % mb, j = e / mb;
      Q[i + (size_t)j * v.M] = q0[i + (size_t)j * v.M];
    }
    off = 0;
    ncol = rb;
    nsrc = base;
  } else {
    const int sl = blockIdx.y - 1;
    off = c.boff[((size_t)t * 2 + side) * v.ns5 + sl];
    if (off < 0) return;
    if (threadIdx.x == 0) sw = ws_block(v, b, sl, side, c.col);
    __syncthreads();
    const WsBlk w = sw;
    for (int e = threadIdx.x; e < w.rows * w.cols; e += blockDim.x) {
      int i = e % w.rows, j = e / w.rows;
      if (side == 0) W[i + (size_t)(off + j) * v.M] = w.src[i + (size_t)j * w.ld];
      else W[j + (size_t)(off + i) * v.M] = w.src[i + (size_t)j * w.ld];
    }
    ncol = side == 0 ? w.cols : w.rows;
    nsrc = W + (size_t)off * v.M;
  }
  __syncthreads();
  // largest squared column norm of the copied columns (m_b rows each)
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  double mx = 0.0;
  for (int j = wp; j < ncol; j += 8) {
    double a = 0.0;
    for (int i = lane; i < mb; i += 32) {
      const double x = nsrc[i + (size_t)j * v.M];
      a += x * x;
    }
    mx = fmax(mx, warp_sum(a));
  }
  if (lane == 0) shm[wp] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int q = 0; q < 8; ++q) a = fmax(a, shm[q]);
    atomicMax(reinterpret_cast<unsigned long long*>(c.tau + t * 2 + side), (unsigned long long)__double_as_longlong(a));
    if (blockIdx.y > 0) atomicAdd(c.flops, 2.0 * mb * (double)ncol);
  }
}

// boxes with nothing pending skip the compression; the others are charged
// the flops of their basis QR (factored for every box when the level
// started: QR and explicit Q, 8 (m - k)(r - k) per column k and side)
__global__ void k_cmp_skip(LV v, Cmp c) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= c.cnt) return;
  int b = cbox(c, v, t);
  int rb = v.r[b];
  const int m = v.m[b];
  const int sk = (m == 0 || (c.nc[2 * t] == rb && (c.sym || c.nc[2 * t + 1] == rb))) ? 1 : 0;
  c.skip[t] = sk;
  if (!sk) {
    double f = 0.0;
    for (int k = 0; k < min(m, rb); ++k) f += 8.0 * (m - k) * (double)(rb - k);
    atomicAdd(c.qflops, f * (c.sym ? 1 : 2));
  }
}

// the basis of every box of the level into W (U_b, side 0; V_b, side 1)
// for the basis QR of the whole level; nc = rold = r_b, skip when there is
// nothing to factor.  grid (nb * sides), 256 threads; c.all = 1
__global__ void k_basis_gather(LV v, Cmp c, int nsides) {
  const int t = blockIdx.x / nsides, side = blockIdx.x % nsides;
  const int b = t;
  const int mb = v.m[b], rb = v.r[b];
  double* W = c.W + ((size_t)t * 2 + side) * v.M * c.WC;
  const double* base = side == 0 ? v.u(b) : v.v(b);
  for (int e = threadIdx.x; e < mb * rb; e += blockDim.x) {
    int i = e % mb, j = e / mb;
    W[i + (size_t)j * v.M] = base[i + (size_t)j * v.M];
  }
  if (threadIdx.x == 0) {
    c.nc[t * 2 + side] = rb;
    if (side == 0) {
      c.rold[t] = rb;
      c.skip[t] = (mb == 0 || rb == 0) ? 1 : 0;
    }
    c.tau[t * 2 + side] = 0.0;
  }
}

// Column-space compression of [U_b | F] in three steps with the same result,
// in exact arithmetic, as one Householder QR whose first r_b columns are
// taken in order and whose later columns are pivoted (reading R3):
//   phase 1  Householder QR of W[:, :nf] = U_b (nf = r_b, no pivoting): Q0,
//            for every box of a level in one launch when the level starts
//            (c.all; the basis of a box is not modified before its own
//            compression); k_cmp_gather copies Q0 into the colour's Q;
//   k_cmp_ptq / k_cmp_pqt   F := F - Q0 (Q0^T F) as tiled GEMMs (the work
//            that the forced reflectors did as rank-1 updates of every
//            fill-in column);
//   phase 2  Householder QR with column pivoting of the projected F: the
//            largest residual column while its norm exceeds
//            tau = eps * max_j ||[U_b | F]_j|| (the column norms of the
//            augmented matrix before the projection, k_cmp_gather: the
//            relative residual of Sec. 3.2.1); Q' = Q[:, nf:rank], then made orthogonal
//            to Q0 once more (the projection leaves Q0 components of size
//            u ||F_j|| / |R_kk|).
// Produces Q[:, :rank] explicitly, rank = nf + (phase-2 columns).
// One thread-block cluster of QC CTAs per (box, side) (QC chosen per level
// by the host so that the colour's clusters fill the GPU); CTA c owns the
// columns j with j % QC == c and keeps their residual norms in shared memory.
// Columns are never swapped: step k takes pivot column p, one warp of every
// CTA builds the reflector from it (rows k..m-1) in the CTA's shared memory,
// and each CTA applies it to its live columns, four per warp at a time; the
// owner stores the reflector into column p one step later (every CTA has read
// the column by then).  Residual norms are downdated (minus the square of the
// new row-k entry) and recomputed exactly when they fall below 1e-8 of their
// last exact value, so a norm compared with the threshold has not lost its
// digits to cancellation.  One cluster barrier per step (two when a pivot is
// searched: the candidates are exchanged through distributed shared memory).
// Every CTA derives the loop exit from the same cluster-wide values, so all
// pass the same barriers.  With sym only side 0 is factored and its rank
// serves both sides.
// grid (QC * sides * cnt), 256 to 1024 threads, cluster size QC; dynamic shared
// memory: 2 M doubles (reflectors k and k-1), M ints (pivot order),
// 2 ceil(WC / QC) doubles (own column norms and their last exact values).
__global__ void __launch_bounds__(1024) k_cmp_qrcp(LV v, Cmp c) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int QC = (int)cl.num_blocks();
  extern __shared__ double dyn[];
  __shared__ double shv[32];
  __shared__ int shi[32];
  __shared__ ArgMax lbest[2];
  const int cr = (int)cl.block_rank();
  const int bs = blockIdx.x / QC;
  const int t = c.sym ? bs : bs >> 1, side = c.sym ? 0 : bs & 1;
  if (c.skip[t]) return;
  int b = cbox(c, v, t);
  const int nf0 = c.rold[t];
  // phase 1: the basis columns only, all taken in order; phase 2: the
  // projected fill-in columns W[:, nf0:], all pivoted, into Q[:, nf0:]
  const int coff = c.phase == 2 ? nf0 : 0;
  const int m = v.m[b], nc_all = c.nc[t * 2 + side];
  const int n = c.phase == 2 ? nc_all - nf0 : nf0, nf = c.phase == 2 ? 0 : nf0;
  const int M = v.M;
  double* W = c.W + ((size_t)t * 2 + side) * M * c.WC + (size_t)coff * M;
  double* Q = c.Q + ((size_t)t * 2 + side) * M * M + (size_t)coff * M;
  const int cw = (c.ccap + QC - 1) / QC;
  double* vbuf = dyn;                                    // [2][M]
  int* pivs = reinterpret_cast<int*>(dyn + 2 * M);       // [M]
  double* cnl = dyn + 2 * M + (M + 1) / 2;               // [cw] squared residual norms (-1: retired)
  double* cref = cnl + cw;                               // [cw] value at the last exact computation
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nloc = n > cr ? (n - cr + QC - 1) / QC : 0;   // own columns j = cr + QC * jl
  // initial residual norms of the own pivoted columns
  for (int jl = w; jl < nloc; jl += nw) {
    int j = cr + QC * jl;
    double acc = 0.0;
    if (j >= nf)
      for (int i = lane; i < m; i += 32) acc += W[i + (size_t)j * M] * W[i + (size_t)j * M];
    acc = warp_sum(acc);
    if (lane == 0) cnl[jl] = cref[jl] = acc;
  }
  const double tau = c.eps * sqrt(c.tau[t * 2 + side]);
  __syncthreads();
  const int kmax = min(m - coff, n);     // the projected columns lie in m - nf0 dimensions
  int k = 0;
  for (; k < kmax; ++k) {
    double* vref = vbuf + (size_t)(k & 1) * M;
    // the owner stores reflector k-1 into its pivot column
    if (k > 0 && pivs[k - 1] % QC == cr) {
      const double* vp = vbuf + (size_t)((k - 1) & 1) * M;
      for (int i = k - 1 + threadIdx.x; i < m; i += blockDim.x) W[i + (size_t)pivs[k - 1] * M] = vp[i];
    }
    int p = k;
    if (k >= nf) {
      ArgMax best;
      best.v = -1.0;
      best.i = -1;
      for (int jl = threadIdx.x; jl < nloc; jl += blockDim.x) {
        int j = cr + QC * jl;
        if (j < nf) continue;
        ArgMax x;
        x.v = cnl[jl];
        x.i = j;
        best = amax_pick(best, x);
      }
      best = block_amax(best, shv, shi);
      if (threadIdx.x == 0) lbest[k & 1] = best;
      cl.sync();
      ArgMax g;
      g.v = -1.0;
      g.i = -1;
      for (int r = 0; r < QC; ++r) g = amax_pick(g, *cl.map_shared_rank(&lbest[k & 1], r));
      if (!(g.i >= 0 && sqrt(fmax(g.v, 0.0)) > tau)) break;
      p = g.i;
    }
    // reflector from W[k:m, p], normalised, built by warp 0
    if (w == 0) {
      double acc = 0.0;
      for (int i = k + lane; i < m; i += 32) {
        double x = W[i + (size_t)p * M];
        vref[i] = x;
        acc += x * x;
      }
      const double a2 = warp_sum(acc);
      const double alpha = sqrt(a2);
      const double x0 = __shfl_sync(0xffffffffu, lane == 0 ? vref[k] : 0.0, 0);
      if (alpha == 0.0) {
        for (int i = k + lane; i < m; i += 32) vref[i] = 0.0;
      } else {
        const double v0 = x0 + (x0 >= 0.0 ? alpha : -alpha);
        const double inv = 1.0 / sqrt(a2 - x0 * x0 + v0 * v0);
        for (int i = k + lane; i < m; i += 32) vref[i] = (i == k ? v0 : vref[i]) * inv;
      }
      if (lane == 0) {
        pivs[k] = p;
        if (p % QC == cr) cnl[p / QC] = -1.0;        // retired
      }
    }
    __syncthreads();
    // apply H_k to the own live columns, four per warp at once (the row loop
    // outside, so the four columns' loads are independent)
    for (int g0 = 4 * w; g0 < nloc; g0 += 4 * nw) {
      bool live[4];
      double* col[4];
      bool any = false;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        int jl = g0 + u, j = cr + QC * jl;
        live[u] = jl < nloc && j != p && cnl[jl] >= 0.0;
        any |= live[u];
        col[u] = W + (size_t)(live[u] ? j : p) * M;   // column p is not written in this step
      }
      if (!any) continue;
      double dt[4] = {0.0, 0.0, 0.0, 0.0};
      for (int i = k + lane; i < m; i += 32) {
        double vi = vref[i];
#pragma unroll
        for (int u = 0; u < 4; ++u) dt[u] += vi * col[u][i];
      }
      warp_sum4(dt);
      double xk[4] = {0.0, 0.0, 0.0, 0.0};
      for (int i = k + lane; i < m; i += 32) {
        double vi = vref[i];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          double x = col[u][i] - 2.0 * dt[u] * vi;
          if (live[u]) col[u][i] = x;
          if (i == k) xk[u] = x;
        }
      }
      // downdate the fill-in columns' norms; recompute where cancellation
      // has eaten most of them (decided by lane 0, the holder of row k)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int jl = g0 + u;
        bool fill = live[u] && cr + QC * jl >= nf;
        double nv = 0.0;
        int redo = 0;
        if (lane == 0 && fill) {
          nv = cnl[jl] - xk[u] * xk[u];
          redo = !(nv > 1e-8 * cref[jl]);
        }
        redo = __shfl_sync(0xffffffffu, redo, 0);
        if (redo) {
          double acc = 0.0;
          for (int i = k + 1 + lane; i < m; i += 32) acc += col[u][i] * col[u][i];
          acc = warp_sum(acc);
          if (lane == 0) cnl[jl] = cref[jl] = acc;
        } else if (lane == 0 && fill) {
          cnl[jl] = nv;
        }
      }
    }
    cl.sync();
  }
  const int rank = k;
  if (rank == kmax && rank > 0 && pivs[rank - 1] % QC == cr) {   // last reflector (a break stored it already)
    const double* vp = vbuf + (size_t)((rank - 1) & 1) * M;
    for (int i = rank - 1 + threadIdx.x; i < m; i += blockDim.x) W[i + (size_t)pivs[rank - 1] * M] = vp[i];
  }
  cl.sync();   // reflectors visible; no CTA leaves while another may read its shared memory
  // form Q[:, :rank] = H_0 ... H_{rank-1} [e_0 .. e_{rank-1}]; reflector kk is
  // stored in column pivs[kk], rows kk..m-1; four columns per warp
  for (int j0 = 4 * (cr + QC * w); j0 < rank; j0 += 4 * QC * nw) {
    double* qc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      int j = min(j0 + u, rank - 1);
      qc[u] = Q + (size_t)j * M;
      if (j0 + u < rank)
        for (int i = lane; i < m; i += 32) qc[u][i] = (i == j) ? 1.0 : 0.0;
    }
    __syncwarp();
    for (int kk = min(j0 + 3, rank - 1); kk >= 0; --kk) {
      const double* vk = W + (size_t)pivs[kk] * M;
      bool on[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) on[u] = j0 + u < rank && kk <= j0 + u;
      double dt[4] = {0.0, 0.0, 0.0, 0.0};
      for (int i = kk + lane; i < m; i += 32) {
        double vi = vk[i];
#pragma unroll
        for (int u = 0; u < 4; ++u) dt[u] += vi * qc[u][i];
      }
      warp_sum4(dt);
      for (int i = kk + lane; i < m; i += 32) {
        double vi = vk[i];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (on[u]) qc[u][i] -= 2.0 * dt[u] * vi;
      }
      __syncwarp();
    }
  }
  if (cr == 0 && threadIdx.x == 0) {
    if (c.phase == 2) {
      c.rk[t * 2 + side] = nf0 + rank;
      if (c.sym) c.rk[t * 2 + 1] = nf0 + rank;
    }
    if (c.phase == 2) {   // phase 1's flops are charged by k_cmp_skip to the boxes compressed
      double f = 2.0 * m * (n - nf);
      for (int kk = 0; kk < rank; ++kk) f += 4.0 * (m - kk) * (double)(n - kk) + 4.0 * (m - kk) * (double)(rank - kk);
      atomicAdd(c.qflops, f);
    }
  }
}

// X := X - Q0 (Q0^T X) with Q0 = Q[:, :nf0] (the orthonormalised basis) and
// X = W[:, nf0:nc] (what 0: the fill-in columns) or X = Q[:, nf0:rank]
// (what 1: the new basis columns, once more).  Two launches: k_cmp_ptq
// T = Q0^T X (each CTA first clears its tile of T), k_cmp_pqt X -= Q0 T.
__device__ inline int proj_cols(const Cmp& c, int t, int side, int nf0, int what) {
  return (what == 0 ? c.nc[t * 2 + side] : c.rk[t * 2 + side]) - nf0;
}

// grid (tiles over X's columns, tiles over nf0, cnt * sides)
template <int PM>
__global__ void __launch_bounds__(256, 2) k_cmp_ptq(LV v, Cmp c, int what) {
  const int nsd = c.sym ? 1 : 2;
  const int t = blockIdx.z / nsd, side = blockIdx.z % nsd;
  if (c.skip[t]) return;
  const int b = cbox(c, v, t);
  const int m = v.m[b], M = v.M, nf0 = c.rold[t];
  const int ncx = proj_cols(c, t, side, nf0, what);
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  if (i0 >= nf0 || j0 >= ncx) return;
  const double* Q0 = c.Q + ((size_t)t * 2 + side) * M * M;
  const double* X = (what == 0 ? c.W + ((size_t)t * 2 + side) * M * c.WC : Q0) + (size_t)nf0 * M;
  double* T = c.T + ((size_t)t * 2 + side) * (size_t)v.R * c.WC + i0 + (size_t)j0 * v.R;
  const int mr = min(64, nf0 - i0), nc = min(64, ncx - j0);
  for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
    int i = e & 63, j = e >> 6;
    if (i < mr && j < nc) T[i + (size_t)j * v.R] = 0.0;
  }
  __syncthreads();
  tile_gemm_tn<PM>(Q0 + (size_t)i0 * M, M, X + (size_t)j0 * M, M, T, v.R, mr, nc, m, 1.0);
  if (threadIdx.x == 0) atomicAdd(c.flops, 2.0 * mr * (double)nc * m);
}

// grid (tiles over X's columns, tiles over m, cnt * sides)
template <int PM>
__global__ void __launch_bounds__(256, 2) k_cmp_pqt(LV v, Cmp c, int what) {
  const int nsd = c.sym ? 1 : 2;
  const int t = blockIdx.z / nsd, side = blockIdx.z % nsd;
  if (c.skip[t]) return;
  const int b = cbox(c, v, t);
  const int m = v.m[b], M = v.M, nf0 = c.rold[t];
  const int ncx = proj_cols(c, t, side, nf0, what);
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  if (nf0 == 0 || i0 >= m || j0 >= ncx) return;
  const double* Q0 = c.Q + ((size_t)t * 2 + side) * M * M;
  double* X = (what == 0 ? c.W + ((size_t)t * 2 + side) * M * c.WC : c.Q + ((size_t)t * 2 + side) * M * M) +
              (size_t)nf0 * M;
  const double* T = c.T + ((size_t)t * 2 + side) * (size_t)v.R * c.WC + (size_t)j0 * v.R;
  const int mr = min(64, m - i0), nc = min(64, ncx - j0);
  tile_gemm<PM>(Q0 + i0, M, T, v.R, X + i0 + (size_t)j0 * M, M, mr, nc, nf0, -1.0);
  if (threadIdx.x == 0) atomicAdd(c.flops, 2.0 * mr * (double)nc * nf0);
}

// equal ranks: the smaller side takes the other side's extra basis columns
// k..rn-1, orthogonalised against its own k columns (classical Gram-Schmidt
// applied twice) and then among themselves.  grid cnt, 256 threads.
__global__ void __launch_bounds__(256) k_cmp_equalise(LV v, Cmp c) {
  __shared__ double shs[32];
  __shared__ double proj[1024];
  int t = blockIdx.x;
  if (c.skip[t]) return;
  int b = cbox(c, v, t);
  const int m = v.m[b], M = v.M;
  int rU = c.rk[2 * t], rV = c.rk[2 * t + 1];
  int rn = max(rU, rV);
  if (threadIdx.x == 0) c.rn[t] = rn;
  for (int side = 0; side < 2; ++side) {
    int k = side == 0 ? rU : rV;
    if (k >= rn) continue;
    double* Qs = c.Q + ((size_t)t * 2 + side) * M * M;
    const double* Qo = c.Q + ((size_t)t * 2 + (1 - side)) * M * M;
    for (int j = k; j < rn; ++j) {
      double* x = Qs + (size_t)j * M;
      for (int i = threadIdx.x; i < m; i += blockDim.x) x[i] = Qo[i + (size_t)j * M];
      __syncthreads();
      double n0 = sqrt(block_sum([&] {
        double a = 0.0;
        for (int i = threadIdx.x; i < m; i += blockDim.x) a += x[i] * x[i];
        return a;
      }(), shs));
      for (int pass = 0; pass < 2; ++pass) {
        // coefficients against the j columns already in the basis
        int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int q = w; q < j; q += nw) {
          double a = 0.0;
          for (int i = lane; i < m; i += 32) a += Qs[i + (size_t)q * M] * x[i];
          a = warp_sum(a);
          if (lane == 0) proj[q] = a;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
          double a = x[i];
          for (int q = 0; q < j; ++q) a -= Qs[i + (size_t)q * M] * proj[q];
          x[i] = a;
        }
        __syncthreads();
      }
      double nx = sqrt(block_sum([&] {
        double a = 0.0;
        for (int i = threadIdx.x; i < m; i += blockDim.x) a += x[i] * x[i];
        return a;
      }(), shs));
      if (!(nx > 1e-8 * n0) || !(nx > 0.0)) {
        if (threadIdx.x == 0) set_err(c.err, DERR_NUMERIC);
        return;
      }
      for (int i = threadIdx.x; i < m; i += blockDim.x) x[i] /= nx;
      __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(c.flops, 8.0 * m * (double)(rn - k) * rn);
  }
}

// L_b = U~^T U_b (side 0), R_b = V~^T V_b (side 1); rn x r_old, ld R.
// grid (tiles over r_old, tiles over rn, 2 * cnt); Lm zeroed beforehand
template <int PM>
__global__ void __launch_bounds__(256, 2) k_cmp_lmat(LV v, Cmp c) {
  int t = blockIdx.z >> 1, side = blockIdx.z & 1;
  if (c.skip[t]) return;
  int b = cbox(c, v, t);
  const int m = v.m[b], M = v.M, rn = c.rn[t], ro = c.rold[t];
  int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  if (i0 >= rn || j0 >= ro) return;
  const double* Q = qbase(c, t, side, M);
  const double* B = side == 0 ? v.u(b) : v.v(b);
  double* Lm = c.Lm + ((size_t)t * 2 + side) * v.R * v.R;
  tile_gemm_tn<PM>(Q + (size_t)i0 * M, M, B + (size_t)j0 * M, M, Lm + i0 + (size_t)j0 * v.R, v.R, rn - i0, ro - j0,
                   m, 1.0);
  if (threadIdx.x == 0) atomicAdd(c.flops, 2.0 * min(64, rn - i0) * (double)min(64, ro - j0) * m);
}

constexpr int TR_CG = 4;   // columns (rows) per pass of the transforms

// blk[0..rn, 0..ncols) := L blk[0..ro, 0..ncols) in place (L rn x ro, ld ldl;
// blk ld ldb), TR_CG columns at a time through shared memory; each output is
// the same p-ordered sum as one column at a time
__device__ inline void transform_cols(double* blk, int ldb, int ncols, const double* L, int ldl, int rn, int ro,
                                      double (*col)[1024]) {
  for (int j0 = 0; j0 < ncols; j0 += TR_CG) {
    const int nj = min(TR_CG, ncols - j0);
    for (int e = threadIdx.x; e < TR_CG * ro; e += blockDim.x) {
      const int u = e / ro, i = e % ro;
      col[u][i] = u < nj ? blk[i + (size_t)(j0 + u) * ldb] : 0.0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < rn; i += blockDim.x) {
      double acc[TR_CG];
#pragma unroll
      for (int u = 0; u < TR_CG; ++u) acc[u] = 0.0;
      for (int p = 0; p < ro; ++p) {
        const double l = L[i + (size_t)p * ldl];
#pragma unroll
        for (int u = 0; u < TR_CG; ++u) acc[u] += l * col[u][p];
      }
#pragma unroll
      for (int u = 0; u < TR_CG; ++u)
        if (u < nj) blk[i + (size_t)(j0 + u) * ldb] = acc[u];
    }
    __syncthreads();
  }
}

// row side: every block of the locals row of b is multiplied by L_b
// (the other-M2L and L2L updates); grid (ns6 + 1, cnt)
// (TR_CG columns per pass, so that L_b is read once per TR_CG columns)
__global__ void __launch_bounds__(256) k_cmp_row_transform(LV v, Cmp c) {
  __shared__ double col[TR_CG][1024];
  int s = blockIdx.x, t = blockIdx.y;
  if (c.skip[t]) return;
  int b = cbox(c, v, t);
  const int rn = c.rn[t], ro = c.rold[t];
  const double* Lm = c.Lm + ((size_t)t * 2) * v.R * v.R;
  double* blk;
  int ncols;
  if (s < v.ns6) {
    int bc[3], q[3];
    morton_coords(b, v.d, v.l, bc);
    slot6_coords(bc, s, v.d, q);
    if (!in_grid(q, v.d, v.n)) return;
    int qb = morton_key(q, v.d, v.l);
    blk = v.ly(b, s);
    ncols = v.r[qb];
  } else {
    if (v.l < 3) return;
    blk = v.ud(b);
    ncols = v.Rp;  // all parent columns (zeros beyond the parent's rank)
  }
  transform_cols(blk, v.R, ncols, Lm, v.R, rn, ro, col);
}

// row side fill-ins: M2P_bq -> A_bq += U~^T M2P_bq ; P2P_bq -> P2L_bq = U~^T P2P_bq
// (the P2L block is zero before b is eliminated).  grid (ns5 * tpc, tiles
// over rn, cnt) with tpc column tiles per block.
template <int PM>
__global__ void __launch_bounds__(256, 2) k_cmp_row_fill(LV v, Cmp c, int tpc) {
  int s = blockIdx.x / tpc, tj = blockIdx.x % tpc, t = blockIdx.z;
  if (c.skip[t]) return;
  int b = cbox(c, v, t);
  int bc[3];
  morton_coords(b, v.d, v.l, bc);
  __shared__ WsBlk sw;
  if (threadIdx.x == 0) sw = ws_block(v, b, s, 0, c.col);
  __syncthreads();
  if (!sw.ok) return;
  const int rn = c.rn[t];
  int i0 = blockIdx.y * 64, j0 = tj * 64;
  if (i0 >= rn || j0 >= sw.cols) return;
  int q[3];
  slot5_coords(bc, s, v.d, q);
  bool elim = colour_of(q, v.d) < c.col;
  double* dst = elim ? v.ly(b, slot6(bc, q, v.d)) : v.lx(b, s);
  const double* Q = c.Q + ((size_t)t * 2) * v.M * v.M;
  tile_gemm_tn<PM>(Q + (size_t)i0 * v.M, v.M, sw.src + (size_t)j0 * sw.ld, sw.ld, dst + i0 + (size_t)j0 * v.R, v.R,
                   rn - i0, sw.cols - j0, sw.rows, 1.0);
  if (threadIdx.x == 0) atomicAdd(c.flops, 2.0 * min(64, rn - i0) * (double)min(64, sw.cols - j0) * sw.rows);
}

// after the row side: clear the redirected fill-in blocks and their flags
// (a P2P_bq leaves a pending P2L_bq for q's column side), U_b := U~,
// r_b := rn.  grid (ns5 + 1, cnt): blockIdx.x = s < ns5 the block of stencil
// slot s (the list made by k_cmp_list before any flag changed), ns5 the basis
__global__ void k_cmp_row_done(LV v, Cmp c) {
  __shared__ WsBlk sw;
  const int sl = blockIdx.x, t = blockIdx.y;
  if (c.skip[t]) return;
  const int b = cbox(c, v, t);
  const int m = v.m[b], M = v.M, rn = c.rn[t];
  if (sl == v.ns5) {
    const double* Q = c.Q + ((size_t)t * 2) * M * M;
    for (int e = threadIdx.x; e < m * rn; e += blockDim.x) {
      int i = e % m, j = e / m;
      v.u(b)[i + (size_t)j * M] = Q[i + (size_t)j * M];
    }
    return;
  }
  if (c.boff[((size_t)t * 2) * v.ns5 + sl] < 0) return;
  if (threadIdx.x == 0) sw = ws_block(v, b, sl, 0, c.col);
  __syncthreads();
  const WsBlk w = sw;
  double* src = const_cast<double*>(w.src);
  for (int e = threadIdx.x; e < w.rows * w.cols; e += blockDim.x) {
    int i = e % w.rows, j = e / w.rows;
    src[i + (size_t)j * w.ld] = 0.0;
  }
  if (threadIdx.x == 0) {
    int bc[3], q[3];
    morton_coords(b, v.d, v.l, bc);
    slot5_coords(bc, sl, v.d, q);
    unsigned* f = v.flag + (size_t)b * v.ns5 + sl;
    atomicAnd(f, ~1u);
    if (colour_of(q, v.d) > c.col) atomicOr(f, 2u);   // a new P2L_bq waits for q's column side
  }
}

// the new rank of every box of the colour, after the row side's blocks are done
__global__ void k_cmp_set_rank(LV v, Cmp c) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= c.cnt || c.skip[t]) return;
  v.r[cbox(c, v, t)] = c.rn[t];
}

// column side: every block of the multipole column of b is multiplied by
// R_b^T (other-M2L and M2M updates); grid (ns6 + 1, cnt)
__global__ void __launch_bounds__(256) k_cmp_col_transform(LV v, Cmp c) {
  __shared__ double row[TR_CG][1024];
  int s = blockIdx.x, t = blockIdx.y;
  if (c.skip[t]) return;
  int b = cbox(c, v, t);
  const int rn = c.rn[t], ro = c.rold[t];
  const double* Rm = c.Lm + ((size_t)t * 2 + 1) * v.R * v.R;
  int bc[3];
  morton_coords(b, v.d, v.l, bc);
  if (s < v.ns6) {
    int q[3];
    slot6_coords(bc, s, v.d, q);   // d in the window of b  <=>  b in the window of d
    if (!in_grid(q, v.d, v.n)) return;
    int db = morton_key(q, v.d, v.l);
    int sd = slot6(q, bc, v.d);
    double* blk = v.ly(db, sd);
    const int nrows = v.r[db];
    // blk[0..nrows, 0..rn) := blk[.., 0..ro) R_b^T, TR_CG rows at a time
    for (int i0 = 0; i0 < nrows; i0 += TR_CG) {
      const int ni = min(TR_CG, nrows - i0);
      for (int e = threadIdx.x; e < TR_CG * ro; e += blockDim.x) {
        const int u = e / ro, p = e % ro;
        row[u][p] = u < ni ? blk[(i0 + u) + (size_t)p * v.R] : 0.0;
      }
      __syncthreads();
      for (int j = threadIdx.x; j < rn; j += blockDim.x) {
        double acc[TR_CG];
#pragma unroll
        for (int u = 0; u < TR_CG; ++u) acc[u] = 0.0;
        for (int p = 0; p < ro; ++p) {
          const double r = Rm[j + (size_t)p * v.R];
#pragma unroll
          for (int u = 0; u < TR_CG; ++u) acc[u] += row[u][p] * r;
        }
#pragma unroll
        for (int u = 0; u < TR_CG; ++u)
          if (u < ni) blk[(i0 + u) + (size_t)j * v.R] = acc[u];
      }
      __syncthreads();
    }
  } else {
    if (v.l < 3) return;
    // V^dag_b (V form, r_old x rp) := R_b V^dag_b ; column-wise
    transform_cols(v.vd(b), v.R, v.Rp, Rm, v.R, rn, ro, row);
  }
}

// Symmetric mode (A = A^T, V~_b = U~_b): the column side of the compression
// as transposes of the row side's results, which hold them already --
//   A_db R_b^T      = (L_b A_bd)^T            for d in the window of b,
//   P2L_qb V~ added = (U~^T M2P_bq)^T added   (q eliminated: part of A_qb),
//   M2P_qb = P2P_qb V~ = (P2L_bq)^T           (q not yet eliminated),
//   V^dag_b         = U^dag_b,
// except where both boxes of a block are compressed in this step (the
// diagonal block A_bb, and M2L blocks between two boxes of the colour): the
// block needs both transforms, and takes the product with R_b^T here after
// its row box's transform.  Runs after the row side (k_cmp_row_done,
// k_cmp_set_rank) and before k_cmp_col_done; replaces k_cmp_col_transform
// and k_cmp_col_fill.  grid (ns6 + 1 + ns5, cnt): window slots, V^dag, and
// stencil slots of the pending column-side blocks.
__global__ void __launch_bounds__(256) k_cmp_col_mirror(LV v, Cmp c) {
  __shared__ double row[TR_CG][1024];
  __shared__ WsBlk sw;
  const int x = blockIdx.x, t = blockIdx.y;
  if (c.skip[t]) return;
  const int b = cbox(c, v, t);
  const int rn = c.rn[t], ro = c.rold[t];
  int bc[3], q[3];
  morton_coords(b, v.d, v.l, bc);
  if (x < v.ns6) {
    slot6_coords(bc, x, v.d, q);   // d in the window of b  <=>  b in the window of d
    if (!in_grid(q, v.d, v.n)) return;
    const int db = morton_key(q, v.d, v.l);
    double* blk = v.ly(db, slot6(q, bc, v.d));
    const int nrows = v.r[db];
    bool both = db == b;
    if (!both && colour_of(q, v.d) == c.col) both = !c.skip[colour_index(q, v.d, v.n)];
    if (!both) {
      // A_db := (A_bd)^T, r_db x rn (the branch is the same for the whole CTA)
      copy_transposed(v.ly(b, x), v.R, blk, v.R, nrows, rn);
      return;
    }
    // blk[0..nrows, 0..rn) := blk[.., 0..ro) R_b^T, TR_CG rows at a time
    const double* Rm = c.Lm + ((size_t)t * 2 + 1) * v.R * v.R;
    for (int i0 = 0; i0 < nrows; i0 += TR_CG) {
      const int ni = min(TR_CG, nrows - i0);
      for (int e = threadIdx.x; e < TR_CG * ro; e += blockDim.x) {
        const int u = e / ro, p = e % ro;
        row[u][p] = u < ni ? blk[(i0 + u) + (size_t)p * v.R] : 0.0;
      }
      __syncthreads();
      for (int j = threadIdx.x; j < rn; j += blockDim.x) {
        double acc[TR_CG];
#pragma unroll
        for (int u = 0; u < TR_CG; ++u) acc[u] = 0.0;
        for (int p = 0; p < ro; ++p) {
          const double r = Rm[j + (size_t)p * v.R];
#pragma unroll
          for (int u = 0; u < TR_CG; ++u) acc[u] += row[u][p] * r;
        }
#pragma unroll
        for (int u = 0; u < TR_CG; ++u)
          if (u < ni) blk[(i0 + u) + (size_t)j * v.R] = acc[u];
      }
      __syncthreads();
    }
    return;
  }
  if (x == v.ns6) {
    if (v.l < 3) return;
    // V^dag_b := U^dag_b (both r_new x r_parent; zeros beyond the parent's rank)
    for (int e = threadIdx.x; e < rn * v.Rp; e += blockDim.x) {
      const int i = e % rn, j = e / rn;
      v.vd(b)[i + (size_t)j * v.R] = v.ud(b)[i + (size_t)j * v.R];
    }
    return;
  }
  // a pending column-side P2P_qb (q not yet eliminated): M2P_qb = (P2L_bq)^T,
  // P2L_bq written into LX(b, s) by the row side
  const int s5 = x - v.ns6 - 1;
  if (threadIdx.x == 0) sw = ws_block(v, b, s5, 1, c.col);
  __syncthreads();
  if (!sw.ok) return;
  slot5_coords(bc, s5, v.d, q);
  if (colour_of(q, v.d) < c.col) return;   // eliminated partner: part of the A_qb mirror
  const int qb = morton_key(q, v.d, v.l);
  const int mq = sw.rows;
  copy_transposed(v.lx(b, s5), v.R, v.xy(qb, slot5(q, bc, v.d)), v.M, mq, rn);
}

// column side fill-ins: P2L_qb -> A_qb += P2L_qb V~ ; P2P_qb -> M2P_qb = P2P_qb V~
// (the M2P block into y_b is zero before b is eliminated).
// grid (ns5 * tpr, tiles over rn, cnt) with tpr row tiles per block.
template <int PM>
__global__ void __launch_bounds__(256, 2) k_cmp_col_fill(LV v, Cmp c, int tpr) {
  int s = blockIdx.x / tpr, ti = blockIdx.x % tpr, t = blockIdx.z;
  if (c.skip[t]) return;
  int b = cbox(c, v, t);
  int bc[3];
  morton_coords(b, v.d, v.l, bc);
  __shared__ WsBlk sw;
  if (threadIdx.x == 0) sw = ws_block(v, b, s, 1, c.col);
  __syncthreads();
  if (!sw.ok) return;
  const int rn = c.rn[t];
  int i0 = ti * 64, j0 = blockIdx.y * 64;
  if (i0 >= sw.rows || j0 >= rn) return;
  int q[3];
  slot5_coords(bc, s, v.d, q);
  int qb = morton_key(q, v.d, v.l);
  bool elim = colour_of(q, v.d) < c.col;
  double* dst;
  int ldd;
  if (elim) {
    dst = v.ly(qb, slot6(q, bc, v.d));
    ldd = v.R;
  } else {
    dst = v.xy(qb, slot5(q, bc, v.d));
    ldd = v.M;
  }
  const double* Q = qbase(c, t, 1, v.M);
  tile_gemm<PM>(sw.src + i0, sw.ld, Q + (size_t)j0 * v.M, v.M, dst + i0 + (size_t)j0 * ldd, ldd,
                min(64, sw.rows - i0), min(64, rn - j0), sw.cols, 1.0);
  if (threadIdx.x == 0) atomicAdd(c.flops, 2.0 * min(64, sw.rows - i0) * (double)min(64, rn - j0) * sw.cols);
}

// after the column side: clear the redirected blocks, the consumed P2L flags
// (a P2P_qb became a pending M2P_qb, which keeps bit 0), V_b := V~.
// grid (ns5 + 1, cnt) as k_cmp_row_done; the pending column-side block of
// slot s is found from the partner's flag, which only this CTA changes
__global__ void k_cmp_col_done(LV v, Cmp c) {
  __shared__ WsBlk sw;
  const int sl = blockIdx.x, t = blockIdx.y;
  if (c.skip[t]) return;
  const int b = cbox(c, v, t);
  const int m = v.m[b], M = v.M, rn = c.rn[t];
  if (sl == v.ns5) {
    const double* Q = qbase(c, t, 1, M);
    for (int e = threadIdx.x; e < m * rn; e += blockDim.x) {
      int i = e % m, j = e / m;
      v.v(b)[i + (size_t)j * M] = Q[i + (size_t)j * M];
    }
    return;
  }
  if (threadIdx.x == 0) sw = ws_block(v, b, sl, 1, c.col);
  __syncthreads();
  const WsBlk w = sw;
  if (!w.ok) return;
  double* src = const_cast<double*>(w.src);
  for (int e = threadIdx.x; e < w.rows * w.cols; e += blockDim.x) {
    int i = e % w.rows, j = e / w.rows;
    src[i + (size_t)j * w.ld] = 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int bc[3], q[3];
    morton_coords(b, v.d, v.l, bc);
    slot5_coords(bc, sl, v.d, q);
    if (colour_of(q, v.d) < c.col) {
      int qb = morton_key(q, v.d, v.l);
      atomicAnd(v.flag + (size_t)qb * v.ns5 + slot5(q, bc, v.d), ~2u);
    }
  }
}

// ============================ pivot, Z and Schur =============================

struct Elim {
  int col, cnt;
  int ncmax;           // capacity of stacked columns
  Coupled* rows;       // [cnt][MAXC]
  Coupled* cols;       // [cnt][MAXC]
  int* nrow;           // [cnt]
  int* ncol;           // [cnt]
  int* totc;           // [cnt] stacked columns
  double* Z;           // [cnt][P * ncmax], ld P
  LuItem* lu;          // [cnt]
  SolveItem* sv;       // [cnt]
  double* colmax;      // [cnt][P]
  int* err;            // device error word
};

// coupled rows / columns of every box of the colour and the LU / solve items
__global__ void k_coupled(LV v, Elim e) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= e.cnt) return;
  int b = colour_box(e.col, t, v.d, v.l);
  int bc[3], q[3];
  morton_coords(b, v.d, v.l, bc);
  int nr = 0, nc = 0, ro = 0, co = 0;
  Coupled* R = e.rows + (size_t)t * MAXC;
  Coupled* C = e.cols + (size_t)t * MAXC;
  int n3 = ipow(3, v.d);
  for (int o = 0; o < n3; ++o) {
    int oo = o;
    for (int k = 0; k < 3; ++k) q[k] = bc[k];
    for (int k = 0; k < v.d; ++k) {
      q[k] = bc[k] + (oo % 3) - 1;
      oo /= 3;
    }
    if (!in_grid(q, v.d, v.n) || (q[0] == bc[0] && q[1] == bc[1] && q[2] == bc[2])) continue;
    int qb = morton_key(q, v.d, v.l);
    bool elim = colour_of(q, v.d) < e.col;
    int sz = elim ? v.r[qb] : v.m[qb];
    if (sz == 0) continue;
    R[nr].box = qb;
    R[nr].type = elim ? 1 : 0;
    R[nr].size = sz;
    R[nr].off = ro;
    ++nr;
    ro += sz;
    C[nc].box = qb;
    C[nc].type = elim ? 1 : 0;
    C[nc].size = sz;
    C[nc].off = co;
    ++nc;
    co += sz;
  }
  int rb = v.r[b], mb = v.m[b];
  if (rb > 0) {
    R[nr].box = b;
    R[nr].type = 2;
    R[nr].size = rb;
    R[nr].off = ro;
    ++nr;
    C[nc].box = b;
    C[nc].type = 2;
    C[nc].size = rb;
    C[nc].off = co;
    ++nc;
    co += rb;
  }
  e.nrow[t] = nr;
  e.ncol[t] = nc;
  e.totc[t] = co;
  LuItem it;
  it.a = v.lu(b);
  it.ipiv = v.piv(b);
  it.colmax = e.colmax + (size_t)t * v.P;
  it.n = mb + rb;
  it.ld = v.P;
  // the coupled columns B (k_z_build) are factored along: the LU leaves
  // L^-1 P B in Z, and only the upper triangular solve remains
  it.b = e.Z + (size_t)t * v.P * e.ncmax;
  it.ldb = v.P;
  it.nb = co;
  e.lu[t] = it;
  SolveItem si;
  si.a = v.lu(b);
  si.ipiv = v.piv(b);
  si.n = mb + rb;
  si.ld = v.P;
  si.x = e.Z + (size_t)t * v.P * e.ncmax;
  si.ldx = v.P;
  si.ncols = co;
  si.perm = nullptr;
  e.sv[t] = si;
}

// net row permutation of each box's pivot LU, for the solve sweeps; one CTA
// per box, through shared memory (dynamic: 2 P ints)
__global__ void k_piv_perm(LV v, int col, int cnt) {
  extern __shared__ int ppsm[];
  const int t = blockIdx.x;
  const int b = colour_box(col, t, v.d, v.l);
  ipiv_to_perm_sm(v.piv(b), v.m[b] + v.r[b], v.pp(b), ppsm, ppsm + v.P);
}

// Piv = [[K_bb, U_b], [V_b^T, 0]] into the LU storage; grid cnt
// grid (cnt, PB_SLICES): slice y takes the columns j = y, y + PB_SLICES, ...
constexpr int PB_SLICES = 16;
__global__ void k_piv_build(LV v, Elim e) {
  int t = blockIdx.x;
  int b = colour_box(e.col, t, v.d, v.l);
  const int m = v.m[b], r = v.r[b], n = m + r, P = v.P, M = v.M;
  double* A = v.lu(b);
  const double* K = v.xx(b, v.centre5());
  const int nj = n > (int)blockIdx.y ? (n - (int)blockIdx.y + PB_SLICES - 1) / PB_SLICES : 0;
  for (int x = threadIdx.x; x < n * nj; x += blockDim.x) {
    int i = x % n, j = (int)blockIdx.y + PB_SLICES * (x / n);
    double val;
    if (i < m && j < m) val = K[i + (size_t)j * M];
    else if (i < m) val = v.u(b)[i + (size_t)(j - m) * M];
    else if (j < m) val = v.v(b)[j + (size_t)(i - m) * M];
    else val = 0.0;
    A[i + (size_t)j * P] = val;
  }
}

// B = A[pivot rows, coupled columns]: [c_C; 0] for x_q / y_q, [0; -I] for y_b,
// in the pivot block's row order (the LU of [Piv | B] interchanges its rows)
// grid (coupled entities, cnt, ZB_SLICES): slice z takes the columns j = z, z + ZB_SLICES, ...
constexpr int ZB_SLICES = 4;
__global__ void k_z_build(LV v, Elim e) {
  int t = blockIdx.y, ci = blockIdx.x;
  if (ci >= e.ncol[t]) return;
  int b = colour_box(e.col, t, v.d, v.l);
  int bc[3], qc[3];
  morton_coords(b, v.d, v.l, bc);
  const int m = v.m[b], r = v.r[b], n = m + r, P = v.P;
  Coupled C = e.cols[(size_t)t * MAXC + ci];
  double* Z = e.Z + (size_t)t * P * e.ncmax + (size_t)C.off * P;
  const int z = blockIdx.z;
  const int nj = C.size > z ? (C.size - z + ZB_SLICES - 1) / ZB_SLICES : 0;
  if (C.type == 2) {
    for (int x = threadIdx.x; x < n * nj; x += blockDim.x) {
      int i = x % n, j = z + ZB_SLICES * (x / n);
      Z[i + (size_t)j * P] = (i - m == j) ? -1.0 : 0.0;
    }
    return;
  }
  morton_coords(C.box, v.d, v.l, qc);
  int s = slot5(bc, qc, v.d);
  const double* src = C.type == 0 ? v.xx(b, s) : v.xy(b, s);
  for (int x = threadIdx.x; x < n * nj; x += blockDim.x) {
    int i = x % n, j = z + ZB_SLICES * (x / n);
    Z[i + (size_t)j * P] = i < m ? src[i + (size_t)j * v.M] : 0.0;
  }
}

// storage of the block (row entity R, column entity C); pc, qc their boxes' coordinates
__device__ inline double* schur_target(const LV& v, int rbox, int rtype, int ctype, const int* pc, const int* qc,
                                       int& ldt) {
  if (rtype == 0) {
    int s = slot5(pc, qc, v.d);
    ldt = v.M;
    return ctype == 0 ? v.xx(rbox, s) : v.xy(rbox, s);
  }
  ldt = v.R;
  return ctype == 0 ? v.lx(rbox, slot5(pc, qc, v.d)) : v.ly(rbox, slot6(pc, qc, v.d));
}

// One work item of the Schur update: box t of the colour, coupled row entity
// ri and column entity cj, and the 64 x 64 output tile (ti, tj) of their
// block; rc = ri | cj << 8 | ti << 16 | tj << 24.
struct SchurItem {
  int t, rc;
};

// The Schur update's work list: for every box of the colour, the (row
// entity, column entity, tile) combinations that exist -- i <= j only with
// sym -- appended to one list (one thread per box, one atomicAdd per box on
// the list's counter, which the caller cleared).  Boxes of one colour update
// disjoint blocks, so the order of the list does not matter.
__global__ void k_schur_items(Elim e, int sym, SchurItem* __restrict__ items, int* __restrict__ count) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= e.cnt) return;
  const Coupled* R = e.rows + (size_t)t * MAXC;
  const Coupled* C = e.cols + (size_t)t * MAXC;
  const int nr = e.nrow[t], nc = e.ncol[t];
  int n = 0;
  for (int ri = 0; ri < nr; ++ri)
    for (int cj = sym ? ri : 0; cj < nc; ++cj) n += ((R[ri].size + 63) / 64) * ((C[cj].size + 63) / 64);
  int o = atomicAdd(count, n);
  for (int ri = 0; ri < nr; ++ri)
    for (int cj = sym ? ri : 0; cj < nc; ++cj) {
      const int tr = (R[ri].size + 63) / 64, tc = (C[cj].size + 63) / 64;
      for (int ti = 0; ti < tr; ++ti)
        for (int tj = 0; tj < tc; ++tj) {
          SchurItem it;
          it.t = t;
          it.rc = ri | (cj << 8) | (ti << 16) | (tj << 24);
          items[o++] = it;
        }
    }
}

// Schur update of one item (one 64 x 64 output tile of one coupled block).
// The row and column lists name the same entities in the same order
// (X_p <-> x_p, Lc_p <-> y_p, Lc_b <-> y_b), so with sym (A = A^T, which the
// elimination keeps: Piv and the Schur complement stay symmetric) the block
// (j, i) is the transpose of (i, j): only i <= j is listed and each
// off-diagonal tile is also stored transposed at its mirror.
// PM: the tile product mode (dense.cuh): FP64 FMAs, the BF16 warp MMAs or
// tcgen05 in FP64 precision, or FP32.  Every thread of the CTA runs it with
// the same item (the tiles synchronise the CTA).
template <int PM>
__device__ __forceinline__ void schur_tile(const LV& v, const Elim& e, const SchurItem item, int sym,
                                           unsigned char* ozs) {
  const int t = item.t;
  const int ri = item.rc & 0xff, cj = (item.rc >> 8) & 0xff, ti = (item.rc >> 16) & 0xff, tj = item.rc >> 24;
  Coupled R = e.rows[(size_t)t * MAXC + ri];
  Coupled C = e.cols[(size_t)t * MAXC + cj];
  int i0 = ti * 64, j0 = tj * 64;
  if (i0 >= R.size || j0 >= C.size) return;
  int b = colour_box(e.col, t, v.d, v.l);
  const int m = v.m[b], P = v.P;
  int bc[3], pc[3], qc[3];
  morton_coords(b, v.d, v.l, bc);
  morton_coords(R.box, v.d, v.l, pc);
  morton_coords(C.box, v.d, v.l, qc);
  const double* Z = e.Z + (size_t)t * P * e.ncmax + (size_t)(C.off + j0) * P;
  int ldt;
  double* T = schur_target(v, R.box, R.type, C.type, pc, qc, ldt);   // sets ldt
  T += i0 + (size_t)j0 * ldt;
  int mr = min(64, R.size - i0), nc = min(64, C.size - j0);
  if (R.type == 2) {
    // (Lc_b, C) += Z[m + i, C]
    for (int x = threadIdx.x; x < mr * nc; x += blockDim.x) {
      int i = x % mr, j = x / mr;
      T[i + (size_t)j * ldt] += Z[m + i0 + i + (size_t)j * P];
    }
    return;
  }
  int sp = slot5(pc, bc, v.d);
  const double* A = R.type == 0 ? v.xx(R.box, sp) : v.lx(R.box, sp);
  int lda = R.type == 0 ? v.M : v.R;
  if (PM == PM_TC05) {
    tile_gemm_64_tc(A + i0, lda, Z, P, T, ldt, mr, nc, m, -1.0, ozs, e.err);
  } else if (PM == PM_OZ) {
    tile_gemm_64_oz(A + i0, lda, Z, P, T, ldt, mr, nc, m, -1.0, ozs);
  } else if (PM == PM_F32) {
    tile_gemm_64<float>(A + i0, lda, Z, P, T, ldt, mr, nc, m, -1.0);
  } else if (PM == PM_TF32) {
    tile_gemm<PM_TF32>(A + i0, lda, Z, P, T, ldt, mr, nc, m, -1.0);
  } else {
    tile_gemm_64(A + i0, lda, Z, P, T, ldt, mr, nc, m, -1.0);
  }
  // a block between well-separated boxes is a pending fill-in unless both
  // boxes are eliminated (an M2L fill-in, kept without compression)
  const bool ws = C.type != 2 && !(R.type == 1 && C.type == 1) && cheb(pc, qc, v.d) == 2;
  if (threadIdx.x == 0 && ti == 0 && tj == 0 && ws)
    atomicOr(v.flag + (size_t)R.box * v.ns5 + slot5(pc, qc, v.d), R.type == 0 ? 1u : 2u);
  if (sym && ri < cj) {
    // mirror: row entity of C, column entity of R (R is never Lc_b here)
    __syncthreads();
    int ldm;
    double* Tm = schur_target(v, C.box, C.type, R.type, qc, pc, ldm);   // sets ldm
    Tm += j0 + (size_t)i0 * ldm;
    for (int x = threadIdx.x; x < mr * nc; x += blockDim.x) {
      int j = x % nc, i = x / nc;
      Tm[j + (size_t)i * ldm] = T[i + (size_t)j * ldt];
    }
    if (threadIdx.x == 0 && ti == 0 && tj == 0 && ws)
      atomicOr(v.flag + (size_t)C.box * v.ns5 + slot5(qc, pc, v.d), C.type == 0 ? 1u : 2u);
  }
}

// Schur update of every coupled block over the colour's work list.
// Persistent: each CTA takes items blockIdx.x, blockIdx.x + gridDim.x, ...
// (grid: the CTAs resident on the device at once), except for the tcgen05
// tile, whose tensor-memory allocation a CTA may make once: there the grid
// covers an upper bound of the list and each CTA takes at most one item.
template <int PM>
__global__ void __launch_bounds__(256, PM == PM_TC05 ? 1 : 2) k_schur(LV v, Elim e, const SchurItem* __restrict__ items,
                                              const int* __restrict__ count, int sym) {
  extern __shared__ __align__(16) unsigned char ozs[];
  const int n = *count;
  if (PM == PM_TC05) {
    if ((int)blockIdx.x < n) schur_tile<PM>(v, e, items[blockIdx.x], sym, ozs);
    return;
  }
  for (int g = blockIdx.x; g < n; g += gridDim.x) {
    schur_tile<PM>(v, e, items[g], sym, ozs);
    __syncthreads();   // the tile's shared memory is reused by the next item
  }
}

// ============================ top (level-1 system) ===========================

__global__ void k_top_assemble(LV v, const int* __restrict__ toff, double* __restrict__ T, int ntop) {
  int b = blockIdx.x, s = blockIdx.y;
  int bc[3], q[3];
  morton_coords(b, v.d, v.l, bc);
  slot6_coords(bc, s, v.d, q);
  if (!in_grid(q, v.d, v.n)) return;
  int qb = morton_key(q, v.d, v.l);
  int rb = v.r[b], rq = v.r[qb];
  const double* src = v.ly(b, s);
  int ob = toff[b], oq = toff[qb];
  for (int x = threadIdx.x; x < rb * rq; x += blockDim.x) {
    int i = x % rb, j = x / rb;
    T[(ob + i) + (size_t)(oq + j) * ntop] = src[i + (size_t)j * v.R];
  }
}

// xoff of each box inside its parent's particles: sum of earlier siblings' ranks
__global__ void k_xoff(int nb, int d, const int* __restrict__ r, int* __restrict__ xoff) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  int off = 0;
  for (int c = (b >> d) << d; c < b; ++c) off += r[c];
  xoff[b] = off;
}

}  // namespace

// ---------------------------------------------------------------------------

// launch kernel template KERN in the product mode pm (PM_FMA, PM_OZ or
// PM_F32), with the dynamic shared memory the mode needs
#define AIFMM_LAUNCH_PM(pm, KERN, grid, ...)                                   \
  do {                                                                         \
    if ((pm) == PM_OZ)                                                         \
      KERN<PM_OZ><<<(grid), 256, OZ_SMEM, st>>>(__VA_ARGS__);                  \
    else if ((pm) == PM_F32)                                                   \
      KERN<PM_F32><<<(grid), 256, 0, st>>>(__VA_ARGS__);                       \
    else if ((pm) == PM_TF32)                                                  \
      KERN<PM_TF32><<<(grid), 256, 0, st>>>(__VA_ARGS__);                      \
    else                                                                       \
      KERN<PM_FMA><<<(grid), 256, 0, st>>>(__VA_ARGS__);                       \
  } while (0)

// product mode of the compress fills and projections, the Schur update
// (unless tcgen05 is chosen there) and, with PM_F32 or PM_TF32, of the Z solve and the
// pivot LU's trailing updates
static int product_mode(const Handle& h) {
  return h.tf32 ? PM_TF32 : h.fp32 ? PM_F32 : h.fma_gemm ? PM_FMA : PM_OZ;
}

// CTAs of the persistent Schur kernel that fit on one SM at once, per
// product mode (queried once per handle)
static int schur_ctas_per_sm(Handle& h, int pm) {
  static thread_local int cache[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  (void)h;
  if (pm < 0 || pm >= 8) return 1;
  if (!cache[pm]) {
    int nb = 0;
    cudaError_t e = pm == PM_OZ   ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_schur<PM_OZ>, 256, OZ_SMEM)
                    : pm == PM_F32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_schur<PM_F32>, 256, 0)
                    : pm == PM_TF32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_schur<PM_TF32>, 256, 0)
                                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_schur<PM_FMA>, 256, 0);
    if (e != cudaSuccess || nb < 1) {
      cudaGetLastError();
      nb = 1;
    }
    cache[pm] = nb;
  }
  return cache[pm];
}

static int alloc_level(Handle& h, FacLevel& F) {
  const size_t nb = F.nb;
  F.m = hnew<int>(h, nb);
  F.r = hnew<int>(h, nb);
  F.xoff = hnew<int>(h, nb);
  F.XX = hnew<double>(h, nb * F.ns5 * F.M * F.M);
  F.XY = hnew<double>(h, nb * F.ns5 * F.M * F.R);
  F.LX = hnew<double>(h, nb * F.ns5 * F.R * F.M);
  F.LY = hnew<double>(h, nb * F.ns6 * F.R * F.R);
  F.U = hnew<double>(h, nb * F.M * F.R);
  F.V = hnew<double>(h, nb * F.M * F.R);
  F.Ud = hnew<double>(h, nb * F.R * std::max(1, F.Rp));
  F.Vd = hnew<double>(h, nb * F.R * std::max(1, F.Rp));
  F.LU = hnew<double>(h, nb * F.P * F.P, false);
  F.ipiv = hnew<int>(h, nb * F.P);
  F.pperm = hnew<int>(h, nb * F.P, false);
  F.flag = hnew<unsigned>(h, nb * F.ns5);
  if (!F.m || !F.r || !F.xoff || !F.XX || !F.XY || !F.LX || !F.LY || !F.U || !F.V || !F.Ud || !F.Vd || !F.LU ||
      !F.ipiv || !F.pperm || !F.flag)
    return HOOM;
  F.bytes = sizeof(double) * nb *
            ((size_t)F.ns5 * (F.M * F.M + 2 * F.M * F.R) + (size_t)F.ns6 * F.R * F.R + 2 * F.M * F.R +
             2 * F.R * std::max(1, F.Rp) + (size_t)F.P * F.P);
  return HOK;
}

static int setup_level(Handle& h, int l) {
  const int d = h.d, L = h.L;
  cudaStream_t st = h.stream;
  FacLevel& F = h.fac[l];
  F.l = l;
  F.nb = 1 << (d * l);
  F.n = 1 << l;
  F.ns5 = ipow(5, d);
  F.ns6 = ipow(6, d);
  const NnLevel& N = h.nn[l];
  F.h_m.assign(F.nb, 0);
  if (l == L) {
    F.h_m = N.h_m;
  } else {
    const FacLevel& C = h.fac[l + 1];
    for (int b = 0; b < F.nb; ++b)
      for (int c = 0; c < (1 << d); ++c) F.h_m[b] += C.h_r[(b << d) + c];
  }
  F.h_r = N.h_rank;
  int M = 1;
  for (int b = 0; b < F.nb; ++b) M = std::max(M, F.h_m[b]);
  F.M = M;
  F.R = M;              // a rank never exceeds the particle count of its box
  F.P = F.M + F.R;
  F.Rp = 1;
  if (l >= 3) {
    const NnLevel& Np = h.nn[l - 1];
    for (int b = 0; b < Np.nb; ++b) F.Rp = std::max(F.Rp, Np.h_rank[b]);
  }
  if (F.R + 1 > 1024) {
    h.err = "rank capacity above 1024 at level " + std::to_string(l);
    return HCAPACITY;
  }
  int e = alloc_level(h, F);
  if (e) return e;
  h.max_m = std::max(h.max_m, F.M);
  AIFMM_CUDA_TRY(h, cudaMemcpyAsync(F.m, F.h_m.data(), sizeof(int) * F.nb, cudaMemcpyHostToDevice, st));
  AIFMM_CUDA_TRY(h, cudaMemcpyAsync(F.r, F.h_r.data(), sizeof(int) * F.nb, cudaMemcpyHostToDevice, st));
  LV v = view(h, F);
  const int n3 = ipow(3, d);
  if (l == L) {
    k_setup_leaf_K<<<dim3(F.nb, n3), 256, 0, st>>>(v, h.start + h.soff[L], h.kp, h.P()); ++h.nlaunch;
    k_setup_leaf_K_mirror<<<dim3(F.nb, n3), 256, 0, st>>>(v, h.start + h.soff[L]); ++h.nlaunch;
    k_copy_basis<<<F.nb, 256, 0, st>>>(v, N.U, N.M, N.R); ++h.nlaunch;
  } else {
    FacLevel& C = h.fac[l + 1];
    LV vc = view(h, C);
    k_setup_parent<<<dim3(F.nb, n3), 256, 0, st>>>(v, vc, C.xoff); ++h.nlaunch;
  }
  k_setup_m2l<<<dim3(F.nb, F.ns6), 128, 0, st>>>(v, N.pivpos, N.R, h.kp, h.P()); ++h.nlaunch;
  k_setup_m2l_mirror<<<dim3(F.nb, F.ns6), 256, 0, st>>>(v); ++h.nlaunch;
  if (l >= 3) {
    const NnLevel& Np = h.nn[l - 1];
    k_setup_udag<<<F.nb, 128, 0, st>>>(v, Np.U, Np.M, Np.R, Np.rank, N.rank); ++h.nlaunch;
  }
  AIFMM_CUDA_TRY(h, cudaGetLastError());
  return HOK;
}

// profile mode: bracket a group of launches with CUDA events on the stream
struct GroupTimer {
  Handle& h;
  int g;
  cudaEvent_t a = nullptr, b = nullptr;
  long long n0;
  GroupTimer(Handle& hh, int gg) : h(hh), g(gg), n0(hh.nlaunch) {
    if (!h.profile) return;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, h.stream);
  }
  ~GroupTimer() {
    if (!h.profile) return;
    cudaEventRecord(b, h.stream);
    h.g_ev.push_back({g, {a, b}});
    h.g_launch[g] += h.nlaunch - n0;
  }
};

// optional per-region timing (environment AIFMM_PROFILE_DETAIL=1): event
// pairs around named regions of the colour loop, summed per level and
// printed to stderr; a diagnostic, off by default
struct DetailProf {
  bool on = false;
  std::vector<std::pair<std::string, std::pair<cudaEvent_t, cudaEvent_t>>> ev;
  cudaEvent_t cur;
  std::string name;
  cudaStream_t st;
  void begin(const char* n) {
    if (!on) return;
    cudaEventCreate(&cur);
    cudaEventRecord(cur, st);
    name = n;
  }
  void end() {
    if (!on) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, st);
    ev.push_back({name, {cur, e}});
  }
  void report(int l) {
    if (!on) return;
    std::vector<std::pair<std::string, double>> tot;
    for (auto& x : ev) {
      float ms = 0.f;
      cudaEventSynchronize(x.second.second);
      cudaEventElapsedTime(&ms, x.second.first, x.second.second);
      bool f = false;
      for (auto& t : tot)
        if (t.first == x.first) {
          t.second += ms;
          f = true;
        }
      if (!f) tot.push_back({x.first, ms});
      cudaEventDestroy(x.second.first);
      cudaEventDestroy(x.second.second);
    }
    ev.clear();
    for (auto& t : tot) std::fprintf(stderr, "DETAIL l=%d %-16s %9.3f ms\n", l, t.first.c_str(), t.second);
  }
};

static void collect_group_times(Handle& h) {
  for (auto& e : h.g_ev) {
    float ms = 0.f;
    cudaEventSynchronize(e.second.second);
    cudaEventElapsedTime(&ms, e.second.first, e.second.second);
    h.g_ms[e.first] += ms;
    cudaEventDestroy(e.second.first);
    cudaEventDestroy(e.second.second);
  }
  h.g_ev.clear();
}

// The register-resident LU panel (k_lu_panel_rg) spread over a thread-block
// cluster of CS CTAs per item, for panels taller than one CTA holds in
// registers (the top system): the FP64 rank-1 updates, which bound such a
// panel on one SM (about two FP64 FMAs per clock per SM), run on CS SMs.
// Measured at 65,536 points: the top system's LU 3.1 -> 2.7 ms against the
// shared-memory panel, but slower than k_lu_panel_rg on panels of up to 512 rows (the
// cluster barrier and the distributed-shared-memory reads cost more per
// column than the FP64 work they spread), so those keep one CTA.
// CTA rank r holds panel rows r * blockDim.x ..., one per thread.  Per
// column, each warp publishes its best candidate (key, position, row and
// pivot reciprocal) in its CTA's double-buffered slots; one cluster barrier;
// then every warp reads all CS x warps candidates through distributed
// shared memory (lane k: candidates k and k + 32), keeps the best (largest
// key, then smallest position) and takes the winning row from its owner's
// slot.  The same operations per entry as k_lu_panel_rg, so the same
// results.  Control flow is uniform over the cluster (the item, and every
// decision, is the same in all its CTAs), and a cluster barrier precedes
// every exit, so no CTA leaves while another may read its shared memory.
// grid (items x CS), cluster CS, blockDim a multiple of 32 with CS x warps <= 64.
constexpr int LU_CL_MAXT = 256;
__global__ void __launch_bounds__(LU_CL_MAXT) k_lu_panel_cl(const LuItem* items, int k0, int* err) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int CS = (int)cl.num_blocks(), cr = (int)cl.block_rank();
  __shared__ long long ck[2][LU_CL_MAXT / 32];
  __shared__ int cp[2][LU_CL_MAXT / 32];
  __shared__ double crow[2][LU_CL_MAXT / 32][LU_NB + 1];
  __shared__ long long thr[LU_NB];
  const LuItem it = items[blockIdx.x / CS];
  const int n = it.n;
  if (k0 >= n) return;   // the whole cluster: same item
  const int h = n - k0;
  const int nbw = min(LU_NB, h);
  const int t = cr * blockDim.x + threadIdx.x;   // panel row of this thread
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int ncand = CS * nw;
  double* A = it.a;
  const int ld = it.ld;
  double a[LU_NB];
#pragma unroll
  for (int j = 0; j < LU_NB; ++j) a[j] = (t < h && j < nbw) ? A[(k0 + t) + (size_t)(k0 + j) * ld] : 0.0;
  if (threadIdx.x < LU_NB)
    thr[threadIdx.x] =
        __double_as_longlong(1e-14 * ((it.colmax && (int)threadIdx.x < nbw) ? it.colmax[k0 + threadIdx.x] : 0.0));
  int pos = t;
  bool live = t < h;
  __syncthreads();
#pragma unroll
  for (int jj = 0; jj < LU_NB; ++jj) {
    if (jj < nbw) {
      const int par = jj & 1;
      long long key = -1;
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
      if (wk >= 0 && pos == wp) {
        double* cw = crow[par][w];
#pragma unroll
        for (int cc = 0; cc < LU_NB; ++cc)
          if (cc >= jj) cw[cc] = a[cc];
        cw[LU_NB] = 1.0 / a[jj];
      }
      if (lane == 0) {
        ck[par][w] = wk;
        cp[par][w] = wp;
      }
      cl.sync();
      long long bk = -1;
      int bp = 0x7fffffff, bs = 0;
      for (int k = lane; k < ncand; k += 32) {
        const int r = k / nw, u = k % nw;
        const long long k2 = *cl.map_shared_rank(&ck[par][u], r);
        const int p2 = *cl.map_shared_rank(&cp[par][u], r);
        if (k2 > bk || (k2 == bk && p2 < bp)) {
          bk = k2;
          bp = p2;
          bs = k;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
        const int op = __shfl_xor_sync(0xffffffffu, bp, o);
        const int os = __shfl_xor_sync(0xffffffffu, bs, o);
        if (ok > bk || (ok == bk && op < bp)) {
          bk = ok;
          bp = op;
          bs = os;
        }
      }
      if (!(bk > thr[jj]) || !(bk >= 0x0010000000000000LL)) {
        if (cr == 0) {
          for (int q = jj + (int)threadIdx.x; q < nbw; q += blockDim.x) it.ipiv[k0 + q] = k0 + q;
          if (threadIdx.x == 0) set_err(err, DERR_SINGULAR);
        }
        cl.sync();
        return;
      }
      const double* pr = cl.map_shared_rank(&crow[par][bs % nw][0], bs / nw);
      const double prl = pr[lane];
      const double rp = pr[LU_NB];
      if (live && pos == bp) {
        it.ipiv[k0 + jj] = k0 + bp;
        live = false;
        pos = jj;
      } else if (pos == jj) {
        pos = bp;
      }
      const double l = live ? a[jj] * rp : 0.0;
      if (live) a[jj] = l;
#pragma unroll
      for (int cc = 0; cc < LU_NB; ++cc)
        if (cc > jj && cc < nbw) {
          const double pc = __shfl_sync(0xffffffffu, prl, cc);
          if (live) a[cc] -= l * pc;
        }
    }
  }
  cl.sync();   // the last column's slots may still be read by the other CTAs
  if (t < h)
#pragma unroll
    for (int j = 0; j < LU_NB; ++j)
      if (j < nbw) A[(k0 + pos) + (size_t)(k0 + j) * ld] = a[j];
}

// CTAs per cluster for the panels of `cnt` items of up to `hc` rows, or 1 for
// one CTA per item: at most LU_CL_MAXT rows per CTA; more CTAs while the
// launch leaves SMs idle and each CTA keeps at least 64 rows
static int lu_panel_cluster(int cnt, int hc, int nsm) {
  int cs = 1;
  while (cs < 8 && (hc + cs - 1) / cs > LU_CL_MAXT) cs *= 2;
  while (cs < 8 && cnt * cs * 2 <= nsm && (hc + 2 * cs - 1) / (2 * cs) >= 64) cs *= 2;
  return cs;
}

// the LU panel of `cnt` items at column k0 (rows up to hc = capacity - k0):
// one CTA with the rows in registers, a cluster per item for taller panels,
// or the shared-memory / global-memory panels
static int lu_panel(Handle& h, const LuItem* items, int cnt, int k0, int hc) {
  cudaStream_t st = h.stream;
  const int cs = lu_panel_cluster(cnt, hc, h.nsm);
  if (hc <= LU_RG_MAXH) {
    k_lu_panel_rg<<<cnt, (hc + 31) / 32 * 32, 0, st>>>(items, k0, h.derr);
    ++h.nlaunch;
  } else if (cs > 1 && (hc + cs - 1) / cs <= LU_CL_MAXT && hc <= h.panel_rows) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cnt * cs);
    cfg.blockDim = dim3(((hc + cs - 1) / cs + 31) / 32 * 32);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    AIFMM_CUDA_TRY(h, cudaLaunchKernelEx(&cfg, k_lu_panel_cl, items, k0, h.derr));
    ++h.nlaunch;
  } else {
    const int hh = std::min(hc, h.panel_rows);
    k_lu_panel_sm<<<cnt, lu_panel_threads(hh), sizeof(double) * (size_t)hh * LU_NB, st>>>(items, k0, h.panel_rows,
                                                                                          h.derr);
    ++h.nlaunch;
    if (hc > h.panel_rows) {
      k_lu_panel_big<<<cnt, 256, 0, st>>>(items, k0, h.panel_rows, h.derr);
      ++h.nlaunch;
    }
  }
  return HOK;
}

// k_cmp_qrcp for c.cnt boxes (nsides each) in clusters of q CTAs; few
// clusters (top levels): wider CTAs, fewer columns per warp
static int launch_qrcp(Handle& h, const LV& v, const Cmp& c, int q, int nsides, const FacLevel& F) {
  cudaLaunchConfig_t cfg = {};
  const int ncta = q * nsides * c.cnt;
  cfg.gridDim = dim3(ncta);
  cfg.blockDim = dim3(ncta <= h.nsm ? 1024 : ncta <= 2 * h.nsm ? 512 : 256);
  cfg.dynamicSmemBytes = sizeof(double) * (2 * (size_t)F.M + (F.M + 1) / 2 + 2 * (size_t)((c.ccap + q - 1) / q));
  if (cfg.dynamicSmemBytes > (size_t)h.smem_optin) {
    h.err = "compress: a box side needs " + std::to_string(cfg.dynamicSmemBytes) + " bytes of shared memory per CTA";
    return HCAPACITY;
  }
  if (cfg.dynamicSmemBytes > 48 * 1024)
    AIFMM_CUDA_TRY(h, cudaFuncSetAttribute(k_cmp_qrcp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)cfg.dynamicSmemBytes));
  cfg.stream = h.stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = q;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  AIFMM_CUDA_TRY(h, cudaLaunchKernelEx(&cfg, k_cmp_qrcp, v, c));
  ++h.nlaunch;
  return HOK;
}

static int factor_level(Handle& h, int l) {
  const int d = h.d;
  cudaStream_t st = h.stream;
  FacLevel& F = h.fac[l];
  LV v = view(h, F);
  const int ncol = ipow(3, d);
  int nws = ipow(5, d) - ipow(3, d);
  const int pm = product_mode(h);
  DetailProf dp;
  dp.on = std::getenv("AIFMM_PROFILE_DETAIL") != nullptr;
  dp.st = st;
  const int nsides = h.sym ? 1 : 2;
  // ---- Householder QR of every box's basis (phase 1 of the column-space
  // compression) in one launch for the whole level: the basis of a box
  // changes only at its own compression, so its Q0 is the same whichever
  // colour step compresses it, and the colour steps no longer wait on a
  // chain of dependent Householder steps each
  double* QB = (double*)hscratch(h, 37, sizeof(double) * (size_t)F.nb * 2 * F.M * F.M);
  {
    Cmp cb = {};
    cb.cnt = F.nb;
    cb.all = 1;
    cb.WC = F.R;
    cb.W = (double*)hscratch(h, 38, sizeof(double) * (size_t)F.nb * 2 * F.M * F.R);
    cb.Q = QB;
    int* ib = (int*)hscratch(h, 39, sizeof(int) * (size_t)F.nb * 8);
    cb.tau = (double*)hscratch(h, 40, sizeof(double) * (size_t)F.nb * 2);
    if (!QB || !cb.W || !ib || !cb.tau) return HOOM;
    cb.nc = ib;
    cb.rk = ib + 2 * F.nb;
    cb.rn = ib + 4 * F.nb;
    cb.rold = ib + 5 * F.nb;
    cb.skip = ib + 6 * F.nb;
    cb.eps = h.ftol;
    cb.flops = h.dacc;
    cb.qflops = h.dacc + 1;
    cb.err = h.derr;
    cb.sym = h.sym ? 1 : 0;
    cb.phase = 1;
    cb.ccap = F.R;
    dp.begin("qr_basis");
    k_basis_gather<<<F.nb * nsides, 256, 0, st>>>(v, cb, nsides); ++h.nlaunch;
    GroupTimer gq(h, Handle::G_QRCP);
    const int rc = launch_qrcp(h, v, cb, 2, nsides, F);
    if (rc != HOK) return rc;
    dp.end();
  }
  for (int col = 0; col < ncol; ++col) {
    int cnt = colour_count(col, d, F.n);
    if (cnt == 0) continue;
    // ---- compress and redirect
    Cmp c;
    c.col = col;
    c.cnt = cnt;
    c.eps = h.ftol;
    c.flops = h.dacc;
    c.qflops = h.dacc + 1;   // the QR steps' flops are counted apart
    c.err = h.derr;
    c.sym = h.sym ? 1 : 0;
    c.all = 0;
    c.QB = QB;
    c.WC = F.R + nws * F.M;
    size_t wsz = (size_t)cnt * 2 * F.M * c.WC;
    c.W = (double*)hscratch(h, 20, sizeof(double) * wsz);
    c.Q = (double*)hscratch(h, 21, sizeof(double) * (size_t)cnt * 2 * F.M * F.M);
    c.cn = (double*)hscratch(h, 22, sizeof(double) * (size_t)cnt * 2 * c.WC);
    int* ib = (int*)hscratch(h, 23, sizeof(int) * (size_t)cnt * 8);
    c.Lm = (double*)hscratch(h, 24, sizeof(double) * (size_t)cnt * 2 * F.R * F.R);
    c.T = (double*)hscratch(h, 32, sizeof(double) * (size_t)cnt * 2 * F.R * c.WC);
    c.tau = (double*)hscratch(h, 33, sizeof(double) * (size_t)cnt * 2);
    c.boff = (int*)hscratch(h, 34, sizeof(int) * (size_t)cnt * 2 * F.ns5);
    if (!c.W || !c.Q || !c.cn || !ib || !c.Lm || !c.T || !c.tau || !c.boff) return HOOM;
    c.nc = ib;
    c.rk = ib + 2 * cnt;
    c.rn = ib + 4 * cnt;
    c.rold = ib + 5 * cnt;
    c.skip = ib + 6 * cnt;
    GroupTimer* gt = new GroupTimer(h, Handle::G_COMPRESS);
    dp.begin("gather");
    k_cmp_list<<<(cnt * nsides * 32 + 127) / 128, 128, 0, st>>>(v, c, nsides); ++h.nlaunch;
    k_cmp_gather<<<dim3(cnt * nsides, F.ns5 + 1), 256, 0, st>>>(v, c, nsides); ++h.nlaunch;
    dp.end();
    k_cmp_skip<<<(cnt + 127) / 128, 128, 0, st>>>(v, c); ++h.nlaunch;
    {
      // Q0 (the basis QR) was copied in by k_cmp_gather: the fill-ins
      // projected off it, then phase 2 (QRCP of the projected fill-ins) in
      // clusters of qc CTAs, qc so that the colour's clusters give about two
      // CTAs per SM, then the new basis columns made orthogonal to Q0 once more
      int qc = 2;
      while (qc < 16 && qc * nsides * cnt < 2 * h.nsm) qc *= 2;
      int maxr = 1;
      for (int b = 0; b < F.nb; ++b) maxr = std::max(maxr, F.h_r[b]);
      const int ptiles_r = (maxr + 63) / 64;
      for (int what = 0; what <= 1; ++what) {
        if (what == 1) {
          c.phase = 2;
          c.ccap = c.WC;
          dp.begin("qrcp_fill");
          delete gt;
          gt = new GroupTimer(h, Handle::G_QRCP);
          const int rc = launch_qrcp(h, v, c, qc, nsides, F);
          if (rc != HOK) {
            delete gt;
            return rc;
          }
          delete gt;
          gt = new GroupTimer(h, Handle::G_COMPRESS);
          dp.end();
        }
        const int ncx = what == 0 ? c.WC : F.M;
        const dim3 g1((ncx + 63) / 64, ptiles_r, cnt * nsides), g2((ncx + 63) / 64, (F.M + 63) / 64, cnt * nsides);
        dp.begin(what == 0 ? "project_fill" : "project_basis");
        AIFMM_LAUNCH_PM(pm, k_cmp_ptq, g1, v, c, what);
        AIFMM_LAUNCH_PM(pm, k_cmp_pqt, g2, v, c, what);
        h.nlaunch += 2;
        dp.end();
      }
    }
    dp.begin("equalise");
    k_cmp_equalise<<<cnt, 256, 0, st>>>(v, c); ++h.nlaunch;
    dp.end();
    dp.begin("lmat");
    AIFMM_CUDA_TRY(h, cudaMemsetAsync(c.Lm, 0, sizeof(double) * (size_t)cnt * 2 * F.R * F.R, st));
    {
      const int rt = (F.R + 63) / 64;
      AIFMM_LAUNCH_PM(pm, k_cmp_lmat, dim3(rt, rt, 2 * cnt), v, c);
      ++h.nlaunch;
    }
    dp.end();
    dp.begin("row_transform");
    k_cmp_row_transform<<<dim3(F.ns6 + 1, cnt), 256, 0, st>>>(v, c); ++h.nlaunch;
    dp.end();
    dp.begin("row_fill");
    const int tpc = (F.M + 63) / 64, rtl = (F.R + 63) / 64;
    AIFMM_LAUNCH_PM(pm, k_cmp_row_fill, dim3(F.ns5 * tpc, rtl, cnt), v, c, tpc);
    ++h.nlaunch;
    dp.end();
    dp.begin("row_done");
    k_cmp_row_done<<<dim3(F.ns5 + 1, cnt), 256, 0, st>>>(v, c); ++h.nlaunch;
    k_cmp_set_rank<<<(cnt + 127) / 128, 128, 0, st>>>(v, c); ++h.nlaunch;
    dp.end();
    if (h.sym) {
      dp.begin("col_mirror");
      k_cmp_col_mirror<<<dim3(F.ns6 + 1 + F.ns5, cnt), 256, 0, st>>>(v, c); ++h.nlaunch;
      dp.end();
    } else {
      dp.begin("col_transform");
      k_cmp_col_transform<<<dim3(F.ns6 + 1, cnt), 256, 0, st>>>(v, c); ++h.nlaunch;
      dp.end();
      dp.begin("col_fill");
      AIFMM_LAUNCH_PM(pm, k_cmp_col_fill, dim3(F.ns5 * tpc, rtl, cnt), v, c, tpc);
      ++h.nlaunch;
      dp.end();
    }
    dp.begin("col_done");
    k_cmp_col_done<<<dim3(F.ns5 + 1, cnt), 256, 0, st>>>(v, c); ++h.nlaunch;
    dp.end();
    delete gt;
    // ---- pivot LU
    Elim e;
    e.col = col;
    e.cnt = cnt;
    e.ncmax = ncol * F.M + F.R;
    e.rows = (Coupled*)hscratch(h, 25, sizeof(Coupled) * (size_t)cnt * MAXC);
    e.cols = (Coupled*)hscratch(h, 26, sizeof(Coupled) * (size_t)cnt * MAXC);
    int* eb = (int*)hscratch(h, 27, sizeof(int) * (size_t)cnt * 3);
    e.Z = (double*)hscratch(h, 28, sizeof(double) * (size_t)cnt * F.P * e.ncmax);
    e.lu = (LuItem*)hscratch(h, 29, sizeof(LuItem) * cnt);
    e.sv = (SolveItem*)hscratch(h, 30, sizeof(SolveItem) * cnt);
    e.colmax = (double*)hscratch(h, 31, sizeof(double) * (size_t)cnt * F.P);
    e.err = h.derr;
    if (!e.rows || !e.cols || !eb || !e.Z || !e.lu || !e.sv || !e.colmax) return HOOM;
    e.nrow = eb;
    e.ncol = eb + cnt;
    e.totc = eb + 2 * cnt;
    k_coupled<<<(cnt + 127) / 128, 128, 0, st>>>(v, e); ++h.nlaunch;
    gt = new GroupTimer(h, Handle::G_PIVLU);
    dp.begin("piv_build");
    k_piv_build<<<dim3(cnt, PB_SLICES), 256, 0, st>>>(v, e); ++h.nlaunch;
    k_z_build<<<dim3(ipow(3, d) + 1, cnt, ZB_SLICES), 256, 0, st>>>(v, e); ++h.nlaunch;
    dp.end();
    k_colmax<<<cnt, 256, 0, st>>>(e.lu, e.colmax, F.P); ++h.nlaunch;
    {
      // LU with partial pivoting of [Piv | B] (B = the coupled columns,
      // k_z_build): the interchanges, the panels' unit-lower solves and the
      // trailing updates also reach B, which ends as L^-1 P B (the forward
      // half of Z = Piv^-1 B), every trailing update a tile GEMM on the
      // tensor cores with 8 digits and the balanced contraction (a column of
      // B mixes entries of very different sizes; see below); fma_gemm: FP64
      // FMAs
      const int maxh = h.panel_rows;
      const int ctot = F.P + e.ncmax;
      const int tiles = (F.P + 63) / 64, ctiles = tiles + (e.ncmax + 63) / 64;
      for (int k0 = 0; k0 < F.P; k0 += LU_NB) {
        dp.begin("lu_panel");
        if (int rc = lu_panel(h, e.lu, cnt, k0, F.P - k0)) return rc;
        dp.end();
        dp.begin("lu_laswp");
        k_lu_laswp<<<dim3((ctot + 127) / 128, cnt), 128, 0, st>>>(e.lu, k0, maxh); ++h.nlaunch;
        dp.end();
        dp.begin("lu_trsm");
        {
          // columns right of the panel, per item, at capacity: n + nb - kend
          // with kend = min(n, k0 + LU_NB), n <= F.P, nb <= ncmax
          const int cols = ctot - k0 - std::min(LU_NB, F.P - k0);
          const int tt = lu_trsm_threads((long long)cnt * cols);
          if (tt)
            k_lu_trsm_t<<<dim3((cols + tt - 1) / tt, cnt), tt, 0, st>>>(e.lu, k0);
          else
            k_lu_trsm<<<dim3((ctot + 3) / 4, cnt), 128, 0, st>>>(e.lu, k0);
          ++h.nlaunch;
        }
        dp.end();
        dp.begin("lu_gemm");
        if (pm == PM_F32)
          k_lu_gemm<PM_F32><<<dim3(ctiles, tiles, cnt), 256, 0, st>>>(e.lu, k0);
        else if (pm == PM_TF32)
          k_lu_gemm<PM_TF32><<<dim3(ctiles, tiles, cnt), 256, 0, st>>>(e.lu, k0);
        else if (pm == PM_OZ)
          k_lu_gemm<PM_OZ8><<<dim3(ctiles, tiles, cnt), 256, OZ_SMEM8, st>>>(e.lu, k0);
        else
          k_lu_gemm<PM_FMA><<<dim3(ctiles, tiles, cnt), 256, 0, st>>>(e.lu, k0);
        ++h.nlaunch;
        dp.end();
      }
    }
    k_piv_perm<<<cnt, 128, sizeof(int) * 2 * (size_t)F.P, st>>>(v, col, cnt); ++h.nlaunch;
    delete gt;
    // ---- Z = U^-1 (L^-1 P B) and the Schur update
    gt = new GroupTimer(h, Handle::G_ZSOLVE);
    {
      // blocked upper triangular solve of Z, upwards, each trailing update a
      // tiled GEMM on the tensor cores with 8 digits (56-bit slices) and the
      // balanced contraction.  A column of Z mixes the x part, of size
      // ~1/A_ii, with the z part, orders of magnitude larger, inside one
      // 64-row chunk: with 7 digits and one exponent per column the small
      // entries kept only 49 - d bits, and the lost accuracy showed up as
      // higher compression ranks at the next level (+16% factor flops, also
      // with the balancing alone); with both, +5% flops for a 1.5x faster
      // solve.  fma_gemm: FP64 FMAs.
      dp.begin("lus");
      const int ctiles = (e.ncmax + 63) / 64;
      const int wstr = (e.ncmax + 3) / 4, cstr = (e.ncmax + 127) / 128;
      const bool wdiag = lus_warp_diag(cnt, e.ncmax);
      for (int k0 = ((F.P - 1) / TB) * TB; k0 >= 0; k0 -= TB) {
        if (wdiag) {
          k_lus_diag_w<0><<<dim3(wstr, cnt), 128, 0, st>>>(e.sv, k0);
        } else {
          k_lus_diag<0><<<dim3(cstr, cnt), 128, 0, st>>>(e.sv, k0);
        }
        ++h.nlaunch;
        if (k0 > 0) {
          const dim3 g(ctiles, (k0 + 63) / 64, cnt);
          if (pm == PM_F32)
            k_lus_update<0, PM_F32><<<g, 256, 0, st>>>(e.sv, k0);
          else if (pm == PM_TF32)
            k_lus_update<0, PM_TF32><<<g, 256, 0, st>>>(e.sv, k0);
          else if (pm == PM_OZ)
            k_lus_update<0, PM_OZ8><<<g, 256, OZ_SMEM8, st>>>(e.sv, k0);
          else
            k_lus_update<0, PM_FMA><<<g, 256, 0, st>>>(e.sv, k0);
          ++h.nlaunch;
        }
      }
      dp.end();
    }
    delete gt;
    int tpb = (F.M + 63) / 64;
    gt = new GroupTimer(h, Handle::G_SCHUR);
    dp.begin("schur");
    {
      // the work list: at most (3^d + 1)^2 entity pairs of tpb^2 tiles per box
      const int ne = ipow(3, d) + 1;
      const size_t cap = (size_t)cnt * ne * ne * tpb * tpb;
      SchurItem* items = (SchurItem*)hscratch(h, 35, sizeof(SchurItem) * cap);
      int* nitems = (int*)hscratch(h, 36, sizeof(int));
      if (!items || !nitems) return HOOM;
      AIFMM_CUDA_TRY(h, cudaMemsetAsync(nitems, 0, sizeof(int), st));
      k_schur_items<<<(cnt + 127) / 128, 128, 0, st>>>(e, h.sym ? 1 : 0, items, nitems); ++h.nlaunch;
      const int sym = h.sym ? 1 : 0;
      if (pm == PM_OZ && h.tc05) {
        k_schur<PM_TC05><<<(unsigned)cap, 256, TC_SMEM, st>>>(v, e, items, nitems, sym);
      } else {
        const int g = h.nsm * schur_ctas_per_sm(h, pm);
        AIFMM_LAUNCH_PM(pm, k_schur, g, v, e, items, nitems, sym);
      }
    }
    ++h.nlaunch;
    dp.end();
    delete gt;
    AIFMM_CUDA_TRY(h, cudaGetLastError());
  }
  AIFMM_CUDA_TRY(h, cudaMemcpyAsync(F.h_r.data(), F.r, sizeof(int) * F.nb, cudaMemcpyDeviceToHost, st));
  AIFMM_CUDA_TRY(h, cudaStreamSynchronize(st));
  int er = check_derr(h);
  if (er) {
    h.err = "factorisation failed at level " + std::to_string(l) +
            (er == DERR_SINGULAR ? ": singular pivot block" : " (device error " + std::to_string(er) + ")");
    return er == DERR_SINGULAR ? HSINGULAR : HCAPACITY;
  }
  dp.report(l);
  k_xoff<<<(F.nb + 127) / 128, 128, 0, st>>>(F.nb, d, F.r, F.xoff); ++h.nlaunch;
  for (int b = 0; b < F.nb; ++b) h.max_rank_factor = std::max(h.max_rank_factor, F.h_r[b]);
  return HOK;
}

// algorithmic FP64 flops of one level (pivot LU, Z and Schur), from the final
// sizes; ranks of boxes eliminated later are their final ranks too, which is
// what the Schur update saw (ranks change only at a box's own compression).
static double level_flops(Handle& h, int l) {
  const int d = h.d;
  FacLevel& F = h.fac[l];
  double fl = 0.0;
  for (int b = 0; b < F.nb; ++b) {
    int bc[3], q[3];
    morton_coords(b, d, l, bc);
    int cb = colour_of(bc, d);
    double m = F.h_m[b], r = F.h_r[b], n = m + r;
    if (m == 0) continue;
    double rows = r, cols = r, ssq = 0.0;
    for (int o = 0; o < ipow(3, d); ++o) {
      int oo = o;
      for (int k = 0; k < d; ++k) {
        q[k] = bc[k] + (oo % 3) - 1;
        oo /= 3;
      }
      if (!in_grid(q, d, F.n) || cheb(bc, q, d) == 0) continue;
      int qb = morton_key(q, d, l);
      double sz = colour_of(q, d) < cb ? F.h_r[qb] : F.h_m[qb];
      rows += sz;
      cols += sz;
      ssq += sz * sz;
    }
    // the forward half of Z = Piv^-1 B runs inside the LU of [Piv | B]
    double flu = 2.0 / 3.0 * n * n * n + n * n * cols, fz = n * n * cols, fs = 2.0 * (rows - r) * m * cols;
    if (h.sym) {
      // blocks (i, j) with i <= j only: neighbour pairs and the y_b column
      double sn = rows - r;
      fs = 2.0 * m * (0.5 * (sn * sn + ssq) + sn * r);
    }
    h.g_flops[Handle::G_PIVLU] += flu;
    h.g_flops[Handle::G_ZSOLVE] += fz;
    h.g_flops[Handle::G_SCHUR] += fs;
    fl += flu + fz + fs;
  }
  return fl;
}

int run_factor(Handle& h) {
  const int L = h.L;
  cudaStream_t st = h.stream;
  h.fac.assign(L + 1, FacLevel());
  h.max_rank_factor = 0;
  h.flops_factor = 0;
  for (int g = 0; g < Handle::G_NG; ++g) h.g_ms[g] = h.g_flops[g] = 0, h.g_launch[g] = 0;
  if (!h.dacc) h.dacc = hnew<double>(h, 4);
  if (!h.dacc) return HOOM;
  AIFMM_CUDA_TRY(h, cudaFuncSetAttribute(k_cmp_qrcp, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  AIFMM_CUDA_TRY(h, cudaFuncSetAttribute(k_schur<PM_OZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
  AIFMM_CUDA_TRY(h, cudaFuncSetAttribute(k_schur<PM_TC05>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
  AIFMM_CUDA_TRY(h, cudaFuncSetAttribute(k_cmp_lmat<PM_OZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
  AIFMM_CUDA_TRY(h, cudaFuncSetAttribute(k_cmp_row_fill<PM_OZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
  AIFMM_CUDA_TRY(h, cudaFuncSetAttribute(k_cmp_col_fill<PM_OZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
  AIFMM_CUDA_TRY(h, cudaFuncSetAttribute(k_cmp_ptq<PM_OZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
  AIFMM_CUDA_TRY(h, cudaFuncSetAttribute(k_cmp_pqt<PM_OZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
  AIFMM_CUDA_TRY(h, cudaFuncSetAttribute(k_lus_update<1, PM_OZ8>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM8));
  AIFMM_CUDA_TRY(h, cudaFuncSetAttribute(k_lu_gemm<PM_OZ8>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM8));
  AIFMM_CUDA_TRY(h, cudaFuncSetAttribute(k_lus_update<0, PM_OZ8>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM8));

  {
    // tallest LU panel kept in shared memory: (rows x 32) doubles within the
    // opt-in limit of the device
    int smax = 0;
    AIFMM_CUDA_TRY(h, cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, h.device));
    h.panel_rows = (smax - 1024) / (int)(sizeof(double) * LU_NB);
    h.smem_optin = smax - 2048;
    AIFMM_CUDA_TRY(h, cudaFuncSetAttribute(k_lu_panel_sm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(sizeof(double) * (size_t)h.panel_rows * LU_NB)));
  }
  AIFMM_CUDA_TRY(h, cudaDeviceGetAttribute(&h.nsm, cudaDevAttrMultiProcessorCount, h.device));
  {
    int l2 = 0;
    AIFMM_CUDA_TRY(h, cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, h.device));
    h.l2_bytes = (size_t)l2;
  }
  DetailProf dpf;   // diagnostic: level set-up, whole level, top LU
  dpf.on = std::getenv("AIFMM_PROFILE_DETAIL") != nullptr;
  dpf.st = st;
  for (int l = L; l >= 2; --l) {
    dpf.begin("setup");
    int e = setup_level(h, l);
    if (e) return e;
    dpf.end();
    dpf.begin("level_total");
    e = factor_level(h, l);
    if (e) return e;
    dpf.end();
    dpf.report(l);
    collect_group_times(h);
    double fc[2] = {0.0, 0.0};
    AIFMM_CUDA_TRY(h, cudaMemcpy(fc, h.dacc, 2 * sizeof(double), cudaMemcpyDeviceToHost));
    AIFMM_CUDA_TRY(h, cudaMemset(h.dacc, 0, 2 * sizeof(double)));
    h.g_flops[Handle::G_COMPRESS] += fc[0];
    h.g_flops[Handle::G_QRCP] += fc[1];
    h.flops_factor += fc[0] + fc[1];
    h.flops_factor += level_flops(h, l);
  }
  // top: dense level-1 system in the level-2 multipoles
  FacLevel& F2 = h.fac[2];
  h.top_off.assign(F2.nb + 1, 0);
  for (int b = 0; b < F2.nb; ++b) h.top_off[b + 1] = h.top_off[b] + F2.h_r[b];
  h.ntop = h.top_off[F2.nb];
  const int nt = std::max(1, h.ntop);
  h.top = hnew<double>(h, (size_t)nt * nt);
  h.top_ipiv = hnew<int>(h, nt);
  h.top_perm = hnew<int>(h, nt, false);
  dpf.begin("top_lu");
  int* toff = hnew<int>(h, F2.nb + 1, false);
  double* cm = hnew<double>(h, nt);
  LuItem* it = hnew<LuItem>(h, 1, false);
  if (!h.top || !h.top_ipiv || !h.top_perm || !toff || !cm || !it) return HOOM;
  AIFMM_CUDA_TRY(h, cudaMemcpyAsync(toff, h.top_off.data(), sizeof(int) * (F2.nb + 1), cudaMemcpyHostToDevice, st));
  LV v2 = view(h, F2);
  k_top_assemble<<<dim3(F2.nb, F2.ns6), 256, 0, st>>>(v2, toff, h.top, h.ntop); ++h.nlaunch;
  LuItem hi;
  hi.a = h.top;
  hi.ipiv = h.top_ipiv;
  hi.colmax = cm;
  hi.n = h.ntop;
  hi.ld = h.ntop;
  hi.b = nullptr;
  hi.ldb = 0;
  hi.nb = 0;
  AIFMM_CUDA_TRY(h, cudaMemcpyAsync(it, &hi, sizeof(hi), cudaMemcpyHostToDevice, st));
  k_colmax<<<1, 256, 0, st>>>(it, cm, nt); ++h.nlaunch;
  for (int k0 = 0; k0 < h.ntop; k0 += LU_NB) {
    if (int rc = lu_panel(h, it, 1, k0, h.ntop - k0)) return rc;
    k_lu_laswp<<<dim3((h.ntop + 127) / 128, 1), 128, 0, st>>>(it, k0, h.panel_rows); ++h.nlaunch;
    k_lu_trsm<<<dim3((h.ntop + 3) / 4, 1), 128, 0, st>>>(it, k0); ++h.nlaunch;
    int tiles = (h.ntop + 63) / 64;
    // trailing updates on the 8-digit tensor-core tile, as in the levels'
    // pivot LUs (FP64 FMAs in the FP32 / FP64-FMA product modes)
    if (product_mode(h) == PM_OZ)
      k_lu_gemm<PM_OZ8><<<dim3(tiles, tiles, 1), 256, OZ_SMEM8, st>>>(it, k0);
    else
      k_lu_gemm<PM_FMA><<<dim3(tiles, tiles, 1), 256, 0, st>>>(it, k0);
    ++h.nlaunch;
  }
  k_ipiv_perm<<<1, 128, h.ntop <= 4096 ? sizeof(int) * 2 * (size_t)h.ntop : 0, st>>>(h.top_ipiv, h.ntop, h.top_perm);
  ++h.nlaunch;
  dpf.end();
  dpf.report(1);
  h.flops_factor += 2.0 / 3.0 * (double)h.ntop * h.ntop * h.ntop;
  AIFMM_CUDA_TRY(h, cudaGetLastError());
  AIFMM_CUDA_TRY(h, cudaStreamSynchronize(st));
  int er = check_derr(h);
  if (er) {
    h.err = "top-level LU: singular";
    return HSINGULAR;
  }
  return HOK;
}

}  // namespace aifmm
