// NNCA operators on the GPU (Sec. 2.3): per box, ACA pivot search on
// A[rows(B), F^{B,i}] (F = points of the interaction-list boxes, eqs. Fj/Fi),
// then U_B = A[rows, s^{B,i}] (A[t^{B,i}, s^{B,i}])^-1 (operator list, Table 2)
// by LU with partial pivoting of the transposed skeleton.  Rows of a non-leaf
// box are its children's row pivots (eq. particleAtNonLeafLevel), which makes
// the bases nested.  Symmetric kernels with sources = targets: V_B = U_B and
// the outgoing pivots are the incoming ones swapped.
//
// The ACA runs in lock-step over all boxes of a level: one iteration is four
// launches (row residual over far-field chunks, column residual per box,
// scaling and dot products over chunks, stopping test per box), so a level
// whose far fields hold tens of thousands of points still fills the GPU.
// Pivot rule: start at row 0; column pivot = largest residual entry of the
// row among unused columns (lowest index on ties); next row = largest entry
// of the residual column among unused rows; a zero residual row is skipped;
// stop at the first term with |u||v| <= eps ||S||_F (term dropped).
#include <algorithm>

#include "internal.h"

namespace aifmm {

namespace {

constexpr int CHUNK = 2048;   // far-field columns per CTA in the chunked kernels
constexpr int ILMAX2 = 27, ILMAX3 = 189;

struct AcaState {
  int k, i, done, phase, jstar;
  double frob2, pivot, nu2;
};

// interaction-list ranges of every box: IL boxes in Morton order with their
// tree-order start and the running column offset.
__global__ void k_il_table(int l, int d, const int* __restrict__ start, int ilmax,
                           int* __restrict__ ils, int* __restrict__ ilo, int* __restrict__ nil) {
  int nb = 1 << (d * l);
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  int n = 1 << l;
  int c[3], q[3];
  morton_coords(b, d, l, c);
  int list[ILMAX3];
  int cnt = 0;
  int ns6 = ipow(6, d);
  for (int s = 0; s < ns6; ++s) {
    slot6_coords(c, s, d, q);
    if (!in_grid(q, d, n) || cheb(c, q, d) <= 1) continue;
    list[cnt++] = morton_key(q, d, l);
  }
  // insertion sort by Morton index (= tree order of the ranges)
  for (int a = 1; a < cnt; ++a) {
    int v = list[a], j = a - 1;
    while (j >= 0 && list[j] > v) {
      list[j + 1] = list[j];
      --j;
    }
    list[j + 1] = v;
  }
  int off = 0;
  for (int a = 0; a < cnt; ++a) {
    int s0 = start[list[a]], e0 = start[list[a] + 1];
    ils[(size_t)b * ilmax + a] = s0;
    ilo[(size_t)b * (ilmax + 1) + a] = off;
    off += e0 - s0;
  }
  ilo[(size_t)b * (ilmax + 1) + cnt] = off;
  nil[b] = cnt;
}

__device__ inline int far_pos(const int* ils, const int* ilo, int cnt, int j) {
  int a = 0;
  while (a + 1 < cnt && ilo[a + 1] <= j) ++a;
  return ils[a] + (j - ilo[a]);
}

struct AcaArgs {
  int nb, M, R, F, ilmax;
  const int* m;
  const int* rows;
  const int* ils;
  const int* ilo;
  const int* nil;
  AcaState* st;
  uint8_t* usedr;
  uint8_t* usedc;
  double* Uv;     // [nb][R+1][M]
  double* Vv;     // [nb][R+1][F]
  double* pv;     // [nb][nchunk] partial argmax values
  int* pi;        // [nb][nchunk] partial argmax indices
  double* pd;     // [nb][nchunk][R+2] partial dots
  double* du;     // [nb][R+1]
  int nchunk;
  int* pivloc;
  int* pivpos;
  int* far;
  int* rank;
  double eps;
  KParams kp;
  Pts P;
};

__global__ void k_aca_init(AcaArgs a) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= a.nb) return;
  AcaState s;
  s.k = 0;
  s.i = 0;
  s.phase = 0;
  s.jstar = -1;
  s.frob2 = 0.0;
  s.pivot = 0.0;
  s.nu2 = 0.0;
  int F = a.ilo[(size_t)b * (a.ilmax + 1) + a.nil[b]];
  s.done = (a.m[b] == 0 || F == 0) ? 1 : 0;
  a.st[b] = s;
  a.rank[b] = 0;
}

// row residual of the current row over one chunk of the far field
__global__ void __launch_bounds__(256) k_aca_row(AcaArgs a) {
  __shared__ double ucol[1024];
  __shared__ double shv[32];
  __shared__ int shi[32];
  int b = blockIdx.y, ch = blockIdx.x;
  AcaState s = a.st[b];
  if (s.done) return;
  const int* ils = a.ils + (size_t)b * a.ilmax;
  const int* ilo = a.ilo + (size_t)b * (a.ilmax + 1);
  int cnt = a.nil[b];
  int F = ilo[cnt];
  int j0 = ch * CHUNK;
  if (j0 >= F) {
    if (threadIdx.x == 0) {
      a.pv[(size_t)b * a.nchunk + ch] = -1.0;
      a.pi[(size_t)b * a.nchunk + ch] = -1;
    }
    return;
  }
  const double* Uv = a.Uv + (size_t)b * (a.R + 1) * a.M;
  double* Vv = a.Vv + (size_t)b * (a.R + 1) * a.F;
  for (int t = threadIdx.x; t < s.k; t += blockDim.x) ucol[t] = Uv[(size_t)t * a.M + s.i];
  __syncthreads();
  int rowpos = a.rows[(size_t)b * a.M + s.i];
  const uint8_t* usedc = a.usedc + (size_t)b * a.F;
  ArgMax best;
  best.v = -1.0;
  best.i = -1;
  int j1 = min(F, j0 + CHUNK);
  for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
    double val = keval(a.kp, a.P, rowpos, far_pos(ils, ilo, cnt, j));
    for (int t = 0; t < s.k; ++t) val = __dsub_rn(val, __dmul_rn(ucol[t], Vv[(size_t)t * a.F + j]));
    Vv[(size_t)s.k * a.F + j] = val;
    if (!usedc[j]) {
      ArgMax c;
      c.v = fabs(val);
      c.i = j;
      best = amax_pick(best, c);
    }
  }
  best = block_amax(best, shv, shi);
  if (threadIdx.x == 0) {
    a.pv[(size_t)b * a.nchunk + ch] = best.v;
    a.pi[(size_t)b * a.nchunk + ch] = best.i;
  }
}

// column residual at the chosen column (one block per box)
__global__ void __launch_bounds__(256) k_aca_col(AcaArgs a) {
  __shared__ double vrow[1024];
  __shared__ double shv[32];
  __shared__ int shi[32];
  __shared__ double shs[32];
  int b = blockIdx.x;
  AcaState s = a.st[b];
  if (s.done) return;
  const int* ils = a.ils + (size_t)b * a.ilmax;
  const int* ilo = a.ilo + (size_t)b * (a.ilmax + 1);
  int cnt = a.nil[b];
  int F = ilo[cnt];
  int m = a.m[b];
  uint8_t* usedr = a.usedr + (size_t)b * a.M;
  ArgMax best;
  best.v = -1.0;
  best.i = -1;
  int nch = (F + CHUNK - 1) / CHUNK;
  for (int c = threadIdx.x; c < nch; c += blockDim.x) {
    ArgMax x;
    x.v = a.pv[(size_t)b * a.nchunk + c];
    x.i = a.pi[(size_t)b * a.nchunk + c];
    best = amax_pick(best, x);
  }
  best = block_amax(best, shv, shi);
  if (!(best.v > 0.0)) {
    // zero residual row: mark it used and move to the lowest unused row
    __syncthreads();
    if (threadIdx.x == 0) {
      usedr[s.i] = 1;
      int nxt = -1;
      for (int r = 0; r < m; ++r)
        if (!usedr[r]) {
          nxt = r;
          break;
        }
      if (nxt < 0) s.done = 1;
      else s.i = nxt;
      s.phase = 0;
      a.st[b] = s;
    }
    return;
  }
  const double* Vv = a.Vv + (size_t)b * (a.R + 1) * a.F;
  double* Uv = a.Uv + (size_t)b * (a.R + 1) * a.M;
  int js = best.i;
  for (int t = threadIdx.x; t < s.k; t += blockDim.x) vrow[t] = Vv[(size_t)t * a.F + js];
  __syncthreads();
  int colpos = far_pos(ils, ilo, cnt, js);
  double nu2 = 0.0;
  for (int r = threadIdx.x; r < m; r += blockDim.x) {
    double u = keval(a.kp, a.P, a.rows[(size_t)b * a.M + r], colpos);
    for (int t = 0; t < s.k; ++t) u = __dsub_rn(u, __dmul_rn(vrow[t], Uv[(size_t)t * a.M + r]));
    Uv[(size_t)s.k * a.M + r] = u;
    nu2 += u * u;
  }
  nu2 = block_sum(nu2, shs);
  __syncthreads();
  // u_t . u_k for t < k, one warp per t
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int t = w; t < s.k; t += nw) {
    double acc = 0.0;
    for (int r = lane; r < m; r += 32) acc += Uv[(size_t)t * a.M + r] * Uv[(size_t)s.k * a.M + r];
    acc = warp_sum(acc);
    if (lane == 0) a.du[(size_t)b * (a.R + 1) + t] = acc;
  }
  if (threadIdx.x == 0) {
    usedr[s.i] = 1;
    s.pivot = Vv[(size_t)s.k * a.F + js];
    s.jstar = js;
    s.nu2 = nu2;
    s.phase = 1;
    a.st[b] = s;
  }
}

// scale the new row by the pivot and form its dot products (chunked)
__global__ void __launch_bounds__(256) k_aca_scale(AcaArgs a) {
  __shared__ double shs[32];
  int b = blockIdx.y, ch = blockIdx.x;
  AcaState s = a.st[b];
  if (s.done || s.phase != 1) return;
  const int* ilo = a.ilo + (size_t)b * (a.ilmax + 1);
  int F = ilo[a.nil[b]];
  int j0 = ch * CHUNK;
  double* pd = a.pd + ((size_t)b * a.nchunk + ch) * (a.R + 2);
  if (j0 >= F) return;
  int j1 = min(F, j0 + CHUNK);
  double* Vv = a.Vv + (size_t)b * (a.R + 1) * a.F;
  double* vk = Vv + (size_t)s.k * a.F;
  double nv2 = 0.0;
  for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
    double v = vk[j] / s.pivot;
    vk[j] = v;
    nv2 += v * v;
  }
  nv2 = block_sum(nv2, shs);
  __syncthreads();
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int t = w; t < s.k; t += nw) {
    double acc = 0.0;
    for (int j = j0 + lane; j < j1; j += 32) acc += Vv[(size_t)t * a.F + j] * vk[j];
    acc = warp_sum(acc);
    if (lane == 0) pd[t] = acc;
  }
  if (threadIdx.x == 0) pd[a.R + 1] = nv2;
}

// stopping test and commit (one block of 32 threads per box)
__global__ void k_aca_commit(AcaArgs a) {
  int b = blockIdx.x;
  AcaState s = a.st[b];
  if (s.done || s.phase != 1) return;
  const int* ils = a.ils + (size_t)b * a.ilmax;
  const int* ilo = a.ilo + (size_t)b * (a.ilmax + 1);
  int cnt = a.nil[b];
  int F = ilo[cnt];
  int nch = (F + CHUNK - 1) / CHUNK;
  int lane = threadIdx.x;
  // reduce chunk partials: nv2 and v_t . v_k
  __shared__ double dv[1024];
  __shared__ double snv2;
  for (int t = lane; t <= s.k; t += 32) {
    int slot = t < s.k ? t : a.R + 1;
    double acc = 0.0;
    for (int c = 0; c < nch; ++c) acc += a.pd[((size_t)b * a.nchunk + c) * (a.R + 2) + slot];
    if (t < s.k) dv[t] = acc;
    else snv2 = acc;
  }
  __syncwarp();
  if (lane != 0) return;
  double cross = 0.0;
  for (int t = 0; t < s.k; ++t) cross += a.du[(size_t)b * (a.R + 1) + t] * dv[t];
  double nu = sqrt(s.nu2), nv = sqrt(snv2);
  s.frob2 += 2.0 * cross + (nu * nv) * (nu * nv);
  int m = a.m[b];
  if (nu * nv <= a.eps * sqrt(fmax(s.frob2, 0.0))) {
    s.done = 1;
    a.st[b] = s;
    a.rank[b] = s.k;
    return;
  }
  int k = s.k;
  a.pivloc[(size_t)b * a.R + k] = s.i;
  a.pivpos[(size_t)b * a.R + k] = a.rows[(size_t)b * a.M + s.i];
  a.far[(size_t)b * a.R + k] = far_pos(ils, ilo, cnt, s.jstar);
  a.usedc[(size_t)b * a.F + s.jstar] = 1;
  s.k = k + 1;
  a.rank[b] = s.k;
  // next row: largest |u_k| among unused rows, lowest index on ties
  const double* uk = a.Uv + ((size_t)b * (a.R + 1) + k) * a.M;
  const uint8_t* usedr = a.usedr + (size_t)b * a.M;
  int best = -1;
  double bv = -1.0;
  for (int r = 0; r < m; ++r) {
    if (usedr[r]) continue;
    double v = fabs(uk[r]);
    if (v > bv) {
      bv = v;
      best = r;
    }
  }
  int kmax = m < F ? m : F;
  if (best < 0 || s.k >= kmax || s.k >= a.R) s.done = 1;
  else s.i = best;
  s.phase = 0;
  a.st[b] = s;
}

__global__ void k_count_active(const AcaState* st, int nb, int* out) {
  int c = 0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) c += st[b].done ? 0 : 1;
  c = __reduce_add_sync(0xffffffffu, c);
  if (threadIdx.x == 0) *out = c;
}

// leaf rows: the box's points in tree order
__global__ void k_leaf_rows(const int* __restrict__ start, int nb, int M, int* __restrict__ m,
                            int* __restrict__ rows) {
  int b = blockIdx.x;
  int s = start[b], e = start[b + 1];
  if (threadIdx.x == 0) m[b] = e - s;
  for (int i = threadIdx.x; i < e - s; i += blockDim.x) rows[(size_t)b * M + i] = s + i;
}

// non-leaf rows: concatenated row pivots of the children (Morton order)
__global__ void k_parent_rows(int d, int nbP, const int* __restrict__ crank, const int* __restrict__ cpiv,
                              int cR, int M, int* __restrict__ m, int* __restrict__ rows) {
  int P = blockIdx.x;
  int nc = 1 << d;
  int off = 0;
  for (int c = 0; c < nc; ++c) {
    int ch = (P << d) + c;
    int r = crank[ch];
    for (int i = threadIdx.x; i < r; i += blockDim.x) rows[(size_t)P * M + off + i] = cpiv[(size_t)ch * cR + i];
    off += r;
  }
  if (threadIdx.x == 0) m[P] = off;
}

// U_B = A[rows, s^i] (A[t^i, s^i])^-1: LU (partial pivoting) of the
// transposed skeleton, then one forward/back substitution per row of U.
__global__ void __launch_bounds__(256) k_nnca_U(int M, int R, const int* __restrict__ m,
                                                const int* __restrict__ rank, const int* __restrict__ rows,
                                                const int* __restrict__ pivpos, const int* __restrict__ far,
                                                double* __restrict__ lu_ws, int* __restrict__ ip_ws,
                                                double* __restrict__ U, KParams kp, Pts P, int* err) {
  __shared__ double shv[32];
  __shared__ int shi[32];
  int b = blockIdx.x;
  int r = rank[b], mb = m[b];
  if (r == 0) return;
  double* A = lu_ws + (size_t)b * R * R;   // A = S^T, column-major ld R: A[a + c*R]
  int* ip = ip_ws + (size_t)b * R;
  const int* tp = pivpos + (size_t)b * R;
  const int* fp = far + (size_t)b * R;
  // S[c][a] = A(t_c, s_a);  S^T[a][c] = S[c][a]
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    int a = e % r, c = e / r;
    A[a + (size_t)c * R] = keval(kp, P, tp[c], fp[a]);
  }
  __syncthreads();
  for (int k = 0; k < r; ++k) {
    ArgMax best;
    best.v = -1.0;
    best.i = -1;
    for (int i = k + threadIdx.x; i < r; i += blockDim.x) {
      ArgMax c;
      c.v = fabs(A[i + (size_t)k * R]);
      c.i = i;
      best = amax_pick(best, c);
    }
    best = block_amax(best, shv, shi);
    int p = best.i;
    if (threadIdx.x == 0) ip[k] = p;
    if (!(best.v > 0.0)) {
      if (threadIdx.x == 0) set_err(err, DERR_SINGULAR);
      return;
    }
    if (p != k)
      for (int c = threadIdx.x; c < r; c += blockDim.x) {
        double t = A[k + (size_t)c * R];
        A[k + (size_t)c * R] = A[p + (size_t)c * R];
        A[p + (size_t)c * R] = t;
      }
    __syncthreads();
    double piv = A[k + (size_t)k * R];
    for (int i = k + 1 + threadIdx.x; i < r; i += blockDim.x) A[i + (size_t)k * R] /= piv;
    __syncthreads();
    int nt = (r - k - 1) * (r - k - 1);
    for (int e = threadIdx.x; e < nt; e += blockDim.x) {
      int i = k + 1 + e % (r - k - 1), c = k + 1 + e / (r - k - 1);
      A[i + (size_t)c * R] -= A[i + (size_t)k * R] * A[k + (size_t)c * R];
    }
    __syncthreads();
  }
  // each row i of U solves S^T u = A(rows_i, s)^T
  double* Ub = U + (size_t)b * M * R;
  for (int i = threadIdx.x; i < mb; i += blockDim.x) {
    int rp = rows[(size_t)b * M + i];
    double z[256];
    if (r > 256) {
      set_err(err, DERR_CAPACITY);
      return;
    }
    for (int a = 0; a < r; ++a) z[a] = keval(kp, P, rp, fp[a]);
    for (int k = 0; k < r; ++k) {
      int p = ip[k];
      if (p != k) {
        double t = z[k];
        z[k] = z[p];
        z[p] = t;
      }
    }
    for (int k = 0; k < r; ++k) {
      double zk = z[k];
      for (int q = k + 1; q < r; ++q) z[q] -= A[q + (size_t)k * R] * zk;
    }
    for (int k = r - 1; k >= 0; --k) {
      double zk = z[k] / A[k + (size_t)k * R];
      z[k] = zk;
      for (int q = 0; q < k; ++q) z[q] -= A[q + (size_t)k * R] * zk;
    }
    for (int a = 0; a < r; ++a) Ub[i + (size_t)a * M] = z[a];
  }
}

}  // namespace

int build_nnca(Handle& h) {
  const int d = h.d, L = h.L;
  cudaStream_t st = h.stream;
  h.nn.assign(L + 1, NnLevel());
  const int ilmax = d == 2 ? ILMAX2 : ILMAX3;
  int* active = hnew<int>(h, 1);
  if (!active) return HOOM;
  for (int l = L; l >= 2; --l) {
    NnLevel& N = h.nn[l];
    N.l = l;
    N.nb = 1 << (d * l);
    const int nb = N.nb;
    const int* startl = h.start + h.soff[l];
    // host-side sizes: rows per box and far-field sizes (from the leaf starts)
    std::vector<int> cnt(nb);
    const int sh = d * (L - l);
    for (int b = 0; b < nb; ++b) cnt[b] = h.h_leaf_start[(size_t)(b + 1) << sh] - h.h_leaf_start[(size_t)b << sh];
    N.h_m.assign(nb, 0);
    if (l == L) {
      for (int b = 0; b < nb; ++b) N.h_m[b] = cnt[b];
    } else {
      const NnLevel& C = h.nn[l + 1];
      for (int b = 0; b < nb; ++b)
        for (int c = 0; c < (1 << d); ++c) N.h_m[b] += C.h_rank[(b << d) + c];
    }
    int Fmax = 0;
    {
      int n = 1 << l;
      for (int b = 0; b < nb; ++b) {
        int c[3], q[3];
        morton_coords(b, d, l, c);
        int f = 0;
        for (int s = 0; s < ipow(6, d); ++s) {
          slot6_coords(c, s, d, q);
          if (!in_grid(q, d, n) || cheb(c, q, d) <= 1) continue;
          f += cnt[morton_key(q, d, l)];
        }
        Fmax = std::max(Fmax, f);
      }
    }
    N.M = std::max(1, *std::max_element(N.h_m.begin(), N.h_m.end()));
    N.F = std::max(1, Fmax);
    N.R = std::max(1, std::min(N.M, N.F));
    const int M = N.M, R = N.R, F = N.F;
    N.m = hnew<int>(h, nb);
    N.rank = hnew<int>(h, nb);
    N.rows = hnew<int>(h, (size_t)nb * M);
    N.pivloc = hnew<int>(h, (size_t)nb * R);
    N.pivpos = hnew<int>(h, (size_t)nb * R);
    N.far = hnew<int>(h, (size_t)nb * R);
    N.U = hnew<double>(h, (size_t)nb * M * R);
    if (!N.m || !N.rank || !N.rows || !N.pivloc || !N.pivpos || !N.far || !N.U) return HOOM;
    if (l == L) {
      k_leaf_rows<<<nb, 128, 0, st>>>(startl, nb, M, N.m, N.rows); ++h.nlaunch;
    } else {
      const NnLevel& C = h.nn[l + 1];
      k_parent_rows<<<nb, 128, 0, st>>>(d, nb, C.rank, C.pivpos, C.R, M, N.m, N.rows); ++h.nlaunch;
    }
    // interaction-list tables
    int* ils = (int*)hscratch(h, 0, sizeof(int) * (size_t)nb * ilmax);
    int* ilo = (int*)hscratch(h, 1, sizeof(int) * (size_t)nb * (ilmax + 1));
    int* nil = (int*)hscratch(h, 2, sizeof(int) * (size_t)nb);
    if (!ils || !ilo || !nil) return HOOM;
    k_il_table<<<(nb + 127) / 128, 128, 0, st>>>(l, d, startl, ilmax, ils, ilo, nil); ++h.nlaunch;
    // ACA workspace
    const int nchunk = (F + CHUNK - 1) / CHUNK;
    AcaArgs a;
    a.nb = nb;
    a.M = M;
    a.R = R;
    a.F = F;
    a.ilmax = ilmax;
    a.m = N.m;
    a.rows = N.rows;
    a.ils = ils;
    a.ilo = ilo;
    a.nil = nil;
    a.nchunk = nchunk;
    a.st = (AcaState*)hscratch(h, 3, sizeof(AcaState) * nb);
    a.usedr = (uint8_t*)hscratch(h, 4, (size_t)nb * M);
    a.usedc = (uint8_t*)hscratch(h, 5, (size_t)nb * F);
    a.Uv = (double*)hscratch(h, 6, sizeof(double) * (size_t)nb * (R + 1) * M);
    a.Vv = (double*)hscratch(h, 7, sizeof(double) * (size_t)nb * (R + 1) * F);
    a.pv = (double*)hscratch(h, 8, sizeof(double) * (size_t)nb * nchunk);
    a.pi = (int*)hscratch(h, 9, sizeof(int) * (size_t)nb * nchunk);
    a.pd = (double*)hscratch(h, 10, sizeof(double) * (size_t)nb * nchunk * (R + 2));
    a.du = (double*)hscratch(h, 11, sizeof(double) * (size_t)nb * (R + 1));
    if (!a.st || !a.usedr || !a.usedc || !a.Uv || !a.Vv || !a.pv || !a.pi || !a.pd || !a.du) return HOOM;
    if (R + 1 > 1024) {
      h.err = "NNCA rank capacity above 1024";
      return HCAPACITY;
    }
    AIFMM_CUDA_TRY(h, cudaMemsetAsync(a.usedr, 0, (size_t)nb * M, st));
    AIFMM_CUDA_TRY(h, cudaMemsetAsync(a.usedc, 0, (size_t)nb * F, st));
    a.pivloc = N.pivloc;
    a.pivpos = N.pivpos;
    a.far = N.far;
    a.rank = N.rank;
    a.eps = h.tol;
    a.kp = h.kp;
    a.P = h.P();
    k_aca_init<<<(nb + 127) / 128, 128, 0, st>>>(a); ++h.nlaunch;
    dim3 gchunk(nchunk, nb);
    int iters = 0;
    const int maxit = M + 2;
    while (iters < maxit) {
      for (int q = 0; q < 8 && iters < maxit; ++q, ++iters) {
        k_aca_row<<<gchunk, 256, 0, st>>>(a); ++h.nlaunch;
        k_aca_col<<<nb, 256, 0, st>>>(a); ++h.nlaunch;
        k_aca_scale<<<gchunk, 256, 0, st>>>(a); ++h.nlaunch;
        k_aca_commit<<<nb, 32, 0, st>>>(a); ++h.nlaunch;
      }
      k_count_active<<<1, 32, 0, st>>>(a.st, nb, active); ++h.nlaunch;
      int hact = 0;
      AIFMM_CUDA_TRY(h, cudaMemcpyAsync(&hact, active, sizeof(int), cudaMemcpyDeviceToHost, st));
      AIFMM_CUDA_TRY(h, cudaStreamSynchronize(st));
      if (hact == 0) break;
    }
    // operators U = A[rows, s] S^-1
    double* lu_ws = (double*)hscratch(h, 12, sizeof(double) * (size_t)nb * R * R);
    int* ip_ws = (int*)hscratch(h, 13, sizeof(int) * (size_t)nb * R);
    if (!lu_ws || !ip_ws) return HOOM;
    k_nnca_U<<<nb, 256, 0, st>>>(M, R, N.m, N.rank, N.rows, N.pivpos, N.far, lu_ws, ip_ws, N.U, h.kp, h.P(),
                                 h.derr); ++h.nlaunch;
    AIFMM_CUDA_TRY(h, cudaGetLastError());
    N.h_rank.assign(nb, 0);
    AIFMM_CUDA_TRY(h, cudaMemcpyAsync(N.h_rank.data(), N.rank, sizeof(int) * nb, cudaMemcpyDeviceToHost, st));
    AIFMM_CUDA_TRY(h, cudaStreamSynchronize(st));
    int e = check_derr(h);
    if (e) {
      h.err = "NNCA failed at level " + std::to_string(l) + " (device error " + std::to_string(e) + ")";
      return e == DERR_SINGULAR ? HSINGULAR : HCAPACITY;
    }
    for (int b = 0; b < nb; ++b) h.max_rank_nnca = std::max(h.max_rank_nnca, N.h_rank[b]);
  }
  return HOK;
}

}  // namespace aifmm
