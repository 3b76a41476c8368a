// Restarted GMRES with right preconditioning by the AIFMM factorisation.
//
// Sec. 4 solves with GMRES (Saad & Schultz) whose product is the NNCA H^2
// matrix-vector product (Experiments 2-4), stopping when the relative
// residual ||A x - b|| / ||b|| reaches eps_GMRES; Experiment 5 uses a
// low-accuracy AIFMM factorisation as the preconditioner.  Here the Krylov
// space is that of A M^-1 (right preconditioning, so the least-squares
// residual is the residual of A x = b itself); M^-1 is the AIFMM solve
// (Algorithm 3) and A the H^2 product.
//
// Every vector operation runs in the kernels below on the handle's stream:
// Arnoldi with classical Gram-Schmidt applied twice (two column-parallel
// passes instead of j dependent dot products), the Givens update of the
// Hessenberg column in one thread, the small triangular solve in one thread.
// The host reads one scalar per iteration (the residual estimate) to decide
// whether to stop.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace aifmm {
namespace {

constexpr int GM_THREADS = 256;
constexpr int GM_MAX_RESTART = 512;

// out[c] = V[:, c] . w for c < ncols; one block per column
__global__ void __launch_bounds__(GM_THREADS) k_gm_dots(const double* __restrict__ V, int64_t ldv, int ncols,
                                                         const double* __restrict__ w, int64_t n,
                                                         double* __restrict__ out) {
  __shared__ double sh[32];
  int c = blockIdx.x;
  if (c >= ncols) return;
  const double* v = V + (size_t)c * ldv;
  double a = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a += v[i] * w[i];
  a = block_sum(a, sh);
  if (threadIdx.x == 0) out[c] = a;
}

// w -= V[:, :ncols] coef (coef on the device)
__global__ void __launch_bounds__(GM_THREADS) k_gm_sub(const double* __restrict__ V, int64_t ldv, int ncols,
                                                        const double* __restrict__ coef, double* __restrict__ w,
                                                        int64_t n) {
  __shared__ double cf[GM_MAX_RESTART + 1];
  for (int c = threadIdx.x; c < ncols; c += blockDim.x) cf[c] = coef[c];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double a = w[i];
    for (int c = 0; c < ncols; ++c) a -= V[i + (size_t)c * ldv] * cf[c];
    w[i] = a;
  }
}

// t = V[:, :ncols] y (y on the device)
__global__ void __launch_bounds__(GM_THREADS) k_gm_gemv(const double* __restrict__ V, int64_t ldv, int ncols,
                                                         const double* __restrict__ yv, double* __restrict__ t,
                                                         int64_t n) {
  __shared__ double cf[GM_MAX_RESTART + 1];
  for (int c = threadIdx.x; c < ncols; c += blockDim.x) cf[c] = yv[c];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double a = 0.0;
    for (int c = 0; c < ncols; ++c) a += V[i + (size_t)c * ldv] * cf[c];
    t[i] = a;
  }
}

// Hessenberg column j: h[0..j] = first pass + second pass coefficients,
// h[j+1] = ||w||; one thread
__global__ void k_gm_hcol(double* __restrict__ H, int ldh, int j, const double* __restrict__ c1,
                          const double* __restrict__ c2, const double* __restrict__ nrm) {
  for (int i = 0; i <= j; ++i) H[i + (size_t)j * ldh] = c1[i] + c2[i];
  H[j + 1 + (size_t)j * ldh] = sqrt(nrm[0]);
}

// y = x / s (s = H[j+1, j] on the device); zero when s == 0
__global__ void k_gm_scale(const double* __restrict__ x, const double* __restrict__ s, double* __restrict__ y,
                           int64_t n) {
  double a = *s;
  double inv = a > 0.0 ? 1.0 / a : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = x[i] * inv;
}

// Givens rotations: apply the j earlier ones to column j of H, build the one
// that zeroes H[j+1, j], rotate g; res = |g[j+1]|.  One thread.
__global__ void k_gm_givens(double* __restrict__ H, int ldh, int j, double* __restrict__ cs,
                            double* __restrict__ sn, double* __restrict__ g, double* __restrict__ res) {
  double* h = H + (size_t)j * ldh;
  for (int i = 0; i < j; ++i) {
    double a = h[i], b = h[i + 1];
    h[i] = cs[i] * a + sn[i] * b;
    h[i + 1] = -sn[i] * a + cs[i] * b;
  }
  double a = h[j], b = h[j + 1];
  double r = hypot(a, b);
  double c = r > 0.0 ? a / r : 1.0, s = r > 0.0 ? b / r : 0.0;
  cs[j] = c;
  sn[j] = s;
  h[j] = r;
  h[j + 1] = 0.0;
  double gj = g[j];
  g[j] = c * gj;
  g[j + 1] = -s * gj;
  res[0] = fabs(g[j + 1]);
}

// y = R^-1 g[0..k) with R the rotated Hessenberg (upper triangular); one thread
__global__ void k_gm_trsv(const double* __restrict__ H, int ldh, int k, const double* __restrict__ g,
                          double* __restrict__ y) {
  for (int i = k - 1; i >= 0; --i) {
    double a = g[i];
    for (int c = i + 1; c < k; ++c) a -= H[i + (size_t)c * ldh] * y[c];
    double d = H[i + (size_t)i * ldh];
    y[i] = d != 0.0 ? a / d : 0.0;
  }
}

// g = [beta, 0, ...] from the squared norm
__global__ void k_gm_g0(double* __restrict__ g, int len, const double* __restrict__ nrm2, double* __restrict__ beta) {
  for (int i = 0; i < len; ++i) g[i] = 0.0;
  double b = sqrt(nrm2[0]);
  g[0] = b;
  beta[0] = b;
}

// r = b - y
__global__ void k_gm_resid(const double* __restrict__ b, const double* __restrict__ y, double* __restrict__ r,
                           int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    r[i] = b[i] - y[i];
}

// x += t
__global__ void k_gm_add(double* __restrict__ x, const double* __restrict__ t, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += t[i];
}

}  // namespace

int run_gmres(Handle& h, const double* b, double* x, double rtol, int maxit, int restart, int prec, int* iters,
              double* relres) {
  const int64_t N = h.N;
  const int m = restart;
  cudaStream_t st = h.stream;
  const int grid = (int)std::min<int64_t>((N + GM_THREADS - 1) / GM_THREADS, 8 * (int64_t)h.nsm);
  double* V = (double*)hscratch(h, 300, sizeof(double) * (size_t)N * (m + 1));
  double* H = (double*)hscratch(h, 301, sizeof(double) * (size_t)(m + 1) * m);
  double* sm = (double*)hscratch(h, 302, sizeof(double) * (size_t)(6 * (m + 1) + 8));
  double* t = (double*)hscratch(h, 303, sizeof(double) * (size_t)N);
  double* w = (double*)hscratch(h, 304, sizeof(double) * (size_t)N);
  if (!V || !H || !sm || !t || !w) return HOOM;
  double* c1 = sm;
  double* c2 = sm + (m + 1);
  double* cs = sm + 2 * (m + 1);
  double* sn = sm + 3 * (m + 1);
  double* g = sm + 4 * (m + 1);
  double* y = sm + 5 * (m + 1);
  double* scal = sm + 6 * (m + 1);   // [0] squared norm, [1] beta, [2] residual estimate
  const int ldh = m + 1;

  auto read = [&](const double* p, double* out) -> int {
    AIFMM_CUDA_TRY(h, cudaMemcpyAsync(out, p, sizeof(double), cudaMemcpyDeviceToHost, st));
    AIFMM_CUDA_TRY(h, cudaStreamSynchronize(st));
    return HOK;
  };
  auto norm2 = [&](const double* v, double* out) {
    k_gm_dots<<<1, GM_THREADS, 0, st>>>(v, N, 1, v, N, out); ++h.nlaunch;
  };
  auto precond = [&](double* v) -> int {
    if (!prec) return HOK;
    return run_solve(h, v, 1, N);
  };

  double hb = 0.0;
  norm2(b, scal);
  int e = read(scal, &hb);
  if (e) return e;
  const double bnorm = std::sqrt(hb);
  AIFMM_CUDA_TRY(h, cudaMemsetAsync(x, 0, sizeof(double) * N, st));
  if (bnorm == 0.0) {
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    return HOK;
  }
  int it = 0;
  bool first = true;
  double rel = 1.0;
  while (true) {
    // r = b - A x (x = 0 on the first cycle), V_0 = r / beta
    if (first) {
      AIFMM_CUDA_TRY(h, cudaMemcpyAsync(w, b, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    } else {
      e = run_h2_matvec(h, x, t, 1, N);
      if (e) return e;
      k_gm_resid<<<grid, GM_THREADS, 0, st>>>(b, t, w, N); ++h.nlaunch;
    }
    first = false;
    norm2(w, scal);
    k_gm_g0<<<1, 1, 0, st>>>(g, m + 1, scal, scal + 1); ++h.nlaunch;
    double beta = 0.0;
    e = read(scal + 1, &beta);
    if (e) return e;
    rel = beta / bnorm;
    if (rel <= rtol || it >= maxit) break;
    k_gm_scale<<<grid, GM_THREADS, 0, st>>>(w, scal + 1, V, N); ++h.nlaunch;
    int k = 0;
    for (int j = 0; j < m; ++j) {
      double* vj = V + (size_t)j * N;
      // w = A M^-1 v_j
      AIFMM_CUDA_TRY(h, cudaMemcpyAsync(t, vj, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
      e = precond(t);
      if (e) return e;
      e = run_h2_matvec(h, t, w, 1, N);
      if (e) return e;
      // classical Gram-Schmidt, twice
      k_gm_dots<<<j + 1, GM_THREADS, 0, st>>>(V, N, j + 1, w, N, c1); ++h.nlaunch;
      k_gm_sub<<<grid, GM_THREADS, 0, st>>>(V, N, j + 1, c1, w, N); ++h.nlaunch;
      k_gm_dots<<<j + 1, GM_THREADS, 0, st>>>(V, N, j + 1, w, N, c2); ++h.nlaunch;
      k_gm_sub<<<grid, GM_THREADS, 0, st>>>(V, N, j + 1, c2, w, N); ++h.nlaunch;
      norm2(w, scal);
      k_gm_hcol<<<1, 1, 0, st>>>(H, ldh, j, c1, c2, scal); ++h.nlaunch;
      k_gm_scale<<<grid, GM_THREADS, 0, st>>>(w, H + (j + 1) + (size_t)j * ldh, V + (size_t)(j + 1) * N, N);
      ++h.nlaunch;
      k_gm_givens<<<1, 1, 0, st>>>(H, ldh, j, cs, sn, g, scal + 2); ++h.nlaunch;
      ++it;
      k = j + 1;
      double est = 0.0;
      e = read(scal + 2, &est);
      if (e) return e;
      if (est / bnorm <= rtol || it >= maxit || est == 0.0) break;
    }
    // x += M^-1 V_k y
    k_gm_trsv<<<1, 1, 0, st>>>(H, ldh, k, g, y); ++h.nlaunch;
    k_gm_gemv<<<grid, GM_THREADS, 0, st>>>(V, N, k, y, t, N); ++h.nlaunch;
    e = precond(t);
    if (e) return e;
    k_gm_add<<<grid, GM_THREADS, 0, st>>>(x, t, N); ++h.nlaunch;
  }
  if (iters) *iters = it;
  if (relres) *relres = rel;
  AIFMM_CUDA_TRY(h, cudaGetLastError());
  return rel <= rtol ? HOK : HNOCONV;
}

}  // namespace aifmm
