// Host-side structures of an AIFMM handle and the launchers each
// translation unit provides.  Device memory is owned by the handle.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "common.cuh"

namespace aifmm {

// NNCA operators of one level (Sec. 2.3).
struct NnLevel {
  int l = 0, nb = 0;
  int M = 0;        // capacity of the box row sets ("particles")
  int R = 0;        // rank capacity
  int F = 0;        // far-field (interaction-list points) capacity
  int* m = nullptr;        // [nb] rows of each box
  int* rank = nullptr;     // [nb] NNCA rank
  int* rows = nullptr;     // [nb][M] tree positions of the rows
  int* pivloc = nullptr;   // [nb][R] local row index of each row pivot
  int* pivpos = nullptr;   // [nb][R] tree positions t^{b,i}
  int* far = nullptr;      // [nb][R] tree positions s^{b,i}
  double* U = nullptr;     // [nb][M*R] column-major, ld M
  std::vector<int> h_rank, h_m;
};

// Extended-system blocks of one level during and after factorisation.
// Row types: X (particle equations, m rows), Lc (locals equations, r rows).
// Column types: x (particles, m), y (multipoles, r).
//   XX[p][s5]: (X_p, x_q)   XY[p][s5]: (X_p, y_q)   LX[p][s5]: (Lc_p, x_q)
//   LY[p][s6]: (Lc_p, y_q)  with s5 the 5^d stencil slot of q around p and
//   s6 the slot of q in the 6^d window (children of N(parent(p))).
struct FacLevel {
  int l = 0, nb = 0, n = 0;
  int M = 0, R = 0, Rp = 0, P = 0;  // P = M + R: pivot capacity
  int ns5 = 0, ns6 = 0;
  int* m = nullptr;      // [nb]
  int* r = nullptr;      // [nb] current rank (grows at compression)
  int* xoff = nullptr;   // [nb] offset of y_b inside x_parent
  double* XX = nullptr;
  double* XY = nullptr;
  double* LX = nullptr;
  double* LY = nullptr;
  double* U = nullptr;   // [nb][M*R]
  double* V = nullptr;   // [nb][M*R]
  double* Ud = nullptr;  // [nb][R*Rp]  U^dag: locals of b from locals of parent
  double* Vd = nullptr;  // [nb][R*Rp]  V^dag (V form, r_b x r_parent)
  double* LU = nullptr;  // [nb][P*P] LU of the pivot block, ld P
  int* ipiv = nullptr;   // [nb][P]
  int* pperm = nullptr;  // [nb][P] net row permutation of each pivot LU
  unsigned* flag = nullptr;  // [nb][ns5] bit0: row-X ws fill-in, bit1: Lc ws fill-in
  std::vector<int> h_m, h_r;
  size_t bytes = 0;
};

struct Handle {
  int64_t N = 0;
  int d = 2, L = 0, leaf = 0;
  KParams kp{};
  double tol = 0;
  double ftol = 0;     // compress threshold of the factorisation
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  int nsm = 152;
  int panel_rows = 0;   // tallest LU panel factored in shared memory
  int smem_optin = 48 * 1024;   // dynamic shared memory a kernel may opt in to
  size_t l2_bytes = 0;
  // tree
  double* pts = nullptr;      // SoA [d][N] in tree order
  int* perm = nullptr;        // [N] tree position -> original index
  int* start = nullptr;       // per level l: start[soff[l] + b], b <= nb(l)
  std::vector<int> soff;
  std::vector<int> h_leaf_start;
  double* bbox = nullptr;     // lo[3], side
  // NNCA per level (index l)
  std::vector<NnLevel> nn;
  // factorisation per level
  std::vector<FacLevel> fac;
  double* top = nullptr;      // dense level-1 system LU
  int* top_ipiv = nullptr;
  int* top_perm = nullptr;
  int ntop = 0;
  std::vector<int> top_off;   // offsets of level-2 boxes in the top system
  bool built = false, factored = false;
  // device error word and scratch
  int* derr = nullptr;
  std::vector<void*> allocs;
  std::vector<std::pair<void*, size_t>> scratch;
  size_t resident = 0;
  std::string err;
  double ms_build = 0, ms_factor = 0, ms_solve = 0, ms_matvec = 0;
  double flops_factor = 0;
  int max_rank_nnca = 0, max_rank_factor = 0, max_m = 0;
  // launch count and optional per-kernel-group event timing (profile mode)
  long long nlaunch = 0;
  double* dacc = nullptr;   // device flop accumulator
  bool profile = false;
  bool sym = true;      // A = A^T exploited by the factorisation
  bool fma_gemm = false;   // Schur tiles on FP64 FMAs instead of the tensor-core emulation
  bool tc05 = false;       // Schur tiles on tcgen05 (TMEM accumulators) instead of the warp MMAs
  bool fp32 = false;       // FP32 products in the factorisation (preconditioner)
  bool tf32 = false;       // TF32 tensor-core products in the factorisation (preconditioner)
  // kernel groups of the factorisation timed in profile mode; G_QRCP and
  // G_SCHUR are single kernels (k_cmp_qrcp, k_schur)
  enum { G_COMPRESS = 0, G_PIVLU = 1, G_ZSOLVE = 2, G_SCHUR = 3, G_QRCP = 4, G_NG = 5 };
  double g_ms[G_NG] = {0, 0, 0, 0, 0};
  double g_flops[G_NG] = {0, 0, 0, 0, 0};
  long long g_launch[G_NG] = {0, 0, 0, 0, 0};
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> g_ev;
  Pts P() const {
    Pts p;
    p.x = pts;
    p.y = pts + N;
    p.z = d == 3 ? pts + 2 * N : pts;
    return p;
  }
};

// ---- allocation (api.cu) ----------------------------------------------------
// Device allocation owned by the handle; returns nullptr on failure and
// records the error.
void* halloc(Handle& h, size_t bytes, bool zero = true);
template <class T>
T* hnew(Handle& h, size_t count, bool zero = true) {
  return static_cast<T*>(halloc(h, count * sizeof(T), zero));
}
void hfree_all(Handle& h);
// grow-only scratch buffer number `slot`
void* hscratch(Handle& h, int slot, size_t bytes);

// status helpers
int check_derr(Handle& h);  // reads and clears the device error word

// ---- tree (tree.cu) -----------------------------------------------------------
int build_tree(Handle& h, const double* pts_dev_aos);

// ---- NNCA (nnca.cu) -----------------------------------------------------------
int build_nnca(Handle& h);

// ---- factorisation (factor.cu) ----------------------------------------------
int run_factor(Handle& h);

// ---- solve and products (solve.cu) -----------------------------------------
int run_solve(Handle& h, double* b_dev, int nrhs, int64_t ld);   // in place, original order
int run_h2_matvec(Handle& h, const double* x_dev, double* y_dev, int nrhs, int64_t ld);
int run_direct_matvec(Handle& h, const double* x_dev, double* y_dev, int nrhs, int64_t ld);
// solve with every temporary in a static device array (no allocation)
int run_solve_noalloc(Handle& h, double* b_dev, int nrhs, int64_t ld);
size_t noalloc_scratch_bytes();

// ---- GMRES (gmres.cu) -------------------------------------------------------
// x = A^-1 b by restarted GMRES on the H^2 product, right-preconditioned by
// the factorisation when prec != 0; b, x device N-vectors in original order
int run_gmres(Handle& h, const double* b_dev, double* x_dev, double rtol, int maxit, int restart, int prec,
              int* iters, double* relres);

// error codes returned by the run_* functions (mapped to aifmm_status)
enum HostErr { HOK = 0, HINVALID = 1, HOOM = 2, HSINGULAR = 3, HSTATE = 4, HNOCONV = 5, HCUDA = 6, HCAPACITY = 8 };

#define AIFMM_CUDA_TRY(h, expr)                                       \
  do {                                                                \
    cudaError_t _e = (expr);                                          \
    if (_e != cudaSuccess) {                                          \
      (h).err = std::string(#expr) + ": " + cudaGetErrorString(_e);   \
      return HCUDA;                                                   \
    }                                                                 \
  } while (0)

}  // namespace aifmm
