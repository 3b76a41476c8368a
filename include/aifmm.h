/*
 * aifmm.h -- C ABI of the GB300 (sm_103a) AIFMM factorisation and solve.
 *
 * The library solves A x = b for a dense N-body interaction matrix A
 * (A_ij = kernel(u_i, v_j), sources = targets) with the Algebraic Inverse
 * Fast Multipole Method of Gujjula & Ambikasaran (arXiv 2301.12704):
 *   build  -- uniform 2^d tree and interaction lists (Sec. 2.1-2.2), NNCA
 *             operators (Sec. 2.3), extended sparse system (Sec. 3.1);
 *   factor -- level-by-level elimination with fill-ins updated first and
 *             compressed/redirected once (Algorithm 2, Sec. 3.2-3.5);
 *   solve  -- right-hand-side Schur operations, top solve, back
 *             substitution (Algorithm 3, Sec. 3.6).
 * Every numerical step runs in CUDA kernels on the current device; the host
 * only sequences launches and reads back a few rank counts per level.
 *
 * Conventions for every entry point
 *   Pointers: a "buffer" argument may point to host or device memory; the
 *     library detects which (cudaPointerGetAttributes) and copies host data
 *     through pinned staging on the handle's stream.  Device buffers must be
 *     on the handle's device (INVALID otherwise).
 *   Device: the handle belongs to the device current at aifmm_build; every
 *     later call makes that device current for its duration and restores the
 *     caller's current device on return.
 *   Streams: work runs on the handle's stream (aifmm_options.stream, or a
 *     non-blocking stream the library creates).  The library does not order
 *     itself after other streams: device buffers must be ready when a call
 *     starts.
 *   Layout: points are row-major N x dim (point-major); right-hand sides and
 *     solutions are column-major N x nrhs with leading dimension ld >= N, in
 *     the caller's original point order.
 *   Ownership: build copies the points; the caller keeps ownership of every
 *     buffer it passes.  The handle owns all device memory it allocates until
 *     aifmm_destroy.
 *   Errors: every call returns an aifmm_status; nothing aborts, traps or
 *     throws across the ABI.  aifmm_last_error(h) gives a message.  Device
 *     kernels report errors through a status word that the host reads after
 *     the call's work completes (calls are synchronous on return).
 *   Threads: one handle is used by one host thread at a time.
 */
#ifndef AIFMM_H
#define AIFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct aifmm_ctx* aifmm_h;

typedef enum {
  AIFMM_OK = 0,
  AIFMM_ERR_INVALID = 1,   /* bad argument: n < 1, dim not 2/3, tol < 0, leaf < 1,
                              duplicate points, null pointer, nrhs < 1, ld < n */
  AIFMM_ERR_OOM = 2,       /* device allocation failed */
  AIFMM_ERR_SINGULAR = 3,  /* a pivot block was numerically singular */
  AIFMM_ERR_STATE = 4,     /* e.g. solve before factor */
  AIFMM_ERR_NOCONV = 5,    /* iterative solve did not converge */
  AIFMM_ERR_CUDA = 6,      /* a CUDA runtime call failed */
  AIFMM_ERR_TIMEOUT = 7,   /* a bounded device wait ran out */
  AIFMM_ERR_CAPACITY = 8   /* a size exceeded a compiled-in capacity */
} aifmm_status;

/* Kernels (Sec. 4): off-diagonal entries as a function of r = |x_i - x_j|.
 *   LOG2D  log r               (Experiment 4 kernel), dim 2
 *   INVR3D 1/r                 dim 3
 *   INVR2D 1/r                 (Experiment 3 kernel), dim 2
 *   GAUSS  exp(-r^2/length^2)  dim 2 or 3
 * The diagonal A_ii is `diag`. */
typedef enum { AIFMM_K_LOG2D = 0, AIFMM_K_INVR3D = 1, AIFMM_K_INVR2D = 2, AIFMM_K_GAUSS = 3 } aifmm_kernel_kind;

typedef struct {
  int kind;        /* aifmm_kernel_kind */
  int dim;         /* 2 or 3 */
  double diag;     /* A_ii; NaN: kernel(0) + nugget (GAUSS only: 1 + nugget;
                      INVALID for the kernels that are infinite at r = 0) */
  double length;   /* Gaussian length scale (GAUSS only) */
  double nugget;   /* added to kernel(0) when diag is NaN (a Gaussian-process
                      noise variance); finite; ignored otherwise */
} aifmm_kernel;

typedef struct {
  int order;       /* 0: distance-2 colour order (default), only value supported */
  int depth;       /* 0: depth from the average-occupancy rule; >= 2: force depth L */
  void* stream;    /* cudaStream_t to run on; NULL = the library's own stream */
  int profile;     /* 1: time the factorisation's kernel groups with CUDA events
                      on the handle's stream (reported by aifmm_stats) */
  int no_symmetry; /* 0 (default): use A = A^T (every built-in kernel is symmetric
                      and sources = targets, so V = U, Sec. 2.3): one RRQR per box
                      gives both bases and the Schur update computes each pair of
                      mirrored blocks once; 1: the general elimination, which
                      compresses rows and columns separately and updates every block */
  double factor_tol; /* > 0: RRQR threshold of the compress-and-redirect steps, in
                      place of tol (the NNCA operators and aifmm_matvec keep tol);
                      a looser value gives the low-accuracy factorisation used as a
                      GMRES preconditioner (Sec. 4, Experiment 5). 0: tol */
  int fma_gemm;    /* 0 (default): the factorisation's tile products -- Schur update,
                      compress fills and projections (7 digits), Z = Piv^-1 B and the
                      pivot LU's trailing updates (8 digits, balanced) -- run on the
                      BF16 tensor cores in FP64 precision (exact 7-bit integer digits,
                      see aifmm_kernels.h); 1: all of them on FP64 FMAs */
  int tcgen05;     /* 1: the Schur-update tiles issue the same digit products on the
                      5th-generation tensor cores (tcgen05.mma, accumulators in tensor
                      memory; aifmm_dgemm_tc05) instead of warp MMAs; same accuracy,
                      slower on the short tiles of these factorisations.  0 (default) */
  int precision;   /* 0 (default): FP64 arithmetic throughout.  1: the tile products of
                      the factorisation (Schur update, Z = Piv^-1 B, the pivot LU's
                      trailing updates, the compress fills and projections) in FP32
                      with FP32 sums, operands and results kept in FP64; the pivoted
                      QR that fixes the compression ranks, the panels and the
                      triangular blocks stay FP64.  A factorisation for preconditioning
                      aifmm_gmres (Sec. 4, AIFMM as a preconditioner); aifmm_solve with
                      it has a relative error of about 1e-6.  2: the same products
                      on the tensor cores in TF32 (10-bit mantissa operands) with FP32
                      accumulation (mma.sync m16n8k8 tiles; FP32 FMAs for products
                      of at most 8 columns); relative error of a solve about 1e-3,
                      a preconditioner only; its compress threshold (factor_tol)
                      must sit above TF32 rounding, ~1e-3 */
  double eta;      /* admissibility parameter of Sec. 2.2 (max diameter <= eta x
                      distance): 0 (default) or any eta >= sqrt(dim), which all give
                      the same lists for the boxes of a uniform tree (neighbours =
                      touching boxes); eta < sqrt(dim) is INVALID (it would need a
                      near field wider than the touching boxes) */
} aifmm_options;

/* Per-handle statistics (aifmm_stats). Times are CUDA-event milliseconds of
 * the last call of each kind. */
typedef struct {
  int64_t n;
  int dim;
  int levels;               /* L */
  int max_rank_nnca;        /* max NNCA rank over levels 2..L */
  int max_rank_factor;      /* r_m: max rank after compress and redirect */
  int max_m;                /* largest pivot x-size over all levels */
  int top_size;             /* size of the dense level-1 system */
  double flops_factor;      /* algorithmic FP64 flops of the last factor */
  double bytes_solve;       /* algorithmic bytes of one solve with nrhs = 1 (after factor):
                               the factor entries both sweeps read once each -- the pivot
                               LUs twice, the coupled blocks of every pivot's rows and
                               columns once, the top LU twice; 0 before factor */
  double bytes_resident;    /* device bytes held by the handle */
  double ms_build, ms_factor, ms_solve, ms_matvec;
  int64_t kernel_launches;  /* kernels launched by the handle so far */
  /* profile mode: CUDA-event time, algorithmic FP64 flops and launches of the
     factorisation's kernel groups, summed over the last aifmm_factor:
     [0] compress and redirect except the pivoted QR, [1] pivot LU,
     [2] Z = Piv^-1 B, [3] Schur update (the one kernel k_schur),
     [4] the pivoted QR of the compression (the one kernel k_cmp_qrcp);
     [5..7] zero */
  double group_ms[8];
  double group_flops[8];
  int64_t group_launches[8];
} aifmm_stats_t;

/* Build the tree, interaction lists, NNCA operators and extended system.
 *   points    N x dim row-major (host or device), copied.
 *   n         number of points N >= 1.
 *   k         kernel description (dim must be 2 or 3).
 *   tol       eps_A >= 0, shared by NNCA and RRQR (Sec. 4, notation table).
 *   leaf_size n_max >= 1, target points per leaf box (the depth rule of Sec. 2.1).
 *   opt       may be NULL (defaults).
 *   out       receives the new handle (NULL on failure).
 * Errors: INVALID, OOM, CUDA, CAPACITY. */
aifmm_status aifmm_build(const double* points, int64_t n, const aifmm_kernel* k, double tol,
                         int leaf_size, const aifmm_options* opt, aifmm_h* out);

/* Algorithm 2: eliminate levels L..2 (distance-2 colour batches), compress
 * and redirect pending well-separated fill-ins once per box, factor the top
 * dense level-1 system.  Independent of any right-hand side (Remark, Sec. 3.6).
 * Errors: STATE (no build), SINGULAR, OOM, CUDA, CAPACITY. */
aifmm_status aifmm_factor(aifmm_h h);

/* Algorithm 3: x = A^-1 rhs through the factorisation.
 *   rhs, x    N x nrhs column-major, leading dimension ld (host or device;
 *             may alias).  Original point order.
 * Errors: STATE (no factor), INVALID, OOM, CUDA. */
aifmm_status aifmm_solve(aifmm_h h, const double* rhs, double* x, int nrhs, int64_t ld);

/* Solve without allocating: the same result as aifmm_solve, for callers that
 * must not call cudaMalloc once their factorisation is resident -- e.g. a
 * request loop serving solves from a thread that runs under a strict
 * allocation budget or alongside code that forbids allocation.  The paper
 * has no counterpart to this call.
 *   rhs, x    DEVICE pointers only (host staging would need an allocation),
 *             N x nrhs column-major, leading dimension ld; may alias.
 * Temporaries live in one static device array of
 * aifmm_noalloc_scratch_bytes() bytes (64 MiB) that every GPU which loads
 * the library holds until the process exits.  The first call on a device
 * looks up that array's device address; make it before any stream capture.
 * The array is shared by all calls and keeps the last call's contents: calls
 * whose work overlaps on the GPU (other streams, other threads) race on it.
 * The call runs with the handle's device current (as every call here does).
 * Errors: STATE (no factor), INVALID (host pointers, nrhs < 1, ld < N),
 * CAPACITY (the problem and nrhs need more than the static array), CUDA. */
aifmm_status aifmm_solve_noalloc(aifmm_h h, const double* rhs, double* x, int nrhs, int64_t ld);

/* Size in bytes of the static array used by aifmm_solve_noalloc. */
int64_t aifmm_noalloc_scratch_bytes(void);

/* y = A_H2 x with the NNCA H^2 representation built by aifmm_build
 * (upward P2M/M2M, M2L, downward L2L/L2P, near-field P2P).
 * Errors: STATE, INVALID, OOM, CUDA. */
aifmm_status aifmm_matvec(aifmm_h h, const double* x, double* y, int nrhs, int64_t ld);

/* y = A x with every entry of A evaluated (exact O(N^2) direct sum on the
 * GPU); used to measure true residuals. Errors: STATE, INVALID, OOM, CUDA. */
aifmm_status aifmm_direct_matvec(aifmm_h h, const double* x, double* y, int nrhs, int64_t ld);

/* Restarted GMRES (Sec. 4: the iterative solver of Experiments 2-4, with the
 * NNCA H^2 product; Experiment 5: a low-accuracy AIFMM factorisation as the
 * preconditioner).  Solves A_H2 x = b with right preconditioning M^-1 = the
 * AIFMM solve (Algorithm 3) when use_precond != 0, none otherwise; starts
 * from x = 0; stops when ||b - A_H2 x|| / ||b|| <= rtol (the residual is
 * recomputed with a product after each restart cycle) or after maxit
 * iterations.  Arnoldi uses classical Gram-Schmidt applied twice.
 *   b, x      N-vectors (host or device), original order; x is output only.
 *   rtol      >= 0; maxit >= 1 total iterations (products); 1 <= restart <= 512.
 *   iters     (may be NULL) iterations done; relres (may be NULL) the final
 *             relative residual of the H^2 system.
 * Device memory: N * (restart + 3) doubles of handle scratch.
 * Errors: STATE (no build, or use_precond without factor), INVALID, NOCONV
 * (x and relres hold the last iterate), OOM, CUDA. */
aifmm_status aifmm_gmres(aifmm_h h, const double* b, double* x, double rtol, int maxit, int restart,
                         int use_precond, int* iters, double* relres);

/* Statistics of the handle. */
aifmm_status aifmm_stats(aifmm_h h, aifmm_stats_t* out);

/* Introspection for parity checks (host buffers only).
 *   aifmm_tree_perm: perm[k] = original index of the k-th point in tree order
 *     (N entries); level_start (may be NULL) receives the leaf-box starts
 *     (2^(dim*L) + 1 entries).
 *   aifmm_level_ranks: for level l in [2, L], NNCA ranks (which = 0) or
 *     ranks after factorisation (which = 1) of the 2^(dim*l) boxes.
 *   aifmm_level_pivots: for level l, the incoming row pivots t^{b,i} of
 *     every box as tree positions, concatenated in box order (sum of NNCA
 *     ranks entries), each box's in the order the pivot search took them.
 *   aifmm_level_far_pivots: the same for the far-field pivots s^{b,i}
 *     (Sec. 2.3, eq. NCA; points of the interaction-list boxes). */
aifmm_status aifmm_tree_perm(aifmm_h h, int64_t* perm, int64_t* level_start);
aifmm_status aifmm_level_ranks(aifmm_h h, int level, int which, int* ranks);
aifmm_status aifmm_level_pivots(aifmm_h h, int level, int64_t* pivots);
aifmm_status aifmm_level_far_pivots(aifmm_h h, int level, int64_t* pivots);

/* Depth L of the handle's tree (0 if h is NULL). */
int aifmm_levels(aifmm_h h);

/* CUDA device index the handle belongs to (the device current at
 * aifmm_build); -1 if h is NULL. */
int aifmm_device(aifmm_h h);

/* Move the handle's later work to a new CUDA stream, created by the library
 * with stream priority `priority` (lower numbers run first; CUDA clamps the
 * value into the device's range, so a large negative value asks for the
 * highest priority).  The handle's current stream is synchronised first, so
 * the caller needs no ordering between the two; a stream the library had
 * created is destroyed, a stream passed in aifmm_options.stream is left to
 * its owner.  For a request loop: factorisations run on default-priority
 * streams (the lowest) and solves against finished factorisations on
 * high-priority ones, so that solve kernels are scheduled ahead of pending
 * factorisation kernels of other handles.  The paper has no counterpart to
 * this call.  INVALID if h is NULL, CUDA if the stream cannot be created (the
 * handle keeps its stream). */
aifmm_status aifmm_set_priority(aifmm_h h, int priority);

/* Message of the last error on h (or of the last failed aifmm_build when h is
 * NULL).  Valid until the next call on the handle. */
const char* aifmm_last_error(aifmm_h h);

/* Free every device and host resource of h. NULL is a no-op. */
void aifmm_destroy(aifmm_h h);

#ifdef __cplusplus
}
#endif
#endif /* AIFMM_H */
