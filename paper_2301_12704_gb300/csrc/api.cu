// C ABI of the library (include/aifmm.h): argument checks, device memory of
// the handle, host/device pointer handling, timing, and the calls into the
// tree, NNCA, factorisation and solve launchers.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <cstdint>
#include <initializer_list>
#include <mutex>
#include <string>

#include "../../include/aifmm.h"
#include "internal.h"

using namespace aifmm;

struct aifmm_ctx {
  Handle h;
};

static std::string g_build_err;

namespace aifmm {

// optional fault injection for tests of the out-of-memory path: the k-th
// device allocation of a handle fails when AIFMM_FAIL_ALLOC_AT=k is set.
static long fail_at() {
  const char* s = std::getenv("AIFMM_FAIL_ALLOC_AT");
  return s ? std::atol(s) : 0;
}

// The library's device memory comes from one stream-ordered pool per GPU
// that keeps freed blocks for later handles (release threshold: unlimited):
// allocations and frees never synchronise the device, so handles driven from
// several host threads (many problems, the serving loop) do not stall each
// other, and a new handle reuses the blocks of destroyed ones instead of
// asking the CUDA driver again.  The pool's memory returns to the CUDA
// driver at process exit.
static cudaMemPool_t lib_pool(int dev) {
  static cudaMemPool_t pools[64] = {};
  static std::mutex mu;
  if (dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> g(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[dev] = p;
  }
  return pools[dev];
}

static cudaError_t dev_alloc(Handle& h, void** p, size_t bytes) {
  cudaMemPool_t pool = lib_pool(h.device);
  return pool ? cudaMallocFromPoolAsync(p, bytes, pool, h.stream) : cudaMallocAsync(p, bytes, h.stream);
}

void* halloc(Handle& h, size_t bytes, bool zero) {
  static thread_local long counter = 0;
  long f = fail_at();
  if (f > 0 && ++counter == f) {
    h.err = "device allocation failed (injected)";
    return nullptr;
  }
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (dev_alloc(h, &p, bytes) != cudaSuccess) {
    cudaGetLastError();
    h.err = "cudaMallocAsync of " + std::to_string(bytes) + " bytes failed";
    return nullptr;
  }
  if (zero && cudaMemsetAsync(p, 0, bytes, h.stream) != cudaSuccess) {
    cudaFreeAsync(p, h.stream);
    h.err = "cudaMemsetAsync failed";
    return nullptr;
  }
  h.allocs.push_back(p);
  h.resident += bytes;
  return p;
}

void* hscratch(Handle& h, int slot, size_t bytes) {
  if ((int)h.scratch.size() <= slot) h.scratch.resize(slot + 1, {nullptr, 0});
  auto& s = h.scratch[slot];
  if (s.second >= bytes && s.first) return s.first;
  if (s.first) {
    // the kernels that used the old buffer were issued on h.stream before
    // this free, so it is ordered after them
    cudaFreeAsync(s.first, h.stream);
    h.resident -= s.second;
    s.first = nullptr;
    s.second = 0;
  }
  void* p = nullptr;
  size_t b = bytes < 16 ? 16 : bytes;
  if (dev_alloc(h, &p, b) != cudaSuccess) {
    cudaGetLastError();
    h.err = "cudaMallocAsync of scratch (" + std::to_string(b) + " bytes) failed";
    return nullptr;
  }
  s.first = p;
  s.second = b;
  h.resident += b;
  return p;
}

void hfree_all(Handle& h) {
  for (void* p : h.allocs) cudaFreeAsync(p, h.stream);
  h.allocs.clear();
  for (auto& s : h.scratch)
    if (s.first) cudaFreeAsync(s.first, h.stream);
  h.scratch.clear();
  h.resident = 0;
  if (h.stream) cudaStreamSynchronize(h.stream);
}

int check_derr(Handle& h) {
  int v = 0;
  cudaMemcpy(&v, h.derr, sizeof(int), cudaMemcpyDeviceToHost);
  if (v) cudaMemset(h.derr, 0, sizeof(int));
  return v;
}

}  // namespace aifmm

static aifmm_status to_status(int e) {
  switch (e) {
    case HOK: return AIFMM_OK;
    case HINVALID: return AIFMM_ERR_INVALID;
    case HOOM: return AIFMM_ERR_OOM;
    case HSINGULAR: return AIFMM_ERR_SINGULAR;
    case HSTATE: return AIFMM_ERR_STATE;
    case HNOCONV: return AIFMM_ERR_NOCONV;
    case HCAPACITY: return AIFMM_ERR_CAPACITY;
    default: return AIFMM_ERR_CUDA;
  }
}

// Where a buffer lives: host memory (pageable or pinned), device memory of
// the handle's GPU (or managed memory), or device memory of another GPU,
// which no call accepts.
enum PtrKind { P_HOST = 0, P_DEVICE = 1, P_OTHER_DEVICE = 2 };

static int ptr_kind(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return P_HOST;
  }
  if (a.type == cudaMemoryTypeDevice) return a.device == dev ? P_DEVICE : P_OTHER_DEVICE;
  if (a.type == cudaMemoryTypeManaged) return P_DEVICE;
  return P_HOST;
}

static bool is_device_ptr(const void* p, int dev) { return ptr_kind(p, dev) == P_DEVICE; }

// true if any of the buffers is device memory of another GPU (message set)
static bool foreign(Handle& h, std::initializer_list<const void*> ps) {
  for (const void* p : ps)
    if (p && ptr_kind(p, h.device) == P_OTHER_DEVICE) {
      h.err = "a buffer is device memory of another GPU than the handle's (device " + std::to_string(h.device) + ")";
      return true;
    }
  return false;
}

// Every call on a handle runs with the handle's device current and restores
// the caller's current device on return, so a call made from a thread whose
// current device is another GPU still launches, allocates and looks up
// device symbols on the handle's GPU.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      cudaGetLastError();
      prev = -1;
      ok = false;
      return;
    }
    if (prev != dev) {
      if (cudaSetDevice(dev) != cudaSuccess) {
        cudaGetLastError();
        ok = false;
      }
    } else {
      prev = -1;   // nothing to restore
    }
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;
};

#define AIFMM_ON_DEVICE(h)                                              \
  DeviceGuard _dg((h).device);                                          \
  if (!_dg.ok) {                                                        \
    (h).err = "cannot make device " + std::to_string((h).device) + " current"; \
    return AIFMM_ERR_CUDA;                                              \
  }

struct Timer {
  cudaEvent_t a, b;
  cudaStream_t s;
  explicit Timer(cudaStream_t st) : s(st) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s);
  }
  double stop() {
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms;
  }
};

extern "C" {

aifmm_status aifmm_build(const double* points, int64_t n, const aifmm_kernel* k, double tol, int leaf_size,
                         const aifmm_options* opt, aifmm_h* out) {
  if (out) *out = nullptr;
  g_build_err.clear();
  if (!points || !k || !out || n < 1 || n > (int64_t)1 << 30 || (k->dim != 2 && k->dim != 3) ||
      !(tol >= 0.0) || leaf_size < 1 || k->kind < 0 || k->kind > 3 || std::isinf(k->diag) ||
      !std::isfinite(k->nugget) || (k->kind == AIFMM_K_GAUSS && !(k->length > 0.0)) ||
      (opt && opt->order != 0) || (opt && opt->depth != 0 && (opt->depth < 2 || opt->depth > 12)) ||
      (opt && !(opt->factor_tol >= 0.0 && std::isfinite(opt->factor_tol))) ||
      (opt && (opt->precision < 0 || opt->precision > 2)) || (opt && !(opt->eta >= 0.0))) {
    g_build_err = "invalid argument";
    return AIFMM_ERR_INVALID;
  }
  // A_ii: diag, or kernel(0) + nugget when diag is NaN (finite only for the
  // Gaussian, whose value at r = 0 is 1)
  double diag = k->diag;
  if (std::isnan(diag)) {
    if (k->kind != AIFMM_K_GAUSS) {
      g_build_err = "invalid argument: diag = NaN asks for kernel(0) + nugget, infinite for this kernel";
      return AIFMM_ERR_INVALID;
    }
    diag = 1.0 + k->nugget;
  }
  // admissibility max(diam X, diam Y) <= eta dist(X, Y) (Sec. 2.2): for
  // boxes of one level, touching boxes are never admissible and boxes one
  // box apart are admissible exactly when eta >= sqrt(d), so every
  // eta >= sqrt(d) gives the lists built here; a smaller eta needs a wider
  // near field, which the library does not build
  if (opt && opt->eta != 0.0 && opt->eta < std::sqrt((double)k->dim) * (1.0 - 1e-12)) {
    g_build_err = "invalid argument: eta below sqrt(dim) needs a near field wider than the neighbouring boxes";
    return AIFMM_ERR_INVALID;
  }
  aifmm_ctx* c = new aifmm_ctx();
  Handle& h = c->h;
  cudaGetDevice(&h.device);
  h.N = n;
  h.d = k->dim;
  h.tol = tol;
  h.ftol = (opt && opt->factor_tol > 0.0) ? opt->factor_tol : tol;
  h.leaf = leaf_size;
  h.kp.kind = k->kind;
  h.kp.dim = k->dim;
  h.kp.diag = diag;
  h.kp.inv_len2 = k->kind == AIFMM_K_GAUSS ? 1.0 / (k->length * k->length) : 0.0;
  h.profile = opt && opt->profile;
  h.sym = !(opt && opt->no_symmetry);
  h.fma_gemm = opt && opt->fma_gemm;
  h.tc05 = opt && opt->tcgen05;
  h.fp32 = opt && opt->precision == 1;
  h.tf32 = opt && opt->precision == 2;
  if (opt && opt->stream) {
    h.stream = (cudaStream_t)opt->stream;
  } else {
    if (cudaStreamCreateWithFlags(&h.stream, cudaStreamNonBlocking) != cudaSuccess) {
      g_build_err = "cudaStreamCreate failed";
      delete c;
      return AIFMM_ERR_CUDA;
    }
    h.own_stream = true;
  }
  // depth: average-occupancy rule L = max(2, min l with (2^d)^l * n_max >= N)
  int L = 2;
  while (((int64_t)1 << (h.d * L)) * leaf_size < n) ++L;
  if (opt && opt->depth) L = opt->depth;
  h.L = L;
  if (h.d * L > 30) {
    g_build_err = "tree too deep";
    aifmm_destroy(c);
    return AIFMM_ERR_CAPACITY;
  }
  Timer tm(h.stream);
  int e = HOK;
  h.derr = hnew<int>(h, 1);
  if (!h.derr) e = HOOM;
  const double* pdev = points;
  const int pk = ptr_kind(points, h.device);
  if (!e && pk == P_OTHER_DEVICE) {
    h.err = "points are device memory of another GPU than the current one";
    e = HINVALID;
  }
  if (!e && pk == P_HOST) {
    double* tmp = hnew<double>(h, (size_t)n * h.d, false);
    if (!tmp) e = HOOM;
    else if (cudaMemcpyAsync(tmp, points, sizeof(double) * n * h.d, cudaMemcpyHostToDevice, h.stream) != cudaSuccess)
      e = HCUDA;
    pdev = tmp;
  }
  if (!e) e = build_tree(h, pdev);
  if (!e) e = build_nnca(h);
  if (!e) {
    cudaError_t ce = cudaStreamSynchronize(h.stream);
    if (ce != cudaSuccess) {
      h.err = cudaGetErrorString(ce);
      e = HCUDA;
    }
  }
  h.ms_build = tm.stop();
  if (e) {
    g_build_err = h.err.empty() ? "build failed" : h.err;
    aifmm_destroy(c);
    return to_status(e);
  }
  h.built = true;
  *out = c;
  return AIFMM_OK;
}

aifmm_status aifmm_factor(aifmm_h c) {
  if (!c) return AIFMM_ERR_INVALID;
  Handle& h = c->h;
  if (!h.built) {
    h.err = "factor before build";
    return AIFMM_ERR_STATE;
  }
  if (h.factored) {
    // refactor from scratch: drop the previous factor storage
    h.err = "handle already factored";
    return AIFMM_ERR_STATE;
  }
  AIFMM_ON_DEVICE(h);
  Timer tm(h.stream);
  int e = run_factor(h);
  if (!e) {
    cudaError_t ce = cudaStreamSynchronize(h.stream);
    if (ce != cudaSuccess) {
      h.err = cudaGetErrorString(ce);
      e = HCUDA;
    }
  }
  h.ms_factor = tm.stop();
  if (e) return to_status(e);
  h.factored = true;
  return AIFMM_OK;
}

// copy a column-major N x nrhs (ld) operand into the device buffer dst (ld)
static int stage_in(Handle& h, const double* src, double* dst, int nrhs, int64_t ld) {
  cudaMemcpyKind kind = is_device_ptr(src, h.device) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (src == dst) return HOK;
  AIFMM_CUDA_TRY(h, cudaMemcpy2DAsync(dst, ld * sizeof(double), src, ld * sizeof(double), h.N * sizeof(double),
                                      nrhs, kind, h.stream));
  return HOK;
}

aifmm_status aifmm_solve(aifmm_h c, const double* rhs, double* x, int nrhs, int64_t ld) {
  if (!c) return AIFMM_ERR_INVALID;
  Handle& h = c->h;
  if (!h.factored) {
    h.err = "solve before factor";
    return AIFMM_ERR_STATE;
  }
  if (!rhs || !x || nrhs < 1 || ld < h.N) {
    h.err = "invalid argument";
    return AIFMM_ERR_INVALID;
  }
  if (foreign(h, {rhs, x})) return AIFMM_ERR_INVALID;
  AIFMM_ON_DEVICE(h);
  Timer tm(h.stream);
  bool xdev = is_device_ptr(x, h.device);
  double* work = xdev ? x : (double*)hscratch(h, 90, sizeof(double) * ld * nrhs);
  if (!work) return AIFMM_ERR_OOM;
  int e = stage_in(h, rhs, work, nrhs, ld);
  if (!e) e = run_solve(h, work, nrhs, ld);
  if (!e && !xdev) {
    if (cudaMemcpy2DAsync(x, ld * sizeof(double), work, ld * sizeof(double), h.N * sizeof(double), nrhs,
                          cudaMemcpyDeviceToHost, h.stream) != cudaSuccess)
      e = HCUDA;
  }
  if (!e && cudaStreamSynchronize(h.stream) != cudaSuccess) {
    h.err = "solve: CUDA error";
    e = HCUDA;
  }
  h.ms_solve = tm.stop();
  if (!e) {
    int de = check_derr(h);
    if (de) {
      h.err = "solve: device error " + std::to_string(de);
      e = HCAPACITY;
    }
  }
  return to_status(e);
}

aifmm_status aifmm_solve_noalloc(aifmm_h c, const double* rhs, double* x, int nrhs, int64_t ld) {
  if (!c) return AIFMM_ERR_INVALID;
  Handle& h = c->h;
  if (!h.factored) {
    h.err = "solve before factor";
    return AIFMM_ERR_STATE;
  }
  if (!rhs || !x || nrhs < 1 || ld < h.N) {
    h.err = "invalid argument";
    return AIFMM_ERR_INVALID;
  }
  if (!is_device_ptr(rhs, h.device) || !is_device_ptr(x, h.device)) {
    h.err = "aifmm_solve_noalloc: rhs and x must be device pointers on the handle's GPU (host staging would "
            "allocate)";
    return AIFMM_ERR_INVALID;
  }
  AIFMM_ON_DEVICE(h);
  int e = HOK;
  if (rhs != x && cudaMemcpy2DAsync(x, ld * sizeof(double), rhs, ld * sizeof(double), h.N * sizeof(double), nrhs,
                                    cudaMemcpyDeviceToDevice, h.stream) != cudaSuccess) {
    h.err = "aifmm_solve_noalloc: copy of rhs failed";
    e = HCUDA;
  }
  if (!e) e = run_solve_noalloc(h, x, nrhs, ld);
  if (!e && cudaStreamSynchronize(h.stream) != cudaSuccess) {
    h.err = "aifmm_solve_noalloc: CUDA error";
    e = HCUDA;
  }
  if (!e) {
    int de = check_derr(h);
    if (de) {
      h.err = "aifmm_solve_noalloc: device error " + std::to_string(de);
      e = HCAPACITY;
    }
  }
  return to_status(e);
}

int64_t aifmm_noalloc_scratch_bytes(void) { return (int64_t)noalloc_scratch_bytes(); }

static aifmm_status product(aifmm_h c, const double* x, double* y, int nrhs, int64_t ld, bool direct) {
  if (!c) return AIFMM_ERR_INVALID;
  Handle& h = c->h;
  if (!h.built) {
    h.err = "matvec before build";
    return AIFMM_ERR_STATE;
  }
  if (!x || !y || nrhs < 1 || ld < h.N) {
    h.err = "invalid argument";
    return AIFMM_ERR_INVALID;
  }
  if (foreign(h, {x, y})) return AIFMM_ERR_INVALID;
  AIFMM_ON_DEVICE(h);
  Timer tm(h.stream);
  bool xdev = is_device_ptr(x, h.device), ydev = is_device_ptr(y, h.device);
  const double* xin = x;
  int e = HOK;
  if (!xdev) {
    double* t = (double*)hscratch(h, 91, sizeof(double) * ld * nrhs);
    if (!t) return AIFMM_ERR_OOM;
    e = stage_in(h, x, t, nrhs, ld);
    xin = t;
  }
  double* yout = ydev ? y : (double*)hscratch(h, 92, sizeof(double) * ld * nrhs);
  if (!yout) return AIFMM_ERR_OOM;
  if (!e) e = direct ? run_direct_matvec(h, xin, yout, nrhs, ld) : run_h2_matvec(h, xin, yout, nrhs, ld);
  if (!e && !ydev) {
    if (cudaMemcpy2DAsync(y, ld * sizeof(double), yout, ld * sizeof(double), h.N * sizeof(double), nrhs,
                          cudaMemcpyDeviceToHost, h.stream) != cudaSuccess)
      e = HCUDA;
  }
  if (!e && cudaStreamSynchronize(h.stream) != cudaSuccess) e = HCUDA;
  h.ms_matvec = tm.stop();
  return to_status(e);
}

aifmm_status aifmm_matvec(aifmm_h c, const double* x, double* y, int nrhs, int64_t ld) {
  return product(c, x, y, nrhs, ld, false);
}

aifmm_status aifmm_direct_matvec(aifmm_h c, const double* x, double* y, int nrhs, int64_t ld) {
  return product(c, x, y, nrhs, ld, true);
}

aifmm_status aifmm_gmres(aifmm_h c, const double* b, double* x, double rtol, int maxit, int restart,
                         int use_precond, int* iters, double* relres) {
  if (!c) return AIFMM_ERR_INVALID;
  Handle& h = c->h;
  if (iters) *iters = 0;
  if (relres) *relres = 0.0;
  if (!h.built || (use_precond && !h.factored)) {
    h.err = use_precond ? "gmres with the preconditioner before factor" : "gmres before build";
    return AIFMM_ERR_STATE;
  }
  if (!b || !x || !(rtol >= 0.0) || maxit < 1 || restart < 1 || restart > 512) {
    h.err = "invalid argument (rtol >= 0, maxit >= 1, 1 <= restart <= 512)";
    return AIFMM_ERR_INVALID;
  }
  if (foreign(h, {b, x})) return AIFMM_ERR_INVALID;
  AIFMM_ON_DEVICE(h);
  Timer tm(h.stream);
  bool xdev = is_device_ptr(x, h.device);
  double* bin = (double*)hscratch(h, 93, sizeof(double) * h.N);
  double* xout = xdev ? x : (double*)hscratch(h, 94, sizeof(double) * h.N);
  if (!bin || !xout) return AIFMM_ERR_OOM;
  int e = stage_in(h, b, bin, 1, h.N);
  if (!e) e = run_gmres(h, bin, xout, rtol, maxit, restart, use_precond ? 1 : 0, iters, relres);
  if ((!e || e == HNOCONV) && !xdev) {
    if (cudaMemcpyAsync(x, xout, sizeof(double) * h.N, cudaMemcpyDeviceToHost, h.stream) != cudaSuccess) e = HCUDA;
  }
  if (cudaStreamSynchronize(h.stream) != cudaSuccess && !e) e = HCUDA;
  h.ms_solve = tm.stop();
  if (e == HNOCONV) h.err = "gmres: relative residual above rtol after maxit iterations";
  if (!e || e == HNOCONV) {
    int de = check_derr(h);
    if (de) {
      h.err = "gmres: device error " + std::to_string(de);
      e = HCAPACITY;
    }
  }
  return to_status(e);
}

aifmm_status aifmm_stats(aifmm_h c, aifmm_stats_t* o) {
  if (!c || !o) return AIFMM_ERR_INVALID;
  Handle& h = c->h;
  std::memset(o, 0, sizeof(*o));
  o->n = h.N;
  o->dim = h.d;
  o->levels = h.L;
  o->max_rank_nnca = h.max_rank_nnca;
  o->max_rank_factor = h.max_rank_factor;
  o->max_m = h.max_m;
  o->top_size = h.ntop;
  o->flops_factor = h.flops_factor;
  // algorithmic bytes of one solve with one right-hand side (Algorithm 3
  // and the right-hand-side Schur operations): every stored factor entry the
  // two sweeps must read, once each -- the pivot block's LU in both sweeps
  // (n^2 entries per sweep), the blocks of the coupled rows in the pivot
  // columns in the forward sweep (K_pb or P2L_pb: rows(p) x m_b) and of the
  // pivot rows in the coupled columns in the backward sweep (K_bq or M2P_bq:
  // m_b x cols(q)), rows/cols(p) = r_p if p was eliminated before b, else
  // m_p -- and the top system's LU twice; vectors are not counted.
  double bytes = 0;
  if (h.factored) {
    for (auto& F : h.fac) {
      if (!F.nb) continue;
      for (int b = 0; b < F.nb; ++b) {
        const double m = F.h_m[b], n = m + F.h_r[b];
        if (m == 0) continue;
        int bc[3], q[3];
        morton_coords(b, h.d, F.l, bc);
        const int cb = colour_of(bc, h.d);
        double coupled = 0.0;
        for (int o = 0; o < ipow(3, h.d); ++o) {
          int oo = o;
          for (int k = 0; k < 3; ++k) q[k] = bc[k];
          for (int k = 0; k < h.d; ++k) {
            q[k] = bc[k] + (oo % 3) - 1;
            oo /= 3;
          }
          if (!in_grid(q, h.d, F.n) || cheb(bc, q, h.d) == 0) continue;
          const int qb = morton_key(q, h.d, F.l);
          coupled += colour_of(q, h.d) < cb ? F.h_r[qb] : F.h_m[qb];
        }
        bytes += 8.0 * (2.0 * n * n + 2.0 * m * coupled);
      }
    }
    bytes += 8.0 * 2.0 * (double)h.ntop * h.ntop;
  }
  o->bytes_solve = bytes;
  o->bytes_resident = (double)h.resident;
  o->ms_build = h.ms_build;
  o->ms_factor = h.ms_factor;
  o->ms_solve = h.ms_solve;
  o->ms_matvec = h.ms_matvec;
  o->kernel_launches = h.nlaunch;
  for (int g = 0; g < Handle::G_NG; ++g) {
    o->group_ms[g] = h.g_ms[g];
    o->group_flops[g] = h.g_flops[g];
    o->group_launches[g] = h.g_launch[g];
  }
  return AIFMM_OK;
}

aifmm_status aifmm_tree_perm(aifmm_h c, int64_t* perm, int64_t* level_start) {
  if (!c || !perm) return AIFMM_ERR_INVALID;
  Handle& h = c->h;
  AIFMM_ON_DEVICE(h);
  std::vector<int> p(h.N);
  if (cudaMemcpy(p.data(), h.perm, sizeof(int) * h.N, cudaMemcpyDeviceToHost) != cudaSuccess) return AIFMM_ERR_CUDA;
  for (int64_t i = 0; i < h.N; ++i) perm[i] = p[i];
  if (level_start)
    for (size_t i = 0; i < h.h_leaf_start.size(); ++i) level_start[i] = h.h_leaf_start[i];
  return AIFMM_OK;
}

aifmm_status aifmm_level_ranks(aifmm_h c, int level, int which, int* ranks) {
  if (!c || !ranks) return AIFMM_ERR_INVALID;
  Handle& h = c->h;
  if (level < 2 || level > h.L) return AIFMM_ERR_INVALID;
  if (which == 0) {
    const auto& v = h.nn[level].h_rank;
    std::memcpy(ranks, v.data(), sizeof(int) * v.size());
    return AIFMM_OK;
  }
  if (!h.factored) return AIFMM_ERR_STATE;
  const auto& v = h.fac[level].h_r;
  std::memcpy(ranks, v.data(), sizeof(int) * v.size());
  return AIFMM_OK;
}

// row pivots (far = false) or far-field pivots (far = true) of every box of a
// level, concatenated in box order, in the order the search took them
static aifmm_status level_pivots(aifmm_h c, int level, int64_t* pivots, bool far) {
  if (!c || !pivots) return AIFMM_ERR_INVALID;
  Handle& h = c->h;
  if (level < 2 || level > h.L) return AIFMM_ERR_INVALID;
  AIFMM_ON_DEVICE(h);
  const NnLevel& N = h.nn[level];
  std::vector<int> p((size_t)N.nb * N.R);
  if (cudaMemcpy(p.data(), far ? N.far : N.pivpos, sizeof(int) * p.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
    return AIFMM_ERR_CUDA;
  size_t o = 0;
  for (int b = 0; b < N.nb; ++b)
    for (int k = 0; k < N.h_rank[b]; ++k) pivots[o++] = p[(size_t)b * N.R + k];
  return AIFMM_OK;
}

aifmm_status aifmm_level_pivots(aifmm_h c, int level, int64_t* pivots) {
  return level_pivots(c, level, pivots, false);
}

aifmm_status aifmm_level_far_pivots(aifmm_h c, int level, int64_t* pivots) {
  return level_pivots(c, level, pivots, true);
}

int aifmm_levels(aifmm_h c) { return c ? c->h.L : 0; }

int aifmm_device(aifmm_h c) { return c ? c->h.device : -1; }

aifmm_status aifmm_set_priority(aifmm_h c, int priority) {
  if (!c) return AIFMM_ERR_INVALID;
  Handle& h = c->h;
  AIFMM_ON_DEVICE(h);
  if (h.stream && cudaStreamSynchronize(h.stream) != cudaSuccess) {
    h.err = std::string("aifmm_set_priority: ") + cudaGetErrorString(cudaGetLastError());
    return AIFMM_ERR_CUDA;
  }
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, priority) != cudaSuccess) {
    h.err = std::string("cudaStreamCreateWithPriority: ") + cudaGetErrorString(cudaGetLastError());
    return AIFMM_ERR_CUDA;
  }
  if (h.own_stream && h.stream) cudaStreamDestroy(h.stream);
  h.stream = s;
  h.own_stream = true;
  return AIFMM_OK;
}

const char* aifmm_last_error(aifmm_h c) {
  if (!c) return g_build_err.c_str();
  return c->h.err.c_str();
}

void aifmm_destroy(aifmm_h c) {
  if (!c) return;
  Handle& h = c->h;
  DeviceGuard dg(h.device);
  hfree_all(h);
  if (h.own_stream && h.stream) cudaStreamDestroy(h.stream);
  delete c;
}

}  // extern "C"
