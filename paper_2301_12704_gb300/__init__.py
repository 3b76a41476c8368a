"""Python binding of the GB300 AIFMM library (include/aifmm.h).

Argument marshalling only: every numerical step runs in the CUDA library
``libaifmm.so`` built in-tree for sm_103a (``_build.build()``).  Importing
this module does not load the library; the first call does, and raises if
the library is missing or no CUDA device is present -- there is no CPU path.

Arrays may be numpy arrays (host memory) or torch tensors (host or device);
float64, C-contiguous points (N x dim) and Fortran-ordered / column-major
right-hand sides (N x nrhs).  Names follow the C ABI: aifmm_build,
aifmm_factor, aifmm_solve, aifmm_matvec, aifmm_direct_matvec, aifmm_stats,
aifmm_tree_perm, aifmm_level_ranks, aifmm_level_pivots, aifmm_destroy.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libaifmm.so")
HEADER = os.path.join(HERE, "..", "include", "aifmm.h")

LOG2D, INVR3D, INVR2D, GAUSS = 0, 1, 2, 3
STATUS = {0: "OK", 1: "ERR_INVALID", 2: "ERR_OOM", 3: "ERR_SINGULAR", 4: "ERR_STATE",
          5: "ERR_NOCONV", 6: "ERR_CUDA", 7: "ERR_TIMEOUT", 8: "ERR_CAPACITY"}


class AifmmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Kernel(C.Structure):
    _fields_ = [("kind", C.c_int), ("dim", C.c_int), ("diag", C.c_double), ("length", C.c_double),
                ("nugget", C.c_double)]


class Options(C.Structure):
    _fields_ = [("order", C.c_int), ("depth", C.c_int), ("stream", C.c_void_p), ("profile", C.c_int),
                ("no_symmetry", C.c_int), ("factor_tol", C.c_double), ("fma_gemm", C.c_int),
                ("tcgen05", C.c_int), ("precision", C.c_int), ("eta", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("dim", C.c_int), ("levels", C.c_int), ("max_rank_nnca", C.c_int),
                ("max_rank_factor", C.c_int), ("max_m", C.c_int), ("top_size", C.c_int),
                ("flops_factor", C.c_double), ("bytes_solve", C.c_double), ("bytes_resident", C.c_double),
                ("ms_build", C.c_double), ("ms_factor", C.c_double), ("ms_solve", C.c_double),
                ("ms_matvec", C.c_double), ("kernel_launches", C.c_int64), ("group_ms", C.c_double * 8),
                ("group_flops", C.c_double * 8), ("group_launches", C.c_int64 * 8)]


_lib = None


def lib():
    """Load libaifmm.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() first")
        L = C.CDLL(LIB_PATH)
        vp, i64, dbl, cint = C.c_void_p, C.c_int64, C.c_double, C.c_int
        L.aifmm_build.argtypes = [vp, i64, C.POINTER(Kernel), dbl, cint, C.POINTER(Options), C.POINTER(vp)]
        L.aifmm_factor.argtypes = [vp]
        L.aifmm_solve.argtypes = [vp, vp, vp, cint, i64]
        L.aifmm_solve_noalloc.argtypes = [vp, vp, vp, cint, i64]
        L.aifmm_set_priority.argtypes = [vp, cint]
        L.aifmm_noalloc_scratch_bytes.argtypes = []
        L.aifmm_noalloc_scratch_bytes.restype = i64
        L.aifmm_matvec.argtypes = [vp, vp, vp, cint, i64]
        L.aifmm_direct_matvec.argtypes = [vp, vp, vp, cint, i64]
        L.aifmm_gmres.argtypes = [vp, vp, vp, dbl, cint, cint, cint, C.POINTER(cint), C.POINTER(dbl)]
        L.aifmm_stats.argtypes = [vp, C.POINTER(Stats)]
        L.aifmm_dgemm_tc.argtypes = [vp, i64, vp, i64, vp, i64, cint, cint, cint, dbl, vp]
        L.aifmm_dgemm_tc.restype = C.c_int
        L.aifmm_dgemm_tc05.argtypes = [vp, i64, vp, i64, vp, i64, cint, cint, cint, dbl, vp]
        L.aifmm_dgemm_tc05.restype = C.c_int
        L.aifmm_dgemm_tc8.argtypes = [vp, i64, vp, i64, vp, i64, cint, cint, cint, dbl, vp]
        L.aifmm_dgemm_tc8.restype = C.c_int
        L.aifmm_gemm_tf32.argtypes = [cint, vp, i64, vp, i64, vp, i64, cint, cint, cint, dbl, vp]
        L.aifmm_gemm_tf32.restype = C.c_int
        L.aifmm_fma_rate.argtypes = [cint, vp, C.POINTER(dbl)]
        L.aifmm_fma_rate.restype = C.c_int
        L.aifmm_tree_perm.argtypes = [vp, vp, vp]
        L.aifmm_level_ranks.argtypes = [vp, cint, cint, vp]
        L.aifmm_level_pivots.argtypes = [vp, cint, vp]
        L.aifmm_level_far_pivots.argtypes = [vp, cint, vp]
        L.aifmm_levels.argtypes = [vp]
        L.aifmm_device.argtypes = [vp]
        L.aifmm_last_error.argtypes = [vp]
        L.aifmm_last_error.restype = C.c_char_p
        L.aifmm_destroy.argtypes = [vp]
        L.aifmm_destroy.restype = None
        for name in ("aifmm_build", "aifmm_factor", "aifmm_solve", "aifmm_solve_noalloc", "aifmm_matvec",
                     "aifmm_direct_matvec", "aifmm_gmres",
                     "aifmm_stats", "aifmm_tree_perm", "aifmm_level_ranks", "aifmm_level_pivots",
                     "aifmm_level_far_pivots", "aifmm_levels", "aifmm_device"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(status, handle=None):
    if status != 0:
        msg = lib().aifmm_last_error(handle)
        raise AifmmError(status, msg.decode() if msg else "")


def _f64(t):
    """A torch tensor as float64 (the ABI's only element type)."""
    import torch
    return t if t.dtype == torch.float64 else t.to(torch.float64)


def _rows(a, n, what):
    """The library reads n rows of every vector or matrix it is given: refuse
    a buffer with another row count before its pointer crosses the ABI."""
    if a.shape[0] != n:
        raise ValueError(f"{what} has {a.shape[0]} rows, the problem has {n} points")


def _ready(h, *arrays):
    """The library runs on the handle's own CUDA stream and does not wait for
    other streams.  Before a torch CUDA tensor's pointer crosses the ABI,
    wait for torch's pending work on its device (the current stream, where
    the tensor was filled or copied), and refuse a tensor on another GPU than
    the handle's."""
    synced = set()
    for a in arrays:
        if a is None or isinstance(a, np.ndarray) or not getattr(a, "is_cuda", False):
            continue
        if h is not None and h.device is not None and a.device.index != h.device:
            raise ValueError(f"tensor on cuda:{a.device.index}, the handle belongs to cuda:{h.device}")
        if a.device.index not in synced:
            import torch
            torch.cuda.current_stream(a.device).synchronize()
            synced.add(a.device.index)


def _ptr(a):
    """(pointer, keepalive) of a float64 numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data, a
    return a.data_ptr(), a


class Handle:
    """Owns one aifmm_h (``device``: the CUDA device index it belongs to)."""

    def __init__(self, raw, n, dim, device=None):
        self.raw, self.n, self.dim, self.device = raw, n, dim, device

    def __del__(self):
        try:
            aifmm_destroy(self)
        except Exception:
            pass


def aifmm_build(points, kernel: int, diag: float, tol: float, leaf_size: int, length: float = 1.0,
                depth: int = 0, stream=None, profile: bool = False, symmetric: bool = True,
                factor_tol: float = 0.0, fma_gemm: bool = False, tcgen05: bool = False,
                fp32: bool = False, nugget: float = 0.0, eta: float = 0.0, tf32: bool = False) -> Handle:
    """Build tree, lists, NNCA operators and the extended system (C: aifmm_build).

    ``symmetric=False`` selects the general elimination (rows and columns
    compressed separately, every Schur block computed); ``factor_tol`` > 0 is
    the compress threshold of the factorisation (default: ``tol``);
    ``fma_gemm`` runs the factorisation's tile products on FP64 FMAs instead of
    the tensor cores;
    ``tcgen05`` issues them on tcgen05.mma instead of warp MMAs; ``fp32``
    makes the factorisation's tile products FP32 (a preconditioner for
    aifmm_gmres), ``tf32`` TF32 tensor-core products (the same use).  ``diag`` = NaN makes A_ii = kernel(0) + ``nugget``
    (Gaussian only); ``eta`` is the admissibility parameter (0 or >= sqrt(dim))."""
    if isinstance(points, np.ndarray):
        points = np.ascontiguousarray(points, dtype=np.float64)
    else:
        points = _f64(points).contiguous()
    if points.ndim != 2:
        raise ValueError("points must be N x dim")
    n, dim = points.shape
    k = Kernel(kernel, dim, float(diag), float(length), float(nugget))
    o = Options(0, int(depth), C.c_void_p(stream) if stream else None, int(bool(profile)), int(not symmetric),
                float(factor_tol), int(bool(fma_gemm)), int(bool(tcgen05)), 2 if tf32 else int(bool(fp32)),
                float(eta))
    out = C.c_void_p()
    _ready(None, points)
    p, keep = _ptr(points)
    _check(lib().aifmm_build(C.c_void_p(p), n, C.byref(k), float(tol), int(leaf_size), C.byref(o), C.byref(out)))
    return Handle(out.value, n, dim, lib().aifmm_device(out.value))


def aifmm_factor(h: Handle) -> None:
    _check(lib().aifmm_factor(h.raw), h.raw)


def _col_major(a):
    """Column-major float64 copy/view of a vector or N x nrhs matrix."""
    if isinstance(a, np.ndarray):
        return np.asfortranarray(a[:, None] if a.ndim == 1 else a, dtype=np.float64)
    t = _f64(a[:, None] if a.dim() == 1 else a)
    return t.t().contiguous().t()


def _empty_cm(a):
    if isinstance(a, np.ndarray):
        return np.empty(a.shape, dtype=np.float64, order="F")
    import torch
    return torch.empty((a.shape[1], a.shape[0]), dtype=a.dtype, device=a.device).t()


def aifmm_solve(h: Handle, rhs):
    """x = A^-1 rhs (C: aifmm_solve); rhs N or N x nrhs, original order."""
    b = _col_major(rhs)
    _rows(b, h.n, "rhs")
    x = _empty_cm(b)
    _ready(h, b, x)
    pb, kb = _ptr(b)
    px, kx = _ptr(x)
    _check(lib().aifmm_solve(h.raw, C.c_void_p(pb), C.c_void_p(px), b.shape[1], h.n), h.raw)
    return x


def aifmm_solve_noalloc(h: Handle, rhs, x):
    """x = A^-1 rhs without any device allocation (C: aifmm_solve_noalloc).
    rhs and x must be column-major float64 CUDA tensors of shape N x nrhs;
    x is written in place and returned."""
    import torch
    if rhs.dim() == 1:
        rhs, x = rhs[:, None], x[:, None]
    if not (rhs.is_cuda and x.is_cuda and rhs.stride(0) == 1 and x.stride(0) == 1):
        raise ValueError("aifmm_solve_noalloc needs column-major CUDA tensors")
    if rhs.dtype != torch.float64 or x.dtype != torch.float64:
        raise ValueError("aifmm_solve_noalloc needs float64 tensors")
    _rows(rhs, h.n, "rhs")
    if tuple(x.shape) != tuple(rhs.shape) or (rhs.shape[1] > 1 and x.stride(1) != rhs.stride(1)):
        raise ValueError("x must have rhs's shape and leading dimension")
    _ready(h, rhs, x)
    _check(lib().aifmm_solve_noalloc(h.raw, C.c_void_p(rhs.data_ptr()), C.c_void_p(x.data_ptr()),
                                     rhs.shape[1], rhs.stride(1) if rhs.shape[1] > 1 else h.n), h.raw)
    return x


def aifmm_noalloc_scratch_bytes() -> int:
    return int(lib().aifmm_noalloc_scratch_bytes())


def _product(fn, h, xv):
    xx = _col_major(xv)
    _rows(xx, h.n, "x")
    y = _empty_cm(xx)
    _ready(h, xx, y)
    px, kx = _ptr(xx)
    py, ky = _ptr(y)
    _check(fn(h.raw, C.c_void_p(px), C.c_void_p(py), xx.shape[1], h.n), h.raw)
    return y


def aifmm_matvec(h: Handle, x):
    """y = A_H2 x with the NNCA operators (C: aifmm_matvec)."""
    return _product(lib().aifmm_matvec, h, x)


def aifmm_direct_matvec(h: Handle, x):
    """y = A x, every entry evaluated (C: aifmm_direct_matvec)."""
    return _product(lib().aifmm_direct_matvec, h, x)


def aifmm_gmres(h: Handle, b, rtol: float = 1e-10, maxit: int = 200, restart: int = 50,
                use_precond: bool = True, raise_noconv: bool = True):
    """Restarted GMRES on the H^2 product, right-preconditioned by the AIFMM
    factorisation when ``use_precond`` (C: aifmm_gmres).  Returns
    (x, iterations, relative residual); x has b's type and device."""
    if isinstance(b, np.ndarray):
        bb = np.ascontiguousarray(b, dtype=np.float64).reshape(-1)
        x = np.empty_like(bb)
    else:
        bb = _f64(b).reshape(-1).contiguous()
        x = torch_empty_like(bb)
    _rows(bb, h.n, "b")
    _ready(h, bb, x)
    pb, kb = _ptr(bb)
    px, kx = _ptr(x)
    it = C.c_int(0)
    rr = C.c_double(0.0)
    st = lib().aifmm_gmres(h.raw, C.c_void_p(pb), C.c_void_p(px), float(rtol), int(maxit), int(restart),
                           int(bool(use_precond)), C.byref(it), C.byref(rr))
    if st != 0 and (st != 5 or raise_noconv):
        _check(st, h.raw)
    return x, it.value, rr.value


def aifmm_dgemm_tc(A, B, C_, alpha: float = 1.0, stream=None, tcgen05: bool = False,
                   digits8: bool = False) -> None:
    """C_ += alpha A B on the tensor cores in FP64 precision (C: aifmm_dgemm_tc,
    aifmm_dgemm_tc05 with ``tcgen05``, aifmm_dgemm_tc8 with ``digits8``).
    A, B, C_ CUDA float64 tensors, column-major (e.g. ``t.t().contiguous().t()``)."""
    import torch
    m, k = A.shape
    k2, n = B.shape
    assert k2 == k and tuple(C_.shape) == (m, n)
    assert A.dtype == B.dtype == C_.dtype == torch.float64, "float64 tensors"
    def ld(t):
        assert t.is_cuda and (t.stride(0) == 1 or t.shape[0] == 1), "column-major CUDA tensors"
        return max(1, t.shape[0], t.stride(1) if t.shape[1] > 1 else 1)

    fn = lib().aifmm_dgemm_tc05 if tcgen05 else lib().aifmm_dgemm_tc8 if digits8 else lib().aifmm_dgemm_tc
    st = fn(C.c_void_p(A.data_ptr()), ld(A), C.c_void_p(B.data_ptr()), ld(B),
                              C.c_void_p(C_.data_ptr()), ld(C_), m, n, k, float(alpha),
                              C.c_void_p(stream) if stream else None)
    if st != 0:
        raise AifmmError(st, "aifmm_dgemm_tc failed")


def aifmm_gemm_tf32(A, B, C_, alpha: float = 1.0, trans_a: bool = False, stream=None) -> None:
    """C_ += alpha op(A) B on the TF32 tensor cores (C: aifmm_gemm_tf32); CUDA
    float64 column-major tensors; op(A) = A^T with ``trans_a``."""
    import torch
    m, n = C_.shape
    k = B.shape[0]
    assert A.dtype == B.dtype == C_.dtype == torch.float64
    def ld(t):
        assert t.is_cuda and (t.stride(0) == 1 or t.shape[0] == 1), "column-major CUDA tensors"
        return max(1, t.shape[0], t.stride(1) if t.shape[1] > 1 else 1)
    st = lib().aifmm_gemm_tf32(int(bool(trans_a)), C.c_void_p(A.data_ptr()), ld(A), C.c_void_p(B.data_ptr()), ld(B),
                               C.c_void_p(C_.data_ptr()), ld(C_), m, n, k, float(alpha),
                               C.c_void_p(stream) if stream else None)
    if st != 0:
        raise AifmmError(st, "aifmm_gemm_tf32 failed")


def aifmm_fma_rate(fp32: bool = False, stream=None) -> float:
    """Measured FMA rate of the current device in TFLOP/s (C: aifmm_fma_rate):
    FP64 by default, FP32 with ``fp32``."""
    r = C.c_double(0.0)
    st = lib().aifmm_fma_rate(int(bool(fp32)), C.c_void_p(stream) if stream else None, C.byref(r))
    if st != 0:
        raise AifmmError(st, "aifmm_fma_rate failed")
    return r.value


def torch_empty_like(t):
    import torch
    return torch.empty_like(t)


def aifmm_stats(h: Handle) -> dict:
    s = Stats()
    _check(lib().aifmm_stats(h.raw, C.byref(s)), h.raw)
    out = {}
    for f, _ in Stats._fields_:
        v = getattr(s, f)
        out[f] = list(v) if hasattr(v, "__len__") else v
    return out


def aifmm_set_priority(h: Handle, priority: int) -> None:
    """Move the handle's later work to a new library stream of this CUDA
    priority (lower runs first; clamped to the device's range)."""
    _check(lib().aifmm_set_priority(h.raw, int(priority)), h.raw)


def aifmm_levels(h: Handle) -> int:
    return lib().aifmm_levels(h.raw)


def aifmm_tree_perm(h: Handle):
    L = aifmm_levels(h)
    perm = np.empty(h.n, dtype=np.int64)
    starts = np.empty((1 << (h.dim * L)) + 1, dtype=np.int64)
    _check(lib().aifmm_tree_perm(h.raw, C.c_void_p(perm.ctypes.data), C.c_void_p(starts.ctypes.data)), h.raw)
    return perm, starts


def aifmm_level_ranks(h: Handle, level: int, which: int = 0):
    r = np.empty(1 << (h.dim * level), dtype=np.int32)
    _check(lib().aifmm_level_ranks(h.raw, level, which, C.c_void_p(r.ctypes.data)), h.raw)
    return r


def aifmm_level_pivots(h: Handle, level: int):
    r = aifmm_level_ranks(h, level, 0)
    p = np.empty(int(r.sum()), dtype=np.int64)
    _check(lib().aifmm_level_pivots(h.raw, level, C.c_void_p(p.ctypes.data)), h.raw)
    return p


def aifmm_level_far_pivots(h: Handle, level: int):
    r = aifmm_level_ranks(h, level, 0)
    p = np.empty(int(r.sum()), dtype=np.int64)
    _check(lib().aifmm_level_far_pivots(h.raw, level, C.c_void_p(p.ctypes.data)), h.raw)
    return p


def aifmm_destroy(h: Handle) -> None:
    if h is not None and h.raw:
        lib().aifmm_destroy(h.raw)
        h.raw = None
