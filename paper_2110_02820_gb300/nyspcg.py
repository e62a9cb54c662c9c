"""Thin Python binding of the C ABI in ``include/nyspcg.h``.

Argument marshalling only: every step of the computation runs in the CUDA
library ``lib/libnyspcg.so``.  Tensors must be CUDA tensors; the current
torch stream is passed to the library.  If the library has not been built
the first call raises ``NysLibraryMissing`` (there is no CPU fallback).

The function names are those of the C ABI: ``nys_sketch``,
``nys_sketch_adaptive``, ``nys_precond_apply``, ``pcg_solve``,
``nys_op_matvec``, ``nys_power_err_est``.
"""

from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass

import torch

NYS_OK, NYS_ERR_ARG, NYS_ERR_NOT_PSD, NYS_ERR_BREAKDOWN, NYS_ERR_MAXIT, NYS_ERR_TIMEOUT, \
    NYS_ERR_CUDA, NYS_ERR_OOM = range(8)
NYS_OP_DENSE, NYS_OP_GRAM, NYS_OP_RBF = range(3)
NYS_F64, NYS_F32 = range(2)
NYS_PREC_F64, NYS_PREC_MIXED = range(2)
NYS_RULE_ERR, NYS_RULE_RATIO = range(2)

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libnyspcg.so")


class NysLibraryMissing(RuntimeError):
    pass


class NysError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: status {status} ({status_str(status)})")
        self.status = status


class _Operator(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dtype", C.c_int32), ("n", C.c_int64), ("m", C.c_int64),
                ("d", C.c_int64), ("ld", C.c_int64), ("data", C.c_void_p), ("sigma", C.c_double)]


class _AdaptInfo(C.Structure):
    _fields_ = [("ell", C.c_int64), ("doublings", C.c_int32), ("estimates", C.c_int32),
                ("err_est", C.c_double), ("lambda_ell", C.c_double), ("kappa_est", C.c_double)]


class _PcgOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxit", C.c_int32), ("precision", C.c_int32),
                ("inner_tol", C.c_double), ("max_refine", C.c_int32), ("use_x0", C.c_int32),
                ("residual_history", C.c_void_p)]


class _PcgResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("refinements", C.c_int32),
                ("escalated", C.c_int32), ("rel_residual", C.c_double)]


_lib = None
_lock = threading.Lock()

EXPORTS = ["nys_sketch", "nys_sketch_adaptive", "nys_precond_apply", "pcg_solve", "nys_factor_get",
           "nys_factor_free", "nys_status_str", "nys_op_matvec", "nys_power_err_est",
           "nys_gemm_tf32_tn"]


def lib() -> C.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise NysLibraryMissing(
                f"{LIB_PATH} is missing: build it with `python -m paper_2110_02820_gb300.build`")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, u64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
        L.nys_sketch.argtypes = [C.POINTER(_Operator), i64, u64, vp, i32, C.POINTER(vp), vp]
        L.nys_sketch_adaptive.argtypes = [C.POINTER(_Operator), i64, i64, i32, dbl, i32, dbl, u64,
                                          vp, vp, i32, C.POINTER(vp), C.POINTER(_AdaptInfo), vp]
        L.nys_precond_apply.argtypes = [vp, C.POINTER(dbl), i64, vp, vp, i32, vp]
        L.pcg_solve.argtypes = [C.POINTER(_Operator), vp, C.POINTER(dbl), i64, vp, vp,
                                C.POINTER(_PcgOpts), C.POINTER(_PcgResult), vp]
        L.nys_factor_get.argtypes = [vp, C.POINTER(vp), C.POINTER(i32), C.POINTER(vp),
                                     C.POINTER(i64), C.POINTER(i64), C.POINTER(dbl)]
        L.nys_factor_free.argtypes = [vp]
        L.nys_factor_free.restype = None
        L.nys_status_str.argtypes = [i32]
        L.nys_status_str.restype = C.c_char_p
        L.nys_op_matvec.argtypes = [C.POINTER(_Operator), dbl, i64, vp, vp, i32, vp]
        L.nys_power_err_est.argtypes = [C.POINTER(_Operator), vp, vp, i32, C.POINTER(dbl), vp]
        L.nys_gemm_tf32_tn.argtypes = [i64, i64, i64, vp, i64, vp, i64, vp, i64, vp]
        L.nys_kernel_launch_count.argtypes = []
        L.nys_kernel_launch_count.restype = C.c_uint64
        L.nys_pcg_graphs.argtypes = [i32]
        L.nys_pcg_graphs.restype = i32
        L.nys_pcg_graph_replays.argtypes = []
        L.nys_pcg_graph_replays.restype = C.c_uint64
        L.nys_autotune.argtypes = [i32]
        L.nys_autotune.restype = i32
        L.nys_autotune_dump.argtypes = [C.c_char_p, i64]
        L.nys_autotune_dump.restype = i64
        L.nys_autotune_clear.argtypes = []
        L.nys_autotune_clear.restype = None
        L.nys_autotune_set.argtypes = [C.c_char_p, i32]
        L.nys_autotune_set.restype = i32
        L.nys_rbf_cross_matvec.argtypes = [vp, i64, i64, vp, i64, i64, i64, dbl, i64, vp, vp, i32,
                                           vp]
        for name in EXPORTS:
            f = getattr(L, name)
            if f.restype is C.c_int:  # default
                f.restype = C.c_int32
        _lib = L
        return _lib


def kernel_launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(lib().nys_kernel_launch_count())


def pcg_graphs(on: int | None = None) -> bool:
    """PCG launch mode: with `on` True/False, capture (or not) the iteration
    loop as a CUDA graph; returns the previous mode.  None only queries."""
    arg = -1 if on is None else (1 if on else 0)
    return bool(lib().nys_pcg_graphs(arg))


def pcg_loop(on: int | None = None) -> bool:
    """Device-side PCG loop (one graph launch per solve; True = on); sets it
    when `on` is 0 or 1 and returns the previous mode."""
    f = lib().nys_pcg_loop
    if f.argtypes is None:
        f.argtypes = [C.c_int32]
        f.restype = C.c_int32
    return bool(f(-1 if on is None else int(on)))


def pcg_reliable(on: int | None = None) -> bool:
    """Reliable-update mode of one-system mixed solves (True = on); sets it when
    `on` is 0 or 1 and returns the previous mode."""
    f = lib().nys_pcg_reliable
    if f.argtypes is None:
        f.argtypes = [C.c_int32]
        f.restype = C.c_int32
    return bool(f(-1 if on is None else int(on)))


def pcg_graph_replays() -> int:
    """PCG iteration graphs replayed so far in this process."""
    return int(lib().nys_pcg_graph_replays())


def autotune(on: bool | None = None) -> bool:
    """Launch-shape autotuner: with `on` True/False, time (or not) the launch
    shapes of unseen problem sizes; returns the previous mode."""
    arg = -1 if on is None else (1 if on else 0)
    return bool(lib().nys_autotune(arg))


def autotune_choices() -> dict:
    """The tuner's current choices, {key: launch shape}."""
    import json
    n = int(lib().nys_autotune_dump(None, 0))
    buf = C.create_string_buffer(n + 1)
    lib().nys_autotune_dump(buf, n + 1)
    return json.loads(buf.value.decode())


def autotune_clear() -> None:
    """Forget every tuned choice of this process."""
    lib().nys_autotune_clear()


def autotune_set(key: str, choice: int) -> None:
    """Pin the launch shape `choice` for `key` (a key of autotune_choices())."""
    _check(lib().nys_autotune_set(key.encode(), int(choice)), "nys_autotune_set")


def status_str(status: int) -> str:
    try:
        return lib().nys_status_str(int(status)).decode()
    except NysLibraryMissing:
        return "?"


def _stream() -> C.c_void_p:
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: torch.Tensor | None) -> C.c_void_p:
    if t is None:
        return C.c_void_p(None)
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _check(status: int, what: str) -> None:
    if status != NYS_OK:
        raise NysError(status, what)


# ---------------------------------------------------------------- operators

class Operator:
    """An operator descriptor; keeps its data tensor alive."""

    def __init__(self, kind: int, data: torch.Tensor, n: int, m: int = 0, d: int = 0,
                 sigma: float = 0.0):
        if not data.is_cuda or not data.is_contiguous():
            raise ValueError("operator data must be a contiguous CUDA tensor")
        self.data = data
        self.kind = kind
        dt = NYS_F64 if data.dtype == torch.float64 else NYS_F32
        ld = data.shape[1]
        self.c = _Operator(kind, dt, n, m, d, ld, data.data_ptr(), float(sigma))
        self.n = n

    @property
    def ref(self):
        return C.byref(self.c)


def dense_operator(A: torch.Tensor) -> Operator:
    """A: n x n symmetric psd, float64, on the GPU."""
    return Operator(NYS_OP_DENSE, A, A.shape[0])


def gram_operator(X: torch.Tensor) -> Operator:
    """A = X^T X for X: m x n float32 on the GPU."""
    return Operator(NYS_OP_GRAM, X, X.shape[1], m=X.shape[0])


def rbf_operator(points: torch.Tensor, sigma: float) -> Operator:
    """Gaussian kernel on n points (n x d float32 on the GPU)."""
    return Operator(NYS_OP_RBF, points, points.shape[0], d=points.shape[1], sigma=sigma)


# ---------------------------------------------------------------- factor

class _CudaArray:
    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (ptr, False), "version": 2, "strides": None}


class Factor:
    """Owns a library factor (U, lambda_hat); freed with nys_factor_free."""

    def __init__(self, handle: C.c_void_p, device: int):
        self.h = handle
        self.device = device
        U, ud, lam = C.c_void_p(), C.c_int32(), C.c_void_p()
        n, ell, nu = C.c_int64(), C.c_int64(), C.c_double()
        _check(lib().nys_factor_get(self.h, C.byref(U), C.byref(ud), C.byref(lam), C.byref(n),
                                    C.byref(ell), C.byref(nu)), "nys_factor_get")
        self._U, self._lam = U.value, lam.value
        self.u_dtype = ud.value
        self.n, self.ell, self.nu = n.value, ell.value, nu.value

    def U(self) -> torch.Tensor:
        """Copy of U (n x ell; float64 or float32)."""
        ts = "<f8" if self.u_dtype == NYS_F64 else "<f4"
        with torch.cuda.device(self.device):
            return torch.as_tensor(_CudaArray(self._U, (self.n, self.ell), ts),
                                   device=f"cuda:{self.device}").clone()

    def lam(self) -> torch.Tensor:
        with torch.cuda.device(self.device):
            return torch.as_tensor(_CudaArray(self._lam, (self.ell,), "<f8"),
                                   device=f"cuda:{self.device}").clone()

    def stats(self) -> dict:
        """Shift escalations, SVD sweeps and refinement steps, lambda_hat_ell."""
        f = lib().nys_factor_stats
        if f.argtypes is None:
            f.argtypes = [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                          C.POINTER(C.c_int32), C.POINTER(C.c_double)]
            f.restype = C.c_int32
        e, sw, rf, le = C.c_int32(), C.c_int32(), C.c_int32(), C.c_double()
        _check(f(self.h, C.byref(e), C.byref(sw), C.byref(rf), C.byref(le)), "nys_factor_stats")
        return {"shift_escalations": e.value, "svd_sweeps": sw.value,
                "svd_refinements": rf.value, "lambda_ell": le.value}

    def free(self) -> None:
        if self.h is not None and self.h.value:
            lib().nys_factor_free(self.h)
        self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ---------------------------------------------------------------- entry points

def nys_sketch(op: Operator, ell: int, seed: int = 0, omega: torch.Tensor | None = None,
               precision: int = NYS_PREC_F64) -> Factor:
    if omega is not None:
        assert omega.dtype == torch.float64 and tuple(omega.shape) == (op.n, ell)
    h = C.c_void_p()
    _check(lib().nys_sketch(op.ref, ell, seed, _ptr(omega), precision, C.byref(h), _stream()),
           "nys_sketch")
    return Factor(h, op.data.device.index or 0)


@dataclass
class AdaptInfo:
    ell: int
    doublings: int
    estimates: int
    err_est: float
    lambda_ell: float
    kappa_est: float


def nys_sketch_columns(op: Operator, ell: int, seed: int = 0, cols: torch.Tensor | None = None,
                       precision: int = NYS_PREC_F64) -> Factor:
    """Column-sampling sketch: Algorithm 1 with Omega = I[:, cols] (cols an
    int64 CUDA tensor of distinct indices, or drawn from `seed` when None)."""
    f = lib().nys_sketch_columns
    if f.argtypes is None:
        f.argtypes = [C.POINTER(_Operator), C.c_int64, C.c_uint64, C.c_void_p, C.c_int32,
                      C.POINTER(C.c_void_p), C.c_void_p]
        f.restype = C.c_int32
    if cols is not None and (cols.dtype != torch.int64 or not cols.is_cuda):
        raise ValueError("cols must be an int64 CUDA tensor")
    h = C.c_void_p()
    _check(f(op.ref, ell, seed, _ptr(cols), precision, C.byref(h), _stream()), "nys_sketch_columns")
    return Factor(h, op.data.device.index or 0)


def nys_sketch_adaptive(op: Operator, ell0: int, ell_max: int, rule: int, tol: float, q: int = 5,
                        mu: float = 0.0, seed: int = 0, omega: torch.Tensor | None = None,
                        g: torch.Tensor | None = None, precision: int = NYS_PREC_F64):
    h = C.c_void_p()
    info = _AdaptInfo()
    _check(lib().nys_sketch_adaptive(op.ref, ell0, ell_max, rule, tol, q, mu, seed, _ptr(omega),
                                     _ptr(g), precision, C.byref(h), C.byref(info), _stream()),
           "nys_sketch_adaptive")
    return Factor(h, op.data.device.index or 0), AdaptInfo(
        info.ell, info.doublings, info.estimates, info.err_est, info.lambda_ell, info.kappa_est)


def nys_precond_apply(f: Factor, mu, v: torch.Tensor) -> torch.Tensor:
    """z = P^{-1} v for each row of v ([nrhs][n] or [n]); mu scalar or per row."""
    vv = v if v.dim() == 2 else v[None]
    nrhs = vv.shape[0]
    mus = [float(mu)] * nrhs if not hasattr(mu, "__len__") else [float(m) for m in mu]
    z = torch.empty_like(vv)
    dt = NYS_F64 if vv.dtype == torch.float64 else NYS_F32
    arr = (C.c_double * nrhs)(*mus)
    _check(lib().nys_precond_apply(f.h, arr, nrhs, _ptr(vv), _ptr(z), dt, _stream()),
           "nys_precond_apply")
    return z if v.dim() == 2 else z[0]


def nys_sketch_solve(f: Factor, mu, b: torch.Tensor) -> torch.Tensor:
    """Algorithm 2: x = (U Lam U^T + mu I)^{-1} b for each row of b ([nrhs][n] or [n])."""
    fn = lib().nys_sketch_solve
    if fn.argtypes is None:
        fn.argtypes = [C.c_void_p, C.POINTER(C.c_double), C.c_int64, C.c_void_p, C.c_void_p,
                       C.c_int32, C.c_void_p]
        fn.restype = C.c_int32
    bb = b if b.dim() == 2 else b[None]
    nrhs = bb.shape[0]
    mus = [float(mu)] * nrhs if not hasattr(mu, "__len__") else [float(m) for m in mu]
    x = torch.empty_like(bb)
    dt = NYS_F64 if bb.dtype == torch.float64 else NYS_F32
    arr = (C.c_double * nrhs)(*mus)
    _check(fn(f.h, arr, nrhs, _ptr(bb), _ptr(x), dt, _stream()), "nys_sketch_solve")
    return x if b.dim() == 2 else x[0]


@dataclass
class PcgResult:
    status: int
    iterations: int
    refinements: int
    rel_residual: float
    escalated: int = 0


def pcg_solve(op: Operator, f: Factor | None, mu, b: torch.Tensor, x: torch.Tensor | None = None,
              tol: float = 1e-8, maxit: int = 500, precision: int = NYS_PREC_F64,
              inner_tol: float = 1e-4, max_refine: int = 20, history: bool = False):
    """Solve (A + mu_s I) x_s = b_s for each row of b ([nsys][n] or [n], float64).

    Returns (x, [PcgResult], history or None).  Statuses MAXIT and BREAKDOWN are
    reported per system in the results; any other failure raises NysError."""
    bb = b if b.dim() == 2 else b[None]
    nsys, n = bb.shape
    mus = [float(mu)] * nsys if not hasattr(mu, "__len__") else [float(m) for m in mu]
    use_x0 = x is not None
    xx = (x if x.dim() == 2 else x[None]).clone() if use_x0 else torch.empty_like(bb)
    hist = torch.empty((nsys, maxit + 1), dtype=torch.float64, device=bb.device) if history else None
    opts = _PcgOpts(tol, maxit, precision, inner_tol, max_refine, int(use_x0),
                    hist.data_ptr() if hist is not None else None)
    res = (_PcgResult * nsys)()
    arr = (C.c_double * nsys)(*mus)
    st = lib().pcg_solve(op.ref, f.h if f is not None else None, arr, nsys, _ptr(bb), _ptr(xx),
                         C.byref(opts), res, _stream())
    if st not in (NYS_OK, NYS_ERR_MAXIT, NYS_ERR_BREAKDOWN):
        raise NysError(st, "pcg_solve")
    out = [PcgResult(r.status, r.iterations, r.refinements, r.rel_residual, r.escalated) for r in res]
    xo = xx if b.dim() == 2 else xx[0]
    return xo, out, hist


def nys_block_pcg(op: Operator, f: Factor | None, mu: float, B: torch.Tensor,
                  X: torch.Tensor | None = None, tol: float = 1e-8, maxit: int = 500,
                  precision: int = NYS_PREC_F64, inner_tol: float = 1e-4, max_refine: int = 20):
    """Block Nystrom PCG for the rows of B ([nrhs][n] float64, nrhs <= 32) with
    one shift mu.  Returns (X, [PcgResult])."""
    fn = lib().nys_block_pcg
    if fn.argtypes is None:
        fn.argtypes = [C.POINTER(_Operator), C.c_void_p, C.c_double, C.c_int64, C.c_void_p,
                       C.c_void_p, C.POINTER(_PcgOpts), C.POINTER(_PcgResult), C.c_void_p]
        fn.restype = C.c_int32
    nrhs = B.shape[0]
    use_x0 = X is not None
    XX = X.clone() if use_x0 else torch.empty_like(B)
    opts = _PcgOpts(tol, maxit, precision, inner_tol, max_refine, int(use_x0), None)
    res = (_PcgResult * nrhs)()
    st = fn(op.ref, f.h if f is not None else None, float(mu), nrhs, _ptr(B), _ptr(XX),
            C.byref(opts), res, _stream())
    if st not in (NYS_OK, NYS_ERR_MAXIT, NYS_ERR_BREAKDOWN):
        raise NysError(st, "nys_block_pcg")
    return XX, [PcgResult(r.status, r.iterations, r.refinements, r.rel_residual, r.escalated) for r in res]


class _PathResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("resketched", C.c_int32),
                ("refinements", C.c_int32), ("ell", C.c_int64), ("err_est", C.c_double),
                ("rel_residual", C.c_double)]


def nys_reg_path(op: Operator, mus, b: torch.Tensor, ell0: int, ell_max: int,
                 err_factor: float = 30.0, q: int = 5, seed: int = 0,
                 omegas: torch.Tensor | None = None, gs: torch.Tensor | None = None,
                 tol: float = 1e-8, maxit: int = 500, precision: int = NYS_PREC_F64,
                 inner_tol: float = 1e-4, max_refine: int = 20):
    """Regularization path (warm starts, factor reuse) for the shifts `mus`.
    Returns (X [count][n], [dict per shift])."""
    fn = lib().nys_reg_path
    if fn.argtypes is None:
        fn.argtypes = [C.POINTER(_Operator), C.c_int64, C.POINTER(C.c_double), C.c_void_p,
                       C.c_void_p, C.c_int64, C.c_int64, C.c_double, C.c_int32, C.c_uint64,
                       C.c_void_p, C.c_void_p, C.POINTER(_PcgOpts), C.POINTER(_PathResult),
                       C.c_void_p]
        fn.restype = C.c_int32
    count = len(mus)
    X = torch.empty((count, b.shape[-1]), dtype=torch.float64, device=b.device)
    arr = (C.c_double * count)(*[float(m) for m in mus])
    opts = _PcgOpts(tol, maxit, precision, inner_tol, max_refine, 0, None)
    res = (_PathResult * count)()
    st = fn(op.ref, count, arr, _ptr(b), _ptr(X), ell0, ell_max, float(err_factor), q, seed,
            _ptr(omegas), _ptr(gs), C.byref(opts), res, _stream())
    if st not in (NYS_OK, NYS_ERR_MAXIT, NYS_ERR_BREAKDOWN):
        raise NysError(st, "nys_reg_path")
    out = [dict(status=r.status, iterations=r.iterations, resketched=bool(r.resketched),
                refinements=r.refinements, ell=r.ell, err_est=r.err_est,
                rel_residual=r.rel_residual) for r in res]
    return X, out


def nys_op_matvec(op: Operator, mu: float, x: torch.Tensor, mode: int = 0) -> torch.Tensor:
    xx = x if x.dim() == 2 else x[None]
    y = torch.empty_like(xx)
    _check(lib().nys_op_matvec(op.ref, float(mu), xx.shape[0], _ptr(xx), _ptr(y), mode, _stream()),
           "nys_op_matvec")
    return y if x.dim() == 2 else y[0]


def nys_gemm_tf32_tn(A: torch.Tensor, B: torch.Tensor) -> torch.Tensor:
    """D = A B^T (TF32 tensor cores, FP32 accumulate) for FP32 CUDA matrices."""
    M, K = A.shape
    N, K2 = B.shape
    assert K == K2 and A.dtype == torch.float32 and B.dtype == torch.float32
    D = torch.empty((M, N), dtype=torch.float32, device=A.device)
    _check(lib().nys_gemm_tf32_tn(M, N, K, _ptr(A), A.stride(0), _ptr(B), B.stride(0), _ptr(D),
                                  N, _stream()), "nys_gemm_tf32_tn")
    return D


def nys_power_err_est(op: Operator, f: Factor, g: torch.Tensor, q: int) -> float:
    est = C.c_double()
    _check(lib().nys_power_err_est(op.ref, f.h, _ptr(g), q, C.byref(est), _stream()),
           "nys_power_err_est")
    return est.value


def timing_start(max_products: int = 8192) -> None:
    """Start CUDA-event timing of the FP32 operator products (diagnostics)."""
    f = lib().nys_timing_start
    if f.argtypes is None:
        f.argtypes = [C.c_int32]
        f.restype = C.c_int32
    _check(f(int(max_products)), "nys_timing_start")


def timing_stop() -> tuple[float, int]:
    """Stop the timing; returns (summed ms, number of products timed)."""
    f = lib().nys_timing_stop
    if f.argtypes is None:
        f.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_int64)]
        f.restype = C.c_int32
    ms, cnt = C.c_double(), C.c_int64()
    _check(f(C.byref(ms), C.byref(cnt)), "nys_timing_stop")
    return ms.value, cnt.value


def nys_gram_matvec_f32_noalloc(op: Operator, mu: float, x: torch.Tensor,
                                y: torch.Tensor) -> None:
    """y = (X^T X + mu I) x (FP32) with no device allocation inside the call.

    For callers that cannot allocate device memory while it runs: the caller
    provides x and y (float32 CUDA tensors of length n); the library's scratch
    is a fixed 4 MiB device array shared by every call (calls that overlap on
    the GPU race).  Raises NysError (NYS_ERR_ARG) for shapes beyond its limit."""
    L = lib()
    f = L.nys_gram_matvec_f32_noalloc
    if f.argtypes is None:
        f.argtypes = [C.POINTER(_Operator), C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]
        f.restype = C.c_int32
    if x.dtype != torch.float32 or y.dtype != torch.float32:
        raise ValueError("x and y must be float32")
    _check(f(op.ref, float(mu), _ptr(x), _ptr(y), _stream()), "nys_gram_matvec_f32_noalloc")


def nys_rbf_cross_matvec(targets: torch.Tensor, points: torch.Tensor, sigma: float,
                         v: torch.Tensor, kind: int = 0) -> torch.Tensor:
    """K(targets, points) v (kind 0) or dK/dsigma v (kind 1), FP64 ([nvec][n] or [n])."""
    vv = v if v.dim() == 2 else v[None]
    nt, d = targets.shape
    n = points.shape[0]
    out = torch.empty((vv.shape[0], nt), dtype=torch.float64, device=v.device)
    _check(lib().nys_rbf_cross_matvec(_ptr(targets), nt, targets.stride(0), _ptr(points), n,
                                      points.stride(0), d, float(sigma), vv.shape[0], _ptr(vv),
                                      _ptr(out), kind, _stream()), "nys_rbf_cross_matvec")
    return out if v.dim() == 2 else out[0]


# stream identifiers of the library's own draws (NYS_STREAM_* in the header)
NYS_STREAM_OMEGA = 0x4F6D656761
NYS_STREAM_ADAPTIVE = 0x4164610000
NYS_STREAM_ESTIMATE = 0x4573740000


def nys_philox4x32_10(ctr: torch.Tensor, key: torch.Tensor) -> torch.Tensor:
    """Philox4x32-10 blocks: ctr [count, 4] and key [count, 2] int32 CUDA
    tensors holding uint32 bit patterns; returns [count, 4] int32 (bits)."""
    f = lib().nys_philox4x32_10
    if f.argtypes is None:
        f.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
        f.restype = C.c_int32
    if ctr.dtype != torch.int32 or key.dtype != torch.int32:
        raise ValueError("ctr and key must be int32 tensors of uint32 bit patterns")
    ctr, key = ctr.contiguous(), key.contiguous()
    count = ctr.shape[0]
    assert ctr.shape == (count, 4) and key.shape == (count, 2)
    out = torch.empty((count, 4), dtype=torch.int32, device=ctr.device)
    _check(f(_ptr(ctr), _ptr(key), count, _ptr(out), _stream()), "nys_philox4x32_10")
    return out


def nys_random_stream(seed: int, stream_id: int, first: int, count: int, words: bool = True,
                      gauss: bool = True, device=None):
    """Elements [first, first + count) of the library's random stream: the raw
    words (int32 tensor of uint32 bit patterns) and the Box-Muller values
    (float64 tensor); either is None when not asked for."""
    f = lib().nys_random_stream
    if f.argtypes is None:
        f.argtypes = [C.c_uint64, C.c_uint64, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p,
                      C.c_void_p]
        f.restype = C.c_int32
    dev = device or torch.device("cuda", torch.cuda.current_device())
    w = torch.empty(count, dtype=torch.int32, device=dev) if words else None
    g = torch.empty(count, dtype=torch.float64, device=dev) if gauss else None
    _check(f(seed, stream_id, first, count, _ptr(w), _ptr(g), _stream()), "nys_random_stream")
    return w, g


def nys_krr_validation(points: torch.Tensor, vpoints: torch.Tensor, sigma: float,
                       alpha: torch.Tensor, yv: torch.Tensor):
    """KRR validation objective: returns (loss, g, ktg) with loss the mean
    squared error of K_v alpha against yv (host float), g = dL/dpred and
    ktg = K_v^T g (FP64 CUDA tensors)."""
    f = lib().nys_krr_validation
    if f.argtypes is None:
        vp, i64 = C.c_void_p, C.c_int64
        f.argtypes = [vp, i64, i64, vp, i64, i64, i64, C.c_double, vp, vp, C.POINTER(C.c_double),
                      vp, vp, vp]
        f.restype = C.c_int32
    n, d = points.shape
    m = vpoints.shape[0]
    g = torch.empty(m, dtype=torch.float64, device=alpha.device)
    ktg = torch.empty(n, dtype=torch.float64, device=alpha.device)
    loss = C.c_double()
    _check(f(_ptr(points), n, points.stride(0), _ptr(vpoints), m, vpoints.stride(0), d,
             float(sigma), _ptr(alpha), _ptr(yv), C.byref(loss), _ptr(g), _ptr(ktg), _stream()),
           "nys_krr_validation")
    return loss.value, g, ktg


def nys_krr_gradients(points: torch.Tensor, vpoints: torch.Tensor | None, sigma: float,
                      alpha: torch.Tensor, lam: torch.Tensor, g: torch.Tensor | None):
    """(dL/dmu, dL/dsigma) of the KRR objective from the training solution
    alpha and the adjoint solution lam (see nys_krr_gradients in the header)."""
    f = lib().nys_krr_gradients
    if f.argtypes is None:
        vp, i64 = C.c_void_p, C.c_int64
        f.argtypes = [vp, i64, i64, vp, i64, i64, i64, C.c_double, vp, vp, vp,
                      C.POINTER(C.c_double), vp]
        f.restype = C.c_int32
    n, d = points.shape
    m = vpoints.shape[0] if vpoints is not None else 0
    ldv = vpoints.stride(0) if vpoints is not None else 0
    out = (C.c_double * 2)()
    _check(f(_ptr(points), n, points.stride(0), _ptr(vpoints), m, ldv, d, float(sigma),
             _ptr(alpha), _ptr(lam), _ptr(g), out, _stream()), "nys_krr_gradients")
    return out[0], out[1]


UNIT_FP64_FMA, UNIT_FP32_FMA, UNIT_MUFU_EX2 = 0, 1, 2


def nys_unit_peak(unit: int) -> float:
    """Measured FLOP/s (FMA pipes) or operations/s (MUFU ex2) of the device."""
    f = lib().nys_unit_peak
    if f.argtypes is None:
        f.argtypes = [C.c_int32, C.POINTER(C.c_double), C.c_void_p]
        f.restype = C.c_int32
    out = C.c_double()
    _check(f(unit, C.byref(out), _stream()), "nys_unit_peak")
    return out.value
