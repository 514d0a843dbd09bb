"""ctypes binding of libmgclover (the C ABI in ``include/mgclover.h``).

Argument marshalling only: every computation runs in the CUDA library.  The
functions carry the C names; buffers may be numpy arrays (host memory,
``MG_HOST``) or torch tensors (CUDA tensors are passed as device pointers,
``MG_DEVICE``; CPU tensors as host pointers).  All buffers are complex128 and
C-contiguous in the layouts the header documents.

If ``libmgclover.so`` has not been built, loading raises: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmgclover.so")

MG_MAX_LEVELS = 4
# status
MG_OK, MG_ERR_ARG, MG_ERR_DIMS, MG_ERR_NV, MG_ERR_STATE = 0, -1, -2, -3, -4
MG_ERR_GS_BREAKDOWN, MG_ERR_SINGULAR_CLOVER, MG_ERR_NOT_CONVERGED, MG_ERR_NAN = -5, -6, -7, -8
MG_ERR_CUDA, MG_ERR_ALLOC = -9, -10
# where
MG_HOST, MG_DEVICE = 0, 1
# operators
MG_OP_D, MG_OP_DP, MG_OP_DR, MG_OP_BR, MG_OP_M, MG_OP_MINV, MG_OP_HOP, MG_OP_R, MG_OP_P, MG_OP_CYCLE, MG_OP_DR_DAG = range(11)
MG_FP64, MG_FP32 = 0, 1
MG_STORE_FP32, MG_STORE_FP16, MG_STORE_BF16 = 0, 1, 2
MG_MODE_MG, MG_MODE_EO_GCR, MG_MODE_BICGSTAB, MG_MODE_CGNR, MG_MODE_BICGSTAB_MP = range(5)
MG_COARSE_DP, MG_COARSE_D = 0, 1
MG_FORCE_SU3, MG_FORCE_WIRTINGER, MG_FORCE_FP32 = 0, 1, 16

MG_KERNEL_DSLASH_CLOVER, MG_KERNEL_DSLASH_XPAY, MG_KERNEL_DR, MG_KERNEL_COARSE_DR, MG_KERNEL_RESTRICT, MG_KERNEL_PROLONG = range(6)

EXPORTED = ["mg_strerror", "mg_last_error", "mg_default_params", "mg_create", "mg_destroy", "mg_load_gauge",
            "mg_set_clover", "mg_set_clover_aniso", "mg_set_params", "mg_get_params", "mg_setup", "mg_set_null_vectors", "mg_get_null_vectors",
            "mg_get_coarse_links", "mg_save_setup", "mg_load_setup", "mg_update_mass", "mg_adapt_setup", "mg_solve", "mg_solve_batch",
            "mg_solve_dagger", "mg_force", "mg_apply", "mg_apply_noalloc", "mg_benchmark_kernel", "mg_benchmark_kernel_nrhs",
            "mg_benchmark_coarse_solve", "mg_benchmark_coarse_floor", "mg_benchmark_fma",
            "mg_level_info"]


class mg_params(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int),
                ("block", (ctypes.c_int * 4) * MG_MAX_LEVELS),
                ("nv", ctypes.c_int * MG_MAX_LEVELS),
                ("setup_iters", ctypes.c_int),
                ("setup_inner", ctypes.c_int),
                ("setup_rq_tol", ctypes.c_double),
                ("nu_pre", ctypes.c_int),
                ("nu_post", ctypes.c_int),
                ("tol_coarse", ctypes.c_double),
                ("maxit_coarse", ctypes.c_int),
                ("restart_coarse", ctypes.c_int),
                ("restart_fine", ctypes.c_int),
                ("maxit_fine", ctypes.c_int),
                ("storage", ctypes.c_int),
                ("coarse_op", ctypes.c_int),
                ("seed", ctypes.c_uint64),
                ("rhs_block", ctypes.c_int),
                ("cuda_graphs", ctypes.c_int),
                ("coarse_impl", ctypes.c_int),
                ("outer_prec", ctypes.c_int),
                ("level_timing", ctypes.c_int)]


class mg_setup_info(ctypes.Structure):
    _fields_ = [("setup_ms", ctypes.c_double),
                ("vectors", ctypes.c_int * MG_MAX_LEVELS),
                ("passes", ctypes.c_int * MG_MAX_LEVELS),
                ("rq_last", ctypes.c_double * MG_MAX_LEVELS),
                ("coarse_sites", ctypes.c_int * MG_MAX_LEVELS)]


class mg_solve_info(ctypes.Structure):
    _fields_ = [("outer_iterations", ctypes.c_int),
                ("restarts", ctypes.c_int),
                ("coarse_iterations", ctypes.c_longlong * MG_MAX_LEVELS),
                ("true_residual", ctypes.c_double),
                ("solve_ms", ctypes.c_double),
                ("dslash_launches", ctypes.c_longlong),
                ("kernel_launches", ctypes.c_longlong),
                ("level_ms", ctypes.c_double * MG_MAX_LEVELS)]


class MGError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {mg_strerror(status)} ({status}): {mg_last_error()}")


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1011_2775_gb300.build.build() "
                               "(nvcc, sm_103a); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.mg_strerror.restype = ctypes.c_char_p
        L.mg_strerror.argtypes = [ip]
        L.mg_last_error.restype = ctypes.c_char_p
        L.mg_last_error.argtypes = []
        sig = {
            "mg_default_params": [ctypes.POINTER(mg_params)],
            "mg_create": [ctypes.POINTER(vp), ctypes.POINTER(ip), ip, vp],
            "mg_destroy": [vp],
            "mg_load_gauge": [vp, vp, ip],
            "mg_set_clover": [vp, dp, dp],
            "mg_set_clover_aniso": [vp, ctypes.POINTER(dp), dp, dp, dp],
            "mg_set_params": [vp, ctypes.POINTER(mg_params)],
            "mg_get_params": [vp, ctypes.POINTER(mg_params)],
            "mg_setup": [vp, ctypes.POINTER(mg_setup_info)],
            "mg_set_null_vectors": [vp, ip, vp, ip, ip],
            "mg_get_null_vectors": [vp, ip, vp, ip, ip],
            "mg_solve": [vp, vp, vp, ip, dp, ip, ip, ctypes.POINTER(mg_solve_info)],
            "mg_solve_dagger": [vp, vp, vp, ip, dp, ip, ip, ctypes.POINTER(mg_solve_info)],
            "mg_force": [vp, vp, vp, vp, ip, ip],
            "mg_get_coarse_links": [vp, ip, vp, vp, ip],
            "mg_save_setup": [vp, ctypes.c_char_p],
            "mg_load_setup": [vp, ctypes.c_char_p, ctypes.POINTER(mg_setup_info)],
            "mg_update_mass": [vp, dp, ctypes.POINTER(mg_setup_info)],
            "mg_adapt_setup": [vp, ip, ip, ip, ctypes.POINTER(mg_setup_info)],
            "mg_solve_batch": [ctypes.POINTER(vp), ip, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(ip), dp,
                               ip, ctypes.POINTER(mg_solve_info)],
            "mg_apply": [vp, ip, ip, vp, vp, ip, ip, ip],
            "mg_benchmark_kernel": [vp, ip, ip, ip, ip, ctypes.POINTER(dp), ctypes.POINTER(dp)],
            "mg_apply_noalloc": [vp, ip, vp, vp, ip],
            "mg_benchmark_kernel_nrhs": [vp, ip, ip, ip, ip, ip, ctypes.POINTER(dp), ctypes.POINTER(dp)],
            "mg_benchmark_coarse_solve": [vp, ip, ip, ctypes.POINTER(dp), ctypes.POINTER(dp), ctypes.POINTER(dp)],
            "mg_benchmark_coarse_floor": [vp, ctypes.POINTER(dp), ctypes.POINTER(dp), ctypes.POINTER(dp),
                                          ctypes.POINTER(ip)],
            "mg_benchmark_fma": [ip, ip, ctypes.POINTER(dp)],
            "mg_level_info": [vp, ip, ctypes.POINTER(ip), ctypes.POINTER(ip)],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ip
        _lib = L
    return _lib


def mg_strerror(status: int) -> str:
    return lib().mg_strerror(int(status)).decode()


def mg_last_error() -> str:
    return lib().mg_last_error().decode()


def _check(status: int, where: str, allow=()):
    if status != MG_OK and status not in allow:
        raise MGError(status, where)
    return status


def _buf(x, writable=False):
    """(pointer, where) of a complex128 C-contiguous numpy array or torch tensor."""
    if isinstance(x, np.ndarray):
        if x.dtype != np.complex128 or not x.flags["C_CONTIGUOUS"]:
            raise TypeError("buffers must be C-contiguous complex128")
        if writable and not x.flags["WRITEABLE"]:
            raise TypeError("output buffer is read-only")
        return ctypes.c_void_p(x.ctypes.data), MG_HOST
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(x, torch.Tensor):
        if x.dtype != torch.complex128 or not x.is_contiguous():
            raise TypeError("tensors must be contiguous complex128")
        return ctypes.c_void_p(x.data_ptr()), (MG_DEVICE if x.is_cuda else MG_HOST)
    raise TypeError(f"unsupported buffer type {type(x)}")


# ----------------------------------------------------------------------------- C names
def mg_default_params() -> mg_params:
    p = mg_params()
    _check(lib().mg_default_params(ctypes.byref(p)), "mg_default_params")
    return p


def mg_create(dims, device: int = 0, stream: int | None = None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    d = (ctypes.c_int * 4)(*[int(v) for v in dims])
    _check(lib().mg_create(ctypes.byref(h), d, int(device), ctypes.c_void_p(stream or 0)), "mg_create")
    return h


def mg_destroy(ctx) -> None:
    _check(lib().mg_destroy(ctx), "mg_destroy")


def mg_load_gauge(ctx, U) -> None:
    p, w = _buf(U)
    _check(lib().mg_load_gauge(ctx, p, w), "mg_load_gauge")


def mg_set_clover(ctx, csw: float, m0: float) -> None:
    _check(lib().mg_set_clover(ctx, float(csw), float(m0)), "mg_set_clover")


def mg_set_clover_aniso(ctx, weights, csw_s: float, csw_t: float, m0: float) -> None:
    w = (ctypes.c_double * 4)(*[float(x) for x in weights])
    _check(lib().mg_set_clover_aniso(ctx, w, float(csw_s), float(csw_t), float(m0)), "mg_set_clover_aniso")


def mg_set_params(ctx, params: mg_params) -> None:
    _check(lib().mg_set_params(ctx, ctypes.byref(params)), "mg_set_params")


def mg_get_params(ctx) -> mg_params:
    p = mg_params()
    _check(lib().mg_get_params(ctx, ctypes.byref(p)), "mg_get_params")
    return p


def mg_setup(ctx) -> mg_setup_info:
    info = mg_setup_info()
    _check(lib().mg_setup(ctx, ctypes.byref(info)), "mg_setup")
    return info


def mg_set_null_vectors(ctx, level: int, V, nv: int) -> None:
    p, w = _buf(V)
    _check(lib().mg_set_null_vectors(ctx, int(level), p, int(nv), w), "mg_set_null_vectors")


def mg_get_null_vectors(ctx, level: int, V, nv: int) -> None:
    p, w = _buf(V, writable=True)
    _check(lib().mg_get_null_vectors(ctx, int(level), p, int(nv), w), "mg_get_null_vectors")


def mg_solve(ctx, psi, eta, nrhs: int, tol: float, mode: int = MG_MODE_MG, allow_not_converged=False):
    """Returns ``(status, mg_solve_info)``."""
    pp, wp = _buf(psi, writable=True)
    pe, we = _buf(eta)
    if wp != we:
        raise TypeError("psi and eta must both be host or both be device buffers")
    info = mg_solve_info()
    st = lib().mg_solve(ctx, pp, pe, int(nrhs), float(tol), int(mode), wp, ctypes.byref(info))
    _check(st, "mg_solve", allow=(MG_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    return st, info


def mg_solve_batch(ctxs, psis, etas, nrhs, tol: float, allow_not_converged=False):
    """Solves several lattices together (one context each); returns ``(status, [mg_solve_info])``."""
    n = len(ctxs)
    bufs = [_buf(p, writable=True) for p in psis]
    ebufs = [_buf(e) for e in etas]
    wheres = {w for _, w in bufs} | {w for _, w in ebufs}
    if len(wheres) != 1:
        raise TypeError("all buffers must be host or all device buffers")
    c_ctx = (ctypes.c_void_p * n)(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in ctxs])
    c_psi = (ctypes.c_void_p * n)(*[p.value for p, _ in bufs])
    c_eta = (ctypes.c_void_p * n)(*[p.value for p, _ in ebufs])
    c_nrhs = (ctypes.c_int * n)(*[int(k) for k in nrhs])
    infos = (mg_solve_info * n)()
    st = lib().mg_solve_batch(c_ctx, n, c_psi, c_eta, c_nrhs, float(tol), wheres.pop(), infos)
    _check(st, "mg_solve_batch", allow=(MG_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    return st, list(infos)


def mg_solve_dagger(ctx, psi, eta, nrhs: int, tol: float, mode: int = MG_MODE_MG, allow_not_converged=False):
    """Solves ``D^dag psi = eta``; returns ``(status, mg_solve_info)``."""
    pp, wp = _buf(psi, writable=True)
    pe, we = _buf(eta)
    if wp != we:
        raise TypeError("psi and eta must both be host or both be device buffers")
    info = mg_solve_info()
    st = lib().mg_solve_dagger(ctx, pp, pe, int(nrhs), float(tol), int(mode), wp, ctypes.byref(info))
    _check(st, "mg_solve_dagger", allow=(MG_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    return st, info


def mg_save_setup(ctx, path: str) -> None:
    _check(lib().mg_save_setup(ctx, os.fsencode(path)), "mg_save_setup")


def mg_load_setup(ctx, path: str) -> mg_setup_info:
    info = mg_setup_info()
    _check(lib().mg_load_setup(ctx, os.fsencode(path), ctypes.byref(info)), "mg_load_setup")
    return info


def mg_update_mass(ctx, m0: float) -> mg_setup_info:
    info = mg_setup_info()
    _check(lib().mg_update_mass(ctx, float(m0), ctypes.byref(info)), "mg_update_mass")
    return info


def mg_adapt_setup(ctx, passes: int = 1, relax: int = 2, transfers: int = 1) -> mg_setup_info:
    info = mg_setup_info()
    _check(lib().mg_adapt_setup(ctx, int(passes), int(relax), int(transfers), ctypes.byref(info)), "mg_adapt_setup")
    return info


def mg_get_coarse_links(ctx, level: int, Y, X) -> None:
    py, wy = _buf(Y, writable=True)
    px, wx = _buf(X, writable=True)
    if wy != wx:
        raise TypeError("Y and X must both be host or both be device buffers")
    _check(lib().mg_get_coarse_links(ctx, int(level), py, px, wy), "mg_get_coarse_links")


def mg_force(ctx, F, lam, psi, kind: int = MG_FORCE_SU3) -> None:
    pf, wf = _buf(F, writable=True)
    pl, wl = _buf(lam)
    pp, wp = _buf(psi)
    if not (wf == wl == wp):
        raise TypeError("F, lambda and psi must all be host or all be device buffers")
    _check(lib().mg_force(ctx, pf, pl, pp, int(kind), wf), "mg_force")


def mg_apply(ctx, op: int, level: int, out, x, nrhs: int = 1, prec: int = MG_FP64) -> None:
    po, wo = _buf(out, writable=True)
    pi, wi = _buf(x)
    if wo != wi:
        raise TypeError("in and out must both be host or both be device buffers")
    _check(lib().mg_apply(ctx, int(op), int(level), po, pi, int(nrhs), int(prec), wo), "mg_apply")


def mg_apply_noalloc(ctx, op: int, out, x, prec: int = MG_FP64) -> None:
    """Allocation-free fine-level operator; ``out`` and ``x`` must be device buffers."""
    po, wo = _buf(out, writable=True)
    pi, wi = _buf(x)
    if wo != MG_DEVICE or wi != MG_DEVICE:
        raise TypeError("mg_apply_noalloc takes device buffers only")
    _check(lib().mg_apply_noalloc(ctx, int(op), po, pi, int(prec)), "mg_apply_noalloc")


def mg_benchmark_kernel(ctx, kernel: int, prec: int = MG_FP32, warmup: int = 5, iters: int = 50):
    """Returns ``(avg_ms_per_launch, algorithmic_bytes_per_launch)``."""
    ms, by = ctypes.c_double(), ctypes.c_double()
    _check(lib().mg_benchmark_kernel(ctx, int(kernel), int(prec), int(warmup), int(iters), ctypes.byref(ms),
                                     ctypes.byref(by)), "mg_benchmark_kernel")
    return ms.value, by.value


def mg_benchmark_kernel_nrhs(ctx, kernel: int, prec: int = MG_FP32, nrhs: int = 1, warmup: int = 5, iters: int = 50):
    """Returns ``(avg_ms_per_launch, algorithmic_bytes_per_launch)`` for nrhs right-hand sides."""
    ms, by = ctypes.c_double(), ctypes.c_double()
    _check(lib().mg_benchmark_kernel_nrhs(ctx, int(kernel), int(prec), int(nrhs), int(warmup), int(iters),
                                          ctypes.byref(ms), ctypes.byref(by)), "mg_benchmark_kernel_nrhs")
    return ms.value, by.value


def mg_benchmark_coarse_floor(ctx):
    """Returns ``(barrier_us, stream_us, stream_bytes, grid)``: one grid barrier and one iteration's link
    stream of the coarsest-level GCR, each timed alone on the streamed solver's grid."""
    b, st, by, g = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    _check(lib().mg_benchmark_coarse_floor(ctx, ctypes.byref(b), ctypes.byref(st), ctypes.byref(by), ctypes.byref(g)),
           "mg_benchmark_coarse_floor")
    return b.value, st.value, by.value, g.value


def mg_benchmark_coarse_solve(ctx, warmup: int = 3, iters: int = 20):
    """Returns ``(avg_ms_per_solve, link_bytes_per_solve, gcr_iterations_per_solve)`` of the coarsest-level solve."""
    ms, by, it = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().mg_benchmark_coarse_solve(ctx, int(warmup), int(iters), ctypes.byref(ms), ctypes.byref(by),
                                           ctypes.byref(it)), "mg_benchmark_coarse_solve")
    return ms.value, by.value, it.value


def mg_benchmark_fma(device: int = 0, prec: int = MG_FP32) -> float:
    """Measured CUDA-core FMA throughput of `device` in TFLOP/s."""
    t = ctypes.c_double()
    _check(lib().mg_benchmark_fma(int(device), int(prec), ctypes.byref(t)), "mg_benchmark_fma")
    return t.value


def mg_level_info(ctx, level: int):
    d = (ctypes.c_int * 4)()
    n = ctypes.c_int()
    _check(lib().mg_level_info(ctx, int(level), d, ctypes.byref(n)), "mg_level_info")
    return tuple(d), n.value
