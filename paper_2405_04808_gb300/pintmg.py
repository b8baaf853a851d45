"""ctypes binding of the pintmg C ABI (include/pintmg.h).

Argument marshalling only: every step of the solver runs in the CUDA library.
The functions keep the ABI's names (mg_setup, mg_vcycle, fgmres_solve,
mg_destroy, mg_status_string).  Device vectors are passed as raw pointers
(e.g. ``tensor.data_ptr()``), streams as ``torch.cuda.Stream.cuda_stream``.
The library must have been built (``python -m paper_2405_04808_gb300.build``);
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB_PATH

MG_OK = 0
MG_NOT_CONVERGED = 1
MG_ERR_ARG = -1
MG_ERR_SINGULAR = -2
MG_ERR_BREAKDOWN = -3
MG_ERR_CUDA = -4
MG_ERR_OOM = -5
MG_ERR_NONFINITE = -7
MG_ERR_UNSUPPORTED = -8

MG_LAYOUT_DENSE = 0
MG_LAYOUT_TRIDIAG = 1
MG_PRECISION_FP64 = 0
MG_PRECISION_FP32 = 1
COARSE_PRECOND = {"sgs": 0, "jacobi": 1, "fgs": 2, "bgs": 3}

#: every symbol include/pintmg.h declares
EXPORTED = ("mg_default_options", "mg_setup", "mg_vcycle", "fgmres_solve", "fgmres_solve_batched",
            "mg_vector_length",
            "mg_launch_count", "mg_profile_enable", "mg_profile_read", "mg_true_residual_noalloc",
            "mg_destroy", "mg_status_string", "mg_last_cuda_error")

_dp = ctypes.POINTER(ctypes.c_double)


class MGProblem(ctypes.Structure):
    _fields_ = [("layout", ctypes.c_int), ("n", ctypes.c_int), ("p", ctypes.c_int), ("q", ctypes.c_int),
                ("theta", ctypes.c_double), ("gamma", ctypes.c_double), ("jz_const", ctypes.c_int),
                ("M", _dp), ("Ju_cur", _dp), ("Ju_prev", _dp), ("Jz_cur", _dp), ("Jz_prev", _dp)]


class MGOptions(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("nu_pre", ctypes.c_int), ("nu_post", ctypes.c_int),
                ("coarse_rtol", ctypes.c_double), ("coarse_maxit", ctypes.c_int),
                ("coarse_fixed_iters", ctypes.c_int), ("end_rule", ctypes.c_int), ("precision", ctypes.c_int),
                ("omega", ctypes.c_double), ("coarse_precond", ctypes.c_int), ("device_loops", ctypes.c_int)]


class MGSolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("vcycles", ctypes.c_int),
                ("coarse_iters", ctypes.c_int),
                ("relres", ctypes.c_double), ("true_relres", ctypes.c_double)]


class PintmgError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {mg_status_string(code)} ({code})")
        self.code = code


_lib = None


def lib():
    """Load libpintmg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libpintmg.so not built at {LIB_PATH}; run python -m paper_2405_04808_gb300.build")
        L = ctypes.CDLL(LIB_PATH)
        L.mg_default_options.argtypes = [ctypes.POINTER(MGOptions)]
        L.mg_default_options.restype = None
        L.mg_setup.argtypes = [ctypes.POINTER(MGProblem), ctypes.POINTER(MGOptions), ctypes.c_void_p,
                               ctypes.POINTER(ctypes.c_void_p)]
        L.mg_setup.restype = ctypes.c_int
        L.mg_vcycle.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.mg_vcycle.restype = ctypes.c_int
        L.fgmres_solve.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                   ctypes.c_int, ctypes.c_int, ctypes.POINTER(MGSolveInfo), ctypes.c_void_p]
        L.fgmres_solve.restype = ctypes.c_int
        L.fgmres_solve_batched.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                           ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(MGSolveInfo), ctypes.c_void_p]
        L.fgmres_solve_batched.restype = ctypes.c_int
        L.mg_vector_length.argtypes = [ctypes.c_void_p]
        L.mg_vector_length.restype = ctypes.c_longlong
        L.mg_launch_count.argtypes = [ctypes.c_void_p]
        L.mg_launch_count.restype = ctypes.c_longlong
        L.mg_profile_enable.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.mg_profile_enable.restype = ctypes.c_int
        L.mg_profile_read.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p),
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong),
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        L.mg_profile_read.restype = ctypes.c_int
        L.mg_true_residual_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_void_p]
        L.mg_true_residual_noalloc.restype = ctypes.c_int
        L.mg_destroy.argtypes = [ctypes.c_void_p]
        L.mg_destroy.restype = None
        L.mg_status_string.argtypes = [ctypes.c_int]
        L.mg_status_string.restype = ctypes.c_char_p
        L.mg_last_cuda_error.argtypes = []
        L.mg_last_cuda_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def mg_status_string(code: int) -> str:
    return lib().mg_status_string(int(code)).decode()


def mg_default_options() -> MGOptions:
    o = MGOptions()
    lib().mg_default_options(ctypes.byref(o))
    return o


def _c(arr):
    a = np.ascontiguousarray(arr, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def mg_setup(prob, levels=2, nu_pre=1, nu_post=1, coarse_rtol=1e-3, coarse_maxit=50,
             coarse_fixed_iters=0, end_rule=0, precision=MG_PRECISION_FP64, omega=1.0, coarse_precond="sgs",
             device_loops=True, stream=0):
    """Build the device hierarchy for a workloads.Problem; returns an opaque handle (int)."""
    keep = []
    P = MGProblem()
    P.layout = MG_LAYOUT_TRIDIAG if prob.kind == "tridiag" else MG_LAYOUT_DENSE
    P.n, P.p, P.q = prob.n, prob.p, prob.q
    P.theta, P.gamma = prob.theta, prob.gamma
    P.jz_const = 1 if prob.jz_const else 0
    for name in ("M", "Ju_cur", "Ju_prev", "Jz_cur", "Jz_prev"):
        a, ptr = _c(getattr(prob, name))
        keep.append(a)
        setattr(P, name, ptr)
    o = MGOptions(levels, nu_pre, nu_post, coarse_rtol, coarse_maxit, coarse_fixed_iters, end_rule, precision, omega,
                  COARSE_PRECOND[coarse_precond], 1 if device_loops else 0)
    h = ctypes.c_void_p()
    code = lib().mg_setup(ctypes.byref(P), ctypes.byref(o), ctypes.c_void_p(stream), ctypes.byref(h))
    if code != MG_OK:
        raise PintmgError(code, "mg_setup")
    return h.value


def mg_vcycle(h, r_ptr: int, y_ptr: int, stream: int = 0) -> int:
    return lib().mg_vcycle(ctypes.c_void_p(h), ctypes.c_void_p(r_ptr), ctypes.c_void_p(y_ptr),
                           ctypes.c_void_p(stream))


def fgmres_solve(h, b_ptr: int, x_ptr: int, rtol: float, maxit: int = 500, restart: int = 100,
                 stream: int = 0):
    """Returns (status, MGSolveInfo).  b_ptr / x_ptr may be host or device addresses."""
    info = MGSolveInfo()
    code = lib().fgmres_solve(ctypes.c_void_p(h), ctypes.c_void_p(b_ptr), ctypes.c_void_p(x_ptr),
                              float(rtol), int(maxit), int(restart), ctypes.byref(info), ctypes.c_void_p(stream))
    return code, info


def fgmres_solve_batched(handles, b_ptrs, x_ptrs, rtol: float, maxit: int = 500, restart: int = 100,
                         stream: int = 0):
    """Solve len(handles) systems in one graph launch; returns (status, [MGSolveInfo])."""
    k = len(handles)
    H = (ctypes.c_void_p * k)(*handles)
    B = (ctypes.c_void_p * k)(*b_ptrs)
    X = (ctypes.c_void_p * k)(*x_ptrs)
    infos = (MGSolveInfo * k)()
    code = lib().fgmres_solve_batched(H, k, B, X, float(rtol), int(maxit), int(restart), infos,
                                      ctypes.c_void_p(stream))
    return code, list(infos)


def mg_vector_length(h) -> int:
    return int(lib().mg_vector_length(ctypes.c_void_p(h)))


def mg_launch_count(h) -> int:
    return int(lib().mg_launch_count(ctypes.c_void_p(h)))


PROFILE_ALL = 0xFFFF
PROFILE_CATEGORIES = ("block_solve", "apply", "residual_restrict", "prolong_add", "sgs_chain", "multidot",
                      "axpy_scale", "arnoldi_scalar", "convert", "setup")


def mg_profile_enable(h, mask: int = PROFILE_ALL) -> None:
    """Time the kernel categories whose bits are set in mask (0 = off)."""
    code = lib().mg_profile_enable(ctypes.c_void_p(h), int(mask))
    if code != MG_OK:
        raise PintmgError(code, "mg_profile_enable")


def mg_profile_read(h) -> dict:
    """{category: (total_ms, launches, algorithmic_bytes, algorithmic_flops)} since mg_profile_enable."""
    k = 16
    names = (ctypes.c_char_p * k)()
    ms = (ctypes.c_double * k)()
    cnt = (ctypes.c_longlong * k)()
    by = (ctypes.c_double * k)()
    fl = (ctypes.c_double * k)()
    n = lib().mg_profile_read(ctypes.c_void_p(h), k, names, ms, cnt, by, fl)
    if n < 0:
        raise PintmgError(n, "mg_profile_read")
    return {names[i].decode(): (ms[i], int(cnt[i]), by[i], fl[i]) for i in range(min(n, k))}


def mg_true_residual_noalloc(h, b_ptr: int, x_ptr: int, out_ptr: int, stream: int = 0) -> int:
    """||b - A x|| and ||b - A x|| / ||b|| into out_ptr[0:2] (device), allocating nothing."""
    return lib().mg_true_residual_noalloc(ctypes.c_void_p(h), ctypes.c_void_p(b_ptr), ctypes.c_void_p(x_ptr),
                                          ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream))


def mg_destroy(h) -> None:
    if h:
        lib().mg_destroy(ctypes.c_void_p(h))


def mg_last_cuda_error() -> str:
    return lib().mg_last_cuda_error().decode()
