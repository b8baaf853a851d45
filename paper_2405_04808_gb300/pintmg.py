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
MG_ERR_TIMEOUT = -6
MG_ERR_NONFINITE = -7
MG_ERR_UNSUPPORTED = -8

MG_LAYOUT_DENSE = 0
MG_LAYOUT_TRIDIAG = 1
MG_PRECISION_FP64 = 0
MG_PRECISION_FP32 = 1
MG_PRECISION_FP32_SMOOTH = 2
MG_PRECISION_BF16_BANDS = 3
COARSE_PRECOND = {"sgs": 0, "jacobi": 1, "fgs": 2, "bgs": 3}
#: storage of the FGMRES basis (mg_krylov_basis)
KRYLOV_BASIS = {"fp64": 0, "pair": 1, "pair_dcgs2": 2}
#: residual restriction of the V-cycle (mg_restrict_rule)
RESTRICT = {"inject": 0, "transpose": 1}

#: every symbol include/pintmg.h declares
EXPORTED = ("mg_default_options", "mg_setup", "mg_vcycle", "fgmres_solve", "fgmres_solve_batched",
            "mg_vector_length",
            "mg_launch_count", "mg_graph_launches", "mg_probe_fma", "mg_profile_enable", "mg_profile_read", "mg_true_residual_noalloc",
            "mg_level_info", "mg_range_sweep", "mg_range_residual", "mg_range_restrict", "mg_range_prolong",
            "mg_coarse_solve", "mg_range_dots", "mg_range_axpy", "mg_range_scale",
            "mg_net_param_count", "mg_net_create", "mg_net_set_params", "mg_net_get_params", "mg_net_get_grad",
            "mg_net_forward", "mg_net_loss_grad", "mg_net_set_metric", "mg_net_adam_step", "mg_net_train",
            "mg_net_destroy",
            "mg_attach_coarse_net", "mg_record_coarse", "mg_recorded_pairs", "mg_coarse_shape", "mg_autotune",
            "mg_block_mapping", "mg_jacobi_radius",
            "mg_destroy", "mg_status_string", "mg_last_cuda_error")

_dp = ctypes.POINTER(ctypes.c_double)


class MGProblem(ctypes.Structure):
    _fields_ = [("layout", ctypes.c_int), ("n", ctypes.c_int), ("p", ctypes.c_int), ("q", ctypes.c_int),
                ("theta", ctypes.c_double), ("gamma", ctypes.c_double), ("jz_const", ctypes.c_int),
                ("M", _dp), ("Ju_cur", _dp), ("Ju_prev", _dp), ("Jz_cur", _dp), ("Jz_prev", _dp),
                ("separable", ctypes.c_int)]


class MGOptions(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("nu_pre", ctypes.c_int), ("nu_post", ctypes.c_int),
                ("coarse_rtol", ctypes.c_double), ("coarse_maxit", ctypes.c_int),
                ("coarse_fixed_iters", ctypes.c_int), ("end_rule", ctypes.c_int), ("precision", ctypes.c_int),
                ("omega", ctypes.c_double), ("coarse_precond", ctypes.c_int), ("device_loops", ctypes.c_int),
                ("krylov_basis", ctypes.c_int), ("restrict_rule", ctypes.c_int)]


class MGSolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("vcycles", ctypes.c_int),
                ("coarse_iters", ctypes.c_int),
                ("relres", ctypes.c_double), ("true_relres", ctypes.c_double), ("coarse_learned", ctypes.c_int)]


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
        L.mg_graph_launches.argtypes = [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_longlong)] * 3
        L.mg_graph_launches.restype = ctypes.c_int
        L.mg_profile_enable.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.mg_profile_enable.restype = ctypes.c_int
        L.mg_profile_read.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p),
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong),
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        L.mg_profile_read.restype = ctypes.c_int
        L.mg_true_residual_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_void_p]
        L.mg_true_residual_noalloc.restype = ctypes.c_int
        vp, ci, cf = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
        cl, cd = ctypes.c_longlong, ctypes.c_double
        fp = ctypes.POINTER(ctypes.c_float)
        for name, args, res in (
                ("mg_net_param_count", [], ctypes.c_longlong),
                ("mg_net_create", [fp, ctypes.POINTER(vp)], ci),
                ("mg_net_set_params", [vp, fp], ci),
                ("mg_net_get_params", [vp, fp], ci),
                ("mg_net_get_grad", [vp, fp], ci),
                ("mg_net_forward", [vp, vp, ci, ci, ci, vp, ci, vp], ci),
                ("mg_net_loss_grad", [vp, vp, vp, ci, ci, ci, fp, vp], ci),
                ("mg_net_adam_step", [vp, cf, cf, cf, cf, vp], ci),
                ("mg_net_train", [vp, vp, vp, ci, ci, ci, ci, ci, cf, ctypes.c_ulonglong, ci, fp, vp], ci),
                ("mg_net_destroy", [vp], None),
                ("mg_net_set_metric", [vp, vp], ci),
                ("mg_attach_coarse_net", [vp, vp, ctypes.c_double, ci], ci),
                ("mg_record_coarse", [vp, vp, vp, ci], ci),
                ("mg_recorded_pairs", [vp], ci),
                ("mg_coarse_shape", [vp, ctypes.POINTER(ci), ctypes.POINTER(ci)], ci),
                ("mg_autotune", [vp, ctypes.POINTER(ci), ctypes.POINTER(ci), vp], ci),
                ("mg_block_mapping", [vp, ci], ci),
                ("mg_jacobi_radius", [vp, ci, ci, ctypes.POINTER(ctypes.c_double), vp], ci),
                ("mg_probe_fma", [ci, ci, ci, vp, vp], ci),
                ("mg_level_info", [vp, ci, ctypes.POINTER(ci), ctypes.POINTER(ctypes.c_longlong)], ci),
                ("mg_range_sweep", [vp, ci, ci, ci, vp, vp, vp, vp], ci),
                ("mg_range_residual", [vp, ci, ci, ci, vp, vp, vp, vp], ci),
                ("mg_range_restrict", [vp, ci, ci, ci, vp, vp, vp], ci),
                ("mg_range_prolong", [vp, ci, ci, ci, vp, vp, vp], ci),
                ("mg_coarse_solve", [vp, vp, vp, vp], ci),
                ("mg_range_dots", [vp, ci, ci, ci, vp, cl, ci, vp, vp, vp], ci),
                ("mg_range_axpy", [vp, ci, ci, ci, vp, cl, ci, vp, cd, vp, vp], ci),
                ("mg_range_scale", [vp, ci, ci, ci, vp, vp, vp, vp], ci)):
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
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
             device_loops=True, krylov_basis="fp64", restrict="inject", separable=True, stream=0):
    """Build the device hierarchy for a workloads.Problem; returns an opaque handle (int).
    krylov_basis: "fp64" (the plain method) or "pair" (FP32-pair basis with compensated dot products).
    restrict: "inject" (Sec. 5.3.1's variable formulas applied to the residual) or "transpose" (R = P^T).
    separable: the caller's assertion that d_u f does not depend on z and f is affine in z (true for both
    workloads), which the rediscretised coarse levels need."""
    keep = []
    P = MGProblem()
    P.layout = MG_LAYOUT_TRIDIAG if prob.kind == "tridiag" else MG_LAYOUT_DENSE
    P.n, P.p, P.q = prob.n, prob.p, prob.q
    P.theta, P.gamma = prob.theta, prob.gamma
    P.jz_const = 1 if prob.jz_const else 0
    P.separable = 1 if separable else 0
    for name in ("M", "Ju_cur", "Ju_prev", "Jz_cur", "Jz_prev"):
        a, ptr = _c(getattr(prob, name))
        keep.append(a)
        setattr(P, name, ptr)
    o = MGOptions(levels, nu_pre, nu_post, coarse_rtol, coarse_maxit, coarse_fixed_iters, end_rule, precision, omega,
                  COARSE_PRECOND[coarse_precond], 1 if device_loops else 0, KRYLOV_BASIS[krylov_basis],
                  RESTRICT[restrict])
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


def mg_graph_launches(h):
    """(status, fixed, per FGMRES iteration, per coarse GMRES iteration) kernel launches of the
    handle's captured solve graph."""
    out = [ctypes.c_longlong(0) for _ in range(3)]
    code = lib().mg_graph_launches(ctypes.c_void_p(h), *[ctypes.byref(o) for o in out])
    return (int(code),) + tuple(int(o.value) for o in out)


PROFILE_ALL = 0xFFFF
PROFILE_CATEGORIES = ("block_solve", "apply", "residual_restrict", "prolong_add", "sgs_chain", "multidot",
                      "axpy_scale", "arnoldi_scalar", "convert", "setup", "net_coarse", "pair_dot", "pair_axpy")


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


# --------------------------------------------------------------------------
# time-range operations (a V-cycle sharded by time: paper_2405_04808_gb300.timeshard)

def mg_level_info(h, level: int):
    """(n_l, vector length) of a level."""
    n, ln = ctypes.c_int(), ctypes.c_longlong()
    _check(lib().mg_level_info(ctypes.c_void_p(h), int(level), ctypes.byref(n), ctypes.byref(ln)), "mg_level_info")
    return n.value, ln.value


def mg_range_sweep(h, level, j0, j1, r_ptr, yold_ptr, y_ptr, stream=0):
    _check(lib().mg_range_sweep(ctypes.c_void_p(h), level, j0, j1, ctypes.c_void_p(r_ptr),
                                ctypes.c_void_p(yold_ptr or 0), ctypes.c_void_p(y_ptr), ctypes.c_void_p(stream)),
           "mg_range_sweep")


def mg_range_residual(h, level, j0, j1, y_ptr, b_ptr, r_ptr, stream=0):
    _check(lib().mg_range_residual(ctypes.c_void_p(h), level, j0, j1, ctypes.c_void_p(y_ptr), ctypes.c_void_p(b_ptr),
                                   ctypes.c_void_p(r_ptr), ctypes.c_void_p(stream)), "mg_range_residual")


def mg_range_dots(h, level, j0, j1, V_ptr, ldv, k, w_ptr, out_ptr, stream=0):
    _check(lib().mg_range_dots(ctypes.c_void_p(h), level, j0, j1, ctypes.c_void_p(V_ptr), ldv, k,
                               ctypes.c_void_p(w_ptr), ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream)),
           "mg_range_dots")


def mg_range_axpy(h, level, j0, j1, V_ptr, ldv, k, c_ptr, sign, w_ptr, stream=0):
    _check(lib().mg_range_axpy(ctypes.c_void_p(h), level, j0, j1, ctypes.c_void_p(V_ptr), ldv, k,
                               ctypes.c_void_p(c_ptr), float(sign), ctypes.c_void_p(w_ptr), ctypes.c_void_p(stream)),
           "mg_range_axpy")


def mg_range_scale(h, level, j0, j1, x_ptr, a_ptr, y_ptr, stream=0):
    _check(lib().mg_range_scale(ctypes.c_void_p(h), level, j0, j1, ctypes.c_void_p(x_ptr), ctypes.c_void_p(a_ptr),
                                ctypes.c_void_p(y_ptr), ctypes.c_void_p(stream)), "mg_range_scale")


def mg_range_restrict(h, level, j0, j1, r_ptr, rc_ptr, stream=0):
    _check(lib().mg_range_restrict(ctypes.c_void_p(h), level, j0, j1, ctypes.c_void_p(r_ptr), ctypes.c_void_p(rc_ptr),
                                   ctypes.c_void_p(stream)), "mg_range_restrict")


def mg_range_prolong(h, level, j0, j1, ec_ptr, y_ptr, stream=0):
    _check(lib().mg_range_prolong(ctypes.c_void_p(h), level, j0, j1, ctypes.c_void_p(ec_ptr), ctypes.c_void_p(y_ptr),
                                  ctypes.c_void_p(stream)), "mg_range_prolong")


def mg_coarse_solve(h, rc_ptr, yc_ptr, stream=0):
    _check(lib().mg_coarse_solve(ctypes.c_void_p(h), ctypes.c_void_p(rc_ptr), ctypes.c_void_p(yc_ptr),
                                 ctypes.c_void_p(stream)), "mg_coarse_solve")


#: threads per CTA and independent FMA chains per thread of mg_probe_fma
PROBE_THREADS = 256
PROBE_CHAINS = 8


def mg_probe_fma(precision: int, blocks: int, iters: int, sink_ptr: int, stream: int = 0) -> float:
    """Launch the FMA-rate probe; returns the floating-point operations the launch performs."""
    _check(lib().mg_probe_fma(int(precision), int(blocks), int(iters), ctypes.c_void_p(sink_ptr),
                              ctypes.c_void_p(stream)), "mg_probe_fma")
    return 2.0 * PROBE_CHAINS * iters * blocks * PROBE_THREADS


def mg_true_residual_noalloc(h, b_ptr: int, x_ptr: int, out_ptr: int, stream: int = 0) -> int:
    """||b - A x|| and ||b - A x|| / ||b|| into out_ptr[0:2] (device), allocating nothing."""
    return lib().mg_true_residual_noalloc(ctypes.c_void_p(h), ctypes.c_void_p(b_ptr), ctypes.c_void_p(x_ptr),
                                          ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream))


# --------------------------------------------------------------------------
# learned coarse-grid correction

def _check(code, what):
    if code != MG_OK:
        raise PintmgError(code, what)


def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def mg_net_param_count() -> int:
    return int(lib().mg_net_param_count())


def mg_net_create(init_params) -> int:
    """A network on the current device from mg_net_param_count() initial parameters (host array)."""
    p = np.ascontiguousarray(init_params, dtype=np.float32)
    if p.size != mg_net_param_count():
        raise PintmgError(MG_ERR_ARG, "mg_net_create")
    net = ctypes.c_void_p()
    _check(lib().mg_net_create(_fptr(p), ctypes.byref(net)), "mg_net_create")
    return net.value


def mg_net_set_params(net, params) -> None:
    p = np.ascontiguousarray(params, dtype=np.float32)
    if p.size != mg_net_param_count():
        raise PintmgError(MG_ERR_ARG, "mg_net_set_params")
    _check(lib().mg_net_set_params(ctypes.c_void_p(net), _fptr(p)), "mg_net_set_params")


def mg_net_get_params(net) -> np.ndarray:
    out = np.empty(mg_net_param_count(), dtype=np.float32)
    _check(lib().mg_net_get_params(ctypes.c_void_p(net), _fptr(out)), "mg_net_get_params")
    return out


def mg_net_get_grad(net) -> np.ndarray:
    out = np.empty(mg_net_param_count(), dtype=np.float32)
    _check(lib().mg_net_get_grad(ctypes.c_void_p(net), _fptr(out)), "mg_net_get_grad")
    return out


def mg_net_forward(net, x_ptr: int, batch: int, T: int, X: int, y_ptr: int, bf16: bool = False,
                   stream: int = 0) -> None:
    _check(lib().mg_net_forward(ctypes.c_void_p(net), ctypes.c_void_p(x_ptr), batch, T, X, ctypes.c_void_p(y_ptr),
                                1 if bf16 else 0, ctypes.c_void_p(stream)), "mg_net_forward")


def mg_net_loss_grad(net, x_ptr: int, t_ptr: int, batch: int, T: int, X: int, stream: int = 0) -> float:
    loss = ctypes.c_float()
    _check(lib().mg_net_loss_grad(ctypes.c_void_p(net), ctypes.c_void_p(x_ptr), ctypes.c_void_p(t_ptr), batch, T, X,
                                  ctypes.byref(loss), ctypes.c_void_p(stream)), "mg_net_loss_grad")
    return float(loss.value)


def mg_net_adam_step(net, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
                     stream: int = 0) -> None:
    _check(lib().mg_net_adam_step(ctypes.c_void_p(net), lr, beta1, beta2, eps, ctypes.c_void_p(stream)),
           "mg_net_adam_step")


def mg_net_train(net, x_ptr: int, y_ptr: int, count: int, T: int, X: int, batch: int, epochs: int, lr: float,
                 seed: int, normalize: bool = True, stream: int = 0) -> np.ndarray:
    """Minibatch Adam over `count` device samples; returns each epoch's mean loss."""
    losses = np.zeros(max(epochs, 1), dtype=np.float32)
    _check(lib().mg_net_train(ctypes.c_void_p(net), ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr), count, T, X,
                              batch, epochs, lr, ctypes.c_ulonglong(seed), 1 if normalize else 0, _fptr(losses),
                              ctypes.c_void_p(stream)), "mg_net_train")
    return losses[:epochs]


def mg_net_set_metric(net, h) -> None:
    """Train `net` on the residual metric of h's coarse operator (h None: mean squared error)."""
    _check(lib().mg_net_set_metric(ctypes.c_void_p(net), ctypes.c_void_p(h) if h else None), "mg_net_set_metric")


def mg_net_destroy(net) -> None:
    if net:
        lib().mg_net_destroy(ctypes.c_void_p(net))


def mg_attach_coarse_net(h, net, admit: float = 0.5, bf16: bool = True) -> None:
    """Use `net` as h's coarse solve (GMRES+SGS measures the proposal and is the fallback); net=None detaches."""
    _check(lib().mg_attach_coarse_net(ctypes.c_void_p(h), ctypes.c_void_p(net or 0), float(admit),
                                      1 if bf16 else 0), "mg_attach_coarse_net")


def mg_record_coarse(h, r_ptr: int, y_ptr: int, max_pairs: int) -> None:
    _check(lib().mg_record_coarse(ctypes.c_void_p(h), ctypes.c_void_p(r_ptr), ctypes.c_void_p(y_ptr),
                                  int(max_pairs)), "mg_record_coarse")


def mg_recorded_pairs(h) -> int:
    return int(lib().mg_recorded_pairs(ctypes.c_void_p(h)))


def mg_coarse_shape(h):
    """(T, X) of the coarse level: the network's sample shape is (5, T, X)."""
    T, X = ctypes.c_int(), ctypes.c_int()
    _check(lib().mg_coarse_shape(ctypes.c_void_p(h), ctypes.byref(T), ctypes.byref(X)), "mg_coarse_shape")
    return T.value, X.value


def mg_jacobi_radius(h, level: int = 0, iters: int = 4000, stream: int = 0) -> float:
    """Spectral radius of the block-Jacobi iteration on a level (Table 2), by power iteration."""
    rho = ctypes.c_double()
    _check(lib().mg_jacobi_radius(ctypes.c_void_p(h), int(level), int(iters), ctypes.byref(rho),
                                  ctypes.c_void_p(stream)), "mg_jacobi_radius")
    return rho.value


SGS_CHAINS = ("scan", "cluster", "serial", "segmented")


def mg_autotune(h, stream: int = 0):
    """Time and select the SGS chain evaluation and dot-product blocking for h
    (cached per shape); returns (chain name, vectors per CTA)."""
    chain, vb = ctypes.c_int(), ctypes.c_int()
    _check(lib().mg_autotune(ctypes.c_void_p(h), ctypes.byref(chain), ctypes.byref(vb), ctypes.c_void_p(stream)),
           "mg_autotune")
    return SGS_CHAINS[chain.value], vb.value


def mg_block_mapping(h, level: int) -> int:
    """Block-solve mapping of a level: 1 = one warp per time block, 2 = two warps per block."""
    code = int(lib().mg_block_mapping(ctypes.c_void_p(h), level))
    if code < 0:
        raise PintmgError(code, "mg_block_mapping")
    return code


def mg_destroy(h) -> None:
    if h:
        lib().mg_destroy(ctypes.c_void_p(h))


def mg_last_cuda_error() -> str:
    return lib().mg_last_cuda_error().decode()
