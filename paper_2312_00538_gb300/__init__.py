"""Python binding of the GB300 ANOVA-NFFT library (libanova.so, C ABI in include/anova.h).

Argument marshalling only: every computation runs in the library's CUDA kernels. Device buffers
are torch CUDA tensors (their data pointers are passed through), host buffers NumPy arrays.
The functions keep the C names. The library must have been built (``__graft_entry__.build()``
or ``python paper_2312_00538_gb300/_build.py``); importing without it raises ImportError.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libanova.so")

ANOVA_OK = 0
ANOVA_ERR_INVALID_ARG = 1
ANOVA_ERR_OUT_OF_RANGE = 2
ANOVA_ERR_NONFINITE = 3
ANOVA_ERR_OOM = 4
ANOVA_ERR_CUDA = 5
ANOVA_ERR_NOT_CONVERGED = 6
ANOVA_ERR_BREAKDOWN = 7
ANOVA_ERR_TIMEOUT = 8
STATUS_NAMES = {0: "ANOVA_OK", 1: "ANOVA_ERR_INVALID_ARG", 2: "ANOVA_ERR_OUT_OF_RANGE",
                3: "ANOVA_ERR_NONFINITE", 4: "ANOVA_ERR_OOM", 5: "ANOVA_ERR_CUDA",
                6: "ANOVA_ERR_NOT_CONVERGED", 7: "ANOVA_ERR_BREAKDOWN", 8: "ANOVA_ERR_TIMEOUT"}

ANOVA_FP32 = 0
ANOVA_FP64 = 1
ANOVA_INTERP_TENSOR = 2
ANOVA_INTERP_SIMT = 4
PCHOL_GREEDY = 0
NYSTROM = 1
PCHOL_RANDOM = 2
PCHOL_PER_WINDOW = 3
NYSTROM_RANDOM = 4
SVM_KRYLOV_MINRES = 0
SVM_KRYLOV_GMRES = 1


class AnovaError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


_lib = None

_c_int = ctypes.c_int
_c_i64 = ctypes.c_int64
_c_dbl = ctypes.c_double
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_lp = ctypes.POINTER(ctypes.c_int64)

_SIGNATURES = {
    "anova_nfft_plan": (_c_int, [_dp, _c_i64, _c_int, _ip, _c_int, _c_dbl, _c_int, _c_int, _c_int,
                                 _vp, ctypes.POINTER(_vp)]),
    "anova_nfft_plan_ex": (_c_int, [_dp, _c_i64, _c_int, _ip, _c_int, _dp, _dp, _c_int, _c_int,
                                    _c_int, _vp, ctypes.POINTER(_vp)]),
    "anova_nfft_plan_tuned": (_c_int, [_dp, _c_i64, _c_int, _ip, _c_int, _dp, _dp, _c_int, _c_int,
                                       _c_int, _vp, _c_int, _c_int, _vp, ctypes.POINTER(_vp)]),
    "anova_matvec": (_c_int, [_vp, _vp, _vp, _c_int]),
    "anova_matvec_batch_create": (_c_int, [_c_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                           ctypes.POINTER(_vp), ctypes.POINTER(_c_int), _vp,
                                           ctypes.POINTER(_vp)]),
    "anova_matvec_batch_run": (_c_int, [_vp]),
    "anova_matvec_batch_destroy": (None, [_vp]),
    "anova_model_create": (_c_int, [_vp, _vp, ctypes.POINTER(_vp)]),
    "anova_model_eval": (_c_int, [_vp, _vp, _vp]),
    "anova_model_destroy": (None, [_vp]),
    "anova_matvec_host": (_c_int, [_vp, _vp, _vp, _c_int]),
    "anova_window_matvec": (_c_int, [_vp, _c_int, _vp, _vp]),
    "anova_spread_grid": (_c_int, [_vp, _c_int, _vp, _vp]),
    "anova_conv_grid": (_c_int, [_vp, _c_int, _vp, _vp]),
    "anova_interp_grid": (_c_int, [_vp, _c_int, _vp, _vp]),
    "anova_spread_grid_noalloc": (_c_int, [_vp, _c_int, _vp, _vp]),
    "anova_plan_info": (_c_int, [_vp, _lp, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int),
                                 ctypes.POINTER(_c_int), _lp]),
    "anova_plan_destroy": (None, [_vp]),
    "anova_plan_check": (_c_int, [_vp]),
    "anova_plan_set_wait_limit": (_c_int, [_vp, _c_i64]),
    "anova_measure_fp32_peak": (_c_int, [_dp]),
    "anova_plan_grid_size": (_c_int, [_vp, _lp]),
    "anova_matvec_grids": (_c_int, [_vp, _vp, _vp, _c_int]),
    "anova_matvec_from_grids": (_c_int, [_vp, _vp, _vp, _c_int]),
    "anova_cross_matvec": (_c_int, [_vp, _vp, _vp, _vp]),
    "anova_plan_set_timing": (_c_int, [_vp, _c_int]),
    "anova_plan_stage_times": (_c_int, [_vp, _dp, _lp]),
    "anova_kernel_coeffs": (_c_int, [_c_dbl, _c_int, _dp]),
    "anova_window_hat": (_c_int, [_c_int, _c_int, _c_int, _dp]),
    "lowrank_precond_build": (_c_int, [_vp, _c_int, _c_int, _c_dbl, ctypes.c_uint64, ctypes.POINTER(_vp)]),
    "lowrank_info": (_c_int, [_vp, ctypes.POINTER(_c_int), _lp]),
    "lowrank_factor": (_c_int, [_vp, _vp]),
    "lowrank_precond_set_theta": (_c_int, [_vp, _vp, _vp]),
    "lowrank_precond_apply": (_c_int, [_vp, _vp, _vp, _vp, _vp]),
    "lowrank_set_core_path": (_c_int, [_vp, _c_int]),
    "lowrank_core": (_c_int, [_vp, _vp, ctypes.POINTER(_c_int)]),
    "lowrank_destroy": (None, [_vp]),
    "svm_opts_default": (None, [_vp]),
    "svm_ipm_solve": (_c_int, [_dp, _c_i64, _c_int, _dp, _c_dbl, _c_dbl, _vp, _dp, _dp, _vp]),
    "svm_ipm_solve_batch": (_c_int, [_vp, _c_int, _c_dbl, _vp, _c_int]),
    "svm_server_create": (_c_int, [_vp, _c_dbl, _c_int, _c_i64, ctypes.POINTER(_vp)]),
    "svm_server_submit": (_c_int, [_vp, _vp, _lp]),
    "svm_server_wait": (_c_int, [_vp, _c_i64]),
    "svm_server_drain": (_c_int, [_vp]),
    "svm_server_get_stats": (_c_int, [_vp, _vp]),
    "svm_request_footprint": (_c_i64, [_c_i64, _c_int, _vp]),
    "svm_server_admission": (_c_int, [_vp, _vp, _c_int, _c_i64, _c_i64, _c_int, _vp]),
    "anova_abi_struct_size": (_c_i64, [ctypes.c_char_p]),
    "svm_server_destroy": (None, [_vp]),
    "anova_last_error": (ctypes.c_char_p, []),
    "anova_version": (ctypes.c_char_p, []),
}


def lib():
    """The loaded library (ctypes.CDLL). Raises ImportError if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libanova.so is not built: run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            if hasattr(L, name):
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    """Names of the C entry points this binding declares."""
    return sorted(_SIGNATURES)


def _check(status):
    if status != ANOVA_OK:
        raise AnovaError(status, lib().anova_last_error().decode())


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _dev_ptr(t):
    """Data pointer of a torch tensor (or an int address)."""
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    if not t.is_contiguous():
        raise ValueError("device buffers must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """Owns an anova_plan_t; destroyed with the object (or by .destroy())."""

    def __init__(self, handle, n, P, precision):
        self.handle = handle
        self.n = n
        self.P = P
        self.precision = precision

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.precision == ANOVA_FP64 else torch.float32

    def destroy(self):
        if self.handle:
            lib().anova_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def anova_nfft_plan(points, windows, sigma, N=32, m=4, flags=ANOVA_FP32, stream=None):
    """anova_nfft_plan: points (n x d, host), windows (P x 3 int32, -1 padded)."""
    X = _f64(points)
    if X.ndim != 2:
        raise ValueError("points must be n x d")
    W = np.ascontiguousarray(windows, dtype=np.int32).reshape(-1, 3)
    h = _vp()
    _check(lib().anova_nfft_plan(_ptr(X, ctypes.c_double), X.shape[0], X.shape[1],
                                 _ptr(W, ctypes.c_int32), W.shape[0], float(sigma), int(N), int(m),
                                 int(flags), _stream_handle(stream), ctypes.byref(h)))
    return Plan(h, X.shape[0], W.shape[0], flags & 1)


def anova_nfft_plan_ex(points, windows, ell, eta=None, N=32, m=4, flags=ANOVA_FP32, stream=None):
    """anova_nfft_plan_ex: one length scale ell_l (and weight eta_l) per window."""
    X = _f64(points)
    W = np.ascontiguousarray(windows, dtype=np.int32).reshape(-1, 3)
    ell = _f64(np.broadcast_to(ell, (W.shape[0],)))
    eta_p = None
    if eta is not None:
        eta = _f64(np.broadcast_to(eta, (W.shape[0],)))
        eta_p = _ptr(eta, ctypes.c_double)
    h = _vp()
    _check(lib().anova_nfft_plan_ex(_ptr(X, ctypes.c_double), X.shape[0], X.shape[1],
                                    _ptr(W, ctypes.c_int32), W.shape[0], _ptr(ell, ctypes.c_double),
                                    eta_p, int(N), int(m), int(flags), _stream_handle(stream),
                                    ctypes.byref(h)))
    return Plan(h, X.shape[0], W.shape[0], flags & 1)


class anova_tune_report(ctypes.Structure):
    _fields_ = [("wi_max", ctypes.c_int), ("interp", ctypes.c_int), ("rhs_chunk", ctypes.c_int),
                ("fork_windows", ctypes.c_int), ("candidates", ctypes.c_int), ("ms", ctypes.c_double),
                ("ms_default", ctypes.c_double), ("conv_lines", ctypes.c_int)]


def anova_nfft_plan_tuned(points, windows, ell, eta=None, N=32, m=4, flags=ANOVA_FP32, nrhs=1, reps=5,
                          stream=None):
    """anova_nfft_plan_tuned: anova_nfft_plan_ex plus the launch-setting search. Returns
    (plan, report dict)."""
    X = _f64(points)
    W = np.ascontiguousarray(windows, dtype=np.int32).reshape(-1, 3)
    ell = _f64(np.broadcast_to(ell, (W.shape[0],)))
    eta_p = None
    if eta is not None:
        eta = _f64(np.broadcast_to(eta, (W.shape[0],)))
        eta_p = _ptr(eta, ctypes.c_double)
    h = _vp()
    rep = anova_tune_report()
    _check(lib().anova_nfft_plan_tuned(_ptr(X, ctypes.c_double), X.shape[0], X.shape[1],
                                       _ptr(W, ctypes.c_int32), W.shape[0], _ptr(ell, ctypes.c_double),
                                       eta_p, int(N), int(m), int(flags), _stream_handle(stream), int(nrhs),
                                       int(reps), ctypes.byref(rep), ctypes.byref(h)))
    return Plan(h, X.shape[0], W.shape[0], flags & 1), {k: getattr(rep, k) for k, _ in rep._fields_}


def anova_matvec(plan, v, Kv, nrhs=1):
    """anova_matvec: v, Kv device tensors holding n x nrhs column-major (i.e. shape (nrhs, n)
    contiguous, or (n,) for one right-hand side)."""
    _check(lib().anova_matvec(plan.handle, _dev_ptr(v), _dev_ptr(Kv), int(nrhs)))


def _host_ptr(a, plan, nrhs):
    if isinstance(a, np.ndarray):
        dt = np.float64 if plan.precision == ANOVA_FP64 else np.float32
        if a.dtype != dt or not (a.flags.f_contiguous or a.ndim == 1) or a.size != plan.n * nrhs:
            raise ValueError("host buffers must be contiguous arrays of the plan's type")
        return ctypes.c_void_p(a.ctypes.data)
    # a torch CPU tensor (e.g. pinned): shape (nrhs, n) or (n,), contiguous
    if a.device.type != "cpu" or not a.is_contiguous() or a.numel() != plan.n * nrhs:
        raise ValueError("host buffers must be contiguous CPU tensors of n * nrhs elements")
    return ctypes.c_void_p(a.data_ptr())


def anova_matvec_host(plan, v, Kv, nrhs=1):
    """anova_matvec_host: v, Kv host buffers (NumPy arrays in column-major order, or contiguous
    torch CPU tensors of shape (nrhs, n)), n * nrhs elements of the plan's type."""
    _check(lib().anova_matvec_host(plan.handle, _host_ptr(v, plan, nrhs), _host_ptr(Kv, plan, nrhs),
                                   int(nrhs)))


def anova_window_matvec(plan, l, v, Kv):
    _check(lib().anova_window_matvec(plan.handle, int(l), _dev_ptr(v), _dev_ptr(Kv)))


def anova_spread_grid(plan, l, v, grid):
    _check(lib().anova_spread_grid(plan.handle, int(l), _dev_ptr(v), _dev_ptr(grid)))


def anova_spread_grid_noalloc(plan, l, v, grid):
    """anova_spread_grid without device allocation in the call (fixed 16 MiB static scratch)."""
    _check(lib().anova_spread_grid_noalloc(plan.handle, int(l), _dev_ptr(v), _dev_ptr(grid)))


def anova_conv_grid(plan, l, grid_in, grid_out):
    _check(lib().anova_conv_grid(plan.handle, int(l), _dev_ptr(grid_in), _dev_ptr(grid_out)))


def anova_interp_grid(plan, l, grid, f):
    _check(lib().anova_interp_grid(plan.handle, int(l), _dev_ptr(grid), _dev_ptr(f)))


def anova_plan_info(plan):
    n = ctypes.c_int64()
    P = ctypes.c_int()
    nos = ctypes.c_int()
    fl = ctypes.c_int()
    nb = ctypes.c_int64()
    _check(lib().anova_plan_info(plan.handle, ctypes.byref(n), ctypes.byref(P), ctypes.byref(nos),
                                 ctypes.byref(fl), ctypes.byref(nb)))
    return dict(n=n.value, P=P.value, n_os=nos.value, flags=fl.value, device_bytes=nb.value)


def anova_cross_matvec(source, target, w, f):
    """f (device, target points) = sum over windows and sources of w_i K(t_j, s_i)."""
    _check(lib().anova_cross_matvec(source.handle, target.handle, _dev_ptr(w), _dev_ptr(f)))


class MatvecBatch:
    """Owns an anova_batch_t (one CUDA graph over several plans' matvecs); keeps the plans and
    vectors alive while it exists."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def run(self):
        _check(lib().anova_matvec_batch_run(self.handle))

    def destroy(self):
        if self.handle:
            lib().anova_matvec_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def anova_matvec_batch_create(plans, vs, kvs, nrhs=None, stream=None):
    """One CUDA graph running anova_matvec(plans[k], vs[k], kvs[k], nrhs[k]) for every k."""
    count = len(plans)
    P = (_vp * count)(*[p.handle for p in plans])
    V = (_vp * count)(*[_dev_ptr(v) for v in vs])
    K = (_vp * count)(*[_dev_ptr(k) for k in kvs])
    R = None if nrhs is None else (_c_int * count)(*[int(x) for x in nrhs])
    h = _vp()
    _check(lib().anova_matvec_batch_create(count, P, V, K, R, _stream_handle(stream), ctypes.byref(h)))
    return MatvecBatch(h, (list(plans), list(vs), list(kvs)))


class Model:
    """Owns an anova_model_t (the kept, convolved source grids); destroyed with the object."""

    def __init__(self, handle, precision):
        self.handle = handle
        self.precision = precision

    def destroy(self):
        if self.handle:
            lib().anova_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def anova_model_create(source, w):
    """Spreads and convolves the weights w (device tensor, source points) once."""
    h = _vp()
    _check(lib().anova_model_create(source.handle, _dev_ptr(w), ctypes.byref(h)))
    return Model(h, source.precision)


def anova_model_eval(model, target, f):
    """f (device, target points) from the model's kept grids."""
    _check(lib().anova_model_eval(model.handle, target.handle, _dev_ptr(f)))


def anova_plan_check(plan):
    _check(lib().anova_plan_check(plan.handle))


def anova_plan_set_wait_limit(plan, polls):
    """Polls of each tensor-core completion wait before it gives up (negative: the default)."""
    _check(lib().anova_plan_set_wait_limit(plan.handle, int(polls)))


def anova_plan_grid_size(plan):
    """Values of one right-hand side's grids (every window's grid back to back)."""
    g = ctypes.c_int64()
    _check(lib().anova_plan_grid_size(plan.handle, ctypes.byref(g)))
    return g.value


def anova_matvec_grids(plan, v, grids, nrhs=1):
    """Spread of v (device) into every window's grid (device, nrhs x grid_total)."""
    _check(lib().anova_matvec_grids(plan.handle, _dev_ptr(v), _dev_ptr(grids), int(nrhs)))


def anova_matvec_from_grids(plan, grids, Kv, nrhs=1):
    """The product at the plan's points from (summed) grids (device) into Kv (device)."""
    _check(lib().anova_matvec_from_grids(plan.handle, _dev_ptr(grids), _dev_ptr(Kv), int(nrhs)))


def anova_measure_fp32_peak():
    """Measured FP32 multiply-add rate of the current GPU (TFLOP/s)."""
    v = ctypes.c_double()
    _check(lib().anova_measure_fp32_peak(ctypes.byref(v)))
    return v.value


def anova_plan_destroy(plan):
    plan.destroy()


STAGES = ("spread", "reduce", "fft", "interp", "sum")


def anova_plan_set_timing(plan, enable=True):
    _check(lib().anova_plan_set_timing(plan.handle, 1 if enable else 0))


def anova_plan_stage_times(plan):
    """Returns (dict stage -> total ms since the last reset, kernel launches since then)."""
    ms = np.zeros(len(STAGES))
    launches = ctypes.c_int64()
    _check(lib().anova_plan_stage_times(plan.handle, _ptr(ms, ctypes.c_double),
                                        ctypes.byref(launches)))
    return dict(zip(STAGES, ms.tolist())), launches.value


def anova_kernel_coeffs(ell, N):
    b = np.zeros(N // 2)
    _check(lib().anova_kernel_coeffs(float(ell), int(N), _ptr(b, ctypes.c_double)))
    return b


def anova_window_hat(m, n_os, count):
    out = np.zeros(count)
    _check(lib().anova_window_hat(int(m), int(n_os), int(count), _ptr(out, ctypes.c_double)))
    return out


def anova_last_error():
    return lib().anova_last_error().decode()


def anova_version():
    return lib().anova_version().decode()


# --------------------------------------------------------------------------- solver (anova_svm.h)
SVM_STOP_GAP = 0
SVM_STOP_ALG1 = 1
SVM_SIGMA_CONSTANT = 0
SVM_SIGMA_ADAPTIVE = 1


class svm_opts(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int), ("sigma_barrier", ctypes.c_double),
                ("gamma", ctypes.c_double), ("sigma_rule", ctypes.c_int), ("alpha0", ctypes.c_double),
                ("stop", ctypes.c_int), ("krylov_max", ctypes.c_int),
                ("krylov_tol", ctypes.c_double), ("refine_max", ctypes.c_int),
                ("precond", ctypes.c_int), ("rank", ctypes.c_int), ("err_tol", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("ell", ctypes.c_double),
                ("windows", ctypes.POINTER(ctypes.c_int32)), ("P", ctypes.c_int),
                ("N", ctypes.c_int), ("m", ctypes.c_int), ("N_precise", ctypes.c_int),
                ("m_precise", ctypes.c_int), ("scale_features", ctypes.c_int),
                ("cuda_stream", ctypes.c_void_p), ("krylov", ctypes.c_int), ("autotune", ctypes.c_int),
                ("m_refine", ctypes.c_int)]


class svm_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("krylov_iterations", ctypes.c_int),
                ("refinements", ctypes.c_int), ("fp64_krylov_iterations", ctypes.c_int),
                ("rank", ctypes.c_int), ("converged", ctypes.c_int),
                ("mu", ctypes.c_double), ("dual", ctypes.c_double), ("primal", ctypes.c_double),
                ("rel_gap", ctypes.c_double), ("xi_alpha", ctypes.c_double),
                ("time_ms", ctypes.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class LowRank:
    """Owns a lowrank_t (and keeps its plan alive)."""

    def __init__(self, handle, plan):
        self.handle = handle
        self.plan = plan

    def destroy(self):
        if self.handle:
            lib().lowrank_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def lowrank_precond_build(plan, kind=PCHOL_GREEDY, r=200, err_tol=1e-5, seed=0):
    h = _vp()
    _check(lib().lowrank_precond_build(plan.handle, int(kind), int(r), float(err_tol),
                                       ctypes.c_uint64(seed), ctypes.byref(h)))
    return LowRank(h, plan)


def lowrank_info(lr):
    rank = ctypes.c_int()
    _check(lib().lowrank_info(lr.handle, ctypes.byref(rank), None))
    piv = np.zeros(rank.value, dtype=np.int64)
    _check(lib().lowrank_info(lr.handle, ctypes.byref(rank), _ptr(piv, ctypes.c_int64)))
    return rank.value, piv


def lowrank_factor(lr, L):
    """Copies the FP64 factor into the device tensor L (n x rank, column-major: shape (rank, n))."""
    _check(lib().lowrank_factor(lr.handle, _dev_ptr(L)))


def lowrank_precond_set_theta(lr, theta, y):
    _check(lib().lowrank_precond_set_theta(lr.handle, _dev_ptr(theta), _dev_ptr(y)))


LOWRANK_CORE_AUTO, LOWRANK_CORE_SIMT, LOWRANK_CORE_TENSOR = 0, 1, 2


def lowrank_set_core_path(lr, path):
    _check(lib().lowrank_set_core_path(lr.handle, int(path)))


def lowrank_core(lr, M=None):
    """Copies the Woodbury core of the last set_theta into M (device, rank x rank) if given;
    returns the path it took (LOWRANK_CORE_SIMT or LOWRANK_CORE_TENSOR)."""
    used = _c_int()
    _check(lib().lowrank_core(lr.handle, None if M is None else _dev_ptr(M), ctypes.byref(used)))
    return used.value


def lowrank_precond_apply(lr, theta, y, g, x):
    _check(lib().lowrank_precond_apply(lr.handle, _dev_ptr(theta), _dev_ptr(y), _dev_ptr(g),
                                       _dev_ptr(x)))


def lowrank_destroy(lr):
    lr.destroy()


def svm_opts_default():
    o = svm_opts()
    lib().svm_opts_default(ctypes.byref(o))
    return o


def svm_ipm_solve(X, y, C, tol, opts=None, windows=None):
    """svm_ipm_solve: host X (n x d) and labels y; returns (alpha, b, stats dict, status).

    Raises AnovaError except for ANOVA_ERR_NOT_CONVERGED, which is returned as the status."""
    X = _f64(X)
    yv = _f64(y)
    n, d = X.shape
    o = opts if opts is not None else svm_opts_default()
    keep = None
    if windows is not None:
        keep = np.ascontiguousarray(windows, dtype=np.int32).reshape(-1, 3)
        o.windows = _ptr(keep, ctypes.c_int32)
        o.P = keep.shape[0]
    alpha = np.zeros(n)
    b = ctypes.c_double()
    st = svm_stats()
    status = lib().svm_ipm_solve(_ptr(X, ctypes.c_double), n, d, _ptr(yv, ctypes.c_double),
                                 float(C), float(tol), ctypes.byref(o),
                                 _ptr(alpha, ctypes.c_double), ctypes.byref(b), ctypes.byref(st))
    if status not in (ANOVA_OK, ANOVA_ERR_NOT_CONVERGED):
        _check(status)
    del keep
    return alpha, b.value, st.as_dict(), status


class svm_problem(ctypes.Structure):
    _fields_ = [("X", ctypes.POINTER(ctypes.c_double)), ("n", ctypes.c_int64), ("d", ctypes.c_int),
                ("y", ctypes.POINTER(ctypes.c_double)), ("C", ctypes.c_double), ("ell", ctypes.c_double),
                ("windows", ctypes.POINTER(ctypes.c_int32)), ("P", ctypes.c_int),
                ("alpha", ctypes.POINTER(ctypes.c_double)), ("b", ctypes.c_double),
                ("stats", svm_stats), ("status", ctypes.c_int)]


def svm_ipm_solve_batch(problems, tol, opts=None, concurrency=8):
    """svm_ipm_solve_batch over a list of dicts with keys X, y, C and optionally ell, windows.

    Returns a list of (alpha, b, stats dict, status) in the input order."""
    keep = []
    arr = (svm_problem * len(problems))()
    alphas = []
    for i, pr in enumerate(problems):
        X = _f64(pr["X"])
        y = _f64(pr["y"])
        al = np.zeros(X.shape[0])
        keep += [X, y]
        alphas.append(al)
        arr[i].X = _ptr(X, ctypes.c_double)
        arr[i].n = X.shape[0]
        arr[i].d = X.shape[1]
        arr[i].y = _ptr(y, ctypes.c_double)
        arr[i].C = float(pr["C"])
        arr[i].ell = float(pr.get("ell", 0.0))
        if pr.get("windows") is not None:
            W = np.ascontiguousarray(pr["windows"], dtype=np.int32).reshape(-1, 3)
            keep.append(W)
            arr[i].windows = _ptr(W, ctypes.c_int32)
            arr[i].P = W.shape[0]
        arr[i].alpha = _ptr(al, ctypes.c_double)
    o = opts if opts is not None else svm_opts_default()
    lib().svm_ipm_solve_batch(ctypes.byref(arr), len(problems), float(tol), ctypes.byref(o),
                              int(concurrency))
    out = []
    for i in range(len(problems)):
        st = arr[i].status
        if st not in (ANOVA_OK, ANOVA_ERR_NOT_CONVERGED):
            raise AnovaError(st, "problem %d of the batch failed" % i)
        out.append((alphas[i], arr[i].b, arr[i].stats.as_dict(), st))
    del keep
    return out


class svm_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("running", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("reserved_bytes", ctypes.c_int64), ("peak_reserved_bytes", ctypes.c_int64),
                ("p50_latency_ms", ctypes.c_double), ("p99_latency_ms", ctypes.c_double),
                ("mean_latency_ms", ctypes.c_double), ("backfilled", ctypes.c_int64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


def _fill_problem(pr, X, y, C, ell, windows):
    """Fill one svm_problem from host arrays; returns the arrays it points into."""
    X = _f64(X)
    y = _f64(y)
    al = np.zeros(X.shape[0])
    keep = [X, y, al]
    pr.X = _ptr(X, ctypes.c_double)
    pr.n = X.shape[0]
    pr.d = X.shape[1]
    pr.y = _ptr(y, ctypes.c_double)
    pr.C = float(C)
    pr.ell = float(ell or 0.0)
    if windows is not None:
        W = np.ascontiguousarray(windows, dtype=np.int32).reshape(-1, 3)
        keep.append(W)
        pr.windows = _ptr(W, ctypes.c_int32)
        pr.P = W.shape[0]
    pr.alpha = _ptr(al, ctypes.c_double)
    return keep


def svm_request_footprint(n, P, opts=None):
    o = opts if opts is not None else svm_opts_default()
    return int(lib().svm_request_footprint(int(n), int(P), ctypes.byref(o)))


def svm_server_admission(footprints, passed, reserved, budget, running):
    """The server's admission rule (host only): index of the queued request to start next, or -1."""
    fp = np.ascontiguousarray(footprints, dtype=np.int64)
    ps = np.ascontiguousarray(passed, dtype=np.int32)
    if fp.ndim != 1 or fp.shape != ps.shape:
        raise ValueError("footprints and passed must be 1-D of equal length")
    pick = ctypes.c_int(-1)
    _check(lib().svm_server_admission(_ptr(fp, ctypes.c_int64) if fp.size else None,
                                      _ptr(ps, ctypes.c_int32) if ps.size else None, int(fp.size),
                                      int(reserved), int(budget), int(running), ctypes.byref(pick)))
    return pick.value


class SvmServer:
    """svm_server_t: queued SVM solves admitted by free slot and device-memory budget.

    submit() returns a ticket at once; wait(ticket) returns (alpha, b, stats dict, status)."""

    def __init__(self, tol, opts=None, slots=8, hbm_budget_bytes=64 << 30):
        self.opts = opts if opts is not None else svm_opts_default()
        h = _vp()
        _check(lib().svm_server_create(ctypes.byref(self.opts), float(tol), int(slots),
                                       int(hbm_budget_bytes), ctypes.byref(h)))
        self.handle = h
        self._pending = {}

    def submit(self, X, y, C, ell=None, windows=None):
        pr = svm_problem()
        keep = _fill_problem(pr, X, y, C, ell, windows)
        t = ctypes.c_int64()
        _check(lib().svm_server_submit(self.handle, ctypes.byref(pr), ctypes.byref(t)))
        self._pending[t.value] = (pr, keep)
        return t.value

    def wait(self, ticket):
        pr, keep = self._pending[ticket]
        st = lib().svm_server_wait(self.handle, int(ticket))
        del self._pending[ticket]
        if st not in (ANOVA_OK, ANOVA_ERR_NOT_CONVERGED):
            raise AnovaError(st, "request %d failed" % ticket)
        return keep[2], pr.b, pr.stats.as_dict(), st

    def drain(self):
        _check(lib().svm_server_drain(self.handle))

    def stats(self):
        s = svm_server_stats()
        _check(lib().svm_server_get_stats(self.handle, ctypes.byref(s)))
        return s.as_dict()

    def destroy(self):
        if self.handle:
            lib().svm_server_destroy(self.handle)
            self.handle = None
            self._pending.clear()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def svm_server_create(tol, opts=None, slots=8, hbm_budget_bytes=64 << 30):
    return SvmServer(tol, opts, slots, hbm_budget_bytes)
