"""ORACLE -- test infrastructure only. The ANOVA kernel by its definition (Sec. 3).

    kappa(x_i, x_j) = sum_l eta_l exp(-||x_j^{W_l} - x_i^{W_l}||^2 / ell_l^2),
    (K v)_j = sum_i v_i kappa(x_i, x_j),   K v = K_1 v + ... + K_P v.

Readings: ell_l = sigma for every window and eta_l = 1 (one shared length scale, unit weights).
"""
import ctypes
import numpy as np

from .build import build_oracle

_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_oracle())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        lp = ctypes.POINTER(ctypes.c_int64)
        lib.oracle_anova_matvec.argtypes = [dp, ctypes.c_int64, ctypes.c_int, ip, ctypes.c_int,
                                            dp, dp, dp, ctypes.c_int, lp, ctypes.c_int64, dp]
        lib.oracle_anova_matvec.restype = None
        lib.oracle_anova_kernel_matrix.argtypes = [dp, ctypes.c_int64, ctypes.c_int, ip,
                                                   ctypes.c_int, dp, dp, dp]
        lib.oracle_anova_kernel_matrix.restype = None
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_set_num_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _prep(X, windows, ell, eta):
    X = np.ascontiguousarray(X, dtype=np.float64)
    W = np.ascontiguousarray(windows, dtype=np.int32).reshape(-1, 3)
    P = W.shape[0]
    ell = np.broadcast_to(np.asarray(ell, dtype=np.float64), (P,)).copy()
    eta = None if eta is None else np.broadcast_to(np.asarray(eta, np.float64), (P,)).copy()
    return X, W, P, ell, eta


def num_threads():
    return _load().oracle_num_threads()


def set_num_threads(t):
    _load().oracle_set_num_threads(int(t))


def anova_matvec(X, windows, ell, V, rows=None, eta=None):
    """Direct FP64 (K V)[rows, :] for V of shape (n,) or (n, nrhs) (nrhs <= 64)."""
    X, W, P, ell, eta = _prep(X, windows, ell, eta)
    n, d = X.shape
    V = np.asarray(V, dtype=np.float64)
    vec = V.ndim == 1
    V2 = V.reshape(n, -1)
    nrhs = V2.shape[1]
    if nrhs > 64:
        raise ValueError("oracle matvec handles at most 64 right-hand sides per call")
    Vc = np.asfortranarray(V2)
    if rows is None:
        rows_arr = None
        nrows = n
    else:
        rows_arr = np.ascontiguousarray(rows, dtype=np.int64)
        if rows_arr.size and (rows_arr.min() < 0 or rows_arr.max() >= n):
            raise ValueError("row index out of range")
        nrows = rows_arr.size
    out = np.zeros((nrows, nrhs), dtype=np.float64, order="F")
    lib = _load()
    lib.oracle_anova_matvec(_ptr(X, ctypes.c_double), n, d, _ptr(W, ctypes.c_int32), P,
                            _ptr(ell, ctypes.c_double),
                            None if eta is None else _ptr(eta, ctypes.c_double),
                            Vc.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nrhs,
                            None if rows_arr is None else _ptr(rows_arr, ctypes.c_int64), nrows,
                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out[:, 0] if vec else out


def anova_kernel_matrix(X, windows, ell, eta=None):
    """Dense FP64 ANOVA kernel matrix K (n x n), entry by entry from the definition."""
    X, W, P, ell, eta = _prep(X, windows, ell, eta)
    n, d = X.shape
    K = np.zeros((n, n), dtype=np.float64)
    _load().oracle_anova_kernel_matrix(_ptr(X, ctypes.c_double), n, d, _ptr(W, ctypes.c_int32),
                                       P, _ptr(ell, ctypes.c_double),
                                       None if eta is None else _ptr(eta, ctypes.c_double),
                                       _ptr(K, ctypes.c_double))
    return K


def window_kernel_matrix(X, window, ell):
    """Dense K_l of one window (a list of 1-3 feature indices) in plain NumPy loops over pairs.

    Used at small n only, as an independent second statement of one window's kernel."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    feats = [k for k in window if k >= 0]
    K = np.empty((n, n))
    for j in range(n):
        diff = X[j, feats][None, :] - X[:, feats]
        K[j] = np.exp(-np.sum(diff * diff, axis=1) / ell ** 2)
    return K


def anova_cross_matvec(Xs, Xt, windows, ell, w, eta=None):
    """Direct FP64 sum with targets distinct from the sources, as in evaluating the decision
    function at new points (Sec. 6): f_j = sum_i w_i kappa(s_i, t_j). Written as the square
    matvec on the stacked point set [sources; targets] with zero weights on the targets, read
    at the target rows, so it is the pinned definition above and nothing else."""
    Xs = np.asarray(Xs, dtype=np.float64)
    Xt = np.asarray(Xt, dtype=np.float64)
    ns = Xs.shape[0]
    X = np.vstack([Xs, Xt])
    v = np.concatenate([np.asarray(w, dtype=np.float64), np.zeros(Xt.shape[0])])
    rows = np.arange(ns, ns + Xt.shape[0])
    return anova_matvec(X, windows, ell, v, rows=rows, eta=eta)
