"""CPU-only checks of the C ABI: the library loads, exports every entry point its headers declare,
and its host-side plan mathematics and argument validation behave (no GPU call is made)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ab():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2312_00538_gb300 as m
    return m


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:anova_status|void|int64_t|const char \*)\s*\*?\s*(\w+)\s*\(", txt, re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol(ab):
    names = _declared()
    assert "anova_nfft_plan" in names and "anova_matvec" in names
    L = ctypes.CDLL(ab.LIB_PATH)
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing
    # the Python binding keeps the C names
    assert set(ab.exported_symbols()) <= names


def test_kernel_coefficients_reproduce_the_gaussian(ab):
    from oracle import nfft as on
    for N, ell, bound in [(32, 0.5, 3e-7), (32, 1.0, 2e-7), (64, 1.0, 1e-11)]:
        b = ab.anova_kernel_coeffs(ell, N)
        t = np.linspace(-0.4, 0.4, 2001)
        approx = b[0] + 2 * np.cos(2 * np.pi * np.outer(t, np.arange(1, N // 2))) @ b[1:]
        assert np.max(np.abs(approx - np.exp(-t ** 2 / ell ** 2))) <= bound
        # and agree with the oracle's independent fit
        assert np.allclose(b, on.trig_coeffs(ell, N), rtol=0, atol=1e-9)


def test_window_transform_matches_bessel_form(ab):
    from oracle import nfft as on
    for m in (4, 6):
        P = ab.anova_window_hat(m, 64, 17)
        c = on.kb_hat_closed_form(np.arange(17), m, 64, on.kb_beta())
        assert np.max(np.abs(P - c) / c) <= (2e-6 if m == 4 else 1e-9)


def test_invalid_arguments_are_rejected_before_any_device_work(ab):
    X = np.zeros((4, 3))
    W = [[0, 1, 2]]
    cases = [
        (dict(points=X, windows=W, sigma=1.0, N=31), ab.ANOVA_ERR_INVALID_ARG),
        (dict(points=X, windows=W, sigma=1.0, N=48), ab.ANOVA_ERR_INVALID_ARG),
        (dict(points=X, windows=W, sigma=-1.0), ab.ANOVA_ERR_INVALID_ARG),
        (dict(points=X, windows=W, sigma=1.0, m=9), ab.ANOVA_ERR_INVALID_ARG),
        (dict(points=X, windows=[[0, 3, -1]], sigma=1.0), ab.ANOVA_ERR_INVALID_ARG),
        (dict(points=X, windows=[[0, -1, 2]], sigma=1.0), ab.ANOVA_ERR_INVALID_ARG),
        (dict(points=X, windows=[[1, 1, -1]], sigma=1.0), ab.ANOVA_ERR_INVALID_ARG),
        (dict(points=X + 0.3, windows=W, sigma=1.0), ab.ANOVA_ERR_OUT_OF_RANGE),
        (dict(points=np.where(np.eye(4, 3) > 0, np.nan, 0.0), windows=W, sigma=1.0),
         ab.ANOVA_ERR_NONFINITE),
        (dict(points=X, windows=W, sigma=1.0, flags=8), ab.ANOVA_ERR_INVALID_ARG),
        (dict(points=X, windows=W, sigma=1.0, flags=ab.ANOVA_INTERP_TENSOR | ab.ANOVA_INTERP_SIMT),
         ab.ANOVA_ERR_INVALID_ARG),
    ]
    for kw, status in cases:
        with pytest.raises(ab.AnovaError) as ei:
            ab.anova_nfft_plan(**kw)
        assert ei.value.status == status, kw
    assert ab.anova_last_error() != ""
    # the tuned plan validates its own arguments, then the plan's
    for kw in (dict(nrhs=0), dict(nrhs=1025), dict(reps=0), dict(N=31)):
        with pytest.raises(ab.AnovaError) as ei:
            ab.anova_nfft_plan_tuned(X, W, 1.0, **kw)
        assert ei.value.status == ab.ANOVA_ERR_INVALID_ARG, kw


def test_model_calls_validate_before_device_work(ab):
    L = ab.lib()
    h = ctypes.c_void_p()
    assert L.anova_model_create(None, None, ctypes.byref(h)) == ab.ANOVA_ERR_INVALID_ARG
    assert L.anova_model_eval(None, None, None) == ab.ANOVA_ERR_INVALID_ARG
    L.anova_model_destroy(None)


def test_matvec_batch_validates_before_device_work(ab):
    L = ab.lib()
    h = ctypes.c_void_p()
    assert L.anova_matvec_batch_create(0, None, None, None, None, None, ctypes.byref(h)) == ab.ANOVA_ERR_INVALID_ARG
    assert L.anova_matvec_batch_create(2, None, None, None, None, None, ctypes.byref(h)) == ab.ANOVA_ERR_INVALID_ARG
    assert L.anova_matvec_batch_run(None) == ab.ANOVA_ERR_INVALID_ARG
    L.anova_matvec_batch_destroy(None)


def test_unused_features_may_lie_outside_the_box(ab):
    # only the features named by a window must lie in [-0.2, 0.2]; validation passes this case
    # and fails later only for want of a device, which this CPU test tolerates
    X = np.zeros((4, 4))
    X[:, 3] = 5.0
    try:
        ab.anova_nfft_plan(X, [[0, 1, 2]], 1.0)
    except ab.AnovaError as e:
        assert e.status == ab.ANOVA_ERR_CUDA


def test_struct_layouts_match_the_headers(ab):
    """The binding's ctypes mirrors of the ABI structs have the C sizes (a field added on one side
    only would shift every later field)."""
    L = ctypes.CDLL(ab.LIB_PATH)
    L.anova_abi_struct_size.restype = ctypes.c_int64
    L.anova_abi_struct_size.argtypes = [ctypes.c_char_p]
    for name in ["anova_tune_report", "svm_opts", "svm_stats", "svm_problem", "svm_server_stats"]:
        c_size = L.anova_abi_struct_size(name.encode())
        assert c_size > 0, name
        assert ctypes.sizeof(getattr(ab, name)) == c_size, name
    assert L.anova_abi_struct_size(b"no_such_struct") == 0
    assert L.anova_abi_struct_size(None) == 0
