"""Parity of the CUDA ANOVA-NFFT matvec with the FP64 oracle (Sec. 3, K v = sum_l K_l v).

Bars: relative l2 error <= 1e-4 for the FP32 plan (N=32, m=4) and <= 1e-9 for the FP64 plan
against the direct sum; the stage entry points against the oracle's plain NFFT stages."""
import numpy as np
import pytest

from oracle import kernel as ok
from oracle import nfft as on
from synth import (config1, config2, matvec_vectors, subsample_rows, minmax_scale,
                   consecutive_windows, SEED_BASE)

from ._gpu_util import require_gpu, rel_l2, to_dev, from_dev

pytestmark = pytest.mark.gpu

FP32_BAR = 1e-4
FP64_BAR = 1e-9


@pytest.fixture(scope="module")
def env():
    return require_gpu()


def _run(torch, ab, plan, V, dtype):
    V = np.asarray(V)
    nrhs = 1 if V.ndim == 1 else V.shape[1]
    v = to_dev(torch, V, dtype)
    out = torch.empty_like(v)
    ab.anova_matvec(plan, v, out, nrhs)
    torch.cuda.synchronize()
    ab.anova_plan_check(plan)  # no kernel-side wait ran out
    return from_dev(out)


def test_config1_fp32_ten_vectors(env):
    torch, ab = env
    cfg = config1()
    V = matvec_vectors(2000, 10, SEED_BASE + 1 + 100)
    plan = ab.anova_nfft_plan(cfg["X"], cfg["windows"], cfg["sigma"], N=32, m=4, flags=ab.ANOVA_FP32)
    got = _run(torch, ab, plan, V, torch.float32)
    ref = ok.anova_matvec(cfg["X"], cfg["windows"], cfg["sigma"], V)
    for r in range(10):
        assert rel_l2(got[:, r], ref[:, r]) <= FP32_BAR


def test_config1_fp64_precise_plan(env):
    torch, ab = env
    cfg = config1()
    V = matvec_vectors(2000, 3, SEED_BASE + 1 + 100)
    plan = ab.anova_nfft_plan(cfg["X"], cfg["windows"], cfg["sigma"], N=64, m=6, flags=ab.ANOVA_FP64)
    got = _run(torch, ab, plan, V, torch.float64)
    ref = ok.anova_matvec(cfg["X"], cfg["windows"], cfg["sigma"], V)
    for r in range(3):
        assert rel_l2(got[:, r], ref[:, r]) <= FP64_BAR


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_matches_plain_nfft_of_the_oracle(env, prec):
    torch, ab = env
    rng = np.random.default_rng(11)
    X = minmax_scale(rng.standard_normal((500, 3)))
    v = rng.standard_normal(500)
    W = np.array([[0, 1, 2]])
    if prec == "fp32":
        plan = ab.anova_nfft_plan(X, W, 0.7, N=32, m=4, flags=ab.ANOVA_FP32)
        got = _run(torch, ab, plan, v, torch.float32)
        ref = on.nfft_fastsum(X, W, 0.7, 32, 4, v)
        assert rel_l2(got, ref) <= 2e-6
    else:
        plan = ab.anova_nfft_plan(X, W, 0.7, N=32, m=4, flags=ab.ANOVA_FP64)
        got = _run(torch, ab, plan, v, torch.float64)
        ref = on.nfft_fastsum(X, W, 0.7, 32, 4, v)
        assert rel_l2(got, ref) <= 1e-12


def _small_plan(ab, prec, N=16, m=4, n=300, seed=5, dw=3):
    rng = np.random.default_rng(seed)
    X = minmax_scale(rng.standard_normal((n, dw)))
    W = np.array([list(range(dw)) + [-1] * (3 - dw)])
    flags = ab.ANOVA_FP64 if prec == "fp64" else ab.ANOVA_FP32
    plan = ab.anova_nfft_plan(X, W, 0.8, N=N, m=m, flags=flags)
    return X, W, plan, rng


@pytest.mark.parametrize("dw", [1, 2, 3])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_stage_spread(env, dw, prec):
    torch, ab = env
    X, W, plan, rng = _small_plan(ab, prec, dw=dw)
    dt = torch.float64 if prec == "fp64" else torch.float32
    v = rng.standard_normal(X.shape[0])
    n_os = 32
    grid = torch.empty((n_os,) * dw, dtype=dt, device="cuda")
    ab.anova_spread_grid(plan, 0, to_dev(torch, v, dt), grid)
    torch.cuda.synchronize()
    ref = on.spread_grid(X[:, :dw], v, n_os, 4)
    tol = 1e-13 if prec == "fp64" else 2e-6
    assert np.max(np.abs(grid.cpu().numpy().astype(np.float64) - ref)) <= tol * np.max(np.abs(ref))


@pytest.mark.parametrize("dw", [1, 2, 3])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_stage_conv(env, dw, prec):
    torch, ab = env
    X, W, plan, rng = _small_plan(ab, prec, dw=dw)
    dt = torch.float64 if prec == "fp64" else torch.float32
    n_os = 32
    g = rng.standard_normal((n_os,) * dw)
    out = torch.empty((n_os,) * dw, dtype=dt, device="cuda")
    ab.anova_conv_grid(plan, 0, torch.tensor(g, dtype=dt, device="cuda"), out)
    torch.cuda.synchronize()
    D1 = on.deconv_diag_1d(0.8, 16, 4, n_os, on.kb_beta())
    ref = on.conv_grid(g, D1)
    tol = 1e-11 if prec == "fp64" else 3e-6
    assert np.max(np.abs(out.cpu().numpy().astype(np.float64) - ref)) <= tol * np.max(np.abs(ref))


@pytest.mark.parametrize("dw", [1, 2, 3])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_stage_interp(env, dw, prec):
    torch, ab = env
    X, W, plan, rng = _small_plan(ab, prec, dw=dw)
    dt = torch.float64 if prec == "fp64" else torch.float32
    n_os = 32
    g = rng.standard_normal((n_os,) * dw)
    f = torch.empty(X.shape[0], dtype=dt, device="cuda")
    ab.anova_interp_grid(plan, 0, torch.tensor(g, dtype=dt, device="cuda"), f)
    torch.cuda.synchronize()
    ref = on.interp_grid(X[:, :dw], g, n_os, 4)
    tol = 1e-13 if prec == "fp64" else 2e-6
    assert np.max(np.abs(from_dev(f) - ref)) <= tol * np.max(np.abs(ref))


def test_mixed_window_sizes_and_per_window_scales(env):
    torch, ab = env
    rng = np.random.default_rng(21)
    X = minmax_scale(rng.standard_normal((3000, 8)))
    W = consecutive_windows(8)            # 3 + 3 + 2 features
    W = np.concatenate([W, [[7, -1, -1]]])  # and a 1-D window
    ell = np.array([0.5, 1.0, 2.0, 0.3])
    eta = np.array([1.0, 0.5, 2.0, -0.25])
    v = rng.standard_normal(3000)
    plan = ab.anova_nfft_plan_ex(X, W, ell, eta, N=32, m=4, flags=ab.ANOVA_FP32)
    got = _run(torch, ab, plan, v, torch.float32)
    ref = ok.anova_matvec(X, W, ell, v, eta=eta)
    assert rel_l2(got, ref) <= FP32_BAR
    # each window alone
    for l in range(4):
        out = torch.empty(3000, dtype=torch.float32, device="cuda")
        ab.anova_window_matvec(plan, l, to_dev(torch, v, torch.float32), out)
        torch.cuda.synchronize()
        refl = ok.anova_matvec(X, W[l:l + 1], ell[l], v, eta=eta[l:l + 1])
        assert rel_l2(from_dev(out), refl) <= FP32_BAR


def test_multi_rhs_equals_single_rhs_bitwise(env):
    torch, ab = env
    rng = np.random.default_rng(31)
    X = minmax_scale(rng.standard_normal((20000, 6)))
    W = consecutive_windows(6)
    plan = ab.anova_nfft_plan(X, W, 1.0, N=32, m=4)
    V = matvec_vectors(20000, 16, 7)
    many = _run(torch, ab, plan, V, torch.float32)
    for r in (0, 5, 15):
        one = _run(torch, ab, plan, V[:, r], torch.float32)
        assert np.array_equal(one, many[:, r])
    # and 20 columns (more than one workspace chunk)
    V20 = matvec_vectors(20000, 20, 8)
    m20 = _run(torch, ab, plan, V20, torch.float32)
    assert np.array_equal(m20[:, 19], _run(torch, ab, plan, V20[:, 19], torch.float32))


def test_deterministic_and_host_entry_point(env):
    torch, ab = env
    cfg = config1()
    v = matvec_vectors(2000, 1, 3)[:, 0]
    p1 = ab.anova_nfft_plan(cfg["X"], cfg["windows"], 1.0)
    p2 = ab.anova_nfft_plan(cfg["X"], cfg["windows"], 1.0)
    a = _run(torch, ab, p1, v, torch.float32)
    b = _run(torch, ab, p1, v, torch.float32)
    c = _run(torch, ab, p2, v, torch.float32)
    assert np.array_equal(a, b) and np.array_equal(a, c)
    vh = np.asfortranarray(v.astype(np.float32))
    kh = np.zeros_like(vh)
    ab.anova_matvec_host(p1, vh, kh, 1)
    assert np.array_equal(kh.astype(np.float64), a)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_host_entry_point_graph_reuse(env, prec):
    """Repeated host-buffer calls with the same buffers replay the captured graph: each call
    reads the buffer's current contents and gives the device path's result bitwise; other
    buffers or another nrhs take the stream path again."""
    torch, ab = env
    cfg = config1()
    n = 2000
    dt = torch.float64 if prec == "fp64" else torch.float32
    plan = (ab.anova_nfft_plan(cfg["X"], cfg["windows"], 1.0, N=64, m=6, flags=ab.ANOVA_FP64) if prec == "fp64"
            else ab.anova_nfft_plan(cfg["X"], cfg["windows"], 1.0))
    V = matvec_vectors(n, 4, 31)
    vh = torch.empty(n, dtype=dt, pin_memory=True)
    kh = torch.empty(n, dtype=dt, pin_memory=True)
    for j in range(3):  # first call captures, the next ones replay
        vh.copy_(torch.from_numpy(V[:, j]).to(dt))
        ab.anova_matvec_host(plan, vh, kh, 1)
        assert np.array_equal(kh.numpy().astype(np.float64), _run(torch, ab, plan, V[:, j], dt))
    vh2 = torch.empty((2, n), dtype=dt, pin_memory=True)
    kh2 = torch.empty((2, n), dtype=dt, pin_memory=True)
    vh2.copy_(torch.from_numpy(np.ascontiguousarray(V[:, 2:4].T)).to(dt))
    for _ in range(2):
        ab.anova_matvec_host(plan, vh2, kh2, 2)
        for r in range(2):
            assert np.array_equal(kh2[r].numpy().astype(np.float64), _run(torch, ab, plan, V[:, 2 + r], dt))
    vh.copy_(torch.from_numpy(V[:, 0]).to(dt))
    ab.anova_matvec_host(plan, vh, kh, 1)
    assert np.array_equal(kh.numpy().astype(np.float64), _run(torch, ab, plan, V[:, 0], dt))


def test_edge_cases(env):
    torch, ab = env
    W = np.array([[0, 1, 2], [3, -1, -1]])
    # n = 1: K v = P v
    x1 = np.array([[0.1, -0.2, 0.2, 0.0]])
    p = ab.anova_nfft_plan(x1, W, 1.0, flags=ab.ANOVA_FP64, N=64, m=6)
    got = _run(torch, ab, p, np.array([1.5]), torch.float64)
    assert abs(got[0] - 3.0) <= 1e-9 * 3.0
    # all points coincident: every entry of K equals P
    Xc = np.tile([[0.05, -0.1, 0.15, -0.2]], (257, 1))
    v = np.random.default_rng(1).standard_normal(257)
    p = ab.anova_nfft_plan(Xc, W, 0.5, flags=ab.ANOVA_FP64, N=64, m=6)
    got = _run(torch, ab, p, v, torch.float64)
    assert np.allclose(got, 2 * v.sum(), rtol=1e-9, atol=1e-9 * np.abs(v).sum())
    # points exactly on grid nodes, on cell edges and on the box corners
    nodes = (np.arange(-12, 13) / 64.0)[:, None]
    Xe = np.concatenate([np.hstack([nodes] * 4), [[0.2, 0.2, -0.2, -0.2], [-0.2, -0.2, 0.2, 0.2]]])
    v = np.random.default_rng(2).standard_normal(Xe.shape[0])
    p = ab.anova_nfft_plan(Xe, W, 0.7, N=32, m=4)
    got = _run(torch, ab, p, v, torch.float32)
    assert rel_l2(got, ok.anova_matvec(Xe, W, 0.7, v)) <= FP32_BAR
    # duplicate-heavy window: three binary features -> 8 distinct points
    rng = np.random.default_rng(3)
    Xb = minmax_scale(rng.integers(0, 2, size=(5000, 3)).astype(float))
    v = rng.standard_normal(5000)
    p = ab.anova_nfft_plan(Xb, np.array([[0, 1, 2]]), 1.0, N=32, m=4)
    got = _run(torch, ab, p, v, torch.float32)
    assert rel_l2(got, ok.anova_matvec(Xb, np.array([[0, 1, 2]]), 1.0, v)) <= FP32_BAR


@pytest.mark.parametrize("sigma,rows", [(1.0, 5000), (0.5, 1000), (2.0, 1000)])
def test_config2_full_size_sampled_rows(env, sigma, rows):
    """n = 1e6, three 3-D windows: rel. l2 error on a seeded row subsample vs the direct sum."""
    torch, ab = env
    cfg = config2()
    X, W = cfg["X"], cfg["windows"]
    v = matvec_vectors(X.shape[0], 1, SEED_BASE + 2 + 100)[:, 0]
    plan = ab.anova_nfft_plan(X, W, sigma, N=32, m=4)
    got = _run(torch, ab, plan, v, torch.float32)
    idx = subsample_rows(X.shape[0], rows, SEED_BASE + 2 + 200)
    ref = ok.anova_matvec(X, W, sigma, v, rows=idx)
    assert rel_l2(got[idx], ref) <= FP32_BAR


def test_config2_sixteen_rhs_sampled_rows(env):
    torch, ab = env
    cfg = config2()
    X, W = cfg["X"], cfg["windows"]
    V = matvec_vectors(X.shape[0], 16, SEED_BASE + 2 + 100)
    plan = ab.anova_nfft_plan(X, W, 1.0, N=32, m=4)
    got = _run(torch, ab, plan, V, torch.float32)
    idx = subsample_rows(X.shape[0], 300, SEED_BASE + 2 + 200)
    ref = ok.anova_matvec(X, W, 1.0, V, rows=idx)
    for r in range(16):
        assert rel_l2(got[idx, r], ref[:, r]) <= FP32_BAR


@pytest.mark.parametrize("prec,m", [("fp32", 2), ("fp32", 3), ("fp32", 5), ("fp32", 6),
                                    ("fp64", 3), ("fp64", 4), ("fp64", 5)])
def test_other_window_cutoffs_match_plain_nfft(env, prec, m):
    """Every compiled cut-off m against the oracle's plain NFFT with the same N and m."""
    torch, ab = env
    rng = np.random.default_rng(100 + m)
    X = minmax_scale(rng.standard_normal((400, 6)))
    W = np.array([[0, 1, 2], [3, 4, -1], [5, -1, -1]])
    v = rng.standard_normal(400)
    fl = ab.ANOVA_FP64 if prec == "fp64" else ab.ANOVA_FP32
    dt = torch.float64 if prec == "fp64" else torch.float32
    plan = ab.anova_nfft_plan(X, W, 0.6, N=16, m=m, flags=fl)
    got = _run(torch, ab, plan, v, dt)
    ref = on.nfft_fastsum(X, W, 0.6, 16, m, v)
    assert rel_l2(got, ref) <= (1e-12 if prec == "fp64" else 3e-6)


def _clustered(n, seed):
    """Points in [-0.2, 0.2]^3 drawn from a few tight clusters, so that cells hold hundreds of
    points (several 256-point segments per cell, several 128-point chunks per column) next to
    sparse cells."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-0.15, 0.15, size=(5, 3))
    lab = rng.integers(0, 5, size=n)
    X = centres[lab] + rng.normal(0.0, 0.004, size=(n, 3))
    X[: n // 10] = rng.uniform(-0.2, 0.2, size=(n // 10, 3))
    return np.clip(X, -0.2, 0.2)


@pytest.mark.parametrize("flags", ["tensor", "simt"])
def test_interpolation_kernels_match_oracle(env, flags):
    """Both FP32 3-D interpolation kernels (tensor-core and FP32-pipe) against the direct sum on
    clustered points (full and ragged chunks, multi-segment cells) and on workload 1."""
    torch, ab = env
    fl = ab.ANOVA_INTERP_TENSOR if flags == "tensor" else ab.ANOVA_INTERP_SIMT
    X = _clustered(12000, SEED_BASE + 50)
    W = np.array([[0, 1, 2]])
    v = matvec_vectors(X.shape[0], 1, SEED_BASE + 51)[:, 0]
    plan = ab.anova_nfft_plan(X, W, 1.0, N=32, m=4, flags=ab.ANOVA_FP32 | fl)
    assert ab.anova_plan_info(plan)["flags"] == fl
    got = _run(torch, ab, plan, v, torch.float32)
    idx = subsample_rows(X.shape[0], 1500, SEED_BASE + 52)
    assert rel_l2(got[idx], ok.anova_matvec(X, W, 1.0, v, rows=idx)) <= FP32_BAR
    cfg = config1()
    V = matvec_vectors(2000, 3, SEED_BASE + 1 + 100)
    plan = ab.anova_nfft_plan(cfg["X"], cfg["windows"], cfg["sigma"], N=32, m=4, flags=ab.ANOVA_FP32 | fl)
    got = _run(torch, ab, plan, V, torch.float32)
    ref = ok.anova_matvec(cfg["X"], cfg["windows"], cfg["sigma"], V)
    for r in range(3):
        assert rel_l2(got[:, r], ref[:, r]) <= FP32_BAR


def test_tensor_and_simt_interpolation_agree(env):
    """The two interpolation kernels compute the same sums: their difference is at the level of
    FP32 rounding (the tensor-core split keeps ~22 significant bits), far below the method's
    error, on clustered points, coincident points and a single point."""
    torch, ab = env
    W = np.array([[0, 1, 2]])
    cases = [_clustered(12000, SEED_BASE + 53), np.full((700, 3), 0.0312), np.array([[0.1, -0.05, 0.2]])]
    for X in cases:
        v = matvec_vectors(X.shape[0], 2, SEED_BASE + 54)
        outs = []
        for fl in (ab.ANOVA_INTERP_TENSOR, ab.ANOVA_INTERP_SIMT):
            plan = ab.anova_nfft_plan(X, W, 1.0, N=32, m=4, flags=ab.ANOVA_FP32 | fl)
            outs.append(_run(torch, ab, plan, v, torch.float32))
        for r in range(2):
            assert rel_l2(outs[0][:, r], outs[1][:, r]) <= 2e-6


def test_tuned_plan_matches_default_and_oracle(env):
    """The autotuned plan (work-item cap, FFT lines per CTA, interpolation form, RHS per pass,
    FP64 window streams) computes the default plan's K v up to the order of sums, and the direct
    sum within the bar."""
    torch, ab = env
    X = _clustered(60000, SEED_BASE + 60)
    X = np.column_stack([X, X[:, ::-1] * 0.9, np.roll(X, 1, axis=1)])
    W = np.array([[0, 1, 2], [3, 4, 5], [6, 7, 8]])
    V = matvec_vectors(X.shape[0], 6, SEED_BASE + 61)
    plan, rep = ab.anova_nfft_plan_tuned(X, W, 1.0, N=32, m=4, flags=ab.ANOVA_FP32, nrhs=6, reps=2)
    assert rep["wi_max"] in (1024, 2048, 4096)
    assert rep["interp"] in (ab.ANOVA_INTERP_TENSOR, ab.ANOVA_INTERP_SIMT)
    assert rep["conv_lines"] in (8, 16, 32)
    # the default setting, then 4 settings on each of 5 plans (default shape, two work-item caps,
    # two FFT line counts)
    assert rep["rhs_chunk"] in (6, 4) and rep["candidates"] == 1 + 5 * 2 * 2
    assert 0 < rep["ms"] <= rep["ms_default"]
    got = _run(torch, ab, plan, V, torch.float32)
    ref_plan = ab.anova_nfft_plan(X, W, 1.0, N=32, m=4, flags=ab.ANOVA_FP32)
    dflt = _run(torch, ab, ref_plan, V, torch.float32)
    idx = subsample_rows(X.shape[0], 800, SEED_BASE + 62)
    ref = ok.anova_matvec(X, W, 1.0, V[:, :2], rows=idx)
    for r in range(6):
        assert rel_l2(got[:, r], dflt[:, r]) <= 2e-6
    for r in range(2):
        assert rel_l2(got[idx, r], ref[:, r]) <= FP32_BAR
    # FP64: the window streams are searched too
    cfg = config1()
    V2 = matvec_vectors(2000, 2, SEED_BASE + 63)
    p64, rep64 = ab.anova_nfft_plan_tuned(cfg["X"], cfg["windows"], cfg["sigma"], N=64, m=6,
                                          flags=ab.ANOVA_FP64, nrhs=2, reps=2)
    assert rep64["interp"] == 0 and rep64["fork_windows"] in (0, 1) and rep64["candidates"] == 1 + 5 * 2
    assert rep64["conv_lines"] in (8, 16, 32)
    got64 = _run(torch, ab, p64, V2, torch.float64)
    ref64 = ok.anova_matvec(cfg["X"], cfg["windows"], cfg["sigma"], V2)
    for r in range(2):
        assert rel_l2(got64[:, r], ref64[:, r]) <= FP64_BAR


def test_matvec_batch_graph_equals_separate_matvecs(env):
    """One CUDA graph over plans of uneven size, window layout and precision gives, bitwise, each
    plan's own matvec, on every launch."""
    torch, ab = env
    rng = np.random.default_rng(SEED_BASE + 90)
    plans, vs, kvs, nrhs, refs = [], [], [], [], []
    specs = [(3000, [[0, 1, 2], [3, 4, 5]], ab.ANOVA_FP32, 1), (17000, [[0, 1, 2]], ab.ANOVA_FP32, 2),
             (800, [[0, -1, -1], [1, 2, -1]], ab.ANOVA_FP32, 1), (2500, [[0, 1, 2], [3, 4, 5]], ab.ANOVA_FP64, 1),
             (40000, [[0, 1, 2], [3, 4, 5]], ab.ANOVA_FP32, 1)]
    for n, W, fl, nr in specs:
        X = minmax_scale(rng.standard_normal((n, 6)))
        N, m = (32, 4) if fl == ab.ANOVA_FP32 else (64, 6)
        p = ab.anova_nfft_plan(X, np.array(W), 0.7, N=N, m=m, flags=fl)
        dt = torch.float32 if fl == ab.ANOVA_FP32 else torch.float64
        v = torch.tensor(rng.standard_normal((nr, n)), dtype=dt, device="cuda")
        if nr == 1:
            v = v.reshape(-1)
        ref = torch.empty_like(v)
        ab.anova_matvec(p, v, ref, nr)
        plans.append(p), vs.append(v), kvs.append(torch.empty_like(v)), nrhs.append(nr), refs.append(ref)
    torch.cuda.synchronize()
    batch = ab.anova_matvec_batch_create(plans, vs, kvs, nrhs)
    for _ in range(2):
        for k in kvs:
            k.zero_()
        batch.run()
        torch.cuda.synchronize()
        for p, k, ref in zip(plans, kvs, refs):
            ab.anova_plan_check(p)
            assert torch.equal(k, ref)
    batch.destroy()
    with pytest.raises(ab.AnovaError):
        ab.anova_matvec_batch_create([plans[0], plans[0]], vs[:1] * 2, kvs[:1] * 2)


def test_matvec_batch_refuses_a_plan_whose_workspace_was_reallocated(env):
    """A batch graph holds the addresses of its plans' workspaces. A later call with more
    right-hand sides reallocates a plan's workspace; the batch must then refuse to run instead of
    launching into freed memory, and a batch created again must run and match."""
    torch, ab = env
    rng = np.random.default_rng(SEED_BASE + 91)
    X = minmax_scale(rng.standard_normal((3000, 6)))
    p = ab.anova_nfft_plan(X, np.array([[0, 1, 2], [3, 4, 5]]), 0.7, N=32, m=4, flags=ab.ANOVA_FP32)
    v = torch.tensor(rng.standard_normal(3000), dtype=torch.float32, device="cuda")
    kv = torch.empty_like(v)
    batch = ab.anova_matvec_batch_create([p], [v], [kv], [1])
    batch.run()
    torch.cuda.synchronize()
    first = kv.clone()
    v4 = torch.tensor(rng.standard_normal((4, 3000)), dtype=torch.float32, device="cuda")
    kv4 = torch.empty_like(v4)
    ab.anova_matvec(p, v4, kv4, 4)          # grows the plan's workspace from 1 to 4 columns
    torch.cuda.synchronize()
    with pytest.raises(ab.AnovaError) as ei:
        batch.run()
    assert ei.value.status == ab.ANOVA_ERR_INVALID_ARG and "workspace" in str(ei.value)
    batch.destroy()
    batch = ab.anova_matvec_batch_create([p], [v], [kv], [1])
    kv.zero_()
    batch.run()
    torch.cuda.synchronize()
    assert torch.equal(kv, first)
    batch.destroy()
