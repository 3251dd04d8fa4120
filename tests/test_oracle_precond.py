"""Pins of the preconditioner oracle (Secs. 4-5): Algorithm 2, Nystrom, Woodbury, the
saddle-point spectrum fact, and preconditioned MINRES."""
import numpy as np
import pytest

from oracle import precond as op
from oracle import kernel as ok
from oracle import minres as om
from synth import minmax_scale, consecutive_windows


def _K(n, d, ell, seed):
    rng = np.random.default_rng(seed)
    X = minmax_scale(rng.standard_normal((n, d)))
    return ok.anova_kernel_matrix(X, consecutive_windows(d), ell), X


def test_full_rank_pivoted_cholesky_reproduces_K():
    K, _ = _K(60, 6, 0.05, 1)      # narrow kernel: well conditioned
    L, piv = op.pivoted_cholesky(K, 60)
    assert L.shape == (60, 60)
    assert np.allclose(L @ L.T, K, rtol=0, atol=1e-12 * np.max(K))
    assert sorted(piv.tolist()) == list(range(60))


def test_first_pivot_tie_goes_to_lowest_index_and_trace_decreases():
    K, _ = _K(80, 6, 0.5, 2)
    traces = []
    for r in range(1, 15):
        L, piv = op.pivoted_cholesky(K, r)
        traces.append(np.trace(K - L @ L.T))
    assert piv[0] == 0            # every diagonal entry equals P
    assert all(t2 <= t1 + 1e-12 for t1, t2 in zip(traces, traces[1:]))
    # the residual stays positive semi-definite
    lam = np.linalg.eigvalsh(K - L @ L.T)
    assert lam.min() >= -1e-10


def test_pivot_is_residual_diagonal_argmax():
    K, _ = _K(50, 3, 0.3, 3)
    L, piv = op.pivoted_cholesky(K, 6)
    for j in range(1, 6):
        res = np.diag(K) - np.sum(L[:, :j] ** 2, axis=1)
        assert piv[j] == int(np.argmax(res))


def test_rank_of_duplicated_points_is_exact():
    # 3 binary features scaled to {-0.2, 0.2}: only 8 distinct points, so rank(K_l) <= 8
    rng = np.random.default_rng(4)
    Xb = minmax_scale(rng.integers(0, 2, size=(200, 3)).astype(float))
    K = ok.anova_kernel_matrix(Xb, np.array([[0, 1, 2]]), 0.3)
    # exact arithmetic stops on a zero residual diagonal; in FP64 it is ~1e-16, so a rounding-level
    # err_tol is needed to see the stop
    L, piv = op.pivoted_cholesky(K, 50, err_tol=1e-10)
    assert L.shape[1] == 8
    assert np.allclose(L @ L.T, K, atol=1e-10)
    Zt = op.nystrom_columns(K, piv)
    assert np.allclose(Zt @ Zt.T, K, atol=1e-8)


def test_err_tol_stops_early():
    K, _ = _K(100, 3, 2.0, 5)      # wide kernel: fast spectral decay
    L, _ = op.pivoted_cholesky(K, 100, err_tol=1e-5)
    assert L.shape[1] < 40
    assert np.max(np.diag(K - L @ L.T)) <= 1e-5 * np.max(np.diag(K)) + 1e-14


def test_nystrom_classic_reproduces_chosen_columns():
    K, _ = _K(70, 6, 0.4, 6)
    idx = [3, 10, 22, 41, 55]
    Zt = op.nystrom_columns(K, idx)
    A = Zt @ Zt.T
    assert np.allclose(A[:, idx], K[:, idx], atol=1e-9)


def test_nystrom_random_full_rank_is_exact():
    K, _ = _K(30, 3, 0.05, 7)
    Zt = op.nystrom_random(K, 30, seed=8)
    assert np.allclose(Zt @ Zt.T, K, atol=1e-8)


def test_woodbury_equals_dense_inverse():
    K, _ = _K(90, 6, 0.5, 9)
    L, _ = op.pivoted_cholesky(K, 12)
    rng = np.random.default_rng(10)
    y = np.where(rng.standard_normal(90) >= 0, 1.0, -1.0)
    theta = rng.uniform(0.01, 50.0, 90)
    g = rng.standard_normal(90)
    x = op.woodbury_apply(L, theta, y, g)
    xd = np.linalg.solve(op.dense_Ahat(L, theta, y), g)
    assert np.allclose(x, xd, rtol=1e-11, atol=1e-12 * np.max(np.abs(xd)))


def test_preconditioned_spectrum_with_exact_block():
    K, _ = _K(40, 3, 0.5, 11)
    rng = np.random.default_rng(12)
    y = np.where(np.arange(40) % 3 == 0, 1.0, -1.0)
    theta = rng.uniform(0.1, 5.0, 40)
    Acal = op.saddle_matrix(K, theta, y)
    A = Acal[:40, :40]
    P = op.triangular_preconditioner(A, y)
    ev = np.sort(np.linalg.eigvals(np.linalg.solve(P, Acal)).real)
    s = y @ np.linalg.solve(A, y)
    expect = np.sort(np.concatenate([np.ones(40), [s]]))
    assert np.allclose(ev, expect, atol=1e-8)


def test_minres_matches_dense_solve_and_exact_blockdiag_converges_fast():
    K, _ = _K(60, 6, 0.5, 13)
    rng = np.random.default_rng(14)
    y = np.where(rng.standard_normal(60) >= 0, 1.0, -1.0)
    theta = rng.uniform(0.1, 2.0, 60)
    Acal = op.saddle_matrix(K, theta, y)
    b = rng.standard_normal(61)
    xd = np.linalg.solve(Acal, b)
    x, info = om.minres(lambda v: Acal @ v, b, rtol=1e-12, max_iter=500)
    assert info["converged"]
    assert np.allclose(x, xd, rtol=1e-8, atol=1e-8 * np.max(np.abs(xd)))
    # exact Ahat = A: blockdiag(A, y^T A^{-1} y) leaves at most 3 distinct eigenvalues
    A = Acal[:60, :60]
    s = y @ np.linalg.solve(A, y)
    Minv = lambda r: np.concatenate([np.linalg.solve(A, r[:60]), [r[60] / s]])
    x2, info2 = om.minres(lambda v: Acal @ v, b, apply_Minv=Minv, rtol=1e-10, max_iter=50)
    assert info2["iterations"] <= 4
    assert np.allclose(x2, xd, rtol=1e-8, atol=1e-8 * np.max(np.abs(xd)))


def test_minres_with_low_rank_preconditioner():
    K, _ = _K(80, 6, 0.5, 15)
    L, _ = op.pivoted_cholesky(K, 20)
    rng = np.random.default_rng(16)
    y = np.where(rng.standard_normal(80) >= 0, 1.0, -1.0)
    theta = rng.uniform(0.01, 1.0, 80)
    Acal = op.saddle_matrix(K, theta, y)
    b = rng.standard_normal(81)
    s = y @ op.woodbury_apply(L, theta, y, y)
    Minv = lambda r: op.blockdiag_apply(L, theta, y, r, s)
    x, info = om.minres(lambda v: Acal @ v, b, apply_Minv=Minv, rtol=1e-11, max_iter=300)
    xd = np.linalg.solve(Acal, b)
    assert info["converged"]
    assert np.allclose(x, xd, rtol=1e-7, atol=1e-7 * np.max(np.abs(xd)))


def test_splitmix64_reference_outputs():
    """The first outputs of SplitMix64 started at 0, as published with the generator."""
    assert [op.splitmix64(0, j) for j in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                       0x06C45D188009454F]
    u = np.array([op.uniform01(123, j) for j in range(20000)])
    assert 0.0 <= u.min() and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01 and abs(u.var() - 1 / 12) < 0.005


def test_rp_cholesky_full_rank_and_triangular_structure():
    rng = np.random.default_rng(5)
    X = rng.uniform(-0.2, 0.2, size=(24, 3))
    K = ok.anova_kernel_matrix(X, np.array([[0, 1, 2]]), 0.3)
    L, piv = op.rp_cholesky(K, 24, seed=7)
    assert len(set(piv.tolist())) == len(piv)                       # no pivot twice
    assert np.allclose(L @ L.T, K, atol=1e-10 * np.max(K)) or len(piv) < 24
    # in pivot order L is lower triangular
    Lp = L[piv, :]
    assert np.max(np.abs(np.triu(Lp, 1))) <= 1e-12
    # at the rank it reached, the residual diagonal is what the factor leaves
    assert np.allclose(np.diag(K - L @ L.T), np.maximum(np.diag(K) - np.sum(L ** 2, axis=1), 0.0),
                       atol=1e-10)


def test_rp_cholesky_draws_in_proportion_to_the_residual_diagonal():
    """Over many seeds the first pivot is uniform (equal diagonal) and the second pivot, given the
    first, follows the residual diagonal after one step."""
    K = np.array([[1.0, 0.9, 0.1, 0.0], [0.9, 1.0, 0.2, 0.1], [0.1, 0.2, 1.0, 0.5], [0.0, 0.1, 0.5, 1.0]])
    first = np.zeros(4)
    second_after0 = np.zeros(4)
    for seed in range(4000):
        _, piv = op.rp_cholesky(K, 2, seed=seed)
        first[piv[0]] += 1
        if piv[0] == 0:
            second_after0[piv[1]] += 1
    assert np.all(np.abs(first / 4000 - 0.25) < 4 * np.sqrt(0.25 * 0.75 / 4000))
    d1 = 1.0 - K[:, 0] ** 2                      # residual diagonal after pivot 0
    p = d1 / d1.sum()
    m = second_after0.sum()
    assert second_after0[0] == 0
    assert np.all(np.abs(second_after0 / m - p) < 4 * np.sqrt(p * (1 - p) / m) + 1e-12)


def test_rp_cholesky_with_argmax_draws_is_algorithm_2():
    """Replacing the draw by the first arg-max of the residual diagonal gives the greedy factor of
    Algorithm 2 (pivots and columns): the column formula is Algorithm 2's."""
    rng = np.random.default_rng(9)
    X = rng.uniform(-0.2, 0.2, size=(40, 3))
    K = ok.anova_kernel_matrix(X, np.array([[0, 1, 2]]), 0.5)
    Lg, pg = op.pivoted_cholesky(K, 12)
    L, piv = op.rp_cholesky(K, 12, seed=0, pick=lambda d, j: int(np.argmax(d)))
    assert piv.tolist() == pg.tolist()
    assert np.allclose(L, Lg, atol=1e-12)


def test_per_window_stacked_factor():
    """Stacking per-window factors: at full rank per window the product is the summed kernel, and
    each block of columns is Algorithm 2 on its own window's matrix."""
    rng = np.random.default_rng(21)
    X = rng.uniform(-0.2, 0.2, size=(30, 6))
    W = np.array([[0, 1, 2], [3, 4, 5]])
    Ks = [ok.window_kernel_matrix(X, w, 0.3) for w in W]
    L, piv = op.per_window_cholesky(Ks, 30)
    assert np.allclose(L @ L.T, ok.anova_kernel_matrix(X, W, 0.3), atol=1e-9)
    L1, p1 = op.pivoted_cholesky(Ks[0], 30)
    assert np.array_equal(piv[: p1.size], p1) and np.allclose(L[:, : p1.size], L1)
    Lk, _ = op.per_window_cholesky(Ks, 5)
    assert Lk.shape == (30, 10)


def test_splitmix64_array_matches_scalar():
    j = np.array([0, 1, 2, 7, 12345, 2 ** 40 + 3], dtype=np.uint64)
    for seed in (0, 99, 2 ** 63 + 7):
        got = op.splitmix64_array(seed, j)
        assert [int(g) for g in got] == [op.splitmix64(seed, int(x)) for x in j]


def test_gaussian_matrix_is_standard_normal():
    """Box-Muller over SplitMix64: moments and the Kolmogorov-Smirnov distance to N(0, 1)."""
    from scipy import stats
    G = op.gaussian_matrix(4000, 5, seed=31)
    assert G.shape == (4000, 5)
    g = G.ravel()
    assert abs(g.mean()) < 0.03 and abs(g.var() - 1.0) < 0.04
    assert stats.kstest(g, "norm").pvalue > 1e-3
    # column-major numbering: column j continues where column j - 1 stopped
    G2 = op.gaussian_matrix(8000, 1, seed=31)
    assert np.array_equal(G2[4000:, 0], G[:, 1])


def test_nystrom_random_depends_on_the_range_only():
    """(K Q)(Q^T K Q)^{-1}(K Q)^T is the same for every orthonormal basis of range(K G); it is a
    lower approximation (K - Z Z^T is PSD); it is exact when k reaches the numerical rank."""
    K, _ = _K(60, 3, 0.5, 13)
    Zt = op.nystrom_random(K, 8, seed=5)
    G = op.gaussian_matrix(60, 8, seed=5)
    R = np.linalg.qr(np.random.default_rng(1).standard_normal((8, 8)))[0]
    Q2 = np.linalg.svd(K @ G @ R, full_matrices=False)[0]
    Z2 = op.nystrom(K, Q2)
    assert np.allclose(Zt @ Zt.T, Z2 @ Z2.T, atol=1e-9)
    assert np.min(np.linalg.eigvalsh(K - Zt @ Zt.T)) > -1e-9
    assert np.trace(K - Zt @ Zt.T) < np.trace(K)
