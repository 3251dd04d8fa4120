"""Seeded input generators (NumPy ``default_rng``, FP64).

Recipes (seed = SEED_BASE + workload number):

* workload 1 (small plain method): n=2000, d=6, X ~ N(0,1); labels from the RAW features,
  y = sign(sin(3 x1) + x2 x3 - x4^2 + 0.5 x5 x6 + 0.1 eps), sign(0) -> +1; windows {0,1,2},{3,4,5};
  sigma = 1, C = 1.
* workload 2 (matvec throughput): n=1e6, d=9, X ~ N(0,1); windows {0-2},{3-5},{6-8}.
* workload 3 (IPM with low-rank preconditioner): n=1e5, d=12 = 8 x N(0,1) + 4 x Bernoulli(1/2) in
  {0,1}; four consecutive 3-D windows; labels from a random two-layer tanh teacher of width 32
  with 5 % of the labels flipped.

Every feature is then min-max scaled into [-0.2, 0.2] = [-1/4 + 0.05, 1/4 - 0.05], the box the
NFFT plan requires; a constant feature maps to 0.
"""
import numpy as np

SEED_BASE = 2312_00538
LO, HI = -0.2, 0.2


def minmax_scale(X):
    """Per-feature affine map of X (n x d) onto [-0.2, 0.2]; constant features map to 0."""
    X = np.asarray(X, dtype=np.float64)
    mn = X.min(axis=0)
    mx = X.max(axis=0)
    span = mx - mn
    out = np.zeros_like(X)
    ok = span > 0
    out[:, ok] = LO + (HI - LO) * (X[:, ok] - mn[ok]) / span[ok]
    return out


def consecutive_windows(d, width=3):
    """Consecutive feature windows of `width` features; the last one may be shorter.

    Returned as a P x 3 int32 array, 0-based, padded with -1."""
    P = (d + width - 1) // width
    W = -np.ones((P, 3), dtype=np.int32)
    for l in range(P):
        feats = list(range(l * width, min(d, (l + 1) * width)))
        W[l, :len(feats)] = feats
    return W


def _sign(z):
    return np.where(z >= 0, 1.0, -1.0)


def config1(n=2000, seed=None):
    """Workload 1. Returns dict(X, y, windows, sigma, C, X_raw)."""
    rng = np.random.default_rng(SEED_BASE + 1 if seed is None else seed)
    d = 6
    Xr = rng.standard_normal((n, d))
    eps = rng.standard_normal(n)
    x1, x2, x3, x4, x5, x6 = (Xr[:, k] for k in range(6))
    y = _sign(np.sin(3 * x1) + x2 * x3 - x4 ** 2 + 0.5 * x5 * x6 + 0.1 * eps)
    return dict(X=minmax_scale(Xr), y=y, windows=consecutive_windows(d), sigma=1.0, C=1.0,
                X_raw=Xr)


def config2(n=1_000_000, seed=None):
    """Workload 2 points (labels are not needed for the matvec benchmark)."""
    rng = np.random.default_rng(SEED_BASE + 2 if seed is None else seed)
    d = 9
    Xr = rng.standard_normal((n, d))
    return dict(X=minmax_scale(Xr), windows=consecutive_windows(d))


def _tanh_teacher(rng, Xr, width=32):
    n, d = Xr.shape
    W1 = rng.standard_normal((width, d)) / np.sqrt(d)
    b1 = 0.1 * rng.standard_normal(width)
    w2 = rng.standard_normal(width) / np.sqrt(width)
    f = np.tanh(Xr @ W1.T + b1) @ w2
    f = f - np.median(f)
    return f


def config3(n=100_000, seed=None, flip=0.05):
    """Workload 3: 8 Gaussian + 4 binary features, tanh teacher, 5 % label flips."""
    rng = np.random.default_rng(SEED_BASE + 3 if seed is None else seed)
    Xg = rng.standard_normal((n, 8))
    Xb = rng.integers(0, 2, size=(n, 4)).astype(np.float64)
    Xr = np.concatenate([Xg, Xb], axis=1)
    f = _tanh_teacher(rng, Xr)
    y = _sign(f)
    nflip = int(round(flip * n))
    idx = rng.choice(n, size=nflip, replace=False)
    y[idx] = -y[idx]
    return dict(X=minmax_scale(Xr), y=y, windows=consecutive_windows(12), sigma=1.0, C=10.0,
                X_raw=Xr)


def small_problem(n, d, seed, binary_features=0):
    """A small labelled problem of the workload-3 kind (Gaussian + binary features, teacher)."""
    rng = np.random.default_rng(seed)
    Xg = rng.standard_normal((n, d - binary_features))
    Xb = rng.integers(0, 2, size=(n, binary_features)).astype(np.float64)
    Xr = np.concatenate([Xg, Xb], axis=1)
    y = _sign(_tanh_teacher(rng, Xr))
    return dict(X=minmax_scale(Xr), y=y, windows=consecutive_windows(d), X_raw=Xr)


def matvec_vectors(n, nrhs, seed):
    """nrhs vectors v ~ N(0,1), returned column-major as an (n, nrhs) Fortran-ordered array."""
    rng = np.random.default_rng(seed)
    V = rng.standard_normal((nrhs, n))
    return np.asfortranarray(V.T)


def subsample_rows(n, k, seed):
    """k distinct row indices of [0, n), sorted."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=min(k, n), replace=False)).astype(np.int64)


C_GRID = (0.1, 1.0, 10.0, 100.0)
SIGMA_GRID = (0.5, 1.0, 2.0, 4.0)


def config4(count=64, n_lo=5_000, n_hi=200_000, seed=None, d=9):
    """Workload 4: `count` independent problems, n log-uniform in [n_lo, n_hi], d = 9 (three 3-D
    windows), labels from the tanh teacher with 5 % flips, (C, sigma) = grid[i mod 16] of
    C in {0.1, 1, 10, 100} x sigma in {0.5, 1, 2, 4}."""
    rng = np.random.default_rng(SEED_BASE + 4 if seed is None else seed)
    ns = np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), size=count)).astype(np.int64)
    probs = []
    for i in range(count):
        sub = np.random.default_rng(SEED_BASE + 4000 + i)
        n = int(ns[i])
        Xr = sub.standard_normal((n, d))
        y = _sign(_tanh_teacher(sub, Xr))
        flip = sub.choice(n, size=int(round(0.05 * n)), replace=False)
        y[flip] = -y[flip]
        g = i % 16
        probs.append(dict(X=minmax_scale(Xr), y=y, windows=consecutive_windows(d),
                          C=C_GRID[g // 4], sigma=SIGMA_GRID[g % 4]))
    return probs


def config5(count, rate, seed=None, n_lo=10_000, n_hi=500_000):
    """Workload 5 (serving): `count` SVM solve requests arriving as a Poisson stream of `rate`
    requests per second. Request i: n log-uniform in [n_lo, n_hi], d uniform in {6, 9, 12, 15, 18}
    (consecutive 3-D windows), (C, sigma) drawn from the grid of workload 4, 8 of every 12 features
    N(0,1) and the rest Bernoulli(1/2) as in workload 3, labels from the tanh teacher with 5 % flips.
    Returns a list of dicts with keys X, y, windows, C, sigma and arrival (seconds from the start)."""
    rng = np.random.default_rng(SEED_BASE + 5 if seed is None else seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=count))
    ns = np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), size=count)).astype(np.int64)
    ds = rng.choice([6, 9, 12, 15, 18], size=count)
    grid = rng.integers(0, 16, size=count)
    reqs = []
    for i in range(count):
        sub = np.random.default_rng(SEED_BASE + 5000 + i)
        n, d = int(ns[i]), int(ds[i])
        nb = d // 3
        Xg = sub.standard_normal((n, d - nb))
        Xb = sub.integers(0, 2, size=(n, nb)).astype(np.float64)
        Xr = np.concatenate([Xg, Xb], axis=1)
        y = _sign(_tanh_teacher(sub, Xr))
        flip = sub.choice(n, size=int(round(0.05 * n)), replace=False)
        y[flip] = -y[flip]
        g = int(grid[i])
        reqs.append(dict(X=minmax_scale(Xr), y=y, windows=consecutive_windows(d), C=C_GRID[g // 4],
                         sigma=SIGMA_GRID[g % 4], arrival=float(arrivals[i])))
    return reqs

