"""ORACLE -- test infrastructure only. Low-rank kernel approximations and the saddle-point
preconditioner, dense FP64 (Secs. 4 and 5).

* pivoted_cholesky: Algorithm 2 (greedy pivoted Cholesky of rank k, outer-product form),
  in place on a dense copy of K. Reading C-13: ties go to the lowest index, and the loop also
  stops once the largest residual diagonal is <= err_tol * max(diag K) (Table 1: err_tol = 1e-5).
* nystrom: K ~ (K Q)(Q^T K Q)^{-1}(K Q)^T (Sec. 4), with the core factored as L D L^T and diagonal
  entries below a threshold replaced by that threshold (reading C-16: 1e-10 * max D).
* woodbury_apply: A^ = Theta + Y Z^T Z Y and A^{-1} = Theta^{-1} - Theta^{-1} Y Z^T
  (I_k + Z Y Theta^{-1} Y Z^T)^{-1} Z Y Theta^{-1} (Sec. 5).
* saddle preconditioner: the paper's P = [[A^, 0], [-y^T, -1]] (Sec. 5), and the block-diagonal
  SPD form blockdiag(A^, y^T A^{-1} y) used with MINRES (reading C-12).
"""
import numpy as np


def pivoted_cholesky(K, k, err_tol=0.0):
    """Algorithm 2 on a dense copy of K. Returns (L, piv): L is n x r with K ~ L L^T in the
    ORIGINAL row order, piv the r pivot indices in the order they were chosen."""
    A = np.array(K, dtype=np.float64, copy=True)
    n = A.shape[0]
    perm = np.arange(n)
    r = 0
    dmax0 = float(np.max(np.diag(A))) if n else 0.0
    for j in range(n):
        diag = np.diag(A)[j:]
        l = j + int(np.argmax(diag))          # first maximal entry: ties -> lowest position
        if not (A[l, l] > 0 and r < k):
            break
        if A[l, l] <= err_tol * dmax0:
            break
        r += 1
        # symmetric swap of rows/columns j and l
        A[[j, l], :] = A[[l, j], :]
        A[:, [j, l]] = A[:, [l, j]]
        perm[[j, l]] = perm[[l, j]]
        A[j, j] = np.sqrt(A[j, j])
        A[j + 1:, j] = A[j + 1:, j] / A[j, j]
        for i in range(j + 1, n):
            A[i:, i] = A[i:, i] - A[i:, j] * A[i, j]
        # keep the trailing block symmetric so its diagonal and later swaps stay consistent
        A[j + 1:, j + 1:] = np.tril(A[j + 1:, j + 1:]) + np.tril(A[j + 1:, j + 1:], -1).T
    Lp = np.tril(A[:, :r])
    L = np.zeros((n, r))
    L[perm, :] = Lp
    return L, perm[:r].copy()


def nystrom(K, Q, rel_threshold=1e-10):
    """K ~ C W^+ C^T with C = K Q and W = Q^T K Q factored as L D L^T (D thresholded).

    Returns a factor Zt (n x k) with K ~ Zt Zt^T."""
    K = np.asarray(K, dtype=np.float64)
    C = K @ Q
    W = Q.T @ C
    W = 0.5 * (W + W.T)
    L, D = ldl_nopivot(W)
    thr = rel_threshold * max(1e-300, float(np.max(np.abs(D))))
    D = np.where(D < thr, thr, D)
    # W^{-1} = L^{-T} D^{-1} L^{-1}  =>  C W^{-1} C^T = (C L^{-T} D^{-1/2})(...)^T
    X = np.linalg.solve(L, C.T)            # L^{-1} C^T
    Zt = (X / np.sqrt(D)[:, None]).T
    return Zt


def ldl_nopivot(W):
    """W = L D L^T with unit lower-triangular L (no pivoting), FP64."""
    n = W.shape[0]
    L = np.eye(n)
    D = np.zeros(n)
    for j in range(n):
        D[j] = W[j, j] - np.sum(L[j, :j] ** 2 * D[:j])
        for i in range(j + 1, n):
            piv = D[j] if D[j] != 0 else 1e-300
            L[i, j] = (W[i, j] - np.sum(L[i, :j] * L[j, :j] * D[:j])) / piv
    return L, D


def nystrom_columns(K, idx, rel_threshold=1e-10):
    """Classic Nystrom: Q = columns idx of the identity."""
    n = K.shape[0]
    Q = np.zeros((n, len(idx)))
    Q[np.asarray(idx), np.arange(len(idx))] = 1.0
    return nystrom(K, Q, rel_threshold)


def nystrom_random(K, k, seed, rel_threshold=1e-10):
    """Q = orth(K G) with the Gaussian G = gaussian_matrix(n, k, seed) (Sec. 4, the randomised
    Nystrom range), orthonormalised by a Householder QR (reading C-16)."""
    G = gaussian_matrix(K.shape[0], k, seed)
    Q, _ = np.linalg.qr(K @ G)
    return nystrom(K, Q, rel_threshold)


def woodbury_apply(Zt, theta, y, g):
    """A^{-1} g for A^ = Theta + Y Z^T Z Y, Z = Zt^T (k x n), by the Woodbury identity."""
    Z = Zt.T
    ti = 1.0 / theta
    core = np.eye(Z.shape[0]) + (Z * (y * ti * y)[None, :]) @ Z.T
    u = Z @ (y * ti * g)
    return ti * g - ti * y * (Z.T @ np.linalg.solve(core, u))


def dense_Ahat(Zt, theta, y):
    return np.diag(theta) + (y[:, None] * (Zt @ Zt.T)) * y[None, :]


def saddle_matrix(K, theta, y):
    """The Newton matrix of eq. (Newton): [[Y K Y + Theta, -y], [-y^T, 0]]."""
    n = y.size
    A = np.zeros((n + 1, n + 1))
    A[:n, :n] = (y[:, None] * K) * y[None, :] + np.diag(theta)
    A[:n, n] = -y
    A[n, :n] = -y
    return A


def triangular_preconditioner(Ahat, y):
    """The paper's P = [[A^, 0], [-y^T, -1]] (Sec. 5)."""
    n = y.size
    P = np.zeros((n + 1, n + 1))
    P[:n, :n] = Ahat
    P[n, :n] = -y
    P[n, n] = -1.0
    return P


def blockdiag_apply(Zt, theta, y, g, s):
    """MINRES preconditioner blockdiag(A^, s)^{-1} g with s = y^T A^{-1} y (reading C-12)."""
    n = y.size
    out = np.empty(n + 1)
    out[:n] = woodbury_apply(Zt, theta, y, g[:n])
    out[n] = g[n] / s
    return out


_GOLDEN_GAMMA = 0x9E3779B97F4A7C15
_MASK64 = (1 << 64) - 1


def splitmix64(seed, j):
    """Output number j (0-based) of SplitMix64 started at `seed` (Steele, Lea and Flood, 2014; the
    generator behind Java's SplittableRandom): the state seed + (j + 1) * 0x9E3779B97F4A7C15 passed
    through the generator's 64-bit finaliser."""
    z = (int(seed) + (int(j) + 1) * _GOLDEN_GAMMA) & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def uniform01(seed, j):
    """The top 53 bits of splitmix64(seed, j) as a double in [0, 1)."""
    return (splitmix64(seed, j) >> 11) * 2.0 ** -53


def _rp_draw(seed):
    def draw(d, j):
        c = np.cumsum(np.maximum(d, 0.0))
        return int(np.searchsorted(c, uniform01(seed, j) * c[-1], side="right"))
    return draw


def rp_cholesky(K, k, seed, err_tol=0.0, pick=None):
    """Randomly pivoted Cholesky (Sec. 4, the variant after Algorithm 2): every pivot is drawn with
    probability proportional to the current residual diagonal d. The draw of step j is the first
    index s (in index order) with cumsum(max(d, 0))[s] > u_j * sum(max(d, 0)), u_j =
    uniform01(seed, j); an entry with d <= 0 is never drawn (the index moves back to the last
    positive entry). Columns as in Algorithm 2: L(:, j) = (K(:, s) - L(:, :j) L(s, :j)^T) /
    sqrt(d_s), d -= L(:, j)^2. Stops at rank k or, as the greedy version, when max(d) <= err_tol *
    max(diag K). Returns (L, piv) with K ~ L L^T in the original row order. `pick(d, j)` replaces
    the draw (tests use the arg-max to recover the greedy Algorithm 2)."""
    pick = _rp_draw(seed) if pick is None else pick
    K = np.asarray(K, dtype=np.float64)
    n = K.shape[0]
    d = np.diag(K).copy()
    dmax0 = float(np.max(d)) if n else 0.0
    L = np.zeros((n, k))
    piv = []
    for j in range(min(k, n)):
        dm = float(np.max(d))
        if not (dm > 0.0) or dm <= err_tol * dmax0:
            break
        s = min(pick(d, j), n - 1)
        # entries with zero weight are never drawn: a target that rounding puts at or past the end
        # of the cumulative sum moves to the last positive entry before it
        while s > 0 and not d[s] > 0.0:
            s -= 1
        col = K[:, s] - L[:, :j] @ L[s, :j]
        L[:, j] = col / np.sqrt(d[s])
        d = d - L[:, j] ** 2
        piv.append(s)
    r = len(piv)
    return L[:, :r].copy(), np.array(piv, dtype=np.int64)


def per_window_cholesky(Ks, k, err_tol=0.0):
    """Per-window stacked factors (Sec. 4, the stacking of per-window low-rank factors):
    sum_l K_l ~ sum_l L_l L_l^T = [L_1 ... L_P][L_1 ... L_P]^T, each L_l the greedy pivoted
    Cholesky (Algorithm 2) of one window's kernel matrix K_l at rank k. Returns the stacked factor
    (n x sum of the ranks reached) and the pivots, window after window."""
    Ls, pivs = [], []
    for K in Ks:
        L, piv = pivoted_cholesky(K, k, err_tol)
        Ls.append(L)
        pivs.append(piv)
    return np.hstack(Ls), np.concatenate(pivs)


def splitmix64_array(seed, j):
    """splitmix64(seed, j) for an integer array j, in wrapping uint64 arithmetic."""
    j = np.asarray(j, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(int(seed) & _MASK64) + (j + np.uint64(1)) * np.uint64(_GOLDEN_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def gaussian_matrix(n, k, seed):
    """Standard normal G (n x k) for the randomised Nystrom range K G (Sec. 4), drawn so that any
    implementation of the same published generators reproduces it: entry (i, j), t = j n + i, is
    the Box-Muller transform (Box and Muller, 1958) sqrt(-2 ln(1 - u)) cos(2 pi u') of the uniforms
    u = uniform01(seed, 2t), u' = uniform01(seed, 2t + 1) (1 - u lies in (0, 1], so the log is
    finite)."""
    t = np.arange(n * k, dtype=np.uint64).reshape(k, n).T          # column-major t = j n + i
    u = (splitmix64_array(seed, 2 * t) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    u2 = (splitmix64_array(seed, 2 * t + 1) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return np.sqrt(-2.0 * np.log(1.0 - u)) * np.cos(2.0 * np.pi * u2)
