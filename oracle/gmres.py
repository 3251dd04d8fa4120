"""ORACLE -- test infrastructure only. Right-preconditioned GMRES (Saad and Schultz, 1986), the
Krylov method the paper applies with its non-symmetric block-triangular preconditioner (Sec. 5).

Solves A x = b from x0 = 0 with A P^{-1} u = b, x = P^{-1} u. Arnoldi with modified Gram-Schmidt
builds an orthonormal basis V of the Krylov space of A P^{-1}; Givens rotations keep the
Hessenberg matrix triangular; after each step |g_{j+1}| is the norm of the true residual
b - A x_j (right preconditioning minimises the unpreconditioned residual). No restart: the loop
stops when that norm is <= rtol ||b|| or after max_iter steps.

Reading: the paper states the spectrum of P^{-1} A (Sec. 5); A P^{-1} is similar to it
(A P^{-1} = P (P^{-1} A) P^{-1}), so with the exact (1,1) block it has n unit eigenvalues and one
equal to y^T A^{-1} y, and GMRES converges in at most two steps.
"""
import numpy as np


def gmres(apply_A, b, apply_Pinv=None, rtol=1e-8, max_iter=100):
    b = np.asarray(b, dtype=np.float64)
    Pinv = apply_Pinv if apply_Pinv is not None else (lambda r: r)
    n = b.size
    beta = float(np.linalg.norm(b))
    if beta == 0.0:
        return np.zeros(n), dict(iterations=0, resid=0.0, converged=True, history=[0.0])
    m = max_iter
    V = np.zeros((n, m + 1))
    H = np.zeros((m + 1, m))
    cs = np.zeros(m)
    sn = np.zeros(m)
    g = np.zeros(m + 1)
    g[0] = beta
    V[:, 0] = b / beta
    history = [beta]
    j = 0
    converged = False
    while j < m:
        w = apply_A(Pinv(V[:, j]))
        for i in range(j + 1):                       # modified Gram-Schmidt
            H[i, j] = V[:, i] @ w
            w = w - H[i, j] * V[:, i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] > 0.0:
            V[:, j + 1] = w / H[j + 1, j]
        for i in range(j):                           # earlier rotations on the new column
            t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
            H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
            H[i, j] = t
        rho = np.hypot(H[j, j], H[j + 1, j])         # new rotation zeroes H[j+1, j]
        cs[j], sn[j] = H[j, j] / rho, H[j + 1, j] / rho
        H[j, j] = rho
        H[j + 1, j] = 0.0
        g[j + 1] = -sn[j] * g[j]
        g[j] = cs[j] * g[j]
        j += 1
        history.append(abs(g[j]))
        if abs(g[j]) <= rtol * beta:
            converged = True
            break
    y = np.linalg.solve(np.triu(H[:j, :j]), g[:j]) if j else np.zeros(0)
    x = Pinv(V[:, :j] @ y)
    return x, dict(iterations=j, resid=history[-1], converged=converged, history=history)


def triangular_apply(apply_Ahat_inv, y, g):
    """P^{-1} g for the paper's P = [[A^, 0], [-y^T, -1]] (Sec. 5): x1 = A^{-1} g1 and, from
    -y^T x1 - x2 = g2, x2 = -(g2 + y^T x1)."""
    n = y.size
    out = np.empty(n + 1)
    out[:n] = apply_Ahat_inv(g[:n])
    out[n] = -(g[n] + y @ out[:n])
    return out
