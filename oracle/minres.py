"""ORACLE -- test infrastructure only. Preconditioned MINRES (Paige and Saunders, 1975), the
Krylov method named for symmetric saddle systems in Sec. 3 and Sec. 5.

Solves A x = b for symmetric A with a symmetric positive definite preconditioner M, given as
apply_Minv(r) = M^{-1} r. Lanczos on the M-inner product, Givens rotations on the tridiagonal,
three-term update of the iterate. The residual estimate is the preconditioned norm
||r||_{M^{-1}}; the loop stops when it drops below rtol times its initial value.
"""
import numpy as np


def minres(apply_A, b, apply_Minv=None, rtol=1e-8, max_iter=1000, x0=None):
    b = np.asarray(b, dtype=np.float64)
    Minv = apply_Minv if apply_Minv is not None else (lambda r: r)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r1 = b - apply_A(x)
    y = Minv(r1)
    beta1 = float(r1 @ y)
    if beta1 < 0:
        raise ValueError("preconditioner is not positive definite")
    beta1 = np.sqrt(beta1)
    if beta1 == 0.0:
        return x, dict(iterations=0, resid=0.0, converged=True)
    # Lanczos vectors (unscaled r, scaled by 1/beta to give v)
    r_prev = np.zeros_like(b)
    r_cur = r1.copy()
    y_cur = y
    beta = beta1
    beta_prev = 0.0
    # rotation and search-direction state
    c_prev2, s_prev2 = 1.0, 0.0   # rotation two steps back (unused at k=1)
    c_prev, s_prev = 1.0, 0.0     # rotation one step back
    phibar = beta1
    w_prev2 = np.zeros_like(b)
    w_prev = np.zeros_like(b)
    it = 0
    resid = beta1
    converged = False
    while it < max_iter:
        it += 1
        v = y_cur / beta
        Av = apply_A(v)
        alpha = float(v @ Av)
        r_next = Av - (alpha / beta) * r_cur - (beta / beta_prev if beta_prev else 0.0) * r_prev
        y_next = Minv(r_next)
        beta_next = float(r_next @ y_next)
        if beta_next < 0:
            raise ValueError("preconditioner is not positive definite")
        beta_next = np.sqrt(beta_next)
        # apply the previous two rotations to the new tridiagonal column (beta, alpha, beta_next)
        eps_k = s_prev2 * beta
        dbar = c_prev2 * beta
        delta_k = c_prev * dbar + s_prev * alpha
        gbar = -s_prev * dbar + c_prev * alpha
        # new rotation annihilating beta_next
        gamma = np.hypot(gbar, beta_next)
        if gamma == 0.0:
            gamma = 1e-300
        c_k, s_k = gbar / gamma, beta_next / gamma
        phi = c_k * phibar
        phibar = -s_k * phibar
        w = (v - eps_k * w_prev2 - delta_k * w_prev) / gamma
        x = x + phi * w
        resid = abs(phibar)
        # shift state
        w_prev2, w_prev = w_prev, w
        c_prev2, s_prev2, c_prev, s_prev = c_prev, s_prev, c_k, s_k
        r_prev, r_cur, y_cur = r_cur, r_next, y_next
        beta_prev, beta = beta, beta_next
        if resid <= rtol * beta1:
            converged = True
            break
        if beta == 0.0:
            converged = True
            break
    return x, dict(iterations=it, resid=resid / beta1, converged=converged)
