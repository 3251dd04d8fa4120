"""ORACLE -- test infrastructure only. Algorithm 1 (interior point method for the SVM dual) with
dense FP64 Newton solves, plus the SVM quantities used to check it.

Problem (Sec. 1, eq. (kernelsvm)): max_alpha e^T alpha - 1/2 alpha^T Y K Y alpha subject to
0 <= alpha_i <= C and y^T alpha = 0.

Barrier Lagrangian and optimality conditions: Sec. 2. Newton system: Sec. 2, eq. (Newton):
    [[Y K Y + Theta, -y], [-y^T, 0]] [d_alpha; d_lambda]
        = [e - Y K Y a + l y + mu e./a - mu e./(C e - a);  y^T a],
    Theta = diag(mu (1/a^2 + 1/(C - a)^2)).

Readings of points the paper leaves open:
* initial point: alpha^0 = min(C/2, 1/2) e, lambda^0 = 0 (the paper only asks for non-zero
  initial infeasibilities); relative infeasibilities are divided by max(1, ||xi^0||) so that a
  zero xi^0 (balanced labels) does not divide by zero.
* barrier schedule: Sec. 2 reduces mu either by a constant sigma or by a sigma_it that changes
  every iteration. sigma_rule="constant" is mu <- 0.6 mu (Table 1); sigma_rule="adaptive" (the
  default) is sigma_it = 1 - (1 - 0.6) s_{it-1} with s_{it-1} the previous step length (s_{-1} =
  1), which equals the constant rule while full steps are taken and keeps mu while the step is
  short. With the constant rule and alpha^0 = C/2 the method stalls at the boundary for C = 10 or
  100 even with exact solves. Either way mu is reduced before the Newton solve, so Theta and the
  right-hand side use mu_{it+1}.
* step lengths (C-9): s = gamma_0 * max{s <= 1 : 0 <= alpha + s d_alpha <= C}; s_lambda = s_alpha.
* stopping: stop="alg1" is Algorithm 1's loop test (continue while mu > tol or either relative
  infeasibility is above tol); stop="gap" is reading C-10 (stop once the relative duality gap
  (P - D) / max(1, |P|) and the relative infeasibility |y^T alpha| / max(1, |xi_alpha^0|) are both
  <= tol). Either way at most max_iter iterations (Table 1: 50). The loop also ends if rounding
  has put an alpha_i exactly on a bound, where Theta is no longer finite (a variable that
  converges to a bound sits at distance ~mu from it, below FP64 resolution for tiny tol).
* bias (C-11): lambda is the multiplier of y^T alpha = 0, so the decision function is
  f(x) = sum_i alpha_i y_i kappa(x_i, x) + b with b = -lambda.
"""
import numpy as np


def dual_objective(K, y, alpha):
    """D(alpha) = e^T alpha - 1/2 alpha^T Y K Y alpha (eq. (kernelsvm))."""
    ya = y * alpha
    return float(alpha.sum() - 0.5 * ya @ (K @ ya))


def primal_objective(K, y, alpha, b, C):
    """Soft-margin primal at w = sum_i alpha_i y_i phi(x_i) and the given bias (Sec. 1):
    1/2 ||w||^2 + C sum_i max(0, 1 - y_i (w^T phi(x_i) + b))."""
    ya = y * alpha
    f = K @ ya
    return float(0.5 * ya @ f + C * np.maximum(0.0, 1.0 - y * (f + b)).sum())


def duality_gap(K, y, alpha, b, C):
    return primal_objective(K, y, alpha, b, C) - dual_objective(K, y, alpha)


def newton_rhs(Q, y, alpha, lam, mu, C):
    """Right-hand side of eq. (Newton) (equivalently xi_lambda, xi_alpha of Algorithm 1)."""
    r1 = 1.0 - Q @ alpha + lam * y + mu / alpha - mu / (C - alpha)
    r2 = float(y @ alpha)
    return r1, r2


def step_to_boundary(alpha, dalpha, C):
    """Largest s in (0, 1] with 0 <= alpha + s dalpha <= C."""
    s = 1.0
    neg = dalpha < 0
    if np.any(neg):
        s = min(s, float(np.min(-alpha[neg] / dalpha[neg])))
    pos = dalpha > 0
    if np.any(pos):
        s = min(s, float(np.min((C - alpha[pos]) / dalpha[pos])))
    return s


def ipm_dense(K, y, C, tol=1e-6, sigma=0.6, gamma0=0.99995, mu0=1.0, max_iter=100,
              record=None, stop="gap", sigma_rule="adaptive", alpha0=None):
    """Algorithm 1 with the Newton system solved by a dense LU (numpy.linalg.solve).

    Returns dict(alpha, lam, b, iterations, mu, history, reason)."""
    K = np.asarray(K, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = y.size
    Q = (y[:, None] * K) * y[None, :]
    alpha = np.full(n, min(C / 2.0, 0.5) if alpha0 is None else alpha0)
    lam = 0.0
    mu = mu0
    s_prev = 1.0
    xl0, xa0 = newton_rhs(Q, y, alpha, lam, mu, C)
    nxl0 = max(1.0, float(np.linalg.norm(xl0)))
    nxa0 = max(1.0, abs(xa0))
    xl, xa = xl0, xa0
    history = []
    it = 0
    reason = "max_iter"

    def done():
        if stop == "alg1":
            return not (mu > tol or abs(xa) / nxa0 > tol or np.linalg.norm(xl) / nxl0 > tol)
        if it == 0:
            return False
        P = primal_objective(K, y, alpha, -lam, C)
        return (P - dual_objective(K, y, alpha)) / max(1.0, abs(P)) <= tol and abs(xa) / nxa0 <= tol

    while it < max_iter:
        if done():
            reason = "converged"
            break
        if np.any(alpha <= 0.0) or np.any(alpha >= C):
            reason = "bound"
            break
        mu = (sigma if sigma_rule == "constant" else 1.0 - (1.0 - sigma) * s_prev) * mu
        theta = mu * (1.0 / alpha ** 2 + 1.0 / (C - alpha) ** 2)
        r1, r2 = newton_rhs(Q, y, alpha, lam, mu, C)
        A = np.zeros((n + 1, n + 1))
        A[:n, :n] = Q + np.diag(theta)
        A[:n, n] = -y
        A[n, :n] = -y
        sol = np.linalg.solve(A, np.concatenate([r1, [r2]]))
        da, dl = sol[:n], sol[n]
        s = gamma0 * step_to_boundary(alpha, da, C)
        s_prev = s
        alpha = alpha + s * da
        lam = lam + s * dl
        xl, xa = newton_rhs(Q, y, alpha, lam, mu, C)
        it += 1
        gap = duality_gap(K, y, alpha, -lam, C)
        history.append(dict(it=it, mu=mu, step=s, xi_alpha=abs(xa) / nxa0,
                            xi_lambda=float(np.linalg.norm(xl)) / nxl0,
                            dual=dual_objective(K, y, alpha), gap=gap))
        if record is not None:
            record(alpha, lam)
    return dict(alpha=alpha, lam=lam, b=-lam, iterations=it, mu=mu, history=history,
                reason=reason)


def kkt_violation(K, y, alpha, b, C, eps_bound=1e-8):
    """Largest violation of the SVM optimality conditions with decision values f = K Y a + b:
    alpha_i = 0 => y_i f_i >= 1;  0 < alpha_i < C => y_i f_i = 1;  alpha_i = C => y_i f_i <= 1."""
    yf = y * (K @ (y * alpha) + b)
    at0 = alpha <= eps_bound * C
    atC = alpha >= C * (1 - eps_bound)
    free = ~(at0 | atC)
    v = 0.0
    if np.any(at0):
        v = max(v, float(np.max(np.maximum(0.0, 1.0 - yf[at0]))))
    if np.any(atC):
        v = max(v, float(np.max(np.maximum(0.0, yf[atC] - 1.0))))
    if np.any(free):
        v = max(v, float(np.max(np.abs(yf[free] - 1.0))))
    return v


def brute_force_dual(K, y, C):
    """Optimal dual value by enumerating every split of the indices into alpha=0 / free / alpha=C
    (3^n splits, n <= 9). On each split, the equality-constrained maximiser of the concave dual over
    the free variables comes from its KKT system; feasible ones are kept and the best value wins."""
    import itertools
    K = np.asarray(K, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = y.size
    if n > 9:
        raise ValueError("brute force is for n <= 9")
    Q = (y[:, None] * K) * y[None, :]
    best = -np.inf
    best_alpha = None
    for split in itertools.product((0, 1, 2), repeat=n):
        split = np.array(split)
        alpha = np.where(split == 2, C, 0.0)
        F = np.flatnonzero(split == 1)
        if F.size:
            # maximise e_F^T a_F - 1/2 a^T Q a  s.t. y^T a = 0, fixed entries outside F
            fixed = np.flatnonzero(split != 1)
            g = 1.0 - Q[np.ix_(F, fixed)] @ alpha[fixed]
            M = np.zeros((F.size + 1, F.size + 1))
            M[:F.size, :F.size] = Q[np.ix_(F, F)]
            M[:F.size, F.size] = -y[F]
            M[F.size, :F.size] = -y[F]
            rhs = np.concatenate([g, [float(y[fixed] @ alpha[fixed])]])
            sol, *_ = np.linalg.lstsq(M, rhs, rcond=None)
            if not np.allclose(M @ sol, rhs, atol=1e-9):
                continue
            alpha[F] = sol[:F.size]
        if abs(y @ alpha) > 1e-9 or np.any(alpha < -1e-12) or np.any(alpha > C + 1e-12):
            continue
        val = dual_objective(K, y, alpha)
        if val > best:
            best, best_alpha = val, alpha.copy()
    return best, best_alpha
