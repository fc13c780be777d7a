"""FP64 CPU oracle for the generalized DWD model solved by the inexact sGS-ADMM.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or run
this module: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code, table or helper with the CUDA library and imports nothing from it.

It is written to be read against the paper (arXiv 2305.12019), not to be fast:

* the problem: generalized DWD, Sec. 2, eq-primal; dual eq-dual; KKT
  eq-optimality; the bounds of Prop. 2 (proof of the second proposition, Sec. 2);
* the method: Algorithm 1 (Sec. 3), steps 1a, 1b, 1c, 2, 3 in that order, on the
  scaled model eq-gen-scale of Sec. 4.2;
* the linear system eq-linsys is solved by the SMW2 formulas of Sec. 3.3.2 as the
  paper prints them (eq-Anew, eq-Ainv, eq-H and the rank-one form of H^{-1}),
  i.e. in d-space with one n x n Cholesky factor;
* the r-subproblem eq-1c / eq-varphi by the Newton iteration of Sec. 3.2, kept
  inside a bracket and bisected when a step leaves it (the paper's fallback);
* the KKT residuals and duality gap of Sec. 4.3 and the sigma rule of Sec. 4.4.

Readings where the paper is silent or garbled (the CUDA path takes the same ones):

R1  D is "a positive multiple of I"; D^2 = mu*I with mu = 1 by default.  The SMW
    matrix called D-hat in eq-Anew holds D^2 (the identity only holds that way).
R3  initial iterate r = xi = 1, w = u = 0, beta = 0, alpha = 0, rho = 0
    (the feasible point used in the proof of Prop. 2).
R4  sigma0 = min(10C, n)^q (Sec. 4.4) unless given.
R5  the sigma rule runs after the KKT evaluation of every iteration k >= 1.
R5b ... unless eta_P or eta_D is below 1e-3 * tol: the rule balances eta_P
    against eta_D, and once one of them is at the level of rounding their
    ratio is noise that would push sigma by 2.2 per iteration.
R6  eta_D also holds eta_D3 = ||Z~ alpha + D rho|| / (1+C), the w-stationarity of
    the Lagrangian of eq-gen-scale; chi = eta_P / max(eta_D, 1e-300).
R7  eta_C3 is the unsquared norm ||alpha - s|| / (1+C).
R8  stopping: kkt = max(eta_P, eta_D, eta_C, eta_gap) <= tol (stricter than the
    paper); stop_rule = 1 applies the paper's rule of Sec. 4.3 instead:
    max(eta_P, eta_D) < tol, min(eta_C, eta_gap) < sqrt(tol),
    max(eta_C, eta_gap) < 0.05.
R9  dual objective kappa * sum(alpha^(q/(q+1))) - Z_scale * ||Z~ alpha||.
R10 prox bracket [lo, hi], lo = max(a, 0), hi = lo + (omega/sigma)^(1/(q+2)).
R11 steps 1a and 1c are solved exactly (direct SMW), so the eps_k schedule is
    not needed and step 1c is always executed.
R15 weights: e = 1 and the r-term weights wt = 1 unless given (wt enters as
    wt_i^q / r_i^q, Sec. 4.5).
"""

from __future__ import annotations

import math

import numpy as np

EPS = np.finfo(np.float64).eps


# --------------------------------------------------------------------------
# model pieces (Sec. 2)
# --------------------------------------------------------------------------

def kappa(q: float) -> float:
    """Dual constant (q+1)/q * q^(1/(q+1)) of eq-dual (Sec. 2)."""
    return (q + 1.0) / q * q ** (1.0 / (q + 1.0))


def primal_objective(r, xi, q, C, e=None, wt=None):
    """Phi(r, xi) = sum wt_i^q / r_i^q + C <e, xi>  (eq-primal; Sec. 4.5 weights)."""
    r = np.asarray(r, dtype=np.float64)
    n = r.size
    e = np.ones(n) if e is None else np.asarray(e, dtype=np.float64)
    wt = np.ones(n) if wt is None else np.asarray(wt, dtype=np.float64)
    if np.any(r <= 0):
        return math.inf
    return float(np.sum(wt ** q / r ** q) + C * np.dot(e, xi))


def primal_value_at(Z, y, w, beta, q, C, e=None, wt=None):
    """Value of eq-primal at a fixed (w, beta) with ||w|| <= 1, minimised over (r, xi).

    For fixed (w, beta), with m_i = y_i (w^T x_i + beta) = (Z^T w + beta y)_i the
    constraint reads r = m + xi, xi >= 0, so each i is a 1-D convex problem
    min_{r > 0, r >= m_i} wt_i^q r^-q + C e_i (r - m_i), solved in closed form by
    r_i = max(m_i, (q wt_i^q / (C e_i))^(1/(q+1))).
    """
    Z = np.asarray(Z, dtype=np.float64)
    n = Z.shape[1]
    e = np.ones(n) if e is None else np.asarray(e, dtype=np.float64)
    wt = np.ones(n) if wt is None else np.asarray(wt, dtype=np.float64)
    m = Z.T @ w + beta * y
    rc = (q * wt ** q / (C * e)) ** (1.0 / (q + 1.0))
    r = np.maximum(m, rc)
    xi = r - m
    return float(np.sum(wt ** q / r ** q) + C * np.dot(e, xi))


def dual_objective(Z, alpha, q, wt=None):
    """-Psi(alpha) = kappa * sum (wt_i alpha_i)^(q/(q+1)) - ||Z alpha||  (eq-dual).

    With wt = 1 this is the paper's dual.  alpha must lie in F_D for it to be a
    lower bound on the primal optimum.
    """
    alpha = np.asarray(alpha, dtype=np.float64)
    wt = np.ones(alpha.size) if wt is None else np.asarray(wt, dtype=np.float64)
    a = np.maximum(alpha, 0.0)
    return float(kappa(q) * np.sum((wt * a) ** (q / (q + 1.0))) - np.linalg.norm(Z @ alpha))


def project_dual_feasible(alpha, y, C, e=None, iters=200):
    """A point of F_D = {0 <= alpha <= Ce, y^T alpha = 0} near alpha (Sec. 2).

    alpha_hat = clip(alpha - lam y, 0, Ce) with lam found by bisection so that
    y^T alpha_hat = 0 (y^T clip(alpha - lam y) is non-increasing in lam).
    """
    alpha = np.asarray(alpha, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    ub = C * (np.ones(alpha.size) if e is None else np.asarray(e, dtype=np.float64))

    def phi(lam):
        return float(y @ np.clip(alpha - lam * y, 0.0, ub))

    lo, hi = -1.0, 1.0
    while phi(lo) < 0:
        lo *= 2.0
    while phi(hi) > 0:
        hi *= 2.0
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if phi(mid) > 0:
            lo = mid
        else:
            hi = mid
    lam = 0.5 * (lo + hi)
    return np.clip(alpha - lam * y, 0.0, ub)


def certified_gap(Z, y, w, beta, alpha, q, C, e=None, wt=None):
    """Weak-duality sandwich D(alpha_hat) <= OPT <= P(w/max(1,||w||), beta).

    Returns (upper, lower, relative gap).  Holds at any size for any (w, beta,
    alpha); it pins the optimum without trusting the solver that produced them.
    """
    w = np.asarray(w, dtype=np.float64)
    wn = np.linalg.norm(w)
    wf = w / max(1.0, wn)
    up = primal_value_at(Z, y, wf, beta, q, C, e, wt)
    ah = project_dual_feasible(alpha, y, C, e)
    lo = dual_objective(Z, ah, q, wt)
    return up, lo, (up - lo) / (1.0 + abs(up) + abs(lo))


def predict(X, w, beta):
    """sgn(beta + x^T w) for the columns of X (training/testing error, Sec. 4.5)."""
    return np.sign(X.T @ w + beta)


# --------------------------------------------------------------------------
# data scaling (Sec. 4.2, eq-gen-scale)
# --------------------------------------------------------------------------

def scale_data(Z):
    """Z_scale = sqrt(||X||_F) (= sqrt(||Z||_F)), Z~ = Z / Z_scale (Sec. 4.2)."""
    Z = np.asarray(Z, dtype=np.float64)
    zs = math.sqrt(np.linalg.norm(Z))
    return Z / zs, zs


# --------------------------------------------------------------------------
# linear system eq-linsys by SMW2 (Sec. 3.3.2)
# --------------------------------------------------------------------------

class SMW2:
    """A^{-1} h for A = [[Z Z^T + D^2, Z y], [(Z y)^T, y^T y]]  (eq-linsys, T = 0).

    Set-up (done once, Sec. 3.3.2): the n x n block I_n + Z^T D^-2 Z of J is
    factored by Cholesky, J^{-1} y-bar is formed, and H^{-1} = J^{-1} -
    (J^{-1} y-bar)(J^{-1} y-bar)^T / (1 + y-bar^T J^{-1} y-bar).  A solve then
    applies eq-Ainv: A^{-1} = Dh^{-1} - Dh^{-1} U H^{-1} U^T Dh^{-1}, with
    Dh = diag(D^2, ||y||^2), U = [[Z, 0], [y^T, ||y||]] (eq-Anew).
    """

    def __init__(self, Z, y, mu):
        self.Z = np.asarray(Z, dtype=np.float64)
        self.y = np.asarray(y, dtype=np.float64)
        self.mu = float(mu)
        d, n = self.Z.shape
        self.d, self.n = d, n
        self.ny = float(np.linalg.norm(self.y))
        G = np.eye(n) + (self.Z.T @ self.Z) / self.mu        # first diagonal block of J (eq-H)
        self.L = np.linalg.cholesky(G)                        # G = L L^T
        ybar = np.concatenate([self.y / self.ny, [1.0]])
        self.Jinv_ybar = self._Jinv(ybar)
        self.coef = 1.0 / (1.0 + ybar @ self.Jinv_ybar)
        self.dhat = np.concatenate([np.full(d, self.mu), [self.ny ** 2]])

    def _Ginv(self, t):
        # forward then backward substitution with the Cholesky factor (Sec. 3.3.2)
        from scipy.linalg import solve_triangular
        z = solve_triangular(self.L, t, lower=True)
        return solve_triangular(self.L.T, z, lower=False)

    def _Jinv(self, t):
        # J = diag(I_n + Z^T D^-2 Z, -1)
        return np.concatenate([self._Ginv(t[: self.n]), [-t[self.n]]])

    def _Hinv(self, t):
        return self._Jinv(t) - self.coef * self.Jinv_ybar * (self.Jinv_ybar @ t)

    def _Ut(self, h):        # U^T h, U = [[Z, 0], [y^T, ||y||]]
        return np.concatenate([self.Z.T @ h[: self.d] + self.y * h[self.d], [self.ny * h[self.d]]])

    def _U(self, s):         # U s
        return np.concatenate([self.Z @ s[: self.n], [self.y @ s[: self.n] + self.ny * s[self.n]]])

    def solve(self, h):
        """[w; beta] = A^{-1} h by eq-Ainv."""
        h1 = h / self.dhat
        s = self._Hinv(self._Ut(h1))
        return h1 - self._U(s) / self.dhat

    def matrix(self):
        """The dense (d+1) x (d+1) A, for tests on tiny sizes only."""
        d = self.d
        A = np.zeros((d + 1, d + 1))
        A[:d, :d] = self.Z @ self.Z.T + self.mu * np.eye(d)
        zy = self.Z @ self.y
        A[:d, d] = zy
        A[d, :d] = zy
        A[d, d] = self.y @ self.y
        return A


class Direct:
    """A^{-1} h for the same A by the direct solver of Sec. 3.3.1 (T = 0, d << n):
    A is formed once ((d+1) x (d+1), 2 n d^2 flops) and factored by Cholesky; a
    solve is two triangular solves."""

    def __init__(self, Z, y, mu):
        self.Z = np.asarray(Z, dtype=np.float64)
        self.y = np.asarray(y, dtype=np.float64)
        self.mu = float(mu)
        d, n = self.Z.shape
        self.d, self.n = d, n
        A = np.zeros((d + 1, d + 1))
        A[:d, :d] = self.Z @ self.Z.T + self.mu * np.eye(d)
        zy = self.Z @ self.y
        A[:d, d] = zy
        A[d, :d] = zy
        A[d, d] = self.y @ self.y
        self.L = np.linalg.cholesky(A)

    def solve(self, h):
        from scipy.linalg import solve_triangular
        z = solve_triangular(self.L, h, lower=True)
        return solve_triangular(self.L.T, z, lower=False)


class LinsysOperator:
    """eq-linsys with T = 0 as a matrix-free operator (Sec. 3.3.3):
    A [w; beta] = [Z (Z^T w + y beta) + mu w; y^T (Z^T w + y beta)], two products
    with Z (4nd flops) per application.  A = U U^T + diag(mu I_d, 0) with
    U = [Z; y^T], so A is symmetric positive definite (for [w; beta] != 0 the
    quadratic form is ||Z^T w + beta y||^2 + mu ||w||^2 > 0)."""

    def __init__(self, Z, y, mu):
        self.Z = np.asarray(Z, dtype=np.float64)
        self.y = np.asarray(y, dtype=np.float64)
        self.mu = float(mu)
        self.d = self.Z.shape[0]

    def matvec(self, v):
        t = self.Z.T @ v[: self.d] + self.y * v[self.d]
        return np.concatenate([self.Z @ t + self.mu * v[: self.d], [self.y @ t]])

    def diagonal(self):
        """diag(A): the Jacobi preconditioner."""
        return np.concatenate([np.sum(self.Z * self.Z, axis=1) + self.mu, [self.y @ self.y]])


def pcg(op, h, x0, tol, max_steps=10000):
    """Preconditioned conjugate gradients (Jacobi: M = diag(A)) for the symmetric
    positive definite eq-linsys, started at x0 and stopped once the residual meets
    the accuracy condition ||h - A x|| <= tol (eq-linsys-tol).  Returns
    (x, ||h - A x||, steps).  The paper's own Krylov solver (PSQMR) is described in
    an appendix that is not part of the text; for an SPD system CG is the method
    of that family with the same cost per step (one product with A)."""
    m = op.diagonal()
    x = np.array(x0, dtype=np.float64)
    r = h - op.matvec(x)
    rn = np.linalg.norm(r)
    steps = 0
    if rn <= tol:
        return x, rn, 0
    z = r / m
    p = z.copy()
    rz = r @ z
    while steps < max_steps:
        Ap = op.matvec(p)
        a = rz / (p @ Ap)
        x += a * p
        r -= a * Ap
        steps += 1
        rn = np.linalg.norm(r)
        if rn <= tol:
            break
        z = r / m
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, np.linalg.norm(h - op.matvec(x)), steps


def eps_schedule(k, c):
    """The summable tolerances of Algorithm 1: eps_k = c / (k + 1)^1.5 (Sec. 3, after
    Algorithm 1; c inversely proportional to the Frobenius norm of the data)."""
    return c / (k + 1.0) ** 1.5


# --------------------------------------------------------------------------
# r-subproblem (Step 1b, eq-1c / eq-varphi, Sec. 3.2)
# --------------------------------------------------------------------------

def prox_r(a, sigma, q, r0=None, omega=None, max_iter=100):
    """Minimiser of phi(s) = (omega/q) s^-q + sigma/2 (s - a)^2 over s > 0, per element.

    With omega = q (the paper's case) this is eq-varphi.  The optimality
    condition s^(q+1) (s - a) = omega / sigma has exactly one positive root, which
    lies in [lo, hi], lo = max(a, 0), hi = lo + (omega/sigma)^(1/(q+2)).  Newton's
    iteration of Sec. 3.2,
        s <- s (omega (q+2)/sigma + a s^(q+1)) / (omega (q+1)/sigma + s^(q+2)),
    is warm-started at r0; a step that leaves the bracket is replaced by bisection
    (the paper's fallback).  Stops when the step is below 4 eps relative.
    """
    a = np.atleast_1d(np.asarray(a, dtype=np.float64)).copy()
    n = a.size
    omega = np.full(n, float(q)) if omega is None else np.broadcast_to(np.asarray(omega, dtype=np.float64), (n,)).copy()
    kq = omega / sigma
    lo = np.maximum(a, 0.0)
    hi = lo + kq ** (1.0 / (q + 2.0))
    if r0 is None:
        s = 0.5 * (lo + hi)
    else:
        s = np.broadcast_to(np.asarray(r0, dtype=np.float64), (n,)).copy()
        bad = ~((s > lo) & (s < hi))
        s[bad] = 0.5 * (lo[bad] + hi[bad])
    active = np.ones(n, dtype=bool)
    for _ in range(max_iter):
        if not active.any():
            break
        i = active
        si = s[i]
        f = si ** (q + 1.0) * (si - a[i]) - kq[i]
        lo_i, hi_i = lo[i], hi[i]
        lo_i = np.where(f < 0, si, lo_i)
        hi_i = np.where(f > 0, si, hi_i)
        lo[i], hi[i] = lo_i, hi_i
        newton = si * (kq[i] * (q + 2.0) + a[i] * si ** (q + 1.0)) / (kq[i] * (q + 1.0) + si ** (q + 2.0))
        # converged: the Newton correction itself is below 4 eps (tested before the
        # bracket safeguard, so rounding noise of f at the root never forces a bisection)
        small = np.abs(newton - si) <= 4.0 * EPS * si
        inside = (newton > lo_i) & (newton < hi_i)
        cand = np.where(inside | small, newton, 0.5 * (lo_i + hi_i))
        done = small | (f == 0)
        s[i] = np.where(f == 0, si, cand)
        idx = np.flatnonzero(i)
        active[idx[done]] = False
    return s


# --------------------------------------------------------------------------
# KKT residuals, gap and sigma rule (Secs. 4.3, 4.4)
# --------------------------------------------------------------------------

def kkt_residuals(Zt, zs, y, q, C, mu, r, w, beta, xi, u, alpha, rho, e=None, wt=None):
    """Relative residuals of Sec. 4.3 for the scaled model eq-gen-scale (readings R6, R7, R9)."""
    n = r.size
    e = np.ones(n) if e is None else e
    wt = np.ones(n) if wt is None else wt
    D = math.sqrt(mu)
    den = 1.0 + C
    s = q * wt ** q / r ** (q + 1.0)
    zta = Zt @ alpha
    eta = {
        "C1": abs(y @ alpha) / den,
        "C2": abs(xi @ (C * e - alpha)) / den,
        "C3": np.linalg.norm(alpha - s) / den,
        "P1": np.linalg.norm(Zt.T @ w + beta * y + xi - r) / den,
        "P2": np.linalg.norm(D * (w - u)) / den,
        "P3": max(np.linalg.norm(w) - zs, 0.0) / den,
        "D1": np.linalg.norm(np.minimum(0.0, alpha)) / den,
        "D2": np.linalg.norm(np.maximum(0.0, alpha - C * e)) / den,
        "D3": np.linalg.norm(zta + D * rho) / den,
    }
    pobj = float(np.sum(wt ** q / r ** q) + C * (e @ xi))
    dobj = float(kappa(q) * np.sum((wt * np.maximum(alpha, 0.0)) ** (q / (q + 1.0))) - zs * np.linalg.norm(zta))
    eta["gap"] = abs(pobj - dobj) / (1.0 + abs(pobj) + abs(dobj))
    eta["P"] = max(eta["P1"], eta["P2"], eta["P3"])
    eta["D"] = max(eta["D1"], eta["D2"], eta["D3"])
    eta["C"] = max(eta["C1"], eta["C2"], eta["C3"])
    eta["kkt"] = max(eta["P"], eta["D"], eta["C"], eta["gap"])
    return eta, pobj, dobj


def sigma_update(sigma, eta_p, eta_d, theta=5.0):
    """Sec. 4.4: chi = eta_P / eta_D; grow sigma by zeta if chi > theta, shrink if 1/chi > theta.

    zeta = 1.1, raised to 1.65 when max(chi, 1/chi) > 50 and to 2.2 when > 500.
    """
    chi = eta_p / max(eta_d, 1e-300)
    big = max(chi, 1.0 / max(chi, 1e-300))
    zeta = 2.2 if big > 500 else (1.65 if big > 50 else 1.1)
    if chi > theta:
        return sigma * zeta
    if 1.0 / max(chi, 1e-300) > theta:
        return sigma / zeta
    return sigma


# --------------------------------------------------------------------------
# weights and the penalty heuristic (Sec. 4.5, Sec. 4.1)
# --------------------------------------------------------------------------

def imbalance_weights(y, q):
    """Sec. 4.5 class-balancing weights: tau_+- = (n_+- / K)^(1/(1+q)) with
    K = n / log(n); tau_i = tau_- / max(tau_+, tau_-) if y_i = +1, tau_+ / max(...) if -1."""
    y = np.asarray(y, dtype=np.float64)
    n = y.size
    n_pos = float(np.sum(y > 0))
    n_neg = float(n - n_pos)
    K = n / math.log(n)
    tau_pos = (n_pos / K) ** (1.0 / (1.0 + q))
    tau_neg = (n_neg / K) ** (1.0 / (1.0 + q))
    top = max(tau_pos, tau_neg)
    return np.where(y > 0, tau_neg / top, tau_pos / top)


def suggest_C(Z, y, q):
    """Sec. 4.1: C = 10^(q+1) max{1, 10^(q-1) log(n) max{1000, d}^(1/3) / dist^(q+1)},
    dist = median Euclidean distance between points of opposite classes (x_i = y_i z_i)."""
    Z = np.asarray(Z, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    d, n = Z.shape
    X = Z * y[None, :]
    P, M = X[:, y > 0], X[:, y < 0]
    dists = [np.linalg.norm(P[:, i] - M[:, j]) for i in range(P.shape[1]) for j in range(M.shape[1])]
    dist = float(np.median(dists))
    t = 10.0 ** (q - 1.0) * math.log(n) * max(1000.0, float(d)) ** (1.0 / 3.0) / dist ** (q + 1.0)
    return 10.0 ** (q + 1.0) * max(1.0, t)


# --------------------------------------------------------------------------
# Algorithm 1
# --------------------------------------------------------------------------

def solve(Z, y, q, C, mu=1.0, tau=1.618, tol=1e-9, max_iter=50000, sigma0=None,
          e=None, wt=None, record=False, stop_rule=0, linsys="smw"):
    """Inexact sGS-ADMM (Algorithm 1) on eq-gen-scale, exact solves of eq-linsys (R11):
    by SMW2 (Sec. 3.3.2, linsys = "smw") or by the direct solver (Sec. 3.3.1,
    linsys = "direct").

    Z is d x n with columns y_i x_i (Sec. 2, eq-r); y in {-1, +1}^n.
    Returns a dict with w (original scale, w~ / Z_scale, Sec. 4.2), beta, r, xi,
    alpha, the scaled u and rho, iteration count, final residuals and objectives.
    """
    Z = np.asarray(Z, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    d, n = Z.shape
    e = np.ones(n) if e is None else np.asarray(e, dtype=np.float64)
    wt = np.ones(n) if wt is None else np.asarray(wt, dtype=np.float64)
    omega = q * wt ** q
    Zt, zs = scale_data(Z)
    smw = SMW2(Zt, y, mu) if linsys == "smw" else Direct(Zt, y, mu)
    D = math.sqrt(mu)

    # R3: feasible start
    r = np.ones(n)
    xi = np.ones(n)
    w = np.zeros(d)
    u = np.zeros(d)
    beta = 0.0
    alpha = np.zeros(n)
    rho = np.zeros(d)
    sigma = float(sigma0) if sigma0 is not None and sigma0 > 0 else min(10.0 * C, n) ** q   # R4
    history = []
    eta = None
    pobj = dobj = float("nan")
    k = 0
    for k in range(max_iter):
        # Step 1a: (w-bar, beta-bar) from eq-linsys with r^k
        v = xi - r - alpha / sigma
        hbar = np.concatenate([-Zt @ v + mu * u + D * rho / sigma, [-(y @ v)]])
        sol = smw.solve(hbar)
        wbar, betabar = sol[:d], sol[d]
        # Step 1b: r^{k+1} by the prox of eq-1c at c^k
        ck = Zt.T @ wbar + y * betabar + xi - alpha / sigma
        r = prox_r(ck, sigma, q, r0=r, omega=omega)
        # Step 1c: (w, beta) from eq-linsys with r^{k+1}
        v = xi - r - alpha / sigma
        h = np.concatenate([-Zt @ v + mu * u + D * rho / sigma, [-(y @ v)]])
        sol = smw.solve(h)
        w, beta = sol[:d], sol[d]
        # Step 2: u = projection of g onto the ball of radius Z_scale; xi = max(0, .)
        g = w - rho / (sigma * D)
        gn = np.linalg.norm(g)
        u = g if gn <= zs else g * (zs / gn)
        ztw = Zt.T @ w
        xi = np.maximum(0.0, r - ztw - y * beta + alpha / sigma - C * e / sigma)
        # Step 3: multipliers
        alpha = alpha - tau * sigma * (ztw + y * beta + xi - r)
        rho = rho - tau * sigma * D * (w - u)
        # Sec. 4.3 residuals
        eta, pobj, dobj = kkt_residuals(Zt, zs, y, q, C, mu, r, w, beta, xi, u, alpha, rho, e, wt)
        if record:
            history.append((sigma, eta["kkt"], eta["P"], eta["D"]))
        if stop_rule == 0 and eta["kkt"] <= tol:                                  # R8
            break
        if stop_rule == 1 and (max(eta["P"], eta["D"]) < tol and min(eta["C"], eta["gap"]) < math.sqrt(tol)
                               and max(eta["C"], eta["gap"]) < 0.05):               # Sec. 4.3
            break
        if k >= 1 and min(eta["P"], eta["D"]) > 1e-3 * tol:   # R5, R5b
            sigma = sigma_update(sigma, eta["P"], eta["D"])
    if stop_rule == 1:
        converged = eta is not None and (max(eta["P"], eta["D"]) < tol and min(eta["C"], eta["gap"]) < math.sqrt(tol)
                                         and max(eta["C"], eta["gap"]) < 0.05)
    else:
        converged = eta is not None and eta["kkt"] <= tol
    return {
        "w": w / zs, "beta": float(beta), "r": r, "xi": xi, "alpha": alpha,
        "w_scaled": w, "u_scaled": u, "rho": rho, "zscale": zs, "sigma": sigma,
        "iters": k + 1, "converged": converged, "eta": eta, "primal": pobj, "dual": dobj,
        "history": history,
    }


def solve_inexact(Z, y, q, C, mu=1.0, tau=1.618, tol=1e-9, max_iter=50000, sigma0=None, e=None, wt=None,
                  eps_c=None, record=False):
    """Algorithm 1 with inexact solves of eq-linsys (Sec. 3, Steps 1a-1c; Sec. 3.3.3,
    the case where d and n are both large, T = 0): no n x n or d x d matrix is formed.

    Step 1a solves eq-linsys by PCG to ||h-bar - A [w-bar; beta-bar]|| <= eps_k
    (eq-linsys-tol), warm-started at the last (w, beta).  Step 1c first tests Step
    1a's solution against the new right-hand side h (r^k replaced by r^{k+1}): if
    ||h - A [w-bar; beta-bar]|| <= 5 eps_k it is kept and the solve is skipped,
    else PCG continues from it to 5 eps_k.  eps_k = c / (k+1)^1.5 with
    c = eps_c, by default 1 / ||Z~||_F (the paper fixes c only up to this
    proportionality).  Returns solve()'s dict plus "cg_steps" (all PCG steps) and
    "step1c_solves" (iterations in which Step 1c had to solve: the paper's
    "double" count).
    """
    Z = np.asarray(Z, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    d, n = Z.shape
    e = np.ones(n) if e is None else np.asarray(e, dtype=np.float64)
    wt = np.ones(n) if wt is None else np.asarray(wt, dtype=np.float64)
    omega = q * wt ** q
    Zt, zs = scale_data(Z)
    op = LinsysOperator(Zt, y, mu)
    D = math.sqrt(mu)
    c_eps = (1.0 / np.linalg.norm(Zt)) if eps_c is None else float(eps_c)

    r = np.ones(n)
    xi = np.ones(n)
    w = np.zeros(d)
    u = np.zeros(d)
    beta = 0.0
    alpha = np.zeros(n)
    rho = np.zeros(d)
    sigma = float(sigma0) if sigma0 is not None and sigma0 > 0 else min(10.0 * C, n) ** q
    history = []
    eta = None
    pobj = dobj = float("nan")
    cg_steps = 0
    solves_1c = 0
    k = 0
    for k in range(max_iter):
        eps_k = eps_schedule(k, c_eps)
        # Step 1a
        v = xi - r - alpha / sigma
        hbar = np.concatenate([-Zt @ v + mu * u + D * rho / sigma, [-(y @ v)]])
        sol, _, st = pcg(op, hbar, np.concatenate([w, [beta]]), eps_k)
        cg_steps += st
        wbar, betabar = sol[:d], sol[d]
        # Step 1b
        ck = Zt.T @ wbar + y * betabar + xi - alpha / sigma
        r = prox_r(ck, sigma, q, r0=r, omega=omega)
        # Step 1c: keep Step 1a's solution if it is accurate enough for the new h
        v = xi - r - alpha / sigma
        h = np.concatenate([-Zt @ v + mu * u + D * rho / sigma, [-(y @ v)]])
        if np.linalg.norm(h - op.matvec(sol)) > 5.0 * eps_k:
            sol, _, st = pcg(op, h, sol, 5.0 * eps_k)
            cg_steps += st
            solves_1c += 1
        w, beta = sol[:d], sol[d]
        # Step 2
        g = w - rho / (sigma * D)
        gn = np.linalg.norm(g)
        u = g if gn <= zs else g * (zs / gn)
        ztw = Zt.T @ w
        xi = np.maximum(0.0, r - ztw - y * beta + alpha / sigma - C * e / sigma)
        # Step 3
        alpha = alpha - tau * sigma * (ztw + y * beta + xi - r)
        rho = rho - tau * sigma * D * (w - u)
        eta, pobj, dobj = kkt_residuals(Zt, zs, y, q, C, mu, r, w, beta, xi, u, alpha, rho, e, wt)
        if record:
            history.append((sigma, eta["kkt"], eta["P"], eta["D"], eps_k))
        if eta["kkt"] <= tol:
            break
        if k >= 1 and min(eta["P"], eta["D"]) > 1e-3 * tol:
            sigma = sigma_update(sigma, eta["P"], eta["D"])
    converged = eta is not None and eta["kkt"] <= tol
    return {
        "w": w / zs, "beta": float(beta), "r": r, "xi": xi, "alpha": alpha,
        "w_scaled": w, "u_scaled": u, "rho": rho, "zscale": zs, "sigma": sigma,
        "iters": k + 1, "converged": converged, "eta": eta, "primal": pobj, "dual": dobj,
        "history": history, "cg_steps": cg_steps, "step1c_solves": solves_1c, "eps_c": c_eps,
    }
