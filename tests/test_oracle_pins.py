"""Pins of two oracle functions that every certificate and every iteration count
rely on, checked against what the paper and the mathematics fix:

* ``project_dual_feasible`` (the feasible point of eq-dual used by the weak-duality
  certificate, Sec. 2): its output lies in F_D = {0 <= alpha <= Ce, y^T alpha = 0},
  it is the Euclidean projection onto F_D (checked against a general-purpose QP
  solve), points of F_D are fixed, and the dual value there never exceeds the
  optimum of eq-dual found by an independent SLSQP maximisation;
* ``sigma_update`` (the sigma rule of Sec. 4.4: theta = 5, zeta = 1.1, 1.65 when
  max(chi, 1/chi) > 50, 2.2 when > 500) on hand-computed cases, and the gate of
  the solver loop (reading R5b: the rule is skipped while min(eta_P, eta_D) is at
  most 1e-3 tol, and runs from the second iteration on, reading R5).
"""
import math

import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import gdwd_oracle as O


def _problem(rng, d, n, n_pos, shift=0.7):
    y = np.where(np.arange(n) < n_pos, 1.0, -1.0)
    X = rng.standard_normal((d, n)) + shift * y[None, :] * np.eye(d, 1)
    return y, X * y[None, :]


def _assert_in_FD(ah, y, C, e):
    ub = C * e
    assert np.all(ah >= 0.0)
    assert np.all(ah <= ub)
    assert abs(y @ ah) <= 1e-12 * max(1.0, float(np.sum(ub)))


# ---------------------------------------------------------------- project_dual_feasible

def _alphas(rng, n, y, C):
    """Random and adversarial starting points."""
    pos = y > 0
    yield rng.uniform(-C, 2 * C, n)                   # anywhere, outside the box too
    yield rng.uniform(0, C, n)                        # inside the box, off the hyperplane
    yield np.zeros(n)                                 # all at 0 (already in F_D)
    yield np.full(n, C)                               # all at C
    yield np.where(pos, C, 0.0)                       # support in the positive class only
    yield np.where(pos, 0.0, C)                       # support in the negative class only
    yield np.where(pos, 3 * C, -2 * C)                # far outside, opposite signs by class
    yield 1e-300 * rng.standard_normal(n)             # tiny values


@pytest.mark.parametrize("n_pos,n", [(5, 10), (3, 12), (1, 7), (8, 9)])
def test_projection_lies_in_FD(n_pos, n):
    rng = np.random.default_rng(100 + n_pos)
    y = np.where(np.arange(n) < n_pos, 1.0, -1.0)
    for C in (0.3, 1.0, 25.0):
        for e in (np.ones(n), rng.uniform(0.2, 1.0, n)):
            for a in _alphas(rng, n, y, C):
                ah = O.project_dual_feasible(a, y, C, e)
                _assert_in_FD(ah, y, C, e)


def test_projection_is_the_euclidean_projection():
    """clip(alpha - lam y, 0, Ce) with y^T alpha_hat = 0 is the closest point of F_D:
    compare with a generic constrained least-squares solve."""
    rng = np.random.default_rng(7)
    n, C = 9, 1.3
    y = np.where(np.arange(n) < 4, 1.0, -1.0)
    e = rng.uniform(0.5, 1.0, n)
    for _ in range(6):
        a = rng.uniform(-C, 2 * C, n)
        ah = O.project_dual_feasible(a, y, C, e)
        sol = minimize(lambda x: 0.5 * np.sum((x - a) ** 2), np.zeros(n), jac=lambda x: x - a,
                       method="SLSQP", bounds=[(0.0, C * ei) for ei in e],
                       constraints=[{"type": "eq", "fun": lambda x: y @ x, "jac": lambda x: y}],
                       options={"ftol": 1e-15, "maxiter": 1000})
        assert sol.success
        assert np.linalg.norm(ah - sol.x) <= 1e-6 * max(1.0, np.linalg.norm(a))
        # no other point of F_D is closer (the solver's point is feasible up to its tolerance)
        assert np.linalg.norm(ah - a) <= np.linalg.norm(sol.x - a) + 1e-9


def test_projection_fixes_points_of_FD():
    rng = np.random.default_rng(8)
    n, C = 10, 2.0
    y = np.where(np.arange(n) < 5, 1.0, -1.0)
    for _ in range(5):
        a = rng.uniform(0, C, n)
        sp, sm = np.sum(a[y > 0]), np.sum(a[y < 0])
        # scale the class with the larger sum down onto the hyperplane (stays in the box)
        if sp > sm:
            a[y > 0] *= sm / sp
        else:
            a[y < 0] *= sp / sm
        assert abs(y @ a) < 1e-12 and np.all(a >= 0) and np.all(a <= C)
        ah = O.project_dual_feasible(a, y, C)
        assert np.max(np.abs(ah - a)) <= 1e-13


@pytest.mark.parametrize("q", [0.5, 1.0, 2.0, 4.0])
def test_projected_dual_value_is_a_lower_bound(q):
    """D(alpha_hat) <= max over F_D of eq-dual, the latter from SLSQP (strong duality
    makes it the primal optimum, which the oracle's solve also gives)."""
    rng = np.random.default_rng(41)
    y, Z = _problem(rng, 5, 10, 5, shift=0.6)
    C = 2.0
    k = O.kappa(q)

    def negdual(a):
        return np.linalg.norm(Z @ a) - k * np.sum(np.maximum(a, 0) ** (q / (q + 1)))

    sol = minimize(negdual, np.full(10, C / 2), method="SLSQP", bounds=[(1e-12, C)] * 10,
                   constraints=[{"type": "eq", "fun": lambda a: y @ a}], options={"ftol": 1e-14, "maxiter": 2000})
    dmax = -sol.fun
    res = O.solve(Z, y, q, C, tol=1e-10, max_iter=400000)
    assert abs(dmax - res["primal"]) <= 1e-6 * abs(res["primal"])
    for a in _alphas(rng, 10, y, C):
        ah = O.project_dual_feasible(a, y, C)
        assert O.dual_objective(Z, ah, q) <= dmax + 1e-9 * abs(dmax)
    # at the oracle's own multipliers the bound is tight
    ah = O.project_dual_feasible(res["alpha"], y, C)
    assert abs(O.dual_objective(Z, ah, q) - dmax) <= 1e-6 * abs(dmax)


def test_certificate_rejects_a_wrong_lower_bound():
    """A point outside F_D can exceed the optimum: the projection is what makes the
    certificate's lower bound valid.  The maximiser of eq-dual without the upper
    bound alpha <= Ce has a dual value above the optimum for a small C; projected
    onto F_D it is a valid lower bound again."""
    rng = np.random.default_rng(5)
    y, Z = _problem(rng, 4, 8, 4, shift=0.5)
    q, C = 1.0, 0.05
    k = O.kappa(q)
    res = O.solve(Z, y, q, C, tol=1e-10, max_iter=400000)

    def negdual(a):
        return np.linalg.norm(Z @ a) - k * np.sum(np.maximum(a, 0) ** (q / (q + 1)))

    sol = minimize(negdual, np.full(8, 1.0), method="SLSQP", bounds=[(1e-12, None)] * 8,
                   constraints=[{"type": "eq", "fun": lambda a: y @ a}], options={"ftol": 1e-14, "maxiter": 2000})
    a = sol.x
    assert a.max() > C                                     # outside the box
    assert O.dual_objective(Z, a, q) > res["primal"] * (1 + 1e-3)
    ah = O.project_dual_feasible(a, y, C)
    assert O.dual_objective(Z, ah, q) <= res["primal"] * (1 + 1e-9)


# ---------------------------------------------------------------- sigma_update

@pytest.mark.parametrize("chi,factor", [
    (6.0, 1.1), (49.0, 1.1), (50.0, 1.1), (50.5, 1.65), (60.0, 1.65), (500.0, 1.65), (501.0, 2.2),
    (600.0, 2.2), (1e12, 2.2),
    (1 / 6.0, 1 / 1.1), (1 / 50.0, 1 / 1.1), (1 / 60.0, 1 / 1.65), (1 / 600.0, 1 / 2.2), (1e-12, 1 / 2.2),
    (5.0, 1.0), (4.999, 1.0), (1.0, 1.0), (0.2, 1.0), (0.21, 1.0),
])
def test_sigma_rule_hand_cases(chi, factor):
    """Sec. 4.4 with theta = 5: grow when chi > 5, shrink when 1/chi > 5, else keep;
    zeta = 1.1, 1.65 when max(chi, 1/chi) > 50, 2.2 when > 500."""
    for sigma in (0.37, 1.0, 1e4):
        eta_d = 1e-4
        eta_p = chi * eta_d
        got = O.sigma_update(sigma, eta_p, eta_d)
        assert got == pytest.approx(sigma * factor, rel=1e-15)


def test_sigma_rule_zero_dual_residual():
    """eta_D = 0 gives an unbounded chi (reading R6): the largest growth factor."""
    assert O.sigma_update(3.0, 1e-3, 0.0) == pytest.approx(3.0 * 2.2, rel=1e-15)


def test_sigma_gate_in_the_solver_loop(monkeypatch):
    """The loop applies the rule from the second iteration on (reading R5) and only
    while min(eta_P, eta_D) > 1e-3 tol (reading R5b)."""
    calls = []
    real = O.sigma_update

    def spy(sigma, ep, ed, theta=5.0):
        calls.append((sigma, ep, ed))
        return real(sigma, ep, ed, theta)

    monkeypatch.setattr(O, "sigma_update", spy)
    rng = np.random.default_rng(12)
    y, Z = _problem(rng, 30, 16, 8, shift=0.8)
    tol = 1e-9
    res = O.solve(Z, y, 1.0, 1.0, tol=tol, max_iter=5000, record=True)
    hist = res["history"]          # (sigma used in iteration k, kkt, eta_P, eta_D)
    assert res["converged"]
    gated = [k for k in range(len(hist) - 1) if k >= 1 and min(hist[k][2], hist[k][3]) > 1e-3 * tol]
    assert len(calls) == len(gated)
    for (sig, ep, ed), k in zip(calls, gated):
        assert (sig, ep, ed) == (hist[k][0], hist[k][2], hist[k][3])
    # sigma only moves where the rule ran, and then by one of the three factors
    for k in range(len(hist) - 1):
        ratio = hist[k + 1][0] / hist[k][0]
        if k not in gated:
            assert ratio == 1.0
        else:
            assert any(math.isclose(ratio, f, rel_tol=1e-14) for f in (1.0, 1.1, 1 / 1.1, 1.65, 1 / 1.65, 2.2,
                                                                         1 / 2.2))


def test_sigma_gate_engages_near_the_rounding_floor(monkeypatch):
    """When a residual sits at the rounding floor (here eta_D is forced to 0 on
    iterations 5 to 12, as the computed eta_D3 can be) the rule must stop moving
    sigma (R5b) instead of pushing it by 2.2 per iteration; outside that window
    the rule runs as before."""
    real = O.kkt_residuals
    it = {"k": -1}

    def fake(*args, **kw):
        eta, pobj, dobj = real(*args, **kw)
        it["k"] += 1
        if 5 <= it["k"] <= 12:
            eta = dict(eta, D=0.0, D1=0.0, D2=0.0, D3=0.0)
        return eta, pobj, dobj

    monkeypatch.setattr(O, "kkt_residuals", fake)
    rng = np.random.default_rng(13)
    y, Z = _problem(rng, 20, 12, 6, shift=0.9)
    res = O.solve(Z, y, 1.0, 1.0, tol=1e-8, max_iter=3000, record=True)
    hist = res["history"]
    assert len(hist) > 14
    for k in range(5, 13):
        assert hist[k + 1][0] == hist[k][0], k
    # without the gate an unbounded chi would have grown sigma by 2.2 on each of them
    assert O.sigma_update(hist[5][0], hist[5][2], 0.0) == pytest.approx(2.2 * hist[5][0])
