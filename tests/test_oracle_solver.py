"""Pins for the oracle's linear solve, its Algorithm-1 loop and its optimality checks.

Each test compares the oracle with something fixed outside it: the dense solve of
eq-linsys, closed-form optima, brute force, an independent library solve of the
dual eq-dual, weak duality, the bounds of Prop. 2 and symmetries of the model.
"""
import math

import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import gdwd_oracle as O


def _two_class(rng, d, n, shift=1.0, n_pos=None):
    n_pos = n // 2 if n_pos is None else n_pos
    y = np.where(np.arange(n) < n_pos, 1.0, -1.0)
    X = rng.standard_normal((d, n))
    X[0] += shift * y
    return X, y, X * y


# ---------------------------------------------------------------- linear system

@pytest.mark.parametrize("d,n,mu", [(7, 4, 1.0), (30, 9, 0.3), (12, 12, 2.5), (5, 11, 1.0)])
def test_smw_matches_dense_solve(d, n, mu):
    """SMW2 (eq-Ainv with the rank-one H^{-1}) equals a dense solve of eq-linsys (T = 0)."""
    rng = np.random.default_rng(d * 100 + n)
    Z = rng.standard_normal((d, n))
    y = np.where(rng.random(n) < 0.5, 1.0, -1.0)
    y[0], y[1] = 1.0, -1.0
    A = np.zeros((d + 1, d + 1))
    A[:d, :d] = Z @ Z.T + mu * np.eye(d)
    A[:d, d] = Z @ y
    A[d, :d] = Z @ y
    A[d, d] = y @ y
    h = rng.standard_normal(d + 1)
    ref = np.linalg.solve(A, h)
    got = O.SMW2(Z, y, mu).solve(h)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref) * np.linalg.cond(A) ** 0.5
    assert np.linalg.norm(A @ got - h) <= 1e-12 * np.linalg.norm(h) * np.linalg.norm(A)


def test_direct_solver_residual_and_toy():
    """The direct solver of Sec. 3.3.1: its solve leaves a residual of eq-linsys at
    rounding level (A assembled here from its blocks), and Algorithm 1 run on it
    reaches the closed-form optimum of the two-point toy and the SMW2 run's
    optimum on a d < n problem."""
    rng = np.random.default_rng(5)
    d, n, mu = 6, 40, 0.7
    Z = rng.standard_normal((d, n))
    y = np.where(np.arange(n) < 15, 1.0, -1.0)
    h = rng.standard_normal(d + 1)
    got = O.Direct(Z, y, mu).solve(h)
    w, b = got[:d], got[d]
    r_w = Z @ (Z.T @ w + y * b) + mu * w - h[:d]          # first block row of eq-linsys
    r_b = y @ (Z.T @ w + y * b) - h[d]                    # last row
    assert np.linalg.norm(np.append(r_w, r_b)) <= 1e-12 * np.linalg.norm(h) * (1 + np.linalg.norm(Z) ** 2)
    # two-point toy (q = 1, separable regime): w* = m / ||m||, beta* = 0
    m = rng.standard_normal(5)
    m *= 1.5 / np.linalg.norm(m)
    yy = np.array([1.0, -1.0])
    res = O.solve(np.stack([m, -m], axis=1) * yy, yy, 1.0, 1.0, tol=1e-10, max_iter=200000, linsys="direct")
    assert res["converged"] and np.linalg.norm(res["w"] - m / 1.5) <= 1e-6 and abs(res["beta"]) <= 1e-7
    # d < n: both solvers reach the same optimum
    X, yv, Zs = _two_class(rng, 4, 60, shift=1.0, n_pos=20)
    a = O.solve(Zs, yv, 2.0, 3.0, tol=1e-10, linsys="direct")
    s_ = O.solve(Zs, yv, 2.0, 3.0, tol=1e-10, linsys="smw")
    assert abs(a["primal"] - s_["primal"]) <= 1e-8 * abs(s_["primal"])
    assert np.linalg.norm(a["w"] - s_["w"]) <= 1e-6 * np.linalg.norm(s_["w"])


# ---------------------------------------------------------------- closed-form toy

@pytest.mark.parametrize("q", [0.5, 1.0, 2.0, 4.0])
@pytest.mark.parametrize("half_gap,C", [(1.5, 1.0), (0.9, 10.0), (0.2, 1.0), (0.3, 0.5)])
def test_two_point_toy(q, half_gap, C):
    """x1 = m, x2 = -m: w* = m/||m||, beta* = 0, r* = max(||m||, r_C), r_C = (q/C)^(1/(q+1))."""
    d = 6
    rng = np.random.default_rng(11)
    m = rng.standard_normal(d)
    m *= half_gap / np.linalg.norm(m)
    X = np.stack([m, -m], axis=1)
    y = np.array([1.0, -1.0])
    Z = X * y
    res = O.solve(Z, y, q, C, tol=1e-10, max_iter=200000)
    assert res["converged"]
    rc = (q / C) ** (1 / (q + 1))
    wstar = m / np.linalg.norm(m)
    assert np.linalg.norm(res["w"] - wstar) <= 1e-6
    if half_gap >= rc:
        obj = 2 * half_gap ** (-q)
        assert abs(res["beta"]) <= 1e-7
        assert np.allclose(res["r"], half_gap, rtol=1e-7)
        assert np.allclose(res["alpha"], q / half_gap ** (q + 1), rtol=1e-6)
    else:
        obj = 2 * (rc ** (-q) + C * (rc - half_gap))
        assert np.allclose(res["alpha"], C, rtol=1e-6)
        assert np.allclose(res["r"], rc, rtol=1e-6)
    assert abs(res["primal"] - obj) <= 1e-7 * obj


def test_two_point_general_offset():
    """Separable pair x1 != -x2: w* = (x1-x2)/Delta, beta* = -w*^T (x1+x2)/2."""
    rng = np.random.default_rng(12)
    x1, x2 = rng.standard_normal(5) + 2.0, rng.standard_normal(5) - 1.0
    X = np.stack([x1, x2], axis=1)
    y = np.array([1.0, -1.0])
    res = O.solve(X * y, y, 1.0, 100.0, tol=1e-11, max_iter=200000)
    delta = np.linalg.norm(x1 - x2)
    ws = (x1 - x2) / delta
    assert delta / 2 >= (1 / 100.0) ** 0.5
    assert np.linalg.norm(res["w"] - ws) <= 1e-6
    assert abs(res["beta"] + ws @ (x1 + x2) / 2) <= 1e-6


# ---------------------------------------------------------------- brute force d = 2

@pytest.mark.parametrize("q,C,seed", [(1.0, 1.0, 0), (2.0, 3.0, 1), (0.5, 0.7, 2), (4.0, 5.0, 3)])
def test_d2_brute_force(q, C, seed):
    """d = 2: grid over the unit disk and beta, refined by Nelder-Mead; the oracle is never worse."""
    rng = np.random.default_rng(100 + seed)
    X, y, Z = _two_class(rng, 2, 9, shift=1.2)
    res = O.solve(Z, y, q, C, tol=1e-10, max_iter=400000)
    assert res["converged"]

    def P(v):
        w = v[:2] / max(1.0, np.linalg.norm(v[:2]))
        return O.primal_value_at(Z, y, w, v[2], q, C)

    best, arg = math.inf, None
    for rad in np.linspace(0, 1, 21):
        for th in np.linspace(0, 2 * np.pi, 181, endpoint=False):
            for b in np.linspace(-4, 4, 81):
                v = np.array([rad * np.cos(th), rad * np.sin(th), b])
                f = P(v)
                if f < best:
                    best, arg = f, v
    ref = minimize(P, arg, method="Nelder-Mead", options={"xatol": 1e-12, "fatol": 1e-14, "maxiter": 20000})
    ref_val = min(ref.fun, best)
    oracle_val = O.primal_value_at(Z, y, res["w"] / max(1, np.linalg.norm(res["w"])), res["beta"], q, C)
    assert oracle_val <= ref_val * (1 + 1e-9)
    assert abs(oracle_val - ref_val) <= 1e-6 * ref_val
    assert abs(res["primal"] - ref_val) <= 1e-6 * ref_val


# ---------------------------------------------------------------- dual by a library solver

@pytest.mark.parametrize("q", [1.0, 2.0])
def test_dual_by_slsqp(q):
    """max of eq-dual over F_D (scipy SLSQP) equals the oracle's primal optimum (strong duality)."""
    rng = np.random.default_rng(21)
    X, y, Z = _two_class(rng, 5, 10, shift=0.6)
    C = 2.0
    res = O.solve(Z, y, q, C, tol=1e-10, max_iter=400000)
    k = O.kappa(q)

    def negdual(a):
        return np.linalg.norm(Z @ a) - k * np.sum(np.maximum(a, 0) ** (q / (q + 1)))

    a0 = np.full(10, C / 2)
    sol = minimize(negdual, a0, method="SLSQP", bounds=[(1e-12, C)] * 10,
                   constraints=[{"type": "eq", "fun": lambda a: y @ a}],
                   options={"ftol": 1e-14, "maxiter": 2000})
    assert abs(-sol.fun - res["primal"]) <= 1e-6 * abs(res["primal"])
    assert np.allclose(sol.x, res["alpha"], atol=1e-3 * C)


# ---------------------------------------------------------------- optimality certificate and bounds

@pytest.mark.parametrize("q", [0.5, 1.0, 2.0, 4.0])
def test_certified_gap_and_prop2(q):
    """Weak duality sandwich below 1e-9, KKT identities, and the Prop. 2 bounds."""
    rng = np.random.default_rng(31)
    X, y, Z = _two_class(rng, 60, 23, shift=0.8, n_pos=9)
    C = 1.5
    res = O.solve(Z, y, q, C, tol=1e-10, max_iter=400000)
    assert res["converged"]
    up, lo, gap = O.certified_gap(Z, y, res["w"], res["beta"], res["alpha"], q, C)
    assert lo <= up + 1e-12 * abs(up)
    assert gap <= 1e-9
    # KKT (eq-optimality)
    assert abs(y @ res["alpha"]) <= 1e-8
    assert np.allclose(res["alpha"], q / res["r"] ** (q + 1), rtol=1e-7)
    za = Z @ res["alpha"]
    assert np.linalg.norm(res["w"] - za / np.linalg.norm(za)) <= 1e-6
    # Prop. 2
    n = y.size
    K = np.linalg.norm(Z, axis=0).max()
    varrho = (n + C * n) / C
    assert res["xi"].max() <= varrho
    assert abs(res["beta"]) <= K + varrho
    assert res["r"].max() <= 2 * (K + varrho)
    assert res["alpha"].min() >= q / (2 * K + 2 * varrho) ** (q + 1)
    assert res["alpha"].max() <= C * (1 + 1e-9)


# ---------------------------------------------------------------- symmetries of the model

def test_invariances():
    rng = np.random.default_rng(41)
    X, y, Z = _two_class(rng, 40, 16, shift=0.7)
    q, C = 1.0, 2.0
    base = O.solve(Z, y, q, C, tol=1e-11, max_iter=400000)
    # flip labels: (w, beta) -> (-w, -beta), r/alpha unchanged
    fl = O.solve(X * (-y), -y, q, C, tol=1e-11, max_iter=400000)
    assert np.linalg.norm(fl["w"] + base["w"]) <= 1e-6
    assert abs(fl["beta"] + base["beta"]) <= 1e-6
    assert np.allclose(fl["alpha"], base["alpha"], rtol=1e-5, atol=1e-9)
    # permute features
    perm = rng.permutation(40)
    pf = O.solve(Z[perm], y, q, C, tol=1e-11, max_iter=400000)
    assert np.linalg.norm(pf["w"] - base["w"][perm]) <= 1e-6
    # orthogonal change of feature coordinates
    Q = np.linalg.qr(rng.standard_normal((40, 40)))[0]
    rot = O.solve(Q @ Z, y, q, C, tol=1e-11, max_iter=400000)
    assert np.linalg.norm(rot["w"] - Q @ base["w"]) <= 1e-6
    assert abs(rot["beta"] - base["beta"]) <= 1e-6
    # permute samples
    ps = rng.permutation(16)
    sp = O.solve(Z[:, ps], y[ps], q, C, tol=1e-11, max_iter=400000)
    assert np.allclose(sp["alpha"], base["alpha"][ps], rtol=1e-5, atol=1e-9)
    assert np.allclose(sp["r"], base["r"][ps], rtol=1e-6)


def test_scaling_invariance_of_solution():
    """Sec. 4.2: the scaled model has the same (r, xi, beta, alpha) and w = w~ / Z_scale."""
    rng = np.random.default_rng(51)
    X, y, Z = _two_class(rng, 30, 12, shift=0.9)
    res = O.solve(Z, y, 1.0, 1.0, tol=1e-11)
    assert abs(np.linalg.norm(res["w_scaled"]) / res["zscale"] - np.linalg.norm(res["w"])) <= 1e-12
    # the constraint of eq-primal holds in original units
    m = Z.T @ res["w"] + res["beta"] * y + res["xi"] - res["r"]
    assert np.linalg.norm(m) <= 1e-8


def test_paper_stopping_rule():
    """Sec. 4.3's rule (stop_rule = 1, tol = 1e-5): the final residuals meet its three
    conditions, it stops no later than the strict max-residual rule at the same tol,
    and its point is a moderately accurate solution (certified gap of the strict
    optimum's order of the tolerance)."""
    rng = np.random.default_rng(61)
    X, y, Z = _two_class(rng, 300, 60, shift=0.8)
    q, C = 2.0, 5.0
    pap = O.solve(Z, y, q, C, tol=1e-5, stop_rule=1, max_iter=2000)
    strict = O.solve(Z, y, q, C, tol=1e-5, stop_rule=0, max_iter=20000)
    assert pap["converged"] and strict["converged"]
    eta = pap["eta"]
    assert max(eta["P"], eta["D"]) < 1e-5
    assert min(eta["C"], eta["gap"]) < np.sqrt(1e-5)
    assert max(eta["C"], eta["gap"]) < 0.05
    assert pap["iters"] <= strict["iters"]
    ref = O.solve(Z, y, q, C, tol=1e-11, max_iter=200000)
    assert abs(pap["primal"] - ref["primal"]) / ref["primal"] <= 0.05
    # strict run at the tighter tolerance meets every residual
    assert strict["eta"]["kkt"] <= 1e-5


def test_imbalance_weights_closed_form():
    """Sec. 4.5: K cancels in the ratio, so the minority class gets weight 1 and the
    majority class (n_min / n_maj)^(1/(1+q)); balanced classes give all ones."""
    y = np.array([1.0] * 3 + [-1.0] * 7)
    w = O.imbalance_weights(y, 1.0)
    assert np.allclose(w[:3], 1.0) and np.allclose(w[3:], 0.6546536707079771)      # sqrt(3/7)
    w2 = O.imbalance_weights(y, 2.0)
    assert np.allclose(w2[3:], 0.7539474411291538)                                  # (3/7)^(1/3)
    assert np.allclose(O.imbalance_weights(np.array([1.0, -1.0] * 5), 4.0), 1.0)


def test_suggest_C_hand_example():
    """Sec. 4.1 on four 1-D points: x_+ = {0, 1}, x_- = {3, 5}; between-class
    distances {3, 5, 2, 4}, median 3.5; n = 4, d = 1 (max{1000, d} = 1000)."""
    x = np.array([[0.0, 1.0, 3.0, 5.0]])
    y = np.array([1.0, 1.0, -1.0, -1.0])
    Z = x * y
    # q = 1: 10^2 max{1, log(4) * 10 / 3.5^2} = 100 * 1.131668...
    assert abs(O.suggest_C(Z, y, 1.0) - 113.1668866220319) <= 1e-9
    # q = 2: 10^3 max{1, 10 log(4) * 10 / 3.5^3} = 1000 * 3.233339...
    assert abs(O.suggest_C(Z, y, 2.0) - 3233.33961777234) <= 1e-7
