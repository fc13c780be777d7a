"""Pins of the oracle's inexact variant of Algorithm 1 (Sec. 3, Steps 1a-1c and
eq-linsys-tol; Sec. 3.3.3, d and n both large, T = 0), checked against what the
mathematics fixes rather than against the code itself:

* the matrix-free operator of eq-linsys equals the dense (d+1) x (d+1) A, and its
  diagonal is A's;
* PCG returns a point whose TRUE residual meets the requested tolerance, and that
  point agrees with a dense direct solve to within the tolerance over the
  smallest eigenvalue of A;
* the tolerances eps_k = c / (k+1)^1.5 are nonincreasing and summable (their sum
  is below c * zeta(1.5));
* with tolerances at the rounding level the inexact algorithm is the exact one:
  same iteration count and the same solution as the SMW2 solve;
* with the default schedule it reaches the same optimum (objective, w, certified
  gap), Step 1a solves every iteration and Step 1c only when Step 1a's solution
  misses 5 eps_k for the new right-hand side (checked call by call).
"""
import math

import numpy as np
import pytest

from oracle import gdwd_oracle as O


def _problem(seed, d, n, n_pos, shift=0.9):
    rng = np.random.default_rng(seed)
    y = np.where(np.arange(n) < n_pos, 1.0, -1.0)
    X = rng.standard_normal((d, n)) + shift * y[None, :] * np.eye(d, 1)
    return X * y[None, :], y, rng


def test_operator_is_eq_linsys():
    Z, y, rng = _problem(1, 9, 7, 3)
    mu = 0.7
    op = O.LinsysOperator(Z, y, mu)
    A = O.SMW2(Z, y, mu).matrix()
    for _ in range(3):
        v = rng.standard_normal(10)
        assert np.allclose(op.matvec(v), A @ v, rtol=1e-13, atol=1e-13)
    assert np.allclose(op.diagonal(), np.diag(A), rtol=1e-14)


@pytest.mark.parametrize("tol", [1e-3, 1e-7, 1e-11])
def test_pcg_meets_its_tolerance(tol):
    Z, y, rng = _problem(2, 40, 25, 10)
    mu = 1.3
    op = O.LinsysOperator(Z, y, mu)
    A = O.SMW2(Z, y, mu).matrix()
    lmin = np.linalg.eigvalsh(A)[0]
    for _ in range(3):
        h = rng.standard_normal(41)
        x, res, steps = O.pcg(op, h, np.zeros(41), tol)
        # the true residual (rounding of h - A x is about 1e-15 of ||h||)
        assert res == pytest.approx(np.linalg.norm(h - A @ x), rel=1e-9, abs=1e-13 * np.linalg.norm(h))
        assert res <= tol
        xs = np.linalg.solve(A, h)
        assert np.linalg.norm(x - xs) <= tol / lmin * (1 + 1e-6)
        # started at the solution it takes no step
        _, _, s0 = O.pcg(op, h, xs, max(tol, 1e-10))
        assert s0 == 0


def test_eps_schedule_is_summable():
    c = 0.37
    eps = np.array([O.eps_schedule(k, c) for k in range(200000)])
    assert np.all(np.diff(eps) <= 0)
    zeta15 = 2.612375348685488
    assert eps.sum() < c * zeta15
    assert eps[0] == c and eps[3] == pytest.approx(c / 8.0)


@pytest.mark.parametrize("q", [1.0, 2.0])
def test_rounding_level_tolerances_reproduce_the_exact_algorithm(q):
    Z, y, _ = _problem(3, 60, 30, 12)
    ex = O.solve(Z, y, q, 1.5, tol=1e-8)
    ix = O.solve_inexact(Z, y, q, 1.5, tol=1e-8, eps_c=1e-13)
    assert ex["converged"] and ix["converged"]
    assert ix["iters"] == ex["iters"]
    assert np.allclose(ix["r"], ex["r"], rtol=1e-7, atol=1e-10)
    assert np.allclose(ix["alpha"], ex["alpha"], rtol=1e-7, atol=1e-10)
    assert abs(ix["primal"] - ex["primal"]) <= 1e-10 * abs(ex["primal"])


@pytest.mark.parametrize("q,C", [(1.0, 2.0), (0.5, 1.0), (2.0, 5.0)])
def test_default_schedule_reaches_the_optimum(q, C, monkeypatch):
    Z, y, _ = _problem(4, 300, 120, 45, shift=0.8)
    calls = []
    real = O.pcg

    def spy(op, h, x0, tol, max_steps=10000):
        before = np.linalg.norm(h - op.matvec(np.asarray(x0, dtype=np.float64)))
        out = real(op, h, x0, tol, max_steps)
        calls.append((tol, before, out[1]))
        return out

    monkeypatch.setattr(O, "pcg", spy)
    ix = O.solve_inexact(Z, y, q, C, tol=1e-7, record=True)
    monkeypatch.undo()
    ex = O.solve(Z, y, q, C, tol=1e-9)
    assert ix["converged"]
    assert abs(ix["primal"] - ex["primal"]) <= 1e-6 * abs(ex["primal"])
    assert np.linalg.norm(ix["w"] - ex["w"]) <= 1e-4 * np.linalg.norm(ex["w"])
    up, lo, gap = O.certified_gap(Z, y, ix["w"], ix["beta"], ix["alpha"], q, C)
    assert gap <= 1e-6
    # one Step 1a solve per iteration at eps_k; Step 1c solves only at 5 eps_k, and
    # only when the reused point missed that accuracy; every solve met its target
    eps = [h[4] for h in ix["history"]]
    a_calls = [c for c in calls if any(math.isclose(c[0], e_, rel_tol=1e-15) for e_ in eps)]
    c_calls = [c for c in calls if c not in a_calls]
    assert len(a_calls) == ix["iters"]
    assert len(c_calls) == ix["step1c_solves"]
    for tol, before, after in calls:
        assert after <= tol
    for tol, before, after in c_calls:
        assert before > tol                       # Step 1c solved only when reuse failed
    assert ix["step1c_solves"] < ix["iters"]      # and the reuse did succeed sometimes
