"""Pins for the oracle's r-subproblem solver (Step 1b, eq-varphi, Sec. 3.2).

None of these re-types the oracle's Newton formula: each checks the root against
something the mathematics fixes independently (the defining polynomial, the
closed-form roots of the q = 1 cubic, a library bracketing root finder, and the
convexity/uniqueness of the minimiser).
"""
import math

import numpy as np
import pytest
from scipy.optimize import brentq, minimize_scalar

from oracle import gdwd_oracle as O

QS = [0.5, 1.0, 2.0, 4.0]


def _grid():
    a = np.concatenate([-np.logspace(3, -3, 25), [0.0], np.logspace(-3, 3, 25)])
    sig = np.logspace(-3, 4, 8)
    return a, sig


@pytest.mark.parametrize("q", QS)
def test_prox_polynomial_residual(q):
    """s^(q+1)(s - a) = q/sigma to 1e-12 relative over a in [-1e3, 1e3], sigma in [1e-3, 1e4]."""
    a, sig = _grid()
    for s_ in sig:
        s = O.prox_r(a, s_, q)
        assert np.all(s > 0)
        lhs = s ** (q + 1) * (s - a)
        scale = np.maximum.reduce([s ** (q + 2), np.abs(a) * s ** (q + 1), np.full_like(s, q / s_)])
        rel = np.abs(lhs - q / s_) / scale
        assert rel.max() <= 1e-12, (q, s_, rel.max())


def _depressed_cubic_max_root(p, qq):
    """Largest real root of t^3 + p t + qq = 0 (Cardano, or the trigonometric form for 3 real roots)."""
    disc = (qq / 2.0) ** 2 + (p / 3.0) ** 3
    if disc > 0:
        # Cardano with the cancellation-free pairing u v = -p/3
        sq = math.sqrt(disc)
        u = np.cbrt(-qq / 2.0 - math.copysign(sq, qq))
        return u - p / (3.0 * u) if u != 0 else 0.0
    m = 2.0 * math.sqrt(-p / 3.0)
    th = math.acos(max(-1.0, min(1.0, 3.0 * qq / (p * m)))) / 3.0
    return max(m * math.cos(th - 2.0 * math.pi * k / 3.0) for k in range(3))


def _cubic_root(a, sigma):
    """Positive root of s^3 - a s^2 - 1/sigma = 0 in closed form.

    Two closed forms: s = t + a/3 with t a root of the depressed cubic, or
    s = 1/x with x the positive root of x^3 + a sigma x - sigma = 0 (already
    depressed; well conditioned when s is small).  The one with the smaller
    relative residual is returned.
    """
    s1 = _depressed_cubic_max_root(-a * a / 3.0, -2.0 * a ** 3 / 27.0 - 1.0 / sigma) + a / 3.0
    s2 = 1.0 / _depressed_cubic_max_root(a * sigma, -sigma)

    def rel(s):
        return abs(s ** 3 - a * s ** 2 - 1.0 / sigma) / max(s ** 3, abs(a) * s ** 2, 1.0 / sigma) if s > 0 else math.inf

    return s1 if rel(s1) <= rel(s2) else s2


def test_prox_q1_closed_form():
    """q = 1: the minimiser is the positive root of the cubic s^3 - a s^2 - 1/sigma (Sec. 3.2)."""
    a, sig = _grid()
    worst = 0.0
    for s_ in sig:
        s = O.prox_r(a, s_, 1.0)
        for ai, si in zip(a, s):
            ref = _cubic_root(ai, s_)
            # one Newton polish of the closed form (cancellation in Cardano for large |a|)
            f = ref ** 3 - ai * ref ** 2 - 1.0 / s_
            ref -= f / (3 * ref ** 2 - 2 * ai * ref)
            worst = max(worst, abs(si - ref) / ref)
    assert worst <= 1e-12


@pytest.mark.parametrize("q", [0.5, 2.0, 4.0])
def test_prox_vs_library_root_finder(q):
    """Matches scipy's brentq on phi'(s) = -q s^-(q+1) + sigma (s - a) inside the bracket."""
    rng = np.random.default_rng(7)
    for _ in range(200):
        a = rng.uniform(-50, 50)
        sig = 10 ** rng.uniform(-2, 3)
        hi = max(a, 0.0) + (q / sig) ** (1 / (q + 2)) + 1e-12
        lo = a if a > 0 else 1e-8 * hi
        ref = brentq(lambda s: -q * s ** (-q - 1) + sig * (s - a), lo, hi,
                     xtol=1e-300, rtol=4 * np.finfo(float).eps, maxiter=500)
        s = O.prox_r(np.array([a]), sig, q)[0]
        assert abs(s - ref) <= 1e-13 * ref, (q, a, sig, s, ref)


@pytest.mark.parametrize("q", QS)
def test_prox_is_minimiser(q):
    """The returned point minimises phi(s) = s^-q + sigma/2 (s-a)^2 (bounded 1-D minimiser)."""
    rng = np.random.default_rng(3)
    for _ in range(50):
        a = rng.uniform(-5, 5)
        sig = 10 ** rng.uniform(-1, 2)
        s = O.prox_r(np.array([a]), sig, q)[0]
        phi = lambda t: t ** (-q) + 0.5 * sig * (t - a) ** 2
        m = minimize_scalar(phi, bounds=(1e-6, max(a, 0) + 10), method="bounded",
                            options={"xatol": 1e-12})
        assert phi(s) <= phi(m.x) + 1e-10 * abs(phi(m.x))


def test_prox_warm_start_and_weights():
    """Warm start anywhere (even outside the bracket) gives the same root; omega scales the constant."""
    rng = np.random.default_rng(5)
    a = rng.uniform(-3, 3, 1000)
    s_cold = O.prox_r(a, 2.0, 2.0)
    s_warm = O.prox_r(a, 2.0, 2.0, r0=rng.uniform(1e-3, 100, 1000))
    assert np.allclose(s_cold, s_warm, rtol=1e-13, atol=0)
    om = rng.uniform(0.1, 3.0, 1000)
    s = O.prox_r(a, 2.0, 2.0, omega=om)
    assert np.allclose(s ** 3 * (s - a), om / 2.0, rtol=1e-11)


@pytest.mark.parametrize("q", QS)
def test_kappa_conjugate(q):
    """inf_{r>0} r^-q + alpha r = kappa alpha^(q/(q+1)) (derivation of eq-dual, Sec. 2)."""
    for alpha in [1e-3, 0.1, 1.0, 7.5, 300.0]:
        f = lambda r: r ** (-q) + alpha * r
        rstar = (q / alpha) ** (1 / (q + 1))
        m = minimize_scalar(f, bounds=(rstar / 10, rstar * 10), method="bounded", options={"xatol": 1e-12})
        assert abs(m.fun - O.kappa(q) * alpha ** (q / (q + 1))) <= 1e-9 * m.fun
