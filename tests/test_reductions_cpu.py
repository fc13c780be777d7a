"""CPU checks of the algebra the CUDA path uses in place of the paper's formulas,
against the oracle (no CUDA code is imported).

* The n-space reduction of eq-linsys (Woodbury on the SMW2 form): x = G^{-1}(b + v),
  beta = -y^T x / s, c = x + beta p, w = g' - Z~ c / mu.
* The border elimination of the direct solver: with G' = I + Z~ Z~^T / mu,
  P = G'^{-1}, b^ = Z~ y, p = P b^, s = b^T p:
  beta = (h_beta - p^T h_w / mu) / (n - s / mu), w = (P h_w - p beta) / mu.
* The kernelized iteration: u, rho, g carried as coefficient vectors in the columns
  of Z~, every d-space norm a quadratic form in K = Z~^T Z~; its iterates equal
  those of Algorithm 1 as the oracle runs it.
* The fused first solve: Step 1a's x-bar from products formed before sigma' is
  known (three vectors in general, two when sigma is kept).
* The residual sums taken about the last theta (eta_P2, eta_D3, ||w||).
"""
import math

import numpy as np

from oracle import gdwd_oracle as O


def _problem(seed, d, n, mu=0.8):
    rng = np.random.default_rng(seed)
    Z = rng.standard_normal((d, n))
    y = np.where(np.arange(n) < n // 3, 1.0, -1.0)
    return Z, y, mu, rng


def test_nspace_reduction_matches_smw2():
    Z, y, mu, rng = _problem(1, 40, 12)
    G = np.eye(12) + Z.T @ Z / mu
    p = np.linalg.solve(G, y)
    s = y @ p
    for _ in range(3):
        u, rho, v = rng.standard_normal(40), rng.standard_normal(40), rng.standard_normal(12)
        sigma = 0.37
        gp = u + rho / (sigma * math.sqrt(mu))
        x = np.linalg.solve(G, Z.T @ gp + v)
        beta = -(y @ x) / s
        c = x + beta * p
        w = gp - Z @ c / mu
        h = np.concatenate([-Z @ v + mu * u + math.sqrt(mu) * rho / sigma, [-(y @ v)]])
        ref = O.SMW2(Z, y, mu).solve(h)
        assert np.allclose(w, ref[:40], rtol=1e-11, atol=1e-11)
        assert abs(beta - ref[40]) <= 1e-11 * (1 + abs(ref[40]))


def test_direct_border_elimination_matches_direct_solve():
    Z, y, mu, rng = _problem(2, 6, 50)
    d, n = Z.shape
    Gp = np.eye(d) + Z @ Z.T / mu
    P = np.linalg.inv(Gp)
    bh = Z @ y
    p = P @ bh
    s = bh @ p
    for _ in range(3):
        h = rng.standard_normal(d + 1)
        beta = (h[d] - p @ h[:d] / mu) / (n - s / mu)
        w = (P @ h[:d] - p * beta) / mu
        ref = O.Direct(Z, y, mu).solve(h)
        assert np.allclose(w, ref[:d], rtol=1e-11, atol=1e-11)
        assert abs(beta - ref[d]) <= 1e-11 * (1 + abs(ref[d]))


def test_kernelized_iterates_equal_algorithm_1():
    """Twenty iterations of the coefficient form against the oracle's own iterates
    (the same sigma: the oracle's sigma path is replayed)."""
    rng = np.random.default_rng(3)
    d, n, q, C, mu, tau = 30, 14, 1.0, 2.0, 1.0, 1.618
    y = np.where(np.arange(n) < 6, 1.0, -1.0)
    Z = rng.standard_normal((d, n)) * y
    ref = O.solve(Z, y, q, C, mu=mu, tau=tau, tol=1e-300, max_iter=60, record=True)
    sigmas = [h[0] for h in ref["history"]]
    Zt, zs = O.scale_data(Z)
    K = Zt.T @ Zt
    G = np.eye(n) + K / mu
    p = np.linalg.solve(G, y)
    s = y @ p
    sq = math.sqrt(mu)
    r, xi, alpha = np.ones(n), np.ones(n), np.zeros(n)
    au, ar = np.zeros(n), np.zeros(n)
    for sigma in sigmas:
        gs = 1.0 / (sigma * sq)
        b = K @ au + (K @ ar) * gs                                    # Z~^T g'
        vbar = xi - r - alpha / sigma
        xb = np.linalg.solve(G, b + vbar)
        betab = -(y @ xb) / s
        cbar = xb + betab * p
        r = O.prox_r(cbar + r, sigma, q, r0=r)                        # Step 1b
        v = xi - r - alpha / sigma
        x = np.linalg.solve(G, b + v)
        beta = -(y @ x) / s
        c = x + beta * p
        ztw = c - v - y * beta                                        # Z~^T w
        ag = au - c / mu                                              # g = Z~ a_g
        gnorm = math.sqrt(max(ag @ K @ ag, 0.0))
        theta = 1.0 if gnorm <= zs else zs / gnorm
        xi = np.maximum(0.0, r - ztw - y * beta + alpha / sigma - C / sigma)   # Step 2
        alpha = alpha - tau * sigma * (ztw + y * beta + xi - r)                # Step 3
        ar = (1.0 - tau) * ar - tau * sigma * sq * (1.0 - theta) * ag
        au = theta * ag
    assert np.allclose(r, ref["r"], rtol=1e-9, atol=1e-12)
    assert np.allclose(alpha, ref["alpha"], rtol=1e-9, atol=1e-12)
    assert np.allclose(xi, ref["xi"], rtol=1e-9, atol=1e-12)
    assert np.allclose(Zt @ au, ref["u_scaled"], rtol=1e-9, atol=1e-12)
    assert np.allclose(Zt @ ar, ref["rho"], rtol=1e-9, atol=1e-12)


def test_fused_first_solve_equals_direct_solve():
    """The Z-streaming kernel forms Step 1a's x-bar = G^{-1} rhs1 of iteration k+1
    from three G^{-1} products taken during iteration k's pass over Z:
        rhs1 = a1 U_g + ((1 - tau) U_rho / sqrt(mu) - alpha) / sigma' + (xi - r),
        a1 = theta - tau (sigma / sigma') (1 - theta),
    with U_g = Z~^T g, U_rho = Z~^T rho of iteration k and sigma' the next sigma.
    When the sigma rule keeps sigma' = sigma this is a1 U_g + W with
    W = ((1 - tau) U_rho / sqrt(mu) - alpha) / sigma + (xi - r) and
    a1 = theta - tau (1 - theta): two products, the form the kernel takes.
    Sixty iterations on the oracle's sigma path: both fused x-bars equal the direct
    one, and the iterates equal the oracle's."""
    rng = np.random.default_rng(4)
    d, n, q, C, mu, tau = 30, 14, 1.0, 2.0, 0.7, 1.618
    y = np.where(np.arange(n) < 6, 1.0, -1.0)
    Z = rng.standard_normal((d, n)) * y
    ref = O.solve(Z, y, q, C, mu=mu, tau=tau, tol=1e-300, max_iter=60, record=True)
    sigmas = [h[0] for h in ref["history"]]
    Zt, zs = O.scale_data(Z)
    G = np.eye(n) + Zt.T @ Zt / mu
    Gi = np.linalg.inv(G)
    p = Gi @ y
    s = y @ p
    sq = math.sqrt(mu)
    r, xi, alpha = np.ones(n), np.ones(n), np.zeros(n)
    u, rho = np.zeros(d), np.zeros(d)
    prev = None   # (X1, X2, X3, XW, theta, sigma) from the last pass
    kept = 0
    for sigma in sigmas:
        gp = u + rho / (sigma * sq)
        b = Zt.T @ gp
        rhs1 = b + xi - r - alpha / sigma
        xb = Gi @ rhs1
        if prev is not None:
            X1, X2, X3, XW, th, sp = prev
            a1 = th - tau * (sp / sigma) * (1.0 - th)
            xf = a1 * X1 + X2 / sigma + X3
            assert np.allclose(xf, xb, rtol=1e-10, atol=1e-12 * np.abs(xb).max())
            if sigma == sp:
                kept += 1
                x2 = (th - tau * (1.0 - th)) * X1 + XW
                assert np.allclose(x2, xb, rtol=1e-10, atol=1e-12 * np.abs(xb).max())
        betab = -(y @ xb) / s
        r = O.prox_r(xb + betab * p + r, sigma, q, r0=r)
        v = xi - r - alpha / sigma
        x = Gi @ (b + v)
        beta = -(y @ x) / s
        c = x + beta * p
        w = gp - Zt @ c / mu
        g = w - rho / (sigma * sq)
        gn = np.linalg.norm(g)
        theta = 1.0 if gn <= zs else zs / gn
        ztw = Zt.T @ w
        xi = np.maximum(0.0, r - ztw - y * beta + alpha / sigma - C / sigma)
        alpha = alpha - tau * sigma * (ztw + y * beta + xi - r)
        # the three right-hand sides the kernel multiplies by G^{-1} during the pass
        V1 = Zt.T @ g
        V2 = (1.0 - tau) * (Zt.T @ rho) / sq - alpha
        V3 = xi - r
        prev = (Gi @ V1, Gi @ V2, Gi @ V3, Gi @ (V2 / sigma + V3), theta, sigma)
        rho = rho - tau * sigma * sq * (w - theta * g)
        u = theta * g
    assert kept >= 10, kept
    assert np.allclose(r, ref["r"], rtol=1e-9, atol=1e-12)
    assert np.allclose(alpha, ref["alpha"], rtol=1e-9, atol=1e-12)
    assert np.allclose(u, ref["u_scaled"], rtol=1e-9, atol=1e-12)


def test_residual_sums_about_the_last_theta():
    """eta_P2 and eta_D3 need ||(1 - theta) g + gs rho||^2 and ||a - kap g||^2
    (kap = tau mu sigma (1 - theta)), with theta known only after the pass that
    forms g.  The kernels sum y = (1 - theta_p) g + gs rho and v = a - khat g
    (khat = tau mu sigma (1 - theta_p)) about the last theta_p and expand in
    eps = theta_p - theta:
        ||w - u+||^2 = ||y||^2 + 2 eps <y, g> + eps^2 ||g||^2,
        ||a - kap g||^2 = ||v||^2 - 2 dlt <v, g> + dlt^2 ||g||^2, dlt = tau mu sigma eps,
        ||w||^2 = ||y||^2 + 2 theta_p <y, g> + theta_p^2 ||g||^2.
    Near convergence (small residuals, theta settled) these keep their relative
    accuracy, while the expansions in ||g||^2, <g, rho>, ||rho||^2 (or ||a||^2,
    <a, g>) lose it to cancellation."""
    rng = np.random.default_rng(11)
    d, tau, mu, sigma = 4000, 1.618, 0.9, 37.0
    gs = 1.0 / (sigma * math.sqrt(mu))
    g = rng.standard_normal(d) * 5.0
    for theta_p, theta in ((0.31, 0.31), (0.31, 0.3100004), (1.0, 1.0), (0.8, 0.7)):
        kap = tau * mu * sigma * (1.0 - theta)
        # rho and a chosen so that both residuals are ~1e-7 of their terms
        rho = -(1.0 - theta) * g / gs + 1e-7 * rng.standard_normal(d)
        a = kap * g + 1e-7 * rng.standard_normal(d)
        true_p2 = np.sum(((1.0 - theta) * g + gs * rho) ** 2)
        true_d3 = np.sum((a - kap * g) ** 2)
        # the kernels' sums and expansion
        y = (1.0 - theta_p) * g + gs * rho
        v = a - tau * mu * sigma * (1.0 - theta_p) * g
        eps = theta_p - theta
        dlt = tau * mu * sigma * eps
        p2 = y @ y + 2.0 * eps * (y @ g) + eps * eps * (g @ g)
        d3 = v @ v - 2.0 * dlt * (v @ g) + dlt * dlt * (g @ g)
        w = g + gs * rho
        w2 = y @ y + 2.0 * theta_p * (y @ g) + theta_p ** 2 * (g @ g)
        assert abs(w2 - w @ w) <= 1e-9 * (w @ w)
        if eps == 0.0:
            # theta settled: the sums are the residuals themselves
            assert abs(p2 - true_p2) <= 1e-9 * true_p2
            assert abs(d3 - true_d3) <= 1e-9 * true_d3
            # while the old expansions about theta = 1 lose them to cancellation
            old_d3 = kap * kap * (g @ g) - 2.0 * kap * (a @ g) + a @ a
            assert abs(old_d3 - true_d3) > 1e-3 * true_d3 or kap == 0.0
        else:
            scale = (1.0 - theta) ** 2 * (g @ g)
            assert abs(p2 - true_p2) <= 1e-12 * scale + 1e-9 * true_p2
