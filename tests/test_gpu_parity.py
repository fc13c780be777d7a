"""GPU parity: the CUDA path through the C-ABI against the FP64 CPU oracle.

Component parity (element by element): the Step-1b prox, the Gram matrix
G = I + Z~^T Z~ / mu of the SMW2 set-up, and the two streaming products
Z~^T x / Z~ x.  Solution parity: gdwd_solve against oracle.solve on seeded
synthetic problems at sizes that span several slabs, tiles and a ragged tail,
then the full spiked FP32 workload (d = 20000, n = 1000) against the oracle and
the weak-duality certificate.

Tolerances (the acceptance bar): |d obj|/|obj| <= 1e-6,
||dw||/||w|| <= 1e-4, identical held-out predictions except near-ties
(|w^T x + beta| < 1e-6 ||x||), kkt <= tol.
"""
import numpy as np
import pytest

from oracle import gdwd_oracle as O
from paper_2305_12019_gb300 import synth

pytestmark = pytest.mark.gpu

OBJ_TOL = 1e-6
W_TOL = 1e-4


def _torch():
    import torch
    return torch


def _predictions_match(Xt, w_gpu, b_gpu, w_ref, b_ref):
    s_gpu = Xt.T @ w_gpu + b_gpu
    s_ref = Xt.T @ w_ref + b_ref
    tie = np.abs(s_ref) < 1e-6 * np.linalg.norm(Xt, axis=0)
    return np.array_equal(np.sign(s_gpu[~tie]), np.sign(s_ref[~tie])), int(tie.sum())


def _compare(res, w, ref, obj_tol=OBJ_TOL, w_tol=W_TOL):
    relobj = abs(res["primal_obj"] - ref["primal"]) / abs(ref["primal"])
    relw = np.linalg.norm(w - ref["w"]) / np.linalg.norm(ref["w"])
    assert relobj <= obj_tol, relobj
    assert relw <= w_tol, relw
    return relobj, relw


# --------------------------------------------------------------------- components

@pytest.mark.parametrize("q", [0.5, 1.0, 2.0, 4.0, 3.0])
def test_prox_parity(gdwd_lib, q):
    torch = _torch()
    rng = np.random.default_rng(int(q * 10))
    n = 20011
    a = np.concatenate([rng.uniform(-1e3, 1e3, n // 2), rng.uniform(-3, 3, n - n // 2)])
    r0 = np.where(rng.random(n) < 0.5, rng.uniform(1e-3, 10, n), -1.0)
    om = rng.uniform(0.2, 5.0, n)
    for sigma in [1e-3, 0.37, 1.0, 250.0]:
        ad, rd, od = (torch.tensor(v, device="cuda") for v in (a, r0, om))
        got = gdwd_lib.prox(ad, sigma, q, r0=rd, omega=od).cpu().numpy()
        ref = O.prox_r(a, sigma, q, r0=np.where(r0 > 0, r0, np.nan), omega=om)
        assert np.all(got > 0)
        rel = np.abs(got - ref) / ref
        assert rel.max() <= 1e-12, (q, sigma, rel.max())
    got0 = gdwd_lib.prox(torch.zeros(0, dtype=torch.float64, device="cuda"), 1.0, q)
    assert got0.numel() == 0


@pytest.mark.parametrize("gram_path", [0, 1])
@pytest.mark.parametrize("store,d,n", [("f64", 3001, 257), ("f32", 3001, 257), ("f32", 9000, 130),
                                       ("f64", 37, 300), ("f64", 2500, 157), ("f32", 1111, 65)])
def test_gram_parity(gdwd_lib, store, d, n, gram_path):
    rng = np.random.default_rng(d + n)
    y = np.where(np.arange(n) % 3 == 0, 1.0, -1.0)
    X = rng.standard_normal((d, n))
    if store == "f32":
        X = X.astype(np.float32).astype(np.float64)
    Z = X * y
    mu = 0.7
    with gdwd_lib.Solver(Z.astype(np.float32) if store == "f32" else Z, y, 1.0, 1.0, store=store, mu=mu,
                         gram_path=gram_path) as s:
        G = s.gram()
        info = s.info()
        zs = info["zscale"]
    assert info["gram_tensor_cores"] == (1 if (store == "f32" and gram_path == 0) else 0)
    Zt, zs_ref = O.scale_data(Z)
    Gref = np.eye(n) + Zt.T @ Zt / mu
    assert abs(zs - zs_ref) <= 1e-13 * zs_ref
    err = np.abs(G - Gref).max() / np.abs(Gref).max()
    # FP32 storage, SIMT kernel: products rounded to FP32 and summed in FP32 over
    # 16-row chunks before the double-float fold, ~16 * 2^-24 per chunk relative,
    # random over d/16 chunks: a few 1e-8 of the largest entry.  FP32 storage,
    # tensor cores: exact products of the BF16 split terms, but the tensor core's
    # FP32 accumulation of a 64-row strip (four roundings of up to 2^-23 each,
    # not necessarily of random sign) plus the dropped terms (below 2^-23 of a
    # product): <= 6e-7 of the largest entry.  FP64 storage: FP64 sums.
    bound = 1e-13 if store == "f64" else (6e-7 if gram_path == 0 else 5e-8)
    assert err <= bound, err
    assert np.array_equal(G, G.T)


@pytest.mark.parametrize("store,d,n", [("f64", 5003, 301), ("f32", 20000, 1000), ("f32", 333, 77)])
def test_apply_parity(gdwd_lib, store, d, n):
    torch = _torch()
    rng = np.random.default_rng(5)
    y = np.where(np.arange(n) < n // 2, 1.0, -1.0)
    X = rng.standard_normal((d, n))
    if store == "f32":
        X = X.astype(np.float32).astype(np.float64)
    Z = X * y
    Zt, _ = O.scale_data(Z)
    with gdwd_lib.Solver(Z.astype(np.float32) if store == "f32" else Z, y, 1.0, 1.0, store=store) as s:
        xd = rng.standard_normal(d)
        xn = rng.standard_normal(n)
        out_n = torch.zeros(n, dtype=torch.float64, device="cuda")
        out_d = torch.zeros(d, dtype=torch.float64, device="cuda")
        s.apply(torch.tensor(xd, device="cuda"), out_n, trans=True)
        s.apply(torch.tensor(xn, device="cuda"), out_d, trans=False)
    ref_n = Zt.T @ xd
    ref_d = Zt @ xn
    # FP32 streams: products rounded to FP32 against an FP64 reference
    tol = 1e-13 if store == "f64" else 2e-6
    scale_n = np.abs(Zt).T @ np.abs(xd)
    scale_d = np.abs(Zt) @ np.abs(xn)
    assert np.max(np.abs(out_n.cpu().numpy() - ref_n) / scale_n) <= tol
    assert np.max(np.abs(out_d.cpu().numpy() - ref_d) / scale_d) <= tol


# --------------------------------------------------------------------- whole solves

def test_plain_fp64_workload(gdwd_lib):
    """d=500, n=100, N(+-0.5 e1, I), q=1, C=1, sigma0=1, tol 1e-9, FP64."""
    inst = synth.plain_fp64()
    ref = O.solve(inst.Z, inst.y, inst.q, inst.C, sigma0=1.0, tol=1e-10)
    with gdwd_lib.Solver(inst.Z, inst.y, inst.q, inst.C, store="f64", sigma0=1.0, tol=inst.tol) as s:
        res, w, alpha = s.solve(alpha=True)
    r = res[0]
    assert r["status"] == 0 and r["kkt"] <= inst.tol, r
    _compare(r, w[:, 0], ref)
    assert abs(r["beta"] - ref["beta"]) <= 1e-5 * (1 + abs(ref["beta"]))
    assert np.allclose(alpha[:, 0], ref["alpha"], rtol=1e-5, atol=1e-8)
    ok, ties = _predictions_match(inst.Xtest, w[:, 0], r["beta"], ref["w"], ref["beta"])
    assert ok
    # the certificate on the GPU output alone
    up, lo, gap = O.certified_gap(inst.Z, inst.y, w[:, 0], r["beta"], alpha[:, 0], inst.q, inst.C)
    assert gap <= 1e-8


@pytest.mark.parametrize("q,store,d,n,n_pos,C", [
    (1.0, "f32", 4001, 203, 101, 10.0),
    (0.5, "f64", 2500, 157, 40, 2.0),
    (2.0, "f32", 6007, 311, 200, 5.0),
    (4.0, "f64", 1201, 96, 70, 1.0),
])
def test_small_solves_match_oracle(gdwd_lib, q, store, d, n, n_pos, C):
    inst = synth.gaussian(seed=d + n, d=d, n=n, shift=1.0, n_pos=n_pos, q=q, C=C, m_test=500,
                          dtype=np.float32 if store == "f32" else np.float64)
    Z = inst.Z
    tol = 1e-8 if store == "f64" else 1e-6
    ref = O.solve(Z.astype(np.float64), inst.y, q, C, tol=1e-9)
    with gdwd_lib.Solver(Z, inst.y, q, C, store=store, tol=tol) as s:
        res, w, alpha = s.solve(alpha=True)
    r = res[0]
    assert r["status"] == 0 and r["kkt"] <= tol, r
    _compare(r, w[:, 0], ref)
    ok, _ = _predictions_match(inst.Xtest.astype(np.float64), w[:, 0], r["beta"], ref["w"], ref["beta"])
    assert ok
    up, lo, gap = O.certified_gap(Z.astype(np.float64), inst.y, w[:, 0], r["beta"], alpha[:, 0], q, C)
    assert gap <= 10 * tol


def test_c_grid_sequential(gdwd_lib):
    """One handle, several C (the factor does not depend on C)."""
    inst = synth.gaussian(seed=77, d=3000, n=150, shift=1.0, q=1.0, C=1.0, dtype=np.float64)
    Cs = [0.1, 1.0, 10.0]
    with gdwd_lib.Solver(inst.Z, inst.y, 1.0, 1.0, store="f64", tol=1e-8) as s:
        res, w, _ = s.solve(Cs=Cs)
    for k, C in enumerate(Cs):
        ref = O.solve(inst.Z, inst.y, 1.0, C, tol=1e-9)
        assert res[k]["status"] == 0
        _compare(res[k], w[:, k], ref)


def test_spiked_fp32_full_size(gdwd_lib):
    """The full d=20000, n=1000 spiked FP32 workload against the oracle and the certificate."""
    inst = synth.spiked_fp32()
    Z = inst.Z
    with gdwd_lib.Solver(Z, inst.y, inst.q, inst.C, store="f32", tol=inst.tol) as s:
        res, w, alpha = s.solve(alpha=True)
        info = s.info()
    r = res[0]
    assert r["status"] == 0 and r["kkt"] <= inst.tol, r
    assert info["slabs"] <= info["grid"] * 2
    Z64 = Z.astype(np.float64)
    up, lo, gap = O.certified_gap(Z64, inst.y, w[:, 0], r["beta"], alpha[:, 0], inst.q, inst.C)
    assert gap <= 1e-5, gap
    ref = O.solve(Z64, inst.y, inst.q, inst.C, tol=1e-8)
    _compare(r, w[:, 0], ref)
    ok, _ = _predictions_match(inst.Xtest.astype(np.float64), w[:, 0], r["beta"], ref["w"], ref["beta"])
    assert ok


def test_invalid_and_edge_cases(gdwd_lib):
    """Two samples (the smallest n), one feature, and a host-side rejection."""
    X = np.array([[1.0, -1.0]])
    y = np.array([1.0, -1.0])
    with gdwd_lib.Solver(X * y, y, 1.0, 10.0, store="f64", tol=1e-9) as s:
        res, w, _ = s.solve()
    assert res[0]["status"] == 0
    assert abs(w[0, 0] - 1.0) <= 1e-6 and abs(res[0]["beta"]) <= 1e-6
    with pytest.raises(gdwd_lib.GdwdError):
        gdwd_lib.Solver(np.ones((3, 2)), np.array([1.0, 1.0]), 1.0, 1.0)


# --------------------------------------------------------------------- low-precision storage

@pytest.mark.parametrize("fmt", ["bf16", "f16", "e4m3"])
def test_quantized_codes_bit_exact(gdwd_lib, fmt):
    """Stored codes and per-column scales equal the independent numpy rounding model."""
    from tests import quantize_ref as QR
    rng = np.random.default_rng(17)
    d, n = 1037, 45
    y = np.where(np.arange(n) < 20, 1.0, -1.0)
    X = rng.standard_t(3, size=(d, n)).astype(np.float32)
    X[:, 3] = 0.0                      # an all-zero column
    X[5, 7] = 1e-30                    # deep subnormal after scaling
    Z = (X * y).astype(np.float32)
    with gdwd_lib.Solver(Z, y, 1.0, 1.0, store=fmt) as s:
        codes, cs = s.stored()
    q_ref, s_ref = QR.quantize(Z.astype(np.float64), fmt)
    assert np.array_equal(cs, s_ref)
    got = QR.decode(codes, fmt)
    assert np.array_equal(got, q_ref), np.argwhere(got != q_ref)[:5]


@pytest.mark.parametrize("fmt,q,C", [("bf16", 1.0, 10.0), ("f16", 2.0, 5.0), ("e4m3", 1.0, 1.0)])
def test_quantized_solve_matches_oracle(gdwd_lib, fmt, q, C):
    """The quantized problem solved on the GPU equals the oracle on the dequantized data."""
    from tests import quantize_ref as QR
    inst = synth.gaussian(seed=31 + len(fmt), d=5003, n=257, shift=1.0, n_pos=100, q=q, C=C, m_test=500)
    Z = inst.Z
    with gdwd_lib.Solver(Z, inst.y, q, C, store=fmt, tol=1e-6) as s:
        res, w, alpha = s.solve(alpha=True)
    r = res[0]
    assert r["status"] == 0 and r["kkt"] <= 1e-6, r
    qv, sc = QR.quantize(Z.astype(np.float64), fmt)
    Zdq = qv * sc[None, :]
    ref = O.solve(Zdq, inst.y, q, C, tol=1e-9)
    _compare(r, w[:, 0], ref)
    up, lo, gap = O.certified_gap(Zdq, inst.y, w[:, 0], r["beta"], alpha[:, 0], q, C)
    assert gap <= 1e-5
    # the quantized optimum against the optimum of the original data (reported, loose bound)
    ref_orig = O.solve(Z.astype(np.float64), inst.y, q, C, tol=1e-9)
    rel = abs(r["primal_obj"] - ref_orig["primal"]) / abs(ref_orig["primal"])
    assert rel <= {"bf16": 1e-2, "f16": 1e-3, "e4m3": 1e-1}[fmt], rel


@pytest.mark.parametrize("fmt", ["bf16", "e4m3"])
def test_refinement_sweep_restores_original_optimum(gdwd_lib, fmt):
    """refine = 1: quantized solve, then the FP32 master warm-started from it; the
    result is the optimum of the ORIGINAL data to the solution tolerance."""
    inst = synth.gaussian(seed=41, d=6007, n=301, shift=1.0, n_pos=120, q=1.0, C=2.0, m_test=500)
    Z = inst.Z
    Cs = [0.5, 2.0]
    with gdwd_lib.Solver(Z, inst.y, 1.0, 2.0, store=fmt, tol=1e-6, refine=1) as s:
        res, w, alpha = s.solve(Cs=Cs, alpha=True)
    for k, C in enumerate(Cs):
        r = res[k]
        assert r["status"] == 0 and r["kkt"] <= 1e-6, r
        ref = O.solve(Z.astype(np.float64), inst.y, 1.0, C, tol=1e-9)
        _compare(r, w[:, k], ref)
        ok, _ = _predictions_match(inst.Xtest.astype(np.float64), w[:, k], r["beta"], ref["w"], ref["beta"])
        assert ok


def test_paper_stopping_rule(gdwd_lib):
    """stop_rule = 1 (Sec. 4.3's rule at tol 1e-5): the reported residuals meet its
    three conditions, it stops no later than the strict rule, and the point is a
    moderately accurate solution of the oracle's problem."""
    inst = synth.gaussian(seed=71, d=6000, n=300, shift=1.0, n_pos=120, q=1.0, C=1.0)
    with gdwd_lib.Solver(inst.Z, inst.y, 1.0, 1.0, store="f32", tol=1e-5, stop_rule=1, max_iter=2000) as s:
        rp, wp, _ = s.solve()
    with gdwd_lib.Solver(inst.Z, inst.y, 1.0, 1.0, store="f32", tol=1e-5) as s:
        rs, ws, _ = s.solve()
    r = rp[0]
    assert r["status"] == 0 and rs[0]["status"] == 0
    assert max(r["eta_p"], r["eta_d"]) < 1e-5
    assert min(r["eta_c"], r["eta_gap"]) < np.sqrt(1e-5)
    assert max(r["eta_c"], r["eta_gap"]) < 0.05
    assert r["iters"] <= rs[0]["iters"]
    ref = O.solve(inst.Z.astype(np.float64), inst.y, 1.0, 1.0, tol=1e-9)
    assert abs(r["primal_obj"] - ref["primal"]) / ref["primal"] <= 0.05


def test_weighted_solve_and_suggest_C(gdwd_lib):
    """Weighted DWD (Sec. 4.5: class-balancing wt and per-sample e) against the
    oracle, and the Sec. 4.1 penalty heuristic against the oracle's direct
    median of between-class distances."""
    inst = synth.gaussian(seed=81, d=3000, n=180, shift=1.0, n_pos=45, q=2.0, C=1.0, dtype=np.float64)
    Z, y = inst.Z, inst.y
    wt = gdwd_lib.imbalance_weights(y, 2.0)
    assert np.allclose(wt, O.imbalance_weights(y, 2.0), rtol=1e-14)
    e = 0.5 + 0.5 * np.random.default_rng(3).random(Z.shape[1])
    with gdwd_lib.Solver(Z, y, 2.0, 3.0, store="f64", tol=1e-8) as s:
        s.set_weights(e=e, wt=wt)
        res, w, alpha = s.solve(alpha=True)
        Cs = s.suggest_C()
    r = res[0]
    assert r["status"] == 0, r
    ref = O.solve(Z, y, 2.0, 3.0, tol=1e-10, e=e, wt=wt)
    _compare(r, w[:, 0], ref)
    assert abs(Cs - O.suggest_C(Z, y, 2.0)) / O.suggest_C(Z, y, 2.0) <= 1e-9


@pytest.mark.parametrize("store,dots_every", [("f32", 1), ("f32", 64), ("bf16", 1), ("f64", 1000)])
def test_column_dot_period(gdwd_lib, store, dots_every):
    """b = Z~^T g' carried in n-space with direct Z~^T u every dots_every iterations
    (1: every iteration; large: almost never) reaches the oracle's solution."""
    from tests import quantize_ref as QR
    inst = synth.gaussian(seed=97, d=4001, n=230, shift=1.0, n_pos=90, q=1.0, C=2.0,
                          dtype=np.float64 if store == "f64" else np.float32)
    tol = 1e-8 if store == "f64" else 1e-6
    with gdwd_lib.Solver(inst.Z, inst.y, 1.0, 2.0, store=store, tol=tol, dots_every=dots_every) as s:
        res, w, _ = s.solve()
    assert res[0]["status"] == 0, res[0]
    Zref = inst.Z.astype(np.float64)
    if store == "bf16":
        qv, sc = QR.quantize(Zref, "bf16")
        Zref = qv * sc[None, :]
    ref = O.solve(Zref, inst.y, 1.0, 2.0, tol=1e-10)
    _compare(res[0], w[:, 0], ref)


def test_large_C_on_the_ball_follows_the_oracle(gdwd_lib):
    """Heavy-tailed data with d >> n at C = 1000: w sits on the ball (theta < 1)
    and the residuals reach 1e-7, where eta_P2 and eta_D3 expanded in sums of g,
    rho and Z~ alpha cancel and the sigma rule then follows rounding.  Both GPU
    loops must follow the FP64 oracle's residuals and stop at its iteration."""
    inst = synth.heavy_tailed(seed=5011, d=20000, n=500, n_pos=125)
    Z = inst.Z.astype(np.float64)
    ref = O.solve(Z, inst.y, 1.0, 1e3, tol=1e-6, max_iter=20000)
    assert ref["converged"]
    for kern in (0, 1):
        with gdwd_lib.Solver(Z, inst.y, 1.0, 1e3, store="f64", tol=1e-6, kernelized=kern) as s:
            res, w, _ = s.solve()
        r = res[0]
        assert r["status"] == 0, (kern, r)
        assert abs(r["iters"] - ref["iters"]) <= max(3, ref["iters"] // 50), (kern, r["iters"], ref["iters"])
        assert abs(r["primal_obj"] - ref["primal"]) <= 1e-6 * (1.0 + abs(ref["primal"]))
        assert np.linalg.norm(w[:, 0] - ref["w"]) <= 1e-4 * np.linalg.norm(ref["w"])
