"""Failure statuses of the library, produced without any GPU fault.

* GDWD_EMAXITER: the iteration limit stops a solve; the last iterate and its
  residuals are still returned and finite.
* GDWD_ETIMEOUT: a bounded device wait runs out.  The test makes the first grid
  barrier of the iteration kernel wait for an arrival that no CTA supplies
  (GDWD_INJECT_STALL), with a short timeout_s; every CTA gives up, waits for its
  own bulk copies still in flight and returns.  The same process then solves
  normally, on the same handle and on a new one, and the results match the FP64
  oracle.
* GDWD_ENOMEM: an allocation of gdwd_create fails (GDWD_INJECT_ALLOC_FAIL, a
  host-side injection into the library's allocation wrapper); no handle is
  returned and the next create succeeds.
"""
import time

import numpy as np
import pytest

from oracle import gdwd_oracle as O

pytestmark = pytest.mark.gpu

ETIMEOUT, ENOMEM, EMAXITER = 6, 2, 4


def _problem(seed=3, d=3000, n=257):
    rng = np.random.default_rng(seed)
    y = np.where(np.arange(n) % 3 == 0, 1.0, -1.0)
    X = rng.standard_normal((d, n)) + 0.8 * y[None, :] * np.eye(d, 1)
    return (X * y).astype(np.float32), y


def _check_solution(res, w, Z, y, q, C):
    ref = O.solve(Z.astype(np.float64), y, q, C, tol=1e-9)
    relobj = abs(res["primal_obj"] - ref["primal"]) / abs(ref["primal"])
    relw = np.linalg.norm(w - ref["w"]) / np.linalg.norm(ref["w"])
    assert res["status"] == 0 and res["kkt"] <= 1e-6
    assert relobj <= 1e-6 and relw <= 1e-4, (relobj, relw)


def test_max_iter_returns_last_iterate(gdwd_lib):
    Z, y = _problem()
    with gdwd_lib.Solver(Z, y, 1.0, 2.0, store="f32", max_iter=3) as s:
        res, w, alpha = s.solve(alpha=True)
    r = res[0]
    assert r["status"] == EMAXITER and r["iters"] == 3
    assert np.all(np.isfinite(w)) and np.all(np.isfinite(alpha)) and np.linalg.norm(w) > 0
    for k in ("kkt", "eta_p", "eta_d", "eta_c", "eta_gap", "primal_obj", "dual_obj"):
        assert np.isfinite(r[k]) and r[k] != 0.0, k
    assert r["kkt"] > 1e-6


def test_bounded_wait_times_out_then_solves(gdwd_lib, monkeypatch):
    Z, y = _problem()
    q, C = 1.0, 2.0
    s = gdwd_lib.Solver(Z, y, q, C, store="f32", timeout_s=0.25)
    try:
        monkeypatch.setenv("GDWD_INJECT_STALL", "1")
        t0 = time.perf_counter()
        with pytest.raises(gdwd_lib.GdwdError) as exc:
            s.solve()
        waited = time.perf_counter() - t0
        assert exc.value.status == ETIMEOUT
        assert 0.2 <= waited < 30.0
        monkeypatch.delenv("GDWD_INJECT_STALL")
        # the context is intact: the same handle solves normally afterwards
        res, w, _ = s.solve()
        _check_solution(res[0], w[:, 0], Z, y, q, C)
    finally:
        s.close()
    with gdwd_lib.Solver(Z, y, q, C, store="f32") as s2:
        res, w, _ = s2.solve()
    _check_solution(res[0], w[:, 0], Z, y, q, C)


@pytest.mark.parametrize("k", [1, 5, 12])
def test_injected_allocation_failure(gdwd_lib, monkeypatch, k):
    Z, y = _problem(d=500, n=64)
    monkeypatch.setenv("GDWD_INJECT_ALLOC_FAIL", str(k))
    with pytest.raises(gdwd_lib.GdwdError) as exc:
        gdwd_lib.Solver(Z, y, 1.0, 1.0, store="f32")
    assert exc.value.status == ENOMEM
    monkeypatch.delenv("GDWD_INJECT_ALLOC_FAIL")
    with gdwd_lib.Solver(Z, y, 1.0, 1.0, store="f32") as s:
        res, w, _ = s.solve()
    assert res[0]["status"] == 0


@pytest.mark.parametrize("store,solver", [("f32", "smw"), ("f64", "smw"), ("bf16", "smw"), ("f32", "direct"),
                                          ("f32", "inexact")])
def test_non_finite_data_refused(gdwd_lib, store, solver):
    """A NaN or Inf in Z is refused with GDWD_EINVAL and no handle, after the
    set-up kernels have run on it (the finiteness flag is read at the single
    synchronisation of gdwd_create); the next create on clean data succeeds."""
    Z, y = _problem(seed=11, d=600, n=120)
    if solver == "direct":
        Z, y = _problem(seed=11, d=40, n=900)
    for bad in (np.nan, np.inf):
        Zb = Z.copy()
        Zb[Z.shape[0] // 2, Z.shape[1] - 1] = bad
        with pytest.raises(gdwd_lib.GdwdError) as exc:
            gdwd_lib.Solver(Zb, y, 1.0, 1.0, store=store, solver=solver)
        assert exc.value.status == 1 and "non-finite" in str(exc.value)
    with gdwd_lib.Solver(Z, y, 1.0, 1.0, store=store, solver=solver) as s:
        res, w, _ = s.solve()
    assert res[0]["status"] == 0
