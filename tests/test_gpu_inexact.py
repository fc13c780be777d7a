"""The inexact solver (solver = 2; Algorithm 1 with Steps 1a-1c solved by
preconditioned CG to eq-linsys-tol, Sec. 3.3.3 with T = 0) against the FP64
oracle: the exact SMW2 solve for the solution (objective, w, held-out
predictions, certified gap) and the oracle's own inexact algorithm for the
same schedule.  No n x n matrix is formed: beyond the stored Z, the handle's
device memory stays far below the 8 n^2 bytes of one n x n FP64 matrix at the
largest case."""
import numpy as np
import pytest

from oracle import gdwd_oracle as O
from paper_2305_12019_gb300 import synth

pytestmark = pytest.mark.gpu


def _pred_match(Xt, w1, b1, w2, b2):
    s1, s2 = Xt.T @ w1 + b1, Xt.T @ w2 + b2
    tie = np.abs(s2) < 1e-6 * np.linalg.norm(Xt, axis=0)
    return np.array_equal(np.sign(s1[~tie]), np.sign(s2[~tie]))


@pytest.mark.parametrize("store,d,n,q,C,tol", [("f32", 3001, 257, 1.0, 2.0, 1e-6), ("f32", 1200, 1500, 2.0, 5.0, 1e-6),
                                               ("f64", 500, 300, 0.5, 1.0, 1e-8), ("f32", 5000, 4000, 1.0, 1.0, 1e-6)])
def test_inexact_solver_against_oracle(gdwd_lib, store, d, n, q, C, tol):
    inst = synth.gaussian(seed=d + n, d=d, n=n, shift=1.0, n_pos=n // 3, q=q, C=C, m_test=400,
                          dtype=np.float64 if store == "f64" else np.float32)
    Z = inst.Z
    with gdwd_lib.Solver(Z, inst.y, q, C, store=store, tol=tol, solver="inexact") as s:
        res, w, alpha = s.solve(alpha=True)
        info = s.info()
    r = res[0]
    assert info["solver"] == 2
    assert r["status"] == 0 and r["kkt"] <= tol, r
    assert r["cg_steps"] > 0 and 0 <= r["step1c_solves"] <= r["iters"]
    if n >= 4000:
        # beyond the stored Z (4 bytes per element, rows padded to the slab
        # height), well under one n x n FP64 matrix
        z_bytes = 4 * n * (d + 1024)
        assert info["device_bytes"] - z_bytes < 8 * n * n / 8, info["device_bytes"]
    Z64 = Z.astype(np.float64)
    ref = O.solve(Z64, inst.y, q, C, tol=1e-9)
    relobj = abs(r["primal_obj"] - ref["primal"]) / abs(ref["primal"])
    relw = np.linalg.norm(w[:, 0] - ref["w"]) / np.linalg.norm(ref["w"])
    assert relobj <= 1e-6, relobj
    assert relw <= (1e-4 if q <= 2 else 1e-3), relw
    assert _pred_match(inst.Xtest.astype(np.float64), w[:, 0], r["beta"], ref["w"], ref["beta"])
    up, lo, gap = O.certified_gap(Z64, inst.y, w[:, 0], r["beta"], alpha[:, 0], q, C)
    assert gap <= 10 * tol
    if n <= 1500:
        # the oracle's inexact algorithm (same eps_k and reuse test) reaches the same point
        ix = O.solve_inexact(Z64, inst.y, q, C, tol=tol)
        assert ix["converged"]
        assert abs(r["primal_obj"] - ix["primal"]) <= 1e-6 * abs(ix["primal"])


def test_inexact_refuses_unsupported_combinations(gdwd_lib):
    inst = synth.gaussian(seed=5, d=100, n=40, shift=1.0, q=1.0, C=1.0)
    for kw in (dict(store="bf16"), dict(kernelized=1), dict(refine=1, store="bf16")):
        with pytest.raises(gdwd_lib.GdwdError) as exc:
            gdwd_lib.Solver(inst.Z, inst.y, 1.0, 1.0, solver="inexact", **kw)
        assert exc.value.status == 8
    with gdwd_lib.Solver(inst.Z, inst.y, 1.0, 1.0, solver="inexact") as s:
        with pytest.raises(gdwd_lib.GdwdError):
            s.gram()
