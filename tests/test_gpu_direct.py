"""GPU parity of the direct solver of eq-linsys (Sec. 3.3.1, solver = "direct") with
the FP64 oracle, for d << n.

The direct solver stores Z^T with samples as rows, factors the d x d matrix
I + Z~ Z~^T / mu once and eliminates the border of the (d+1) x (d+1) system in
closed form.  The oracle runs Algorithm 1 with its own direct solve (the dense
Cholesky of A); both must reach the same optimum (|d obj|/|obj| <= 1e-6,
||dw||/||w|| <= 1e-4) and the certified gap on the data.
"""
import numpy as np
import pytest

from oracle import gdwd_oracle as O
from paper_2305_12019_gb300 import synth

pytestmark = pytest.mark.gpu

OBJ_TOL = 1e-6
W_TOL = 1e-4


def _compare(res, w, ref):
    relobj = abs(res["primal_obj"] - ref["primal"]) / abs(ref["primal"])
    relw = np.linalg.norm(w - ref["w"]) / np.linalg.norm(ref["w"])
    assert relobj <= OBJ_TOL, relobj
    assert relw <= W_TOL, relw


@pytest.mark.parametrize("q,store,d,n,n_pos,C", [
    (1.0, "f64", 30, 3001, 1000, 1.0),
    (2.0, "f32", 100, 20011, 8000, 5.0),
    (0.5, "f64", 7, 999, 500, 2.0),
    (1.0, "f32", 257, 5000, 2500, 10.0),
])
def test_direct_matches_oracle(gdwd_lib, q, store, d, n, n_pos, C):
    inst = synth.gaussian(seed=d * 7 + n, d=d, n=n, shift=0.5, n_pos=n_pos, q=q, C=C,
                          dtype=np.float32 if store == "f32" else np.float64)
    tol = 1e-8 if store == "f64" else 1e-6
    Z64 = inst.Z.astype(np.float64)
    ref = O.solve(Z64, inst.y, q, C, tol=1e-9, linsys="direct")
    with gdwd_lib.Solver(inst.Z, inst.y, q, C, store=store, tol=tol, solver="direct") as s:
        info = s.info()
        res, w, alpha = s.solve(alpha=True)
    assert info["solver"] == 1
    r = res[0]
    assert r["status"] == 0 and r["kkt"] <= tol, r
    _compare(r, w[:, 0], ref)
    up, lo, gap = O.certified_gap(Z64, inst.y, w[:, 0], r["beta"], alpha[:, 0], q, C)
    assert gap <= 10 * tol


def test_direct_equals_smw_path(gdwd_lib):
    """On a problem both can take (d = 300, n = 1500) the two solvers of eq-linsys
    reach the same solution."""
    inst = synth.gaussian(seed=3, d=300, n=1500, shift=1.0, n_pos=600, q=1.0, C=2.0, dtype=np.float64)
    out = []
    for sv in ("smw", "direct"):
        with gdwd_lib.Solver(inst.Z, inst.y, 1.0, 2.0, store="f64", tol=1e-8, solver=sv) as s:
            res, w, _ = s.solve()
        assert res[0]["status"] == 0, (sv, res[0])
        out.append((res[0], w[:, 0]))
    (a, wa), (b, wb) = out
    assert abs(a["primal_obj"] - b["primal_obj"]) / abs(a["primal_obj"]) <= 1e-7
    assert np.linalg.norm(wa - wb) / np.linalg.norm(wa) <= 1e-5


def test_direct_weights_cgrid_and_limits(gdwd_lib):
    """Weighted DWD and several C on one direct-solver handle; the options and
    entry points it does not take are refused."""
    inst = synth.gaussian(seed=9, d=40, n=4000, shift=0.5, n_pos=1000, q=1.0, C=1.0, dtype=np.float64)
    Z, y = inst.Z, inst.y
    wt = gdwd_lib.imbalance_weights(y, 1.0)
    Cs = [0.3, 3.0]
    with gdwd_lib.Solver(Z, y, 1.0, 1.0, store="f64", tol=1e-8, solver="direct") as s:
        s.set_weights(wt=wt)
        res, w, _ = s.solve(Cs=Cs)
        G = s.gram()
        with pytest.raises(gdwd_lib.GdwdError, match="EUNSUPPORTED"):
            s.suggest_C()
    for k, C in enumerate(Cs):
        assert res[k]["status"] == 0, res[k]
        _compare(res[k], w[:, k], O.solve(Z, y, 1.0, C, tol=1e-10, wt=wt, linsys="direct"))
    Zt, _ = O.scale_data(Z)
    assert np.abs(G - (np.eye(40) + Zt @ Zt.T)).max() <= 1e-12 * np.abs(G).max()
    for kw in ({"refine": 1}, {"kernelized": 1}, {"store": "bf16"}):
        with pytest.raises(gdwd_lib.GdwdError, match="EUNSUPPORTED"):
            gdwd_lib.Solver(Z, y, 1.0, 1.0, **dict({"store": "f64", "solver": "direct"}, **kw))


def test_direct_edge_cases(gdwd_lib):
    """n = 2, d = 1."""
    X = np.array([[1.0, -1.0]])
    y = np.array([1.0, -1.0])
    with gdwd_lib.Solver(X * y, y, 1.0, 10.0, store="f64", tol=1e-9, solver="direct") as s:
        res, w, _ = s.solve()
    assert res[0]["status"] == 0, res[0]
    assert abs(w[0, 0] - 1.0) <= 1e-6 and abs(res[0]["beta"]) <= 1e-6
