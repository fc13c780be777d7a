"""GPU tests of the joint C-grid kernel: several values of C iterated in
lock-step by one persistent launch (each pass over Z serves all of them).

Each instance must match the FP64 oracle for its own C, and the joint result
must equal the sequential one (one C per launch) within the solution tolerance.
"""
import numpy as np
import pytest

from oracle import gdwd_oracle as O
from paper_2305_12019_gb300 import synth

pytestmark = pytest.mark.gpu


def _cmp(res, w, ref, obj_tol=1e-6, w_tol=1e-4):
    relobj = abs(res["primal_obj"] - ref["primal"]) / abs(ref["primal"])
    relw = np.linalg.norm(w - ref["w"]) / np.linalg.norm(ref["w"])
    assert relobj <= obj_tol and relw <= w_tol, (relobj, relw)


@pytest.mark.parametrize("store,d,n,q,Cs", [
    ("f64", 3000, 150, 1.0, [0.1, 1.0, 10.0]),            # K = 3 (one frozen slot)
    ("f32", 6007, 301, 1.0, [0.05, 0.5, 5.0, 50.0]),      # K = 4
    ("f32", 2511, 97, 2.0, [0.3, 3.0]),                    # K = 2
])
def test_joint_cgrid_matches_oracle(gdwd_lib, store, d, n, q, Cs):
    inst = synth.gaussian(seed=d + n, d=d, n=n, shift=1.0, n_pos=n // 3, q=q, C=1.0,
                          dtype=np.float64 if store == "f64" else np.float32)
    Z = inst.Z
    # FP32 products put a noise floor of ~1e-7 under the residuals of FP32 / BF16
    # storage, so those solve to the workload tolerance 1e-6
    tol = 1e-8 if store == "f64" else 1e-6
    with gdwd_lib.Solver(Z, inst.y, q, 1.0, store=store, tol=tol) as s:
        res, w, alpha = s.solve(Cs=Cs, alpha=True)
    for k, C in enumerate(Cs):
        r = res[k]
        assert r["status"] == 0 and r["kkt"] <= tol, (k, r)
        ref = O.solve(Z.astype(np.float64), inst.y, q, C, tol=1e-9, max_iter=200000)
        _cmp(r, w[:, k], ref)
        up, lo, gap = O.certified_gap(Z.astype(np.float64), inst.y, w[:, k], r["beta"], alpha[:, k], q, C)
        assert gap <= 1e-6


def test_joint_equals_sequential_bf16_six_c(gdwd_lib):
    """Six C values in BF16 storage: a group of four and a group of two, against
    the one-C-per-launch path on the same stored (quantized) problem."""
    inst = synth.gaussian(seed=77, d=5003, n=257, shift=1.0, n_pos=100, q=1.0, C=1.0)
    Cs = list(np.logspace(-1, 2, 6))
    with gdwd_lib.Solver(inst.Z, inst.y, 1.0, 1.0, store="bf16", tol=1e-6) as s:
        rj, wj, _ = s.solve(Cs=Cs)
    with gdwd_lib.Solver(inst.Z, inst.y, 1.0, 1.0, store="bf16", tol=1e-6, cgrid_sequential=1) as s:
        rs, ws, _ = s.solve(Cs=Cs)
    for k in range(len(Cs)):
        assert rj[k]["status"] == 0 and rs[k]["status"] == 0
        relobj = abs(rj[k]["primal_obj"] - rs[k]["primal_obj"]) / abs(rs[k]["primal_obj"])
        relw = np.linalg.norm(wj[:, k] - ws[:, k]) / np.linalg.norm(ws[:, k])
        assert relobj <= 1e-6 and relw <= 1e-4, (k, relobj, relw)


def test_cgrid_full_size_certificates(gdwd_lib):
    """The C-grid workload at its full size (d = 50000, n = 2000, BF16 storage, the
    joint kernel), on four of its 32 values of C: every solve reaches kkt <= 1e-6
    on the stored problem, and the weak-duality certificate on the ORIGINAL data
    (an FP64 host computation that holds at any size) stays at the level the BF16
    quantization allows."""
    inst = synth.gaussian(seed=3001, d=50000, n=2000, shift=1.5, q=1.0, C=1.0)
    Cs = list(np.logspace(-2, 3, 32)[[4, 12, 20, 28]])
    with gdwd_lib.Solver(inst.Z, inst.y, 1.0, 1.0, store="bf16", tol=1e-6) as s:
        res, w, alpha = s.solve(Cs=Cs, alpha=True)
    Z64 = inst.Z.astype(np.float64)
    for k, C in enumerate(Cs):
        r = res[k]
        assert r["status"] == 0 and r["kkt"] <= 1e-6, (k, r)
        up, lo, gap = O.certified_gap(Z64, inst.y, w[:, k], r["beta"], alpha[:, k], 1.0, C)
        assert gap <= 1e-5, (k, gap)
