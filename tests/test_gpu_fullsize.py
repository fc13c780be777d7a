"""Parity at the full sizes of the batched, served and largest workloads.

* Uneven batch (64 instances, d log-uniform 5k-50k, n 200-2000, q in {0.5, 1, 2,
  4}, classes 1:1 to 1:4, BF16 storage): eight of the 64 seeded instances spread
  over the size range, solved together through gdwd_solve_batch, each against
  the FP64 oracle on the dequantized data (objective, w, held-out predictions).
* Served stream (Poisson arrivals, d 1k-100k, n 50-5000, q in {1, 2}, C
  0.1-100, FP16 storage, data drawn on the device from each request's seed): a
  seeded sample of the stream's requests (d n <= 4e6, so the oracle finishes),
  regenerated the same way, submitted to one server together, each against the
  oracle on its dequantized data (where the oracle reaches the optimum within
  the same iteration limit).
* Largest instance (d = 200000, n = 5000, Student-t columns, classes 1:3, E4M3
  storage with the FP32 refinement sweep, 16 values of C): the weak-duality
  certificate on the ORIGINAL data for every C; and the same recipe at d = 20000,
  n = 500 solved at C = 0.01 and C = 100, against a full oracle solve of the
  original data, with identical held-out predictions.

The oracle solves (tol 1e-7) run in spawned worker processes (eight at a time,
two BLAS threads each), started before the GPU work they are compared with.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

from oracle import gdwd_oracle as O
from paper_2305_12019_gb300 import synth

pytestmark = pytest.mark.gpu

# The stop rule's gap (Sec. 4.3) is relative to 1 + |pobj| + |dobj|, so a solve
# stopped at tol = 1e-6 pins the objective to about 1e-6 on that scale, not
# relative to |pobj| (small for q = 4 or large C): compare on the same scale.
OBJ_TOL = 2e-6


def _w_tol(q):
    # at tol 1e-6 the flat objectives of large q leave w less determined (q = 4:
    # up to ~1.2e-3 on the BF16 batch instances, where objective and predictions
    # still agree to 1e-6 and exactly)
    return 1e-4 if q <= 2.0 else 2e-3


def _oracle_job(job):
    """One oracle solve in a worker: regenerate the data, apply the storage
    rounding the library applies, solve in FP64."""
    from tests import quantize_ref as QR
    kind = job["kind"]
    if kind == "gaussian":
        inst = synth.gaussian(seed=job["seed"], d=job["d"], n=job["n"], shift=job["shift"], n_pos=job["n_pos"],
                              q=job["q"], C=job["C"])
        Z = inst.Z.astype(np.float64)
        y = inst.y
    elif kind == "given":
        Z = np.asarray(job["Z"], dtype=np.float64)
        y = job["y"]
    else:
        inst = synth.heavy_tailed(seed=job["seed"], d=job["d"], n=job["n"], n_pos=job["n_pos"])
        Z = inst.Z.astype(np.float64)
        y = inst.y
    if job.get("fmt"):
        qv, sc = QR.quantize(Z, job["fmt"])
        Z = qv * sc[None, :]
    r = O.solve(Z, y, job["q"], job["C"], tol=job.get("tol", 1e-7), max_iter=job.get("max_iter", 60000))
    return {"primal": r["primal"], "w": r["w"], "beta": r["beta"], "iters": r["iters"], "converged": r["converged"],
            "kkt": r["eta"]["kkt"]}


class _Pool:
    """Spawned workers with a few BLAS threads each (set before numpy loads in them)."""

    def __init__(self, workers=8, threads=2):
        keys = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")
        old = {k: os.environ.get(k) for k in keys}
        for k in keys:
            os.environ[k] = str(threads)
        try:
            self.pool = mp.get_context("spawn").Pool(workers)
        finally:
            for k, v in old.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def submit(self, jobs):
        return self.pool.map_async(_oracle_job, jobs)

    def close(self):
        self.pool.close()
        self.pool.join()


def _predictions_match(Xt, w_gpu, b_gpu, w_ref, b_ref):
    s_gpu = Xt.T @ w_gpu + b_gpu
    s_ref = Xt.T @ w_ref + b_ref
    tie = np.abs(s_ref) < 1e-6 * np.linalg.norm(Xt, axis=0)
    return np.array_equal(np.sign(s_gpu[~tie]), np.sign(s_ref[~tie]))


def _check(res, w, ref, q, Xt=None, w_tol=None):
    assert res["status"] == 0 and res["kkt"] <= 1e-6, res
    # the reference is solved to 1e-7; where the FP64 iteration needs more than
    # its iteration limit for that (large C), it must at least be 5x tighter
    # than the GPU's stop
    assert ref["converged"] or ref["kkt"] <= 2e-7, ref["kkt"]
    relobj = abs(res["primal_obj"] - ref["primal"]) / (1.0 + abs(ref["primal"]))
    relw = np.linalg.norm(w - ref["w"]) / np.linalg.norm(ref["w"])
    assert relobj <= OBJ_TOL, relobj
    assert relw <= (_w_tol(q) if w_tol is None else w_tol), (q, relw)
    if Xt is not None:
        assert _predictions_match(Xt, w, res["beta"], ref["w"], ref["beta"])


# --------------------------------------------------------------------- uneven batch

def test_uneven_batch_instances_against_oracle(gdwd_lib):
    shapes = synth.uneven_batch(4001, count=64)
    order = sorted(range(64), key=lambda k: shapes[k]["d"] * shapes[k]["n"])
    pick = [order[i] for i in range(4, 64, 8)]          # eight instances across the size range
    jobs, reqs, keeps, tests = [], [], [], []
    for k in pick:
        sh = shapes[k]
        inst = synth.gaussian(seed=sh["seed"], d=sh["d"], n=sh["n"], shift=sh["shift"], n_pos=sh["n_pos"], q=sh["q"],
                              C=sh["C"], m_test=500)
        r, kp = gdwd_lib.make_request(inst.Z, inst.y, inst.q, inst.C, store="bf16", tol=1e-6, want_alpha=True)
        reqs.append(r)
        keeps.append(kp)
        tests.append(inst.Xtest)
        jobs.append(dict(kind="gaussian", seed=sh["seed"], d=sh["d"], n=sh["n"], shift=sh["shift"], n_pos=sh["n_pos"],
                         q=sh["q"], C=sh["C"], fmt="bf16"))
    pool = _Pool()
    try:
        pending = pool.submit(jobs)
        res, lat, st = gdwd_lib.solve_batch(reqs, slots=4)
        refs = pending.get()
    finally:
        pool.close()
    for j, k in enumerate(pick):
        _check(res[j], keeps[j]["w"], refs[j], shapes[k]["q"], tests[j])


# --------------------------------------------------------------------- served stream

def _served_specs(seed=5001, T=10.0, lam=200.0):
    """The request shapes of the served stream (as the served benchmark draws them)."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / lam, size=int(lam * T * 1.5) + 16))
    arrivals = arrivals[arrivals < T]
    specs = []
    for k in range(arrivals.size):
        d = int(round(np.exp(rng.uniform(np.log(1e3), np.log(1e5)))))
        n = int(round(np.exp(rng.uniform(np.log(50), np.log(5000)))))
        q = float(rng.choice([1.0, 2.0]))
        C = float(np.exp(rng.uniform(np.log(0.1), np.log(100))))
        specs.append((d, n, q, C, 6000 + k))
    return specs


def _served_data(d, n, seed):
    """A served request's data, drawn on the device from its seed as the stream does."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    v = torch.randn(d, device="cuda", generator=g, dtype=torch.float32)
    v /= v.norm()
    y = torch.where(torch.arange(n, device="cuda") < n // 2, 1.0, -1.0)
    X = torch.randn(n, d, device="cuda", generator=g, dtype=torch.float32) + 1.5 * y[:, None] * v[None, :]
    Zrows = (X * y[:, None]).contiguous()          # n x d: row i = column i of Z
    return Zrows.cpu().numpy().T.copy(), y.double().cpu().numpy()


def test_served_requests_against_oracle(gdwd_lib):
    specs = _served_specs()
    small = [s for s in specs if s[0] * s[1] <= 4e6]          # oracle cost bound
    rng = np.random.default_rng(77)
    sample = [small[i] for i in sorted(rng.choice(len(small), size=6, replace=False))]
    datas = [_served_data(d, n, seed) for d, n, q, C, seed in sample]
    jobs = [dict(kind="given", Z=Z, y=y, q=q, C=C, fmt="f16", max_iter=20000)
            for (Z, y), (d, n, q, C, seed) in zip(datas, sample)]
    pool = _Pool()
    try:
        pending = pool.submit(jobs)
        srv = gdwd_lib.Server(slots=4)
        tickets, keeps = [], []
        for (Z, y), (d, n, q, C, seed) in zip(datas, sample):
            r, kp = gdwd_lib.make_request(Z, y, q, C, store="f16", tol=1e-6)
            tickets.append(srv.submit(r, kp))
            keeps.append(kp)
        outs = [srv.poll(t, wait=True) for t in tickets]
        srv.close()
        refs = pending.get()
    finally:
        pool.close()
    # A request that the FP64 oracle itself cannot bring to 2e-7 within the
    # GPU's iteration limit (in this sample: n = 52 samples against d = 59349
    # features at C = 0.13, where eta_C converges very slowly) has no reference
    # to compare with; every other request must match it.
    compared = 0
    for (res, _), kp, ref, s in zip(outs, keeps, refs, sample):
        if not (ref["converged"] or ref["kkt"] <= 2e-7):
            continue
        # few samples in many dimensions at a large C leave w loosely fixed by a
        # stop at kkt 1e-6: on a request like (d = 4940, n = 59, q = 2, C = 77) the
        # FP64 oracle's own w at tol 1e-6 differs from its w at tol 1e-9 by 8.8e-4
        _check(res, kp["w"], ref, s[2], w_tol=2e-3 if s[1] < 100 else None)
        compared += 1
    assert compared >= 4, compared


# --------------------------------------------------------------------- largest instance

def test_largest_fp8_certified_on_original_data(gdwd_lib):
    """d = 200000, n = 5000: every one of the 16 C values certified on the original
    (unquantized) data by weak duality, after the FP32 refinement sweep."""
    import torch
    inst = synth.heavy_tailed(seed=5001, d=200000, n=5000, n_pos=1250)
    Cs = np.logspace(-2, 3, 16)
    Zf = inst.Z                                                   # float32, 4 GB
    Zd = torch.as_strided(torch.from_numpy(np.ascontiguousarray(Zf.T)).cuda(), Zf.shape, (1, Zf.shape[0]))
    with gdwd_lib.Solver(Zd, inst.y, 1.0, 1.0, store="e4m3", tol=1e-6, refine=1) as s:
        res, w, alpha = s.solve(Cs=Cs, alpha=True)
    del Zd
    torch.cuda.empty_cache()
    Z64 = Zf.astype(np.float64)
    del Zf
    for k, C in enumerate(Cs):
        r = res[k]
        assert r["status"] == 0 and r["kkt"] <= 1e-6, (C, r)
        up, lo, gap = O.certified_gap(Z64, inst.y, w[:, k], r["beta"], alpha[:, k], 1.0, C)
        assert lo <= up * (1 + 1e-12)
        assert gap <= 1e-6, (C, gap)
        assert abs(r["primal_obj"] - up) <= 1e-5 * abs(up), (C, r["primal_obj"], up)


def test_largest_fp8_recipe_reduced_size_against_oracle(gdwd_lib):
    """The same recipe at d = 20000, n = 500 (the full instance's d : n = 40, 1:3),
    E4M3 + refinement, at C = 0.01 (the grid's low end) and C = 100, against full
    oracle solves of the original data; held-out points (a second draw of the
    recipe) get identical predictions.  (At C = 1000 this smaller instance's
    FP32 master cannot reach kkt 1e-6: its products, rounded at 1e-7 of
    |Z~| |alpha| with alpha up to C, leave a floor near 5e-6 that FP64 storage
    does not have; the full instance's 16 values of C up to 1000 are certified
    in the test above.)"""
    d, n = 20000, 500
    inst = synth.heavy_tailed(seed=5011, d=d, n=n, n_pos=n // 4)
    Xt = synth.heavy_tailed(seed=5012, d=d, n=500, n_pos=125).X.astype(np.float64)
    Cs = [1e-2, 1e2]
    jobs = [dict(kind="heavy", seed=5011, d=d, n=n, n_pos=n // 4, q=1.0, C=C) for C in Cs]
    pool = _Pool(workers=2, threads=8)
    try:
        pending = pool.submit(jobs)
        with gdwd_lib.Solver(inst.Z, inst.y, 1.0, 1.0, store="e4m3", tol=1e-6, refine=1) as s:
            res, w, _ = s.solve(Cs=np.array(Cs))
        refs = pending.get()
    finally:
        pool.close()
    for k in range(len(Cs)):
        _check(res[k], w[:, k], refs[k], 1.0, Xt)
