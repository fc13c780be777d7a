"""Measurements of the other workloads (run through ``bench.py --workload NAME``).

Each prints one JSON line with its own metric.  All inputs are seeded synthetic
stand-ins for the paper's data sets (see paper_2305_12019_gb300/synth.py).

  plain_fp64    d=500, n=100, FP64, tol 1e-9: solves/s (latency-bound, L2-resident)
  cgrid_bf16    d=50000, n=2000, 32 values of C (logspace(-2, 3)), BF16 storage,
                joint C-grid launches: C-solves/s, against the plain FP32
                one-C-at-a-time path on the same data
  uneven_batch  64 instances, d log-uniform 5k-50k, n 200-2000, q in {0.5,1,2,4},
                classes 1:1-1:4, BF16 storage, gdwd_solve_batch: instances/s
  served        Poisson arrivals (200/s for 10 s by default) of FP16 problems with
                d log-uniform 1k-100k, n 50-5000, q in {1,2}, C 0.1-100, generated
                on the device per request seed: p50 / p99 latency and solves/s
                (uneven_batch, served, largest_fp8: --kern 1 runs the kernelized iteration)
  direct_fp32   d=200, n=1e6 FP32 through the direct solver of eq-linsys (d << n):
                solves/s, iterations, streaming-pass bandwidth
  largest_fp8   d=200000, n=5000, Student-t columns, 1:3, 16 values of C, E4M3
                storage with the FP32 refinement sweep: C-solves/s
  kernelized    the kernelized n-space iteration (no pass over Z per iteration)
                against the Z-streaming one: the spiked FP32 bench instance
                (d=20000, n=1000), a wide spiked FP32 instance (d=200000,
                n=1000, Z 800 MB > L2) and the cgrid_bf16 grid (32 C, one at a
                time): solves/s of both, per-iteration time, iterations
"""
from __future__ import annotations

import json
import os
import time

import numpy as np

from oracle import gdwd_oracle as O


def _torch():
    import torch
    return torch


def _hbm_peak():
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _roofline(kernel, bytes_per_iter, iters, solve_ms, formula):
    peak, kind = _hbm_peak()
    achieved = bytes_per_iter * iters / (solve_ms * 1e-3) / 1e9
    return {"kernel": kernel, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": kind, "bytes_per_iteration": bytes_per_iter,
            "bytes_formula": formula}


def _device_colmajor(Z):
    torch = _torch()
    d, n = Z.shape
    t = torch.from_numpy(np.ascontiguousarray(Z.T)).cuda()
    return torch.as_strided(t, (d, n), (1, d))


def plain_fp64(args, gdwd, synth):
    torch = _torch()
    inst = synth.plain_fp64()
    Zd = _device_colmajor(inst.Z)
    for _ in range(args.warmup):
        with gdwd.Solver(Zd, inst.y, 1.0, 1.0, store="f64", tol=1e-9, sigma0=1.0) as s:
            s.solve()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        with gdwd.Solver(Zd, inst.y, 1.0, 1.0, store="f64", tol=1e-9, sigma0=1.0) as s:
            res, w, _ = s.solve()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / args.steps
    ref = O.solve(inst.Z, inst.y, 1.0, 1.0, sigma0=1.0, tol=1e-10)
    return {"metric": "gDWD solves/s at KKT<=1e-9", "value": 1.0 / dt, "unit": "solves/s", "ms_per_step": dt * 1e3,
            "config": {"workload": "plain_fp64 d=500 n=100 q=1 C=1 sigma0=1 tol=1e-9", "store": "f64"},
            "iters": res[0]["iters"], "kkt": res[0]["kkt"],
            "err_vs_oracle": {"rel_obj": abs(res[0]["primal_obj"] - ref["primal"]) / ref["primal"],
                              "rel_w": float(np.linalg.norm(w[:, 0] - ref["w"]) / np.linalg.norm(ref["w"]))}}


def cgrid_bf16(args, gdwd, synth):
    torch = _torch()
    d, n = args.cg_d, args.cg_n
    inst = synth.gaussian(seed=3001, d=d, n=n, shift=1.5, q=1.0, C=1.0)
    Cs = np.logspace(-2, 3, 32)
    Zd = _device_colmajor(inst.Z)
    with gdwd.Solver(Zd, inst.y, 1.0, 1.0, store="bf16", tol=1e-6) as s:   # warm-up
        s.solve(Cs=Cs[:4])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with gdwd.Solver(Zd, inst.y, 1.0, 1.0, store="bf16", tol=1e-6) as s:
        res, w, alpha = s.solve(Cs=Cs, alpha=True)
        info = s.info()
    torch.cuda.synchronize()
    t_joint = time.perf_counter() - t0
    # plain FP32 path, one C per launch, on the first four values of C (per-solve time)
    t0 = time.perf_counter()
    with gdwd.Solver(Zd, inst.y, 1.0, 1.0, store="f32", tol=1e-6, cgrid_sequential=1) as s:
        rf, wf, _ = s.solve(Cs=Cs[:4])
    torch.cuda.synchronize()
    t_f32_per = (time.perf_counter() - t0) / 4
    Z64 = inst.Z.astype(np.float64)
    gaps = [O.certified_gap(Z64, inst.y, w[:, k], res[k]["beta"], alpha[:, k], 1.0, Cs[k])[2] for k in range(0, 32, 4)]
    return {"metric": "gDWD C-solves/s at KKT<=1e-6 (quantized problem)", "value": 32 / t_joint, "unit": "solves/s",
            "ms_per_step": t_joint * 1e3,
            "config": {"workload": f"cgrid_bf16 d={d} n={n} 32 C logspace(-2,3) q=1", "store": "bf16"},
            "vs_fp32_single": (32 / t_joint) / (1.0 / t_f32_per), "fp32_single_solves_per_s": 1.0 / t_f32_per,
            "setup_ms": info["t_setup_ms"], "gram_tensor_cores": info["gram_tensor_cores"],
            "iters": [r["iters"] for r in res], "kkt": [r["kkt"] for r in res],
            "all_converged": all(r["status"] == 0 for r in res),
            "certified_gap_original_data_every_4th_C": gaps}


def uneven_batch(args, gdwd, synth):
    shapes = synth.uneven_batch(4001, count=args.batch_count)
    reqs, keeps, insts = [], [], []
    for sh in shapes:
        inst = synth.gaussian(seed=sh["seed"], d=sh["d"], n=sh["n"], shift=1.5, n_pos=sh["n_pos"], q=sh["q"],
                              C=sh["C"])
        r, k = gdwd.make_request(inst.Z, inst.y, inst.q, inst.C, store="bf16", tol=1e-6, want_alpha=True,
                                 kernelized=args.kern)
        reqs.append(r)
        keeps.append(k)
        insts.append(inst)
    t0 = time.perf_counter()
    res, lat, st = gdwd.solve_batch(reqs, slots=args.slots)
    dt = time.perf_counter() - t0
    # certificate on the original data for a sample of instances
    gaps = []
    for k in range(0, len(insts), 8):
        inst = insts[k]
        gaps.append(O.certified_gap(inst.Z.astype(np.float64), inst.y, keeps[k]["w"], res[k]["beta"],
                                    keeps[k]["alpha"], inst.q, inst.C)[2])
    return {"metric": "gDWD instances/s (uneven batch)", "value": len(reqs) / dt, "unit": "solves/s",
            "ms_per_step": dt * 1e3,
            "config": {"workload": f"uneven_batch {len(reqs)} instances d 5k-50k n 200-2000 q in 0.5,1,2,4",
                       "store": "bf16", "slots": args.slots,
                       "iteration": {1: "kernelized", 0: "Z-streaming", -1: "chosen per problem by bytes per iteration"}[args.kern]},
            "status": int(st), "converged": int(sum(r["status"] == 0 for r in res)),
            "not_converged": [{"k": k, "d": shapes[k]["d"], "n": shapes[k]["n"], "q": shapes[k]["q"], "iters": r["iters"],
                               "kkt": r["kkt"], "status": r["status"]} for k, r in enumerate(res) if r["status"] != 0],
            "latency_ms_p50": float(np.percentile(lat, 50)), "latency_ms_p99": float(np.percentile(lat, 99)),
            "certified_gap_original_data_every_8th": gaps}


def served(args, gdwd, synth):
    """Poisson arrivals; each request's data is drawn on the device from its seed
    when the client hands it to the server.  Requests still waiting after
    --serve-wall seconds are not served (counted in the line).  The client keeps at most
    2 x slots requests generated-but-unfinished (the rest wait as seeds), so
    device memory holds only what is in flight; latency runs from the arrival
    time to the moment the client sees the result."""
    torch = _torch()
    rng = np.random.default_rng(5001)
    T, lam = args.serve_seconds, args.serve_rate
    arrivals = np.cumsum(rng.exponential(1.0 / lam, size=int(lam * T * 1.5) + 16))
    arrivals = arrivals[arrivals < T]
    specs = []
    for k in range(arrivals.size):
        d = int(round(np.exp(rng.uniform(np.log(1e3), np.log(1e5)))))
        n = int(round(np.exp(rng.uniform(np.log(50), np.log(5000)))))
        q = float(rng.choice([1.0, 2.0]))
        C = float(np.exp(rng.uniform(np.log(0.1), np.log(100))))
        specs.append((d, n, q, C, 6000 + k))
    gen_stream = torch.cuda.Stream()
    srv = gdwd.Server(slots=args.slots)
    max_out = 2 * args.slots
    pending = {}          # ticket -> (request index, data kept alive until it completes)
    lat_e2e, lat_srv, stats, iters = [], [], [], []
    dn_done = 0.0
    t_start = time.perf_counter()
    nxt = 0
    wall_limit = args.serve_wall
    while (nxt < len(specs) and time.perf_counter() - t_start < wall_limit) or pending:
        for t in list(pending):
            out = srv.poll(t, wait=False)
            if out is not None:
                k, _ = pending.pop(t)
                res, lsrv = out
                lat_e2e.append((time.perf_counter() - t_start - arrivals[k]) * 1e3)
                lat_srv.append(lsrv)
                stats.append(res["status"])
                iters.append(res["iters"])
                dn_done += specs[k][0] * specs[k][1]
        now = time.perf_counter() - t_start
        if nxt < len(specs) and now < wall_limit and len(pending) < max_out and arrivals[nxt] <= now:
            d, n, q, C, seed = specs[nxt]
            with torch.cuda.stream(gen_stream):
                g = torch.Generator(device="cuda")
                g.manual_seed(seed)
                v = torch.randn(d, device="cuda", generator=g, dtype=torch.float32)
                v /= v.norm()
                y = torch.where(torch.arange(n, device="cuda") < n // 2, 1.0, -1.0)
                X = torch.randn(n, d, device="cuda", generator=g, dtype=torch.float32) + 1.5 * y[:, None] * v[None, :]
                Zrows = X * y[:, None]                     # n x d: row i = column i of Z
                del X
            gen_stream.synchronize()
            yh = y.double().cpu().numpy()
            o = gdwd.default_options()
            o.tol, o.store, o.kernelized = 1e-6, gdwd.F16, args.kern
            w = np.zeros(d)
            r = gdwd.Request(Z=Zrows.data_ptr(), zdt=gdwd.F32, z_on_device=1, d=d, n=n, ldz=d,
                             y=yh.ctypes.data, q=q, C=C, opts=o, w=w.ctypes.data, alpha=None)
            t = srv.submit(r, (Zrows, yh, w))
            pending[t] = (nxt, (Zrows, yh, w))
            nxt += 1
            continue
        time.sleep(0.0005)
    t_total = time.perf_counter() - t_start
    srv.close()
    ok = sum(1 for st in stats if st == 0)
    return {"metric": "served gDWD requests: p50/p99 latency, solves/s", "value": len(stats) / t_total,
            "unit": "solves/s", "latency_ms_p50": float(np.percentile(lat_e2e, 50)),
            "latency_ms_p99": float(np.percentile(lat_e2e, 99)),
            "server_latency_ms_p50": float(np.percentile(lat_srv, 50)),
            "server_latency_ms_p99": float(np.percentile(lat_srv, 99)),
            "requests": len(stats), "arrived": int(arrivals.size), "not_served_by_wall_limit": int(arrivals.size - nxt),
            "converged": ok, "wall_s": t_total, "wall_limit_s": wall_limit,
            "offered_rate": lam, "mean_iters": float(np.mean(iters)),
            "z_bytes_per_iteration_mean_fp16": 2.0 * dn_done / max(1, len(stats)),
            "config": {"workload": f"served Poisson {lam}/s for {T} s, d 1k-100k, n 50-5000, q in 1,2, C 0.1-100",
                       "store": "f16", "slots": args.slots, "client_in_flight_max": max_out,
                       "iteration": {1: "kernelized", 0: "Z-streaming", -1: "chosen per problem by bytes per iteration"}[args.kern]}}


def largest_fp8(args, gdwd, synth):
    torch = _torch()
    d, n = args.big_d, args.big_n
    inst = synth.heavy_tailed(seed=5001, d=d, n=n, n_pos=n // 4, q=1.0, C=1.0)
    Cs = np.logspace(-2, 3, 16)
    Zd = _device_colmajor(inst.Z)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with gdwd.Solver(Zd, inst.y, 1.0, 1.0, store="e4m3", tol=1e-6, refine=1, kernelized=args.kern) as s:
        res, w, alpha = s.solve(Cs=Cs, alpha=True)
        info = s.info()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    Z64 = inst.Z.astype(np.float64)
    gaps = [O.certified_gap(Z64, inst.y, w[:, k], res[k]["beta"], alpha[:, k], 1.0, Cs[k])[2] for k in (0, 15)]
    return {"metric": "gDWD C-solves/s at KKT<=1e-6 on the original data (FP8 + FP32 refinement)",
            "value": 16 / dt, "unit": "solves/s", "ms_per_step": dt * 1e3,
            "config": {"workload": f"largest_fp8 d={d} n={n} Student-t 1:3 16 C", "store": "e4m3+refine",
                       "iteration": {1: "kernelized", 0: "Z-streaming", -1: "chosen per problem by bytes per iteration"}[args.kern]},
            "setup_ms": info["t_setup_ms"], "gram_tensor_cores": info["gram_tensor_cores"],
            "iters": [r["iters"] for r in res],
            "converged": int(sum(r["status"] == 0 for r in res)), "certified_gap_C_ends": gaps}


def hbm_stream(gdwd, synth, C=1.0, reps=2):
    """The Z-streaming iteration where Z does stream from HBM: the C-grid instance
    (d=50000, n=2000, Gaussian two-class with mean shift 1.5, BF16 storage: 200 MB,
    above the 129 MB L2), one value of C per solve.  Returns the iteration kernel's
    algorithmic bytes per iteration over its CUDA-event time against the measured
    HBM copy bandwidth, with the per-phase split of the last solve."""
    torch = _torch()
    d, n = 50000, 2000
    inst = synth.gaussian(seed=3001, d=d, n=n, shift=1.5, q=1.0, C=C)
    Zd = _device_colmajor(inst.Z)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    with gdwd.Solver(Zd, inst.y, 1.0, C, store="bf16", tol=1e-6) as s:
        s.solve()                                             # warm-up
        runs = []
        for k in range(reps):
            flush.fill_(float(k))
            torch.cuda.synchronize()
            res, _, _ = s.solve()
            runs.append(res[0])
        info = s.info()
        ph = s.phase_times()
    iters = float(np.mean([r["iters"] for r in runs]))
    t_ms = float(np.mean([r["t_solve_ms"] for r in runs]))
    slabs = info["slabs"]
    bpi = d * n * 2 + 16 * n * n + 64 * d + 160 * n + 8 * n * slabs / 4
    roof = _roofline("iterate_kernel<__nv_bfloat16>", bpi, iters, t_ms,
                     "d*n*2 + 16n^2 + 64d + 160n + 8n*slabs/4 (Z once, G^-1 twice, vectors, column dots every 4th)")
    del Zd
    torch.cuda.empty_cache()
    return {"workload": f"cgrid_bf16 instance d={d} n={n} mu-shift 1.5, C={C}, BF16 Z 200 MB (> L2)",
            "iterations": iters, "solve_ms": t_ms, "us_per_iteration": 1e3 * t_ms / iters,
            "status": [r["status"] for r in runs], "kkt": [r["kkt"] for r in runs], "grid": info["grid"],
            "roofline": roof, "phase_us_per_iter": {k: v / 1e3 / runs[-1]["iters"] for k, v in ph.items() if v > 0}}


def _timed_steps(gdwd, Zd, inst, steps, **kw):
    """Full create + solve + free steps (one warm-up): mean seconds, last result."""
    torch = _torch()
    out = None
    times = []
    for k in range(steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with gdwd.Solver(Zd, inst.y, inst.q, inst.C, tol=inst.tol, **kw) as s:
            res, w, _ = s.solve()
            info = s.info()
            ph = s.phase_times()
        torch.cuda.synchronize()
        if k:
            times.append(time.perf_counter() - t0)
        out = (res[0], w[:, 0], info, ph)
    return float(np.mean(times)), out


def kernelized(args, gdwd, synth):
    torch = _torch()
    line = {"metric": "gDWD solves/s at KKT<=1e-6, kernelized n-space iteration", "unit": "solves/s"}
    cases = {}
    for name, d in (("spiked_fp32_d20000_n1000", 20000), ("spiked_fp32_d200000_n1000", args.kern_wide_d)):
        inst = synth.spiked_fp32(d=d, m_test=0)
        Zd = _device_colmajor(inst.Z)
        row = {}
        for label, k in (("streaming", 0), ("kernelized", 1)):
            t, (r, w, info, ph) = _timed_steps(gdwd, Zd, inst, args.kern_steps, store="f32", kernelized=k)
            row[label] = {"solves_per_s": 1.0 / t, "step_ms": t * 1e3, "iters": r["iters"], "kkt": r["kkt"],
                          "status": r["status"], "solve_ms": r["t_solve_ms"], "setup_ms": info["t_setup_ms"],
                          "us_per_iter": 1e3 * r["t_solve_ms"] / max(1, r["iters"]),
                          "phase_us_per_iter": {kk: v / 1e3 / max(1, r["iters"]) for kk, v in ph.items() if v}}
            row[label + "_w"] = w
        row["rel_w_kernelized_vs_streaming"] = float(np.linalg.norm(row["kernelized_w"] - row["streaming_w"]) /
                                                     np.linalg.norm(row["streaming_w"]))
        del row["kernelized_w"], row["streaming_w"]
        row["speedup"] = row["kernelized"]["solves_per_s"] / row["streaming"]["solves_per_s"]
        cases[name] = row
        del Zd
        torch.cuda.empty_cache()
    # the C grid of cgrid_bf16, one C after the other on the kernelized iteration
    inst = synth.gaussian(seed=3001, d=args.cg_d, n=args.cg_n, shift=1.5, q=1.0, C=1.0)
    Cs = np.logspace(-2, 3, 32)
    Zd = _device_colmajor(inst.Z)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with gdwd.Solver(Zd, inst.y, 1.0, 1.0, store="bf16", tol=1e-6, kernelized=1) as s:
        res, w, alpha = s.solve(Cs=Cs, alpha=True)
    torch.cuda.synchronize()
    t_grid = time.perf_counter() - t0
    Z64 = inst.Z.astype(np.float64)
    gaps = [O.certified_gap(Z64, inst.y, w[:, k], res[k]["beta"], alpha[:, k], 1.0, Cs[k])[2] for k in range(0, 32, 8)]
    cases[f"cgrid_bf16_d{args.cg_d}_n{args.cg_n}_32C"] = {
        "C_solves_per_s": 32 / t_grid, "ms": t_grid * 1e3, "iters": [r["iters"] for r in res],
        "converged": int(sum(r["status"] == 0 for r in res)), "certified_gap_original_data_every_8th_C": gaps}
    head = cases["spiked_fp32_d20000_n1000"]["kernelized"]
    n0 = 1000
    kb = 24.0 * n0 * (n0 + 1) + 200.0 * n0      # G^-1 twice and K once (double-float rows), n-vectors
    line["roofline"] = _roofline("iterate_kern_kernel", kb, head["iters"], head["solve_ms"],
                                 "24 n (n+1) + 200 n bytes per iteration (two G^-1 GEMVs, one K GEMV)")
    line.update({"value": head["solves_per_s"], "ms_per_step": head["step_ms"],
                 "config": {"workload": "kernelized iteration: spiked_fp32 d=20000 n=1000 q=1 C=10 tol=1e-6 "
                                        "(value); wide d=200000 and the BF16 C grid alongside", "store": "f32"},
                 "cases": cases})
    return line


def direct_fp32(args, gdwd, synth):
    """d << n through the direct solver of eq-linsys: the n x n Gram of the SMW
    path would not fit (n = 1e6 -> 8 TB), the d x d one is 320 KB."""
    torch = _torch()
    d, n = args.dir_d, args.dir_n
    inst = synth.gaussian(seed=7001, d=d, n=n, shift=0.3, n_pos=n // 2, q=1.0, C=1.0)
    Zd = _device_colmajor(inst.Z)
    times, out = [], None
    for k in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with gdwd.Solver(Zd, inst.y, 1.0, 1.0, store="f32", tol=1e-6, solver="direct") as s:
            res, w, alpha = s.solve(alpha=True)
            info = s.info()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        out = (res[0], w[:, 0], alpha[:, 0], info)
    r, w, al, info = out
    gap = O.certified_gap(inst.Z.astype(np.float64), inst.y, w, r["beta"], al, 1.0, 1.0)[2]
    zbytes = 4.0 * d * n
    return {"metric": "gDWD solves/s at KKT<=1e-6, direct solver (d << n)", "value": 1.0 / times[-1],
            "unit": "solves/s", "ms_per_step": times[-1] * 1e3,
            "config": {"workload": f"direct_fp32 d={d} n={n} q=1 C=1 tol=1e-6", "store": "f32", "solver": "direct"},
            "iters": r["iters"], "kkt": r["kkt"], "status": r["status"], "setup_ms": info["t_setup_ms"],
            "solve_ms": r["t_solve_ms"], "us_per_iter": 1e3 * r["t_solve_ms"] / max(1, r["iters"]),
            "z_reads_per_iter": 4, "z_gbs": 4 * zbytes * r["iters"] / (r["t_solve_ms"] * 1e-3) / 1e9,
            "roofline": _roofline("direct iteration (four reads of Z^T)", 4 * zbytes + 24.0 * d * d + 64.0 * n,
                                  r["iters"], r["t_solve_ms"],
                                  "4 d n 4 (five products with Z^T, the last two in one read) + 24 d^2 + 64 n "
                                  "bytes per iteration"),
            "certified_gap": gap}


WORKLOADS = {"plain_fp64": plain_fp64, "cgrid_bf16": cgrid_bf16, "uneven_batch": uneven_batch, "served": served,
             "largest_fp8": largest_fp8, "kernelized": kernelized, "direct_fp32": direct_fp32,
             "hbm_stream": lambda args, gdwd, synth: dict(metric="Z-stream GB/s of the iteration kernel (BF16 Z 200 MB)", **hbm_stream(gdwd, synth))}


def run(name, args):
    import torch
    torch.cuda.set_device(0)
    from paper_2305_12019_gb300 import build as b
    b.build()
    from paper_2305_12019_gb300 import gdwd, synth
    line = WORKLOADS[name](args, gdwd, synth)
    line.update({"n_gpus": 1, "data": "synthetic", "higher_is_better": True})
    print(json.dumps(line), flush=True)
    return 0
