"""Benchmark: generalized-DWD solves/s at KKT <= 1e-6 on the spiked FP32 workload.

Workload: d = 20000 features, n = 1000 samples (balanced), x = +-2 v + N(0, I +
49 S S^T) with 5 spike directions, q = 1, C = 10, FP32 data, stop at
kkt <= 1e-6 (seeded synthetic stand-in for the paper's UCI/LIBSVM sets).

One step = one complete solve through the C-ABI: gdwd_create (ingest into the
slab layout, Z_scale, Gram, Cholesky, inverse), gdwd_solve (the persistent
iteration kernel until kkt <= tol, then w), gdwd_free.

  value   solves/s with Z already resident in HBM (a CUDA tensor) when timed
  e2e     the same with Z in pinned host memory: the host->device copy of Z and
          y and the device->host copy of w and the result inside every step
  roofline  the persistent iteration kernel: algorithmic bytes per launch
          (iterations x (1 read of Z + 2 reads of the double-float G^{-1} +
          vector traffic)) / its CUDA-event duration, against the measured HBM peak
  cpu_baseline  the FP64 CPU oracle (oracle/) on the host cores, one full solve

--impl reference times the oracle itself as the reference arm.
Multi-GPU: the workload does not shard; with torchrun each rank runs an
independent replica and value = total solves / max-over-ranks time ("replicas").
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "gDWD solves/s at KKT<=1e-6"
UNIT = "solves/s"
WORKLOAD = "spiked_fp32 d=20000 n=1000 q=1 C=10 tol=1e-6"
CONFIG = {"workload": WORKLOAD, "d": 20000, "n": 1000, "q": 1.0, "C": 10.0, "tol": 1e-6, "store": "f32",
          "seed": 2001, "l2": "flushed between steps (Z is 80 MB < 129 MB L2); Z stays L2-resident within a solve"}
# gdwd_create launches 9 kernels (3 fills, one-pass ingest, scale, BF16 split, tensor-core
# Gram, Gram finish, factor), gdwd_solve 4 (2 fills, iteration, w finish)
LAUNCHES_PER_STEP = 13


# sources of the iteration kernel: the DRAM traffic recorded under profiles/ is
# used only while their hash matches the one recorded with the counters
KERNEL_SOURCES = ["common.cuh", "solver.cuh", "passes.cuh", "nspace.cuh", "iterate.cu"]
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "iterate_kernel_spiked_fp32.md")


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2305_12019_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """dram__bytes_read.sum + dram__bytes_write.sum of one iteration-kernel launch
    from the committed ncu summary, or None if the kernel changed since."""
    try:
        fields = {}
        with open(TRAFFIC_PROFILE) as f:
            for line in f:
                if ":" in line and line.startswith("- "):
                    k, v = line[2:].split(":", 1)
                    fields[k.strip()] = v.strip().strip("`")
        if fields.get("source_hash") != kernel_source_hash():
            return None
        return int(fields["traffic_bytes_per_launch"])
    except Exception:
        return None


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def max_over_ranks(t_ms, ws, device="cuda"):
    """The largest of the ranks' timed milliseconds (all_reduce MAX), the same on
    every rank; t_ms itself on one rank."""
    if ws <= 1:
        return float(t_ms)
    import torch
    import torch.distributed as dist
    tt = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def replica_rate(units_per_rank, t_ms_max, ws):
    """Whole-job rate of ws independent replicas: all units over the slowest rank's time."""
    return ws * units_per_rank / (t_ms_max / 1e3)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, gpu_index=0):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"gdwd_clocks_{os.getpid()}.csv")
        self.gpu = gpu_index

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 7 and parts[0].replace(".", "").isdigit():
                    rows.append(parts)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[0]) for r in rows]
        mx = max(float(r[1]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = [nm for k, nm in enumerate(names) if any(r[3 + k].lower() == "active" for r in rows)]
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": reasons, "samples": len(rows)}


def algorithmic_bytes_per_iteration(d, n, zbytes, slabs, dots_every=16):
    """Per ADMM iteration: Z read once (b = Z~^T g' is carried in n-space), the
    double-float G^{-1} read twice (8 n^2 B each), d-vectors (u, rho, g read/written:
    8 x 8d), n-vectors (~20 x 8n), and every dots_every-th iteration the column-dot
    partials (written and read: 2 x 4 n slabs)."""
    return d * n * zbytes + 2 * 8 * n * n + 64 * d + 160 * n + 8 * n * slabs / dots_every


def run_oracle_solve(inst):
    from oracle import gdwd_oracle as O
    t = time.perf_counter()
    res = O.solve(inst.Z.astype(np.float64), inst.y, inst.q, inst.C, tol=inst.tol)
    return time.perf_counter() - t, res


def reference_arm(args):
    ws, rank = _dist()
    if rank != 0:
        return 0
    from paper_2305_12019_gb300 import synth
    inst = synth.spiked_fp32()
    # Every step, warm-up included, is one full oracle solve of the same instance
    # to kkt <= 1e-6 (about 10 s on 16 host cores), so the run's wall time is
    # what the line reports.
    for _ in range(args.warmup):
        run_oracle_solve(inst)
    times, iters = [], []
    for _ in range(args.steps):
        t, res = run_oracle_solve(inst)
        times.append(t)
        iters.append(res["iters"])
        if not res["converged"]:
            raise SystemExit("oracle solve did not converge")
    t = statistics.mean(times)
    cores = len(os.sched_getaffinity(0))
    val = 1.0 / t
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": CONFIG,
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"one full FP64 oracle solve of the same instance per step "
                                       f"({iters[0]} iterations to kkt<=1e-6)"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gdwd", choices=["gdwd", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the HBM-streaming and served blocks of the default line (profiling runs)")
    ap.add_argument("--extras-serve-seconds", type=float, default=1.0)
    ap.add_argument("--d", type=int, default=20000, help="feature count (profiling of other sizes only)")
    ap.add_argument("--n", type=int, default=1000, help="sample count (profiling of other sizes only)")
    ap.add_argument("--workload", default="spiked_fp32",
                    help="spiked_fp32 (default line) | plain_fp64 | cgrid_bf16 | uneven_batch | served | largest_fp8 | "
                         "kernelized | direct_fp32 | hbm_stream")
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-wall", type=float, default=300.0, help="served: stop admitting after this many seconds")
    ap.add_argument("--cg-d", type=int, default=50000)
    ap.add_argument("--cg-n", type=int, default=2000)
    ap.add_argument("--big-d", type=int, default=200000)
    ap.add_argument("--big-n", type=int, default=5000)
    ap.add_argument("--kern-wide-d", type=int, default=200000)
    ap.add_argument("--kern-steps", type=int, default=3)
    ap.add_argument("--kern", type=int, default=0, help="uneven_batch / served / largest_fp8: 1 = kernelized iteration, -1 = chosen per problem")
    ap.add_argument("--dir-d", type=int, default=200)
    ap.add_argument("--dir-n", type=int, default=1000000)
    args = ap.parse_args()
    if args.workload != "spiked_fp32" and args.impl != "reference":
        import bench_workloads
        return bench_workloads.run(args.workload, args)
    if args.impl == "reference":
        return reference_arm(args)

    import torch
    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2305_12019_gb300 import build as b
    b.build()
    from paper_2305_12019_gb300 import gdwd, synth

    inst = synth.spiked_fp32(d=args.d, n=args.n)
    d, n = inst.d, inst.n
    if (d, n) != (20000, 1000):
        CONFIG.update(workload=f"spiked_fp32 d={d} n={n} q=1 C=10 tol=1e-6 (profiling size)", d=d, n=n)
    Zh = inst.Z                                   # d x n float32 (host)
    # device-resident input, column-major (stride(0) == 1)
    Zd = torch.from_numpy(np.asfortranarray(Zh)).T.contiguous().T.cuda()
    Zd = torch.as_strided(Zd, (d, n), (1, d))
    Zp = torch.from_numpy(np.ascontiguousarray(Zh.T)).pin_memory()   # n x d rows = columns of Z
    Zp_view = torch.as_strided(Zp, (d, n), (1, d))
    y = inst.y
    stream = torch.cuda.current_stream().cuda_stream
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    wdev = torch.empty(d, dtype=torch.float64, device="cuda")

    def step_device():
        with gdwd.Solver(Zd, y, inst.q, inst.C, store="f32", tol=inst.tol, stream=stream) as s:
            res, _, _ = s.solve(w_out=wdev)
            info = s.info()
            info["phase_ns"] = s.phase_times()
        return res[0], info

    def step_e2e():
        with gdwd.Solver(Zp_view, y, inst.q, inst.C, store="f32", tol=inst.tol, stream=stream) as s:
            res, w, _ = s.solve()
        return res[0], w

    for _ in range(args.warmup):
        step_device()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    results = []
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(float(k))                   # evict Z from L2 between steps
            ev[k][0].record()
            r, info = step_device()
            ev[k][1].record()
            results.append(r)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    if ws > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b2) for a, b2 in ev]
    t_ms = max_over_ranks(sum(step_ms), ws)
    ms_per_step = t_ms / args.steps
    value = replica_rate(args.steps, t_ms, ws)
    for r in results:
        if r["status"] != 0 or r["kkt"] > inst.tol:
            raise SystemExit(f"solve did not converge: {r}")

    # roofline of the persistent iteration kernel (library CUDA events on the launch stream)
    iters = statistics.mean(r["iters"] for r in results)
    t_iter_ms = statistics.mean(r["t_solve_ms"] for r in results)
    t_setup_ms = statistics.mean(r["t_setup_ms"] for r in results)
    bytes_it = algorithmic_bytes_per_iteration(d, n, 4, info["slabs"])
    peak, peak_kind = _peaks()
    achieved = iters * bytes_it / (t_iter_ms * 1e-3) / 1e9
    roof = {"kernel": "iterate_kernel<float>", "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": peak_kind, "traffic": None,
            "bytes_per_iteration": bytes_it, "iterations": iters, "launch_ms": t_iter_ms}
    roof["traffic"] = profiled_traffic()

    # end to end through the public API with host buffers
    e2e_ms = []
    for k in range(max(1, args.steps)):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r, w = step_e2e()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        assert r["status"] == 0
    e2e_val = replica_rate(len(e2e_ms), max_over_ranks(sum(e2e_ms), ws), ws)
    h2d = d * n * 4 + n * 8
    d2h = d * 8 + 256

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak" if ws > 1 else "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": CONFIG, "parallelism": f"replicas{ws}",
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": LAUNCHES_PER_STEP * args.steps,
            "roofline": roof, "clocks": clk.summary(),
            "detail": {"setup_ms": t_setup_ms, "iterate_ms": t_iter_ms, "iterations": iters,
                       "step_ms": step_ms, "wall_s": wall, "grid": info["grid"], "slabs": info["slabs"],
                       "block_rows": info["block_rows"], "kkt": [r["kkt"] for r in results],
                       "setup_stages_ms": {k: info[k] for k in ("t_ingest_ms", "t_gram_ms", "t_factor_ms")},
                       "phase_us_per_iter": {k: v / 1e3 / iters for k, v in info["phase_ns"].items()}}}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        t_or, ref = run_oracle_solve(inst)
        line["cpu_baseline"] = {"value": 1.0 / t_or, "unit": UNIT, "cores": len(os.sched_getaffinity(0)),
                                "kind": "oracle", "sample": "one full FP64 oracle solve of the same instance "
                                f"({ref['iters']} iterations to kkt<=1e-6)"}
        # error of the GPU result against the oracle (last device step)
        with gdwd.Solver(Zd, y, inst.q, inst.C, store="f32", tol=inst.tol, stream=stream) as s:
            res, w, _ = s.solve()
        line["detail"]["err_vs_oracle"] = {
            "rel_obj": abs(res[0]["primal_obj"] - ref["primal"]) / abs(ref["primal"]),
            "rel_w": float(np.linalg.norm(w[:, 0] - ref["w"]) / np.linalg.norm(ref["w"]))}
    if rank == 0 and ws == 1 and not args.no_extras:
        # the two other halves of the metric: Z streamed from HBM (the C-grid
        # instance, 200 MB of BF16) and a short served stream (Poisson arrivals,
        # latency from arrival)
        import bench_workloads
        line["detail"]["hbm_stream"] = bench_workloads.hbm_stream(gdwd, synth)
        sargs = argparse.Namespace(**vars(args))
        sargs.serve_seconds, sargs.kern = args.extras_serve_seconds, -1
        sv = bench_workloads.served(sargs, gdwd, synth)
        line["detail"]["served"] = {k: sv[k] for k in ("value", "unit", "latency_ms_p50", "latency_ms_p99",
                                                      "server_latency_ms_p50", "server_latency_ms_p99", "requests",
                                                      "arrived", "converged", "wall_s", "offered_rate", "mean_iters",
                                                      "config")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
