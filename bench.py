"""Benchmark of the IFEAST hot path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload lap2d_50|lap3d_64]

One step = one full IFEAST solve (Algorithm 2 from the seeded initial subspace
until ||R_F|| <= 1e-10) of the workload, inputs resident on the device. The
metric is converged eigenpairs per second (pairs inside the interval with
relative residual <= 1e-10, times steps, over the device time of the steps).
Under torchrun every rank solves its own replica of the workload (no data
exchange: "weak" scaling) and rank 0 prints one JSON line.

--impl reference times the CPU oracle (the plain FP64 numpy/scipy
FEAST/IFEAST of the paper's Algorithm 2) on the host cores, on a bounded
sample of the same workload, and prints the same JSON line with
"impl": "reference".
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "converged eigenpairs/s at residual<=1e-10"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="lap2d_50", choices=["lap2d_50"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    return p.parse_args()


def make_workload(name):
    from paper_1706_00692_gb300 import inputs
    if name == "lap2d_50":
        return inputs.workload_lap2d_50(seed=0)
    raise ValueError(name)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 7:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(self.samples)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        n = max((d.get("num_threads", 1) for d in threadpool_info()), default=1)
        return int(n)
    except Exception:
        return os.cpu_count() or 1


def oracle_sample(wl, budget_s=20.0):
    """Times the CPU oracle (Algorithm 2, per-node GMRES) on the workload until
    it converges or the time budget runs out; returns (pairs/s, sample text)."""
    from oracle import ifeast_oracle as orc
    z, w = orc.contour_nodes(wl.rule, wl.nc, wl.emin, wl.emax)
    A = wl.A.to_scipy()
    t0 = time.perf_counter()
    iters = [0]

    def cb(it, lam, X, res, ins):
        iters[0] = it
        if time.perf_counter() - t0 > budget_s:
            raise TimeoutError

    try:
        out = orc.ifeast(A, wl.X0(), wl.emin, wl.emax, z, w, inner="gmres", k=wl.inner_iters,
                         alpha=wl.alpha, tol=1e-10, max_outer=200, callback=cb)
        dt = time.perf_counter() - t0
        pairs = int((out["inside"] & (out["res"] <= 1e-10)).sum()) if out["converged"] else 0
        return pairs / dt, f"full solve of {wl.name}: {iters[0]} outer iterations, {pairs} pairs, {dt:.1f} s"
    except TimeoutError:
        dt = time.perf_counter() - t0
        return 0.0, f"{wl.name}: {iters[0]} outer iterations in {dt:.1f} s without converging"


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    wl = make_workload(args.workload)
    vals = []
    sample = ""
    for _ in range(args.warmup):
        oracle_sample(wl, budget_s=5.0)
    for _ in range(args.steps):
        v, sample = oracle_sample(wl, budget_s=30.0)
        vals.append(v)
    value = float(np.mean(vals))
    cores = cpu_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "eigenpairs/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl.name, "n": wl.A.n, "m0": wl.m0,
                                             "nc": wl.nc, "inner_iters": wl.inner_iters},
            "cpu_baseline": {"value": value, "unit": "eigenpairs/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "eigenpairs/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    from paper_1706_00692_gb300 import Solver
    from paper_1706_00692_gb300.build import build

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    build()
    wl = make_workload(args.workload)
    dev = torch.device("cuda", torch.cuda.current_device())
    X0 = torch.as_tensor(wl.X0(), device=dev)
    S = Solver(wl.A, wl.emin, wl.emax, wl.m0, nc=wl.nc, rule=wl.rule, inner_iters=wl.inner_iters,
               alpha=wl.alpha, device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def step():
        rc = S.solve(X0)
        if rc != 0:
            raise RuntimeError(f"solve status {rc}")

    for _ in range(max(args.warmup, 3) if args.warmup >= 0 else 3):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    times = []
    stats = []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1)  # L2 flushed between timed steps (outside the events)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            stats.append(S.stats())
    torch.cuda.synchronize()
    total_ms = float(sum(times))
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    lam, X, res = S.eigenpairs()
    pairs = int((res <= 1e-10).sum())
    value = pairs * args.steps * world / (total_ms / 1e3)

    # end to end through the C ABI with host buffers: create (A host->device),
    # solve (X0 host->device), eigenpairs (device->host), destroy
    X0h = torch.from_numpy(wl.X0()).pin_memory().numpy()
    csr_bytes = wl.A.rowptr.nbytes + wl.A.colidx.nbytes + wl.A.val.nbytes
    e2e_times = []
    for _ in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S2 = Solver(wl.A, wl.emin, wl.emax, wl.m0, nc=wl.nc, rule=wl.rule,
                    inner_iters=wl.inner_iters, alpha=wl.alpha, device=dev)
        rc = S2.solve(X0h)
        l2, x2, r2 = S2.eigenpairs()
        S2.close()
        e2e_times.append(time.perf_counter() - t0)
        assert rc == 0
    e2e_pairs = int((r2 <= 1e-10).sum())
    e2e_value = e2e_pairs * world / statistics.mean(e2e_times)
    d2h = l2.nbytes + x2.nbytes + r2.nbytes

    if rank == 0:
        st = stats[-1]
        line = {"metric": METRIC, "value": value, "unit": "eigenpairs/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": wl.name, "n": wl.A.n, "nnz": wl.A.nnz, "m0": wl.m0,
                           "nc": wl.nc, "contour": wl.rule, "inner": "gmres",
                           "inner_iters": wl.inner_iters, "alpha": wl.alpha,
                           "l2": "flushed between steps (256 MB write)",
                           "outer_iters": st["outer_iters"], "pairs": pairs},
                "e2e": {"value": e2e_value, "unit": "eigenpairs/s",
                        "h2d_bytes_per_step": int(csr_bytes + X0h.nbytes),
                        "d2h_bytes_per_step": int(d2h)},
                "gpu_launches": None,
                "clocks": clk.summary()}
        if not args.no_cpu_baseline and world == 1:
            v, sample = oracle_sample(wl, budget_s=30.0)
            line["cpu_baseline"] = {"value": v, "unit": "eigenpairs/s", "cores": cpu_threads(),
                                    "kind": "oracle", "sample": sample}
        print(json.dumps(line), flush=True)
    S.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
