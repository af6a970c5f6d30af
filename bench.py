"""Benchmark of the IFEAST hot path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload lap3d_64|lap3d_64_fp16|lap3d_64_bf16|lap3d_64_twopass|
                                lap3d_64_fp64|
                                lap2d_50|fem3d_64|fem3d_64_fp64|fem3d_48|fem3d_128|serve]

One step = one full IFEAST solve (Algorithm 2 from the seeded initial subspace
until ||R_F|| <= 1e-10) of the workload, inputs resident on the device. The
default workload is the 3D 7-point Laplacian on 64^3 plus a U[0,1) potential
(n = 262,144), interior window with 56 eigenvalues, m0 = 80, 8 contour nodes,
shared-basis MINRES inner solves in FP32 with the FP64 outer iteration. The
fem3d workloads are generalized problems (Q1 finite elements, K x = lambda M x,
lowest eigenvalues) with per-node GMRES inner solves. The
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
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="lap3d_64", choices=["lap3d_64", "lap3d_64_fp16",
                                                                 "lap3d_64_bf16",
                                                                 "lap3d_64_twopass",
                                                                 "lap3d_64_fp64", "lap2d_50",
                                                                 "fem3d_64", "fem3d_64_fp64",
                                                                 "fem3d_48", "fem3d_128",
                                                                 "serve"])
    p.add_argument("--requests", type=int, default=64, help="serving stream length")
    p.add_argument("--rate", type=float, default=8.0, help="serving arrivals per second")
    p.add_argument("--n-max", type=float, default=1e6, help="largest serving request size")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp64-form", action="store_true",
                   help="lap3d_64: skip the one timed solve of the same workload with FP64 "
                        "inner arithmetic and storage (about 13 s)")
    p.add_argument("--two-pass-gb", type=float, default=80.0,
                   help="serving: a request whose stored FP32 Lanczos basis would exceed this "
                        "many GB runs in the two-pass mode")
    p.add_argument("--rate-sweep", default="",
                   help="serving: comma-separated multiples of the one-at-a-time service rate "
                        "(e.g. 0.5,0.8,1.2); each runs the stream with Poisson arrivals at that rate")
    return p.parse_args()


def make_workload(name):
    from paper_1706_00692_gb300 import inputs
    if name == "lap2d_50":
        return inputs.workload_lap2d_50(seed=0)
    if name == "lap3d_64":
        return inputs.workload_lap3d_64_interior(seed=0, precision="fp32")
    if name == "lap3d_64_fp64":
        return inputs.workload_lap3d_64_interior(seed=0, precision="fp64")
    if name == "lap3d_64_fp16":
        return inputs.workload_lap3d_64_interior(seed=0, precision="fp16")
    if name == "lap3d_64_bf16":
        return inputs.workload_lap3d_64_interior(seed=0, precision="bf16")
    if name == "lap3d_64_twopass":
        return inputs.workload_lap3d_64_interior(seed=0, precision="fp32", two_pass=True)
    if name == "fem3d_64":  # generalized K x = lambda M x, per-node FP32 GMRES
        return inputs.workload_fem3d(64, 50, precision="fp32")
    if name == "fem3d_64_fp64":
        return inputs.workload_fem3d(64, 50, precision="fp64")
    if name == "fem3d_48":
        return inputs.workload_fem3d(48, 40, precision="fp32")
    if name == "fem3d_128":  # 128^3 pencil, 102 lowest pairs, two nodes per GMRES pass
        return inputs.workload_fem3d_128()
    raise ValueError(name)


def measured_peaks():
    """HBM copy bandwidth from MEASURED_PEAKS.json next to this script, else
    the 6.8 TB/s fallback; FP64 FMA peak from the same file or 1.2 TFLOP/s."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# DRAM bytes per launch of the FP32 fixed-width Lanczos step kernel on the 64^3
# workload (m0 = 80): dram__bytes_read.sum + dram__bytes_write.sum of one ncu
# capture of that kernel at the bench's launch shape. Re-measure when the
# kernel changes (None: not measured for the workload).
ELL_STEP_TRAFFIC_LAP3D64 = 312.7e6

# the per-step kernels of the Lanczos loop (step, coefficients) are timed in one
# step of PROFILE_EVERY: an event pair around a launch stops it from overlapping
# the previous kernel (programmatic dependent launch), which costs the solve
# ~10 us per sampled step; 1 in 32 still samples ~290 launches per solve
PROFILE_EVERY = 32


def step_bytes(wl, elem):
    """Algorithmic bytes of one Lanczos step launch (s > 0): read w_{s-1} and
    v_{s-1} (the gathered rows counted once), write v_s and w_s (elem bytes per
    stored entry), read the CSR structure and values once (FP32 values unless
    the inner arithmetic is FP64)."""
    n, m0, nnz = wl.A.n, wl.m0, wl.A.nnz
    val_elem = 8 if wl.precision == "fp64" else 4
    return 4 * n * m0 * elem + 4 * (n + 1) + nnz * (4 + val_elem)


def kernel_stats(ktimes, klaunch):
    """{class: (all launches, timed launches, ms per timed launch)} from the
    library's timed launches and their summed ms, and its launch counts."""
    return {k: (klaunch.get(k, c), c, t / c) for k, (c, t) in ktimes.items() if c > 0}


def lanczos_roofline(kstat, wl, peak, peak_kind):
    """Roofline entry of the Lanczos step kernel when it is the class with the
    most estimated device time (all launches x ms per timed launch), else None:
    algorithmic bytes per launch over the mean timed launch, against the peak."""
    top = max(kstat.items(), key=lambda kv: kv[1][0] * kv[1][2]) if kstat else None
    if top is None or top[0] != "lanczos_step":
        return None
    elem = {"fp16": 2, "bf16": 2, "fp32": 4}.get(wl.precision, 8)
    launches, timed, ms_each = top[1]
    nbytes = step_bytes(wl, elem)
    achieved = nbytes / (ms_each * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": "k_lanczos_step", "achieved": achieved,
            "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_source": f"{peak_kind} copy bandwidth",
            "traffic": (ELL_STEP_TRAFFIC_LAP3D64
                        if wl.name.startswith("lap3d_64") and wl.precision == "fp32" else None),
            "bytes_per_launch": nbytes, "launches": launches,
            "launches_timed": timed, "us_per_launch": 1e3 * ms_each}


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
    from paper_1706_00692_gb300.replicas import dist_env as env
    return env()


def cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        n = max((d.get("num_threads", 1) for d in threadpool_info()), default=1)
        return int(n)
    except Exception:
        return os.cpu_count() or 1


def reduced_instance(wl):
    """The oracle's sample of a workload too large for it: the same generator
    at a size the CPU oracle solves completely in seconds. lap3d: the 3D 7-point
    Laplacian + U[0,1) potential on 10^3 with the window at the same relative
    position (first eigenvalue 0.4% into the spectrum; endpoints at the widest
    gap within three eigenvalues of the targets), 10 pairs, m0 = 16, 8
    trapezoid half-circle nodes, alpha = 3e-2, inner solves of at most 150
    steps in residual form from the second iteration on. fem3d: the Q1 pencil
    on 10^3, lowest eigenvalues to the first gap at or after 8, 12 GL nodes,
    per-node GMRES (32 steps, alpha = 1e-2), residual form below ||R_F|| = 1e-3.
    The window endpoints come from a dense eigvalsh of the small matrix."""
    from paper_1706_00692_gb300 import inputs
    if wl.B is not None:
        K, M = inputs.fem_q1((10, 10, 10))
        ev = inputs.fem_q1_eigs((10, 10, 10))
        cnt = inputs._gap_count(ev, 8)
        emin, emax = 0.0, 0.5 * (ev[cnt - 1] + ev[cnt])
        m0 = int(1.5 * cnt) + 2
        return dict(name=f"fem3d_10^3_lowest{cnt}_m0_{m0}_gl12_gmres32", A=K, B=M, emin=emin,
                    emax=emax, m0=m0, rule="gl_half", nc=12, k=32, alpha=1e-2,
                    correction_rf=1e-3, count=cnt)
    N = 10
    A = inputs.add_diagonal_fast(inputs.laplacian((N, N, N)), inputs.random_potential(N ** 3, 1))
    ev = np.linalg.eigvalsh(A.to_scipy().toarray())

    def gap_at(i):
        g = max(range(max(1, i - 3), i + 4), key=lambda c: ev[c] - ev[c - 1])
        return g, 0.5 * (ev[g - 1] + ev[g])

    i0, emin = gap_at(4)
    i1, emax = gap_at(12)
    m0 = int(np.ceil(1.43 * (i1 - i0) / 4) * 4)
    return dict(name=f"lap3d_10^3_pot_interior{i1 - i0}_m0_{m0}_trap8", A=A, B=None, emin=emin,
                emax=emax, m0=m0, rule="trap_half", nc=8, k=150, alpha=3e-2,
                correction_rf=np.inf, count=i1 - i0)


def oracle_sample(wl):
    """Times the CPU oracle (the plain FP64 numpy/scipy Algorithm 2) on one
    complete solve, from the seeded initial subspace to ||R_F|| <= 1e-10:
    of the workload itself when it is the 50x50 one, else of its reduced
    instance (reduced_instance). The per-node GMRES inner solver of the
    oracle equals the shared-basis solver in exact arithmetic (Section 3).
    Returns (converged pairs/s, text)."""
    from oracle import ifeast_oracle as orc
    if wl.A.n > 100000:
        r = reduced_instance(wl)
        A = r["A"].to_scipy()
        B = None if r["B"] is None else r["B"].to_scipy()
        z, w = orc.contour_nodes(r["rule"], r["nc"], r["emin"], r["emax"])
        X0 = inputs_subspace(A.shape[0], r["m0"], 0)
        t0 = time.perf_counter()
        out = orc.ifeast(A, X0, r["emin"], r["emax"], z, w, inner="gmres", k=r["k"],
                         alpha=r["alpha"], tol=1e-10, max_outer=60, B=B,
                         correction_rf=r["correction_rf"])
        dt = time.perf_counter() - t0
        pairs = int((out["inside"] & (out["res"] <= 1e-10)).sum()) if out["converged"] else 0
        return pairs / dt, (f"complete oracle solve of the reduced instance {r['name']} "
                            f"(n = {A.shape[0]}; the {wl.A.n}-row workload takes the oracle days): "
                            f"{out['iters']} outer iterations, {pairs} pairs, {dt:.1f} s")
    z, w = orc.contour_nodes(wl.rule, wl.nc, wl.emin, wl.emax)
    A = wl.A.to_scipy()
    t0 = time.perf_counter()
    out = orc.ifeast(A, wl.X0(), wl.emin, wl.emax, z, w, inner="gmres", k=wl.inner_iters,
                     alpha=wl.alpha, tol=1e-10, max_outer=200)
    dt = time.perf_counter() - t0
    pairs = int((out["inside"] & (out["res"] <= 1e-10)).sum()) if out["converged"] else 0
    return pairs / dt, (f"complete oracle solve of {wl.name}: {out['iters']} outer iterations, "
                        f"{pairs} pairs, {dt:.1f} s")


def oracle_reference_eigs(wl):
    """The eigenvalues the workload's interval holds, from outside the CUDA
    path: the oracle-written golden file for the 64^3 window (shift-invert
    Lanczos), the closed-form spectra for the 50x50 Laplacian and the Q1
    pencils. (values, source) or (None, reason)."""
    from paper_1706_00692_gb300 import inputs
    if wl.name.startswith("lap3d_64"):
        path = os.path.join(ROOT, "tests", "golden", "lap3d64_window.txt")
        try:
            data = np.loadtxt(path)
        except OSError:
            return None, "golden file missing"
        return data[data[:, 2] == 1, 0], "CPU oracle, shift-invert Lanczos (tests/golden/lap3d64_window.txt)"
    if wl.name.startswith("lap2d_50"):
        ev = inputs.laplacian_eigs((50, 50))
        return ev[(ev > wl.emin) & (ev < wl.emax)], "closed form"
    if wl.B is not None and wl.name.startswith("fem3d_"):
        N = round(wl.A.n ** (1.0 / 3.0))
        ev = inputs.fem_q1_eigs((N, N, N))
        return ev[(ev > wl.emin) & (ev < wl.emax)], "closed form"
    return None, "no reference for this workload"


def error_vs_reference(wl, lam, res):
    ref, source = oracle_reference_eigs(wl)
    out = {"pairs": int(lam.size), "max_resid": float(res.max()) if res.size else None,
           "source": source}
    if ref is None:
        return out
    out["reference_pairs"] = int(ref.size)
    if ref.size == lam.size and ref.size:
        err = np.abs(lam - ref) / np.abs(ref)
        out["max_rel_eig_err"] = float(err.max())
        out["per_pair_rel_eig_err"] = [float(f"{e:.2e}") for e in err]
    return out


def fp64_form_solve(args, dev):
    """One solve of the 64^3 workload with FP64 Krylov vectors and arithmetic
    (stored basis ~250 GB), timed with CUDA events on its stream after an L2
    flush; the eigenvalues are compared with the oracle's like the main line's."""
    import gc
    import torch
    from paper_1706_00692_gb300 import Solver
    gc.collect()
    torch.cuda.empty_cache()  # the FP32 solvers' workspaces go back to the device
    wl = make_workload("lap3d_64_fp64")
    X0 = torch.as_tensor(wl.X0(), device=dev)
    S = Solver(wl.A, wl.emin, wl.emax, wl.m0, nc=wl.nc, rule=wl.rule, inner=wl.inner,
               inner_iters=wl.inner_iters, alpha=wl.alpha, precision=wl.precision,
               two_pass=wl.two_pass, B=wl.B, node_chunk=wl.node_chunk, device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    flush.fill_(1)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rc = S.solve(X0)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    if rc != 0:
        S.close()
        return {"status": int(rc)}
    st = S.stats()
    lam, _, res = S.eigenpairs()
    S.close()
    del flush
    torch.cuda.empty_cache()
    pairs = int((res <= 1e-10).sum())
    return {"workload": wl.name, "value": pairs / (ms / 1e3), "unit": "eigenpairs/s",
            "ms_per_solve": ms, "pairs": pairs, "outer_iters": st["outer_iters"],
            "krylov_steps_total": st["total_matvecs"], "dtype": "f64",
            "timing": "one solve after the timed FP32 steps, CUDA events, L2 flushed before it",
            "error_vs_reference": error_vs_reference(wl, lam, res)}


def inputs_subspace(n, m0, seed):
    from paper_1706_00692_gb300 import inputs
    return inputs.initial_subspace(n, m0, seed)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    wl = make_workload(args.workload)
    vals = []
    sample = ""
    for _ in range(args.warmup):
        oracle_sample(wl)
    for _ in range(args.steps):
        v, sample = oracle_sample(wl)
        vals.append(v)
    value = float(np.mean(vals))
    cores = cpu_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "eigenpairs/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl.name, "n": wl.A.n, "m0": wl.m0,
                                             "nc": wl.nc, "contour": wl.rule,
                                             "inner": wl.inner, "inner_iters": wl.inner_iters},
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
    skw = dict(nc=wl.nc, rule=wl.rule, inner=wl.inner, inner_iters=wl.inner_iters,
               alpha=wl.alpha, precision=wl.precision, two_pass=wl.two_pass, B=wl.B,
               node_chunk=wl.node_chunk, device=dev)
    S = Solver(wl.A, wl.emin, wl.emax, wl.m0, **skw)
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
    # kernel timing with CUDA events on the handle's stream: every launch, except
    # that the per-step Lanczos kernels are timed one step in PROFILE_EVERY
    # (events between them would stop their programmatic overlap in every step)
    S.set_profiling(PROFILE_EVERY)
    S.kernel_times(reset=True)
    S.kernel_launches(reset=True)
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
    ktimes = S.kernel_times(reset=True)
    klaunch = S.kernel_launches(reset=True)
    S.set_profiling(False)
    kstat = kernel_stats(ktimes, klaunch)
    lam, X, res = S.eigenpairs()
    pairs = int((res <= 1e-10).sum())
    accuracy = error_vs_reference(wl, lam, res)
    # replicas: converged pairs of every rank over the slowest rank's time
    from paper_1706_00692_gb300.replicas import job_throughput
    _, total_s, value = job_throughput(pairs * args.steps, float(sum(times)) / 1e3, device=dev)
    total_ms = total_s * 1e3
    # the end-to-end solver below holds a workspace of its own (the FP64 basis
    # alone is ~250 GB at this size): release this one first
    S.close()
    del flush
    torch.cuda.empty_cache()

    # end to end through the C ABI with host buffers: create (A host->device),
    # solve (X0 host->device), eigenpairs (device->host), destroy
    X0h = torch.from_numpy(wl.X0()).pin_memory().numpy()
    csr_bytes = sum(M.rowptr.nbytes + M.colidx.nbytes + M.val.nbytes
                    for M in (wl.A, wl.B) if M is not None)
    e2e_times = []
    for _ in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S2 = Solver(wl.A, wl.emin, wl.emax, wl.m0, **skw)
        rc = S2.solve(X0h)
        l2, x2, r2 = S2.eigenpairs()
        S2.close()
        e2e_times.append(time.perf_counter() - t0)
        assert rc == 0
    e2e_pairs = int((r2 <= 1e-10).sum())
    _, _, e2e_value = job_throughput(e2e_pairs * len(e2e_times), float(sum(e2e_times)), device=dev)
    d2h = l2.nbytes + x2.nbytes + r2.nbytes

    # the same workload with FP64 Krylov arithmetic and storage (the plain-precision
    # form of the same algorithm): one solve, timed on the device like the steps above
    fp64_form = None
    if args.workload == "lap3d_64" and not args.no_fp64_form and world == 1:
        fp64_form = fp64_form_solve(args, dev)

    # roofline of the dominant kernel class, from the live event timings
    peak, peak_kind = measured_peaks()
    roofline = lanczos_roofline(kstat, wl, peak, peak_kind)
    gpu_launches = int(sum(klaunch.values()))
    if rank == 0:
        st = stats[-1]
        line = {"metric": METRIC, "value": value, "unit": "eigenpairs/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if wl.precision == "fp64" else "f32",
                "data": "synthetic",
                "config": {"workload": wl.name, "n": wl.A.n, "nnz": wl.A.nnz, "m0": wl.m0,
                           "nc": wl.nc, "contour": wl.rule, "inner": wl.inner,
                           "inner_precision": wl.precision,
                           "inner_storage": {"fp16": "f16", "bf16": "bf16",
                                             "fp32": "f32"}.get(wl.precision, "f64"),
                           "inner_iters": wl.inner_iters,
                           "alpha": wl.alpha, "l2": "flushed between steps (256 MB write)",
                           "outer_iters": st["outer_iters"], "pairs": pairs,
                           "krylov_steps_total": st["total_matvecs"],
                           "krylov_steps_seq": st["seq_matvecs"]},
                "e2e": {"value": e2e_value, "unit": "eigenpairs/s",
                        "h2d_bytes_per_step": int(csr_bytes + X0h.nbytes),
                        "d2h_bytes_per_step": int(d2h)},
                "gpu_launches": gpu_launches,
                "roofline": roofline,
                "kernel_ms": {k: {"launches": n, "timed": c, "ms_per_launch": round(e, 6),
                                  "ms": round(n * e, 3)} for k, (n, c, e) in kstat.items()},
                "kernel_timing": f"CUDA events per launch; the chained Lanczos-loop kernels "
                                 f"(step, coefficient reduction, Givens batch) timed at one "
                                 f"launch in {PROFILE_EVERY} of each",
                "error_vs_reference": accuracy,
                "clocks": clk.summary()}
        if fp64_form is not None:
            line["fp64_form"] = fp64_form
        if not args.no_cpu_baseline and world == 1:
            v, sample = oracle_sample(wl)
            line["cpu_baseline"] = {"value": v, "unit": "eigenpairs/s", "cores": cpu_threads(),
                                    "kind": "oracle", "sample": sample}
        print(json.dumps(line), flush=True)
    S.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def run_serve(args):
    """Serving stream: Poisson arrivals of eigen-requests (2D/3D Laplacians with a
    potential, n log-uniform 1e3..n_max, m0 16..128), submitted at their arrival
    times to one server (memory budget 160 GB, 8 running at once). A request
    whose stored Lanczos basis would exceed --two-pass-gb (80 GB) runs in the
    two-pass mode (three basis vectors). Reports converged eigenpairs/s over the makespan and
    p50/p99 request latency, and the same stream served one request at a time
    for comparison. A second, smaller stream (16 requests, n up to 5e4) is run
    three ways: served (mixed precision, 8 at once), one at a time in the same
    form, and one at a time in the plain FP64 form of Algorithm 2 (per-node
    GMRES, at most 32 steps, alpha = 1e-2), all to residual 1e-10."""
    import torch
    from paper_1706_00692_gb300 import Server, inputs
    from paper_1706_00692_gb300.build import build
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl")
    build()
    reqs = inputs.serving_requests(args.requests, seed=1234, rate=args.rate, n_max=args.n_max)
    K = 300
    # FP32 basis of K + 1 vectors over --two-pass-gb (default half the 160 GB budget, so
    # that two such requests can be resident at once): keep three vectors and rebuild
    # them in a second pass
    two_pass = [(K + 1) * r.A.n * r.m0 * 4 > args.two_pass_gb * 2**30 for r in reqs]
    warm = inputs.serving_requests(3, seed=999, n_max=2e4)

    mixed = dict(inner="minres", inner_iters=K, alpha=3e-2, precision="fp32")
    plain = dict(inner="gmres", inner_iters=32, alpha=1e-2, precision="fp64")

    def serve(max_active, timed_arrivals, reqs=reqs, two_pass=two_pass, form=mixed,
              arrival_scale=1.0):
        srv = Server(160 << 30, max_active=max_active, device=local)
        for r in warm:  # load kernels, warm the allocator
            srv.wait(srv.submit(r.A, r.emin, r.emax, r.m0, r.X0, rule="trap_half", **form))
        ids = []
        t0 = time.perf_counter()
        for r, tp in zip(reqs, two_pass):
            if timed_arrivals:
                dt = r.arrival * arrival_scale - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
            ids.append(srv.submit(r.A, r.emin, r.emax, r.m0, r.X0, rule="trap_half",
                                  two_pass=tp, **form))
        outs = [srv.wait(i) for i in ids]
        span = time.perf_counter() - t0
        srv.close()
        lat = np.array([o[4]["submit_to_done_ms"] for o in outs])
        svc = np.array([o[4]["submit_to_done_ms"] - o[4]["submit_to_start_ms"] for o in outs])
        pairs = sum(int((o[3] <= 1e-10).sum()) for o in outs if o[0] == 0)
        failed = {}
        for r, o in zip(reqs, outs):
            if o[0] != 0:
                failed[str(o[0])] = failed.get(str(o[0]), 0) + 1
        serve.svc = svc  # start-to-done time of each request (its service time when alone)
        return pairs, span, lat, failed

    with ClockSampler(local) as clk:
        pairs, span, lat, failed = serve(8, True)
    pairs1, span1, lat1, failed1 = serve(1, False)
    # share of the one-at-a-time service time by request size class
    sizes = np.array([r.A.n for r in reqs])
    svc1 = serve.svc
    share = {name: float(svc1[(sizes >= lo) & (sizes < hi)].sum() / svc1.sum())
             for name, lo, hi in [("n<1e4", 0, 1e4), ("1e4<=n<1e5", 1e4, 1e5),
                                  ("n>=1e5", 1e5, np.inf)]}
    count = {name: int(((sizes >= lo) & (sizes < hi)).sum())
             for name, lo, hi in [("n<1e4", 0, 1e4), ("1e4<=n<1e5", 1e4, 1e5),
                                  ("n>=1e5", 1e5, np.inf)]}
    # arrival-rate sweep: multiples f of the one-at-a-time service rate mu (requests/s);
    # the stream's exponential inter-arrival times are rescaled from rate args.rate to f mu
    sweep = []
    mu = len(reqs) / span1
    for f in [float(x) for x in args.rate_sweep.split(",") if x.strip()]:
        with ClockSampler(local) as clk_f:
            pr, sp, la, fa = serve(8, True, arrival_scale=args.rate / (f * mu))
        sweep.append({"rate_factor": f, "arrival_rate_per_s": f * mu, "value": pr / sp,
                      "pairs": pr, "makespan_s": sp, "failed": fa,
                      "p50_ms": float(np.percentile(la, 50)),
                      "p99_ms": float(np.percentile(la, 99)), "clocks": clk_f.summary()})
    # the mixed-precision served form against the plain FP64 form, one request at a time
    small = inputs.serving_requests(16, seed=1234, rate=args.rate, n_max=5e4)
    nosplit = [False] * len(small)
    cmp = {}
    for name, ma, timed, form in [("served_mixed", 8, True, mixed),
                                  ("one_at_a_time_mixed", 1, False, mixed),
                                  ("one_at_a_time_plain_fp64", 1, False, plain)]:
        pr, sp, la, fa = serve(ma, timed, small, nosplit, form)
        cmp[name] = {"value": pr / sp, "pairs": pr, "makespan_s": sp, "failed": fa,
                     "p50_ms": float(np.percentile(la, 50)),
                     "p99_ms": float(np.percentile(la, 99))}
    from paper_1706_00692_gb300.replicas import job_throughput
    _, _, value = job_throughput(pairs, span, device=torch.device("cuda", local))
    if rank == 0:
        line = {"metric": "served eigenpairs/s (Poisson stream); p50/p99 latency",
                "value": value, "unit": "eigenpairs/s", "n_gpus": world,
                "steps": 1, "warmup": len(warm), "ms_per_step": span * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": f"serve_{args.requests}_poisson_rate{args.rate:g}"
                                       f"_n1e3-{args.n_max:.0e}_m0_16-128",
                           "max_active": 8, "budget_gb": 160, "inner": "minres",
                           "inner_precision": "fp32", "contour": "trap_half",
                           "two_pass_requests": int(sum(two_pass)),
                           "two_pass_above_gb": args.two_pass_gb,
                           "n_max_seen": int(max(r.A.n for r in reqs))},
                "latency_ms": {"p50": float(np.percentile(lat, 50)),
                               "p99": float(np.percentile(lat, 99))},
                "failed": failed, "pairs": pairs, "requests": len(reqs),
                "one_at_a_time": {"value": pairs1 / span1, "makespan_s": span1,
                                  "failed": failed1, "service_rate_per_s": mu,
                                  "service_time_share_by_size": share,
                                  "requests_by_size": count},
                "rate_sweep": sweep,
                "vs_plain_fp64": {"stream": "16 requests, n 1e3-5e4, m0 16-128, seed 1234",
                                  "plain_form": "per-node GMRES FP64, <= 32 steps, alpha 1e-2",
                                  "mixed_form": "shared-basis MINRES FP32, <= 300 steps, "
                                                "alpha 3e-2", **cmp},
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.workload == "serve" and args.impl == "ours":
        run_serve(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
