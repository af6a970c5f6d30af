"""Run one IFEAST solve of a named synthetic workload and report the result.

    python -m paper_1706_00692_gb300.cli [--workload lap3d_64|lap3d_64_fp16|lap3d_64_bf16|
                                                     lap3d_64_twopass|lap3d_64_fp64|lap2d_50|
                                                     fem3d_64|fem3d_64_fp64|fem3d_48|fem3d_128]
                                         [--max-outer M] [--inner-iters K] [--alpha A] [--verbose]
                                         [--rr-calls R] [--plain-loads]

Prints one JSON line: status, eigenpairs found, largest residual, outer
iterations, Krylov steps and wall time. Exit status 0 whenever the library
calls succeed (a solve stopped by --max-outer before convergence, or one whose
interval holds no Ritz value yet, included).
With --rr-calls R it runs no solve: R Rayleigh-Ritz calls (Algorithm 2, steps
3-4) on the workload's matrix and a seeded random subspace of its m0 columns,
and prints the per-kernel CUDA-event times of those calls.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import inputs
from .solver import Solver


def workload(name: str):
    if name == "lap2d_50":
        return inputs.workload_lap2d_50(seed=0)
    if name == "lap3d_64":
        return inputs.workload_lap3d_64_interior(seed=0, precision="fp32")
    if name == "lap3d_64_fp64":
        return inputs.workload_lap3d_64_interior(seed=0, precision="fp64")
    if name == "lap3d_64_fp16":
        return inputs.workload_lap3d_64_interior(seed=0, precision="fp16")
    if name == "lap3d_64_twopass":
        return inputs.workload_lap3d_64_interior(seed=0, precision="fp32", two_pass=True)
    if name == "fem3d_64":
        return inputs.workload_fem3d(64, 50, precision="fp32")
    if name == "fem3d_64_fp64":
        return inputs.workload_fem3d(64, 50, precision="fp64")
    if name == "fem3d_48":
        return inputs.workload_fem3d(48, 40, precision="fp32")
    if name == "fem3d_128":
        return inputs.workload_fem3d_128()
    if name == "lap3d_64_bf16":
        return inputs.workload_lap3d_64_interior(seed=0, precision="bf16")
    if name.startswith("convdiff_"):  # convdiff_N: N x N upwind convection-diffusion
        return inputs.workload_convdiff(int(name.split("_")[1]))
    raise SystemExit(f"unknown workload {name}")


def main(argv=None) -> int:
    p = argparse.ArgumentParser()
    p.add_argument("--workload", default="lap3d_64")
    p.add_argument("--max-outer", type=int, default=100)
    p.add_argument("--inner-iters", type=int, default=0, help="override the workload's cap")
    p.add_argument("--alpha", type=float, default=-1.0,
                   help="override the workload's inner tolerance factor (alpha of Algorithm 2)")
    p.add_argument("--verbose", action="store_true")
    p.add_argument("--plain-loads", action="store_true",
                   help="FP32 per-node GMRES: read the basis with plain loads, not TMA")
    p.add_argument("--rr-calls", type=int, default=0,
                   help="time this many Rayleigh-Ritz calls instead of a solve")
    a = p.parse_args(argv)
    import torch
    wl = workload(a.workload)
    if a.rr_calls > 0:
        return rr_calls(wl, a.rr_calls)
    k = a.inner_iters or wl.inner_iters
    alpha = a.alpha if a.alpha >= 0.0 else wl.alpha
    S = Solver(wl.A, wl.emin, wl.emax, wl.m0, nc=wl.nc, rule=wl.rule, inner=wl.inner,
               inner_iters=k, alpha=alpha, precision=wl.precision, two_pass=wl.two_pass,
               max_outer=a.max_outer, B=wl.B, node_chunk=wl.node_chunk,
               verbose=a.verbose, plain_loads=a.plain_loads, nonsymmetric=wl.nonsym,
               nonsym_correction=wl.nonsym_correction)
    X0 = torch.as_tensor(wl.X0(), device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc = S.solve(X0)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    st = S.stats()
    out = {"workload": wl.name, "status": rc, "seconds": dt, "outer_iters": st["outer_iters"],
           "found": st["found"], "RF": st["RF"], "krylov_steps_total": st["total_matvecs"],
           "krylov_steps_seq": st["seq_matvecs"]}
    if rc in (0, 4) and wl.nonsym:  # complex Ritz pairs; the upwind spectrum is real
        lam, X, res = S.eigenpairs_complex()
        out["max_residual"] = float(res.max()) if res.size else None
        N = round(wl.A.n ** 0.5)
        ref = inputs.upwind_convection_diffusion_eigs((N, N), 10.0)
        ref = ref[(ref > wl.emin) & (ref < wl.emax)]
        out["reference_pairs"] = int(ref.size)
        if ref.size == lam.size and ref.size:
            out["max_rel_eig_err_vs_closed_form"] = float(
                np.max(np.abs(np.sort(lam.real) - ref)) / ref.max())
            out["max_abs_imag_rel"] = float(np.abs(lam.imag).max() / ref.max())
    elif rc in (0, 4):
        lam, X, res = S.eigenpairs()
        out["max_residual"] = float(res.max()) if res.size else None
        if wl.B is not None and wl.name.startswith("fem3d_"):  # closed-form Q1 spectrum
            N = round(wl.A.n ** (1.0 / 3.0))
            ev = inputs.fem_q1_eigs((N, N, N))
            ref = ev[(ev > wl.emin) & (ev < wl.emax)]
            out["reference_pairs"] = int(ref.size)
            if ref.size == lam.size and ref.size:
                out["max_rel_eig_err_vs_closed_form"] = float(np.max(np.abs(lam - ref) / ref))
    S.close()
    print(json.dumps(out), flush=True)
    return 0 if rc in (0, 4, 6) else 1


def rr_calls(wl, calls: int) -> int:
    """Time `calls` Rayleigh-Ritz calls on a seeded N(0,1) subspace."""
    import torch
    S = Solver(wl.A, wl.emin, wl.emax, wl.m0, nc=wl.nc, rule=wl.rule, inner=wl.inner,
               inner_iters=wl.inner_iters, alpha=wl.alpha, precision=wl.precision, B=wl.B)
    Q = torch.as_tensor(inputs.initial_subspace(wl.A.n, wl.m0, 3), device="cuda")
    S.set_profiling(True)
    for _ in range(calls):
        X, lam, res = S.rayleigh_ritz(Q)
    torch.cuda.synchronize()
    kt = S.kernel_times()
    out = {"workload": wl.name, "rr_calls": calls,
           "ms_per_call": {k: t / c for k, (c, t) in kt.items()},
           "res_range": [float(res.min()), float(res.max())]}
    S.close()
    print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
