"""Parity of the shared-basis (Lanczos / multi-shift MINRES) inner solver with
the oracle's GMRES on the shift-independent Krylov basis (Section 3), and of
its full solves (FP64 and FP32 inner arithmetic) with brute force.

Tolerances: with few steps the Lanczos basis is orthonormal to rounding, so
the filtered block equals the oracle's (Arnoldi + least squares) to 1e-9
relative in FP64, 2e-5 in FP32 (about 300 times FP32's unit roundoff; measured
worst 2.7e-6 over k <= 10), 1e-2 in FP16 storage and 6e-2 in BF16; converged
eigenvalues agree to 1e-10 relative and residuals are <= 1e-10 in every
precision (the outer iteration is FP64)."""
import os

import numpy as np
import pytest

from oracle import ifeast_oracle as orc
from paper_1706_00692_gb300 import inputs

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
# FP16 storage rounds every Lanczos vector entry to 2^-11 relative; over a few
# steps the filtered block then differs from the FP64 oracle by a few 1e-3 of
# its largest entry
FP16_TOL = 1e-2
# BF16 keeps 8 significant bits (u = 3.9e-3), eight times FP16's rounding
BF16_TOL = 6e-2
# FP32 Lanczos vectors, products and dots (u = 6.0e-8); the recurrence over
# k <= 10 steps and the FP64 least squares on FP32-rounded alpha, beta carry
# the rounding into the coefficients with a growth of a few units per step:
# about 300 u of the block's largest entry
FP32_TOL = 2e-5


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1706_00692_gb300.build import build
    build()
    return t


def _solver(A, emin, emax, m0, **kw):
    from paper_1706_00692_gb300 import Solver
    return Solver(A, emin, emax, m0, inner="minres", **kw)


def _interior_problem():
    A = inputs.add_diagonal(inputs.laplacian((12, 12, 12)), inputs.random_potential(1728, 0))
    ev = np.linalg.eigvalsh(A.to_scipy().toarray())
    i0, cnt = 40, 30
    return A, ev, 0.5 * (ev[i0 - 1] + ev[i0]), 0.5 * (ev[i0 + cnt - 1] + ev[i0 + cnt]), i0, cnt


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", FP32_TOL)])
@pytest.mark.parametrize("k", [1, 4, 10])
def test_filter_matches_oracle_shared_basis(torch, precision, tol, k):
    A = inputs.add_diagonal(inputs.laplacian((13, 11, 7)), inputs.random_potential(1001, 5))
    m0, nc, emin, emax = 7, 5, 0.9, 1.4
    X = inputs.initial_subspace(A.n, m0, 21)
    S = _solver(A, emin, emax, m0, nc=nc, inner_iters=k, precision=precision)
    Q, steps = S.apply_filter(torch.as_tensor(X, device="cuda"))
    z, w = orc.contour_nodes("gl_half", nc, emin, emax)
    stats = {"inner_steps": []}
    Qr = orc._filtered_subspace_shared(A.to_scipy(), X, z, w, True, k, 0.0, stats)
    assert np.abs(Q.cpu().numpy() - Qr).max() <= tol * np.abs(Qr).max()
    assert (steps.cpu().numpy() == k).all()
    S.close()


def test_filter_tolerance_steps_match_oracle(torch):
    A = inputs.add_diagonal(inputs.laplacian((13, 11, 7)), inputs.random_potential(1001, 5))
    m0, nc, emin, emax = 6, 4, 0.9, 1.4
    X = inputs.initial_subspace(A.n, m0, 22)
    S = _solver(A, emin, emax, m0, nc=nc, inner_iters=40, alpha=0.5)
    Q, steps = S.apply_filter(torch.as_tensor(X, device="cuda"), RF=0.2)
    z, w = orc.contour_nodes("gl_half", nc, emin, emax)
    stats = {"inner_steps": []}
    orc._filtered_subspace_shared(A.to_scipy(), X, z, w, True, 40, 0.1, stats)
    st = steps.cpu().numpy()
    ref = np.array(stats["inner_steps"])
    # the stop decision compares |g_{s+1}| with 0.1 ||x_j||; both sides take it in
    # FP64 but on differently rounded least-squares problems, so a pair whose
    # residual sits within rounding of the bound may stop one step apart
    assert np.abs(st - ref).max() <= 1
    assert (st == ref).mean() >= 0.9
    assert st.max() < 40
    S.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16", "bf16"])
def test_solve_lap2d_50(torch, precision):
    wl = inputs.workload_lap2d_50()
    S = _solver(wl.A, wl.emin, wl.emax, wl.m0, nc=wl.nc, inner_iters=200, alpha=1e-2,
                precision=precision)
    rc = S.solve(wl.X0())
    assert rc == 0, rc
    lam, X, res = S.eigenpairs()
    ref = np.loadtxt(os.path.join(GOLDEN, "lap2d_50x50_lowest11.txt"))[:10]
    assert lam.size == 10
    assert np.abs(lam - ref).max() / np.abs(ref).max() <= 1e-10
    assert res.max() <= 1e-10
    AX = wl.A.to_scipy() @ X
    assert (np.linalg.norm(AX - X * lam, axis=0) / np.linalg.norm(AX, axis=0)).max() <= 2e-10
    S.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16", "bf16"])
def test_solve_interior_window_brute_force(torch, precision):
    A, ev, emin, emax, i0, cnt = _interior_problem()
    m0 = 48
    # BF16's outer iteration count is erratic (10, 16 and 35 for three seeds of
    # this problem): its inner solves stall at the 8-bit rounding floor
    S = _solver(A, emin, emax, m0, nc=8, inner_iters=400, alpha=1e-3, precision=precision,
                max_outer=60 if precision == "bf16" else 30)
    rc = S.solve(inputs.initial_subspace(A.n, m0, 1))
    assert rc == 0, (rc, S.stats())
    lam, X, res = S.eigenpairs()
    assert lam.size == cnt
    assert np.abs(lam - ev[i0:i0 + cnt]).max() / np.abs(ev).max() <= 1e-10
    assert res.max() <= 1e-10
    st = S.stats()
    # 16-bit storage stagnates the inner solves above their target more often;
    # with BF16's 8-bit significands most iterations do (converged within the cap)
    assert st["outer_iters"] <= {"fp64": 12, "fp32": 12, "fp16": 20, "bf16": 60}[precision]
    S.close()


def _arrow_matrix(n, seed):
    """Random symmetric sparse matrix plus a dense first row and column: rows of
    every length from 1 to n non-zeros (the long row is split into chunks by
    the SpMM kernels)."""
    B = inputs.random_sparse_symmetric(n, 4, seed).to_scipy().tolil()
    g = np.random.default_rng(seed)
    v = g.standard_normal(n) * 0.1
    B[0, :] = v
    B[:, 0] = v.reshape(-1, 1)
    B[0, 0] = 3.0
    B = B.tocsr()
    B.sort_indices()
    return inputs.CSR(n, B.indptr.astype(np.int32), B.indices.astype(np.int32), B.data.astype(np.float64))


@pytest.mark.parametrize("m0,precision,tol", [(8, "fp32", FP32_TOL), (8, "fp64", 1e-9),
                                              (7, "fp32", FP32_TOL), (36, "fp32", FP32_TOL),
                                              (8, "fp16", FP16_TOL), (8, "bf16", BF16_TOL)])
def test_filter_long_and_short_rows(torch, m0, precision, tol):
    A = _arrow_matrix(517, 3)
    assert np.diff(A.rowptr).max() > 64 and np.diff(A.rowptr).min() <= 4
    nc, emin, emax = 3, 0.5, 1.5
    X = inputs.initial_subspace(A.n, m0, 23)
    S = _solver(A, emin, emax, m0, nc=nc, inner_iters=5, precision=precision)
    Q, steps = S.apply_filter(torch.as_tensor(X, device="cuda"))
    z, w = orc.contour_nodes("gl_half", nc, emin, emax)
    Qr = orc._filtered_subspace_shared(A.to_scipy(), X, z, w, True, 5, 0.0, {"inner_steps": []})
    assert np.abs(Q.cpu().numpy() - Qr).max() <= tol * np.abs(Qr).max()
    S.close()


def _ell_case(kind):
    """Matrices for the fixed-width FP32 step kernel (m0 % 4 == 0, rows of at
    most 16 slots): rows without a stored diagonal entry (slot 0 then holds a
    zero), rows filling all 8 slots, and 9-point rows (16 slots)."""
    import scipy.sparse as sp
    if kind == "no_diag":
        B = inputs.random_sparse_symmetric(1001, 1, 7).to_scipy().tolil()
        for i in range(0, 1001, 3):
            B[i, i] = 0.0
        B = B.tocsr()
        B.eliminate_zeros()
    elif kind == "full8":
        L = inputs.add_diagonal(inputs.laplacian((13, 11, 7)), inputs.random_potential(1001, 5))
        n = L.n
        i = np.arange(n // 2)
        far = sp.coo_matrix((np.full(i.size, 0.3), (i, n - 1 - i)), shape=(n, n))
        B = (L.to_scipy() + far + far.T).tocsr()
    else:
        B = inputs.fem_q1((23, 19))[0].to_scipy()
    B.sort_indices()
    return inputs.CSR(B.shape[0], B.indptr.astype(np.int32), B.indices.astype(np.int32),
                      B.data.astype(np.float64))


@pytest.mark.parametrize("kind", ["no_diag", "full8", "fem9"])
@pytest.mark.parametrize("m0,precision", [(12, "fp32"), (40, "fp32"), (12, "fp16"),
                                          (12, "bf16")])
def test_filter_fixed_width_rows(torch, kind, m0, precision):
    A = _ell_case(kind)
    lens = np.diff(A.rowptr)
    if kind == "no_diag":
        diag = np.array([(A.colidx[A.rowptr[r]:A.rowptr[r + 1]] == r).any() for r in range(A.n)])
        assert (~diag).any() and (lens + ~diag).max() <= 8
    elif kind == "full8":
        assert lens.max() == 8
    else:
        assert 8 < lens.max() <= 16
    nc = 4
    Sd = A.to_scipy()
    ev = np.linalg.eigvalsh(Sd.toarray())
    emin, emax = 0.5 * (ev[10] + ev[11]), 0.5 * (ev[30] + ev[31])
    X = inputs.initial_subspace(A.n, m0, 24)
    S = _solver(A, emin, emax, m0, nc=nc, inner_iters=6, precision=precision)
    Q, steps = S.apply_filter(torch.as_tensor(X, device="cuda"))
    z, w = orc.contour_nodes("gl_half", nc, emin, emax)
    Qr = orc._filtered_subspace_shared(Sd, X, z, w, True, 6, 0.0, {"inner_steps": []})
    tol = {"fp32": FP32_TOL, "fp16": FP16_TOL, "bf16": BF16_TOL}[precision]
    assert np.abs(Q.cpu().numpy() - Qr).max() <= tol * np.abs(Qr).max()
    assert (steps.cpu().numpy() == 6).all()
    S.close()


@pytest.mark.parametrize("k", [1, 4, 10])
def test_filter_fp16_storage_matches_oracle(torch, k):
    A = inputs.add_diagonal(inputs.laplacian((13, 11, 7)), inputs.random_potential(1001, 5))
    m0, nc, emin, emax = 8, 5, 0.9, 1.4
    X = inputs.initial_subspace(A.n, m0, 21)
    S = _solver(A, emin, emax, m0, nc=nc, inner_iters=k, precision="fp16")
    Q, steps = S.apply_filter(torch.as_tensor(X, device="cuda"))
    z, w = orc.contour_nodes("gl_half", nc, emin, emax)
    Qr = orc._filtered_subspace_shared(A.to_scipy(), X, z, w, True, k, 0.0, {"inner_steps": []})
    err = np.abs(Q.cpu().numpy() - Qr).max() / np.abs(Qr).max()
    assert err <= FP16_TOL, err
    assert (steps.cpu().numpy() == k).all()
    S.close()


@pytest.mark.parametrize("case,precision,m0,alpha", [
    ("lap2d", "fp32", 20, 0.0),       # fixed-width rows, fixed step count
    ("ragged", "fp32", 12, 0.5),      # tolerance mode: columns stop at different steps
    ("arrow", "fp32", 8, 0.0),        # CSR kernel (rows longer than 16)
    ("ragged", "fp16", 8, 0.5),       # FP16 storage
])
def test_two_pass_filter_is_bit_identical(torch, case, precision, m0, alpha):
    if case == "lap2d":
        A = inputs.workload_lap2d_50().A
        emin, emax = 0.0, 0.07
    elif case == "ragged":
        A = inputs.add_diagonal(inputs.laplacian((13, 11, 7)), inputs.random_potential(1001, 5))
        emin, emax = 0.9, 1.4
    else:
        A = _arrow_matrix(517, 3)
        emin, emax = 0.5, 1.5
    X = torch.as_tensor(inputs.initial_subspace(A.n, m0, 31), device="cuda")
    out = []
    for two_pass in (False, True):
        S = _solver(A, emin, emax, m0, nc=5, inner_iters=60, alpha=alpha, precision=precision,
                    two_pass=two_pass)
        Q, steps = S.apply_filter(X, RF=0.2)
        out.append((Q.cpu().numpy(), steps.cpu().numpy()))
        S.close()
    assert np.array_equal(out[0][1], out[1][1])
    if alpha > 0:
        assert out[0][1].min() < out[0][1].max()  # the columns stopped at different steps
    assert np.array_equal(out[0][0], out[1][0])


def test_two_pass_solve_is_bit_identical(torch):
    A, ev, emin, emax, i0, cnt = _interior_problem()
    m0 = 48
    res = []
    for two_pass in (False, True):
        S = _solver(A, emin, emax, m0, nc=8, inner_iters=400, alpha=1e-3, precision="fp32",
                    max_outer=30, two_pass=two_pass)
        assert S.solve(inputs.initial_subspace(A.n, m0, 1)) == 0
        lam, X, r = S.eigenpairs()
        res.append((lam, X, S.stats()["outer_iters"]))
        S.close()
    assert res[0][2] == res[1][2]
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1], res[1][1])
    assert np.abs(res[1][0] - ev[i0:i0 + cnt]).max() / np.abs(ev).max() <= 1e-10


def test_sampled_profiling_counts(torch):
    """set_profiling(N): the chained Lanczos-loop kernels (the step kernel, the
    reduction of its partials to alpha_s, beta_{s+1}, and the Givens batches)
    are timed at launches 1, 1 + N, ... of each class, every other kernel at
    every launch, and all launches are counted; one Givens batch covers at
    most 16 steps."""
    from paper_1706_00692_gb300 import Solver
    A, ev, emin, emax, i0, cnt = _interior_problem()
    S = Solver(A, emin, emax, 2 * cnt, nc=8, rule="trap_half", inner="minres", inner_iters=300,
               alpha=3e-2, precision="fp32", max_outer=3)
    S.set_profiling(4)
    S.kernel_times(reset=True)
    S.kernel_launches(reset=True)
    S.solve(inputs.initial_subspace(A.n, 2 * cnt, 0))
    timed = S.kernel_times(reset=True)
    launches = S.kernel_launches(reset=True)
    S.set_profiling(False)
    for k, n in launches.items():
        c = timed[k][0]
        if k in ("lanczos_step", "lanczos_reduce", "lanczos_givens"):
            assert c == (n + 3) // 4, (k, n, c)
        else:
            assert c == n, (k, n, c)
    assert launches["lanczos_step"] > 8
    assert launches["lanczos_reduce"] == launches["lanczos_step"]
    assert launches["lanczos_step"] <= 16 * launches["lanczos_givens"]
    S.close()


def _golden_window():
    path = os.path.join(GOLDEN, "lap3d64_window.txt")
    data = np.loadtxt(path)
    return data[data[:, 2] == 1, 0]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_full_size_lap3d_64_against_oracle(torch, precision):
    """The bench's 64^3 workload in the bench's configuration (n = 262,144,
    m0 = 80, 8 trapezoid nodes, shared-basis MINRES, FP32 inner or the plain
    FP64 form): the 56 eigenvalues of the window equal the CPU oracle's
    (shift-invert Lanczos, tests/golden/lap3d64_window.txt) to 1e-10 relative,
    each pair has an independent FP64 residual ||A x - lam x|| / ||A x|| <= 2e-10
    recomputed on the CPU, and the vectors are orthonormal."""
    from paper_1706_00692_gb300 import Solver
    wl = inputs.workload_lap3d_64_interior(precision=precision)
    if precision == "fp64":
        # the stored FP64 basis (1501 x n x m0 doubles) needs ~252 GB of the device
        torch.cuda.empty_cache()
        free, _ = torch.cuda.mem_get_info()
        need = 1501 * wl.A.n * wl.m0 * 8 + (8 << 30)
        if free < need:
            pytest.skip(f"FP64 basis needs {need / 2**30:.0f} GiB, {free / 2**30:.0f} GiB free")
    S = Solver(wl.A, wl.emin, wl.emax, wl.m0, nc=wl.nc, rule=wl.rule, inner=wl.inner,
               inner_iters=wl.inner_iters, alpha=wl.alpha, precision=wl.precision)
    rc = S.solve(wl.X0())
    lam, X, res = S.eigenpairs()
    S.close()
    del S
    torch.cuda.empty_cache()
    assert rc == 0, rc
    ref = _golden_window()
    assert lam.size == ref.size == wl.expected_count == 56
    assert np.abs(lam - ref).max() <= 1e-10 * np.abs(ref).max()
    assert res.max() <= 1e-10
    As = wl.A.to_scipy()
    AX = As @ X
    r = np.linalg.norm(AX - X * lam[None, :], axis=0) / np.linalg.norm(AX, axis=0)
    assert r.max() <= 2e-10
    assert np.abs(X.T @ X - np.eye(lam.size)).max() <= 1e-9
