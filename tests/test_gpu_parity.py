"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: the GPU and the oracle evaluate the same FP64 formulas in a
different order (classical Gram-Schmidt applied twice vs modified
Gram-Schmidt; blocked vs sequential sums), so step outputs agree to a few
hundred units in the last place of the largest entry: 1e-11 relative to the
block's max norm for the filter, 1e-12 for products. Converged eigenvalues
must agree to 1e-10 relative and residuals be <= 1e-10 (the target of the
method's stop test)."""
import os

import numpy as np
import pytest

from oracle import ifeast_oracle as orc
from paper_1706_00692_gb300 import inputs

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


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
    return Solver(A, emin, emax, m0, **kw)


def _ragged_problem():
    # n = 1001 rows (ragged against every tiling), 3D stencil with potential
    A = inputs.add_diagonal(inputs.laplacian((13, 11, 7)), inputs.random_potential(1001, 5))
    return A


# ------------------------------------------------------------------ SpMM (row a3)

@pytest.mark.parametrize("shape", [((50, 50), 20, 8), ((13, 11, 7), 7, 5), ((9,), 1, 1)])
def test_spmm_shift_matches_oracle(torch, shape):
    grid, m0, nc = shape
    A = inputs.laplacian(grid)
    A = inputs.add_diagonal(A, inputs.random_potential(A.n, 2))
    S = _solver(A, 0.0, 1.0, m0, nc=nc)
    C = m0 * nc
    g = np.random.default_rng(1)
    V = g.standard_normal((A.n, C)) + 1j * g.standard_normal((A.n, C))
    z = g.standard_normal(nc) + 1j * g.standard_normal(nc)
    W = S.spmm_shift(torch.as_tensor(V, device="cuda"), z).cpu().numpy()
    ref = orc.ref_spmm_shift(A.to_scipy(), V, np.repeat(z, m0))
    assert np.abs(W - ref).max() <= 1e-13 * np.abs(ref).max()
    S.close()


def test_spmm_shift_random_ragged_rows(torch):
    A = inputs.random_sparse_symmetric(777, 6, 3)
    assert (np.diff(A.rowptr) == 1).any()  # rows holding only the diagonal
    S = _solver(A, 0.0, 1.0, 3, nc=11)
    g = np.random.default_rng(4)
    V = g.standard_normal((A.n, 33)) + 1j * g.standard_normal((A.n, 33))
    z = g.standard_normal(11) + 1j * g.standard_normal(11)
    W = S.spmm_shift(torch.as_tensor(V, device="cuda"), z).cpu().numpy()
    ref = orc.ref_spmm_shift(A.to_scipy(), V, np.repeat(z, 3))
    assert np.abs(W - ref).max() <= 1e-13 * np.abs(ref).max()
    S.close()


# ------------------------------------------------------------------ filter (rows a2-a6)

@pytest.mark.parametrize("case", ["lap2d", "ragged"])
@pytest.mark.parametrize("k", [1, 5, 10])
def test_filter_fixed_k_matches_oracle(torch, case, k):
    if case == "lap2d":
        wl = inputs.workload_lap2d_50()
        A, emin, emax, m0, nc = wl.A, wl.emin, wl.emax, wl.m0, wl.nc
    else:
        A, emin, emax, m0, nc = _ragged_problem(), 0.9, 1.4, 7, 5
    X = inputs.initial_subspace(A.n, m0, 11)
    S = _solver(A, emin, emax, m0, nc=nc, inner_iters=k)
    Q, steps = S.apply_filter(torch.as_tensor(X, device="cuda"))
    Q = Q.cpu().numpy()
    z, w = orc.contour_nodes("gl_half", nc, emin, emax)
    stats = {"inner_steps": []}
    Qr = orc._filtered_subspace_gmres(A.to_scipy(), X, z, w, True, k, 0.0, stats)
    assert np.abs(Q - Qr).max() <= 1e-11 * np.abs(Qr).max()
    assert (steps.cpu().numpy() == np.array(stats["inner_steps"])).all()
    S.close()


def test_filter_tolerance_mode_steps_match_oracle(torch):
    A = _ragged_problem()
    m0, nc, emin, emax = 6, 4, 0.9, 1.4
    X = inputs.initial_subspace(A.n, m0, 12)
    S = _solver(A, emin, emax, m0, nc=nc, inner_iters=24, alpha=0.5)
    RF = 0.2  # tolerance alpha * RF = 0.1 of ||x_j||
    Q, steps = S.apply_filter(torch.as_tensor(X, device="cuda"), RF=RF)
    z, w = orc.contour_nodes("gl_half", nc, emin, emax)
    stats = {"inner_steps": []}
    Qr = orc._filtered_subspace_gmres(A.to_scipy(), X, z, w, True, 24, 0.5 * RF, stats)
    st = steps.cpu().numpy()
    ref = np.array(stats["inner_steps"])
    assert (st == ref).all(), (st, ref)
    assert st.min() < 24  # the tolerance, not the cap, stopped the solves
    assert np.abs(Q.cpu().numpy() - Qr).max() <= 1e-11 * np.abs(Qr).max()
    S.close()


# ------------------------------------------------------------------ Rayleigh-Ritz (rows a7-a8)

@pytest.mark.parametrize("n_grid,m0", [((50, 50), 20), ((13, 11, 7), 7), ((13, 11, 7), 1), ((16, 16), 33)])
def test_rayleigh_ritz_matches_oracle(torch, n_grid, m0):
    A = inputs.laplacian(n_grid)
    Q = inputs.initial_subspace(A.n, m0, 3)
    S = _solver(A, 0.0, 8.0, m0)
    X, lam, res = S.rayleigh_ritz(torch.as_tensor(Q, device="cuda"))
    X, lam, res = X.cpu().numpy(), lam.cpu().numpy(), res.cpu().numpy()
    As = A.to_scipy()
    lr, XQ = orc.rayleigh_ritz(Q, As @ Q)
    Xr = Q @ XQ
    rr = orc.eigen_residuals(As @ Xr, Xr, lr)
    assert np.abs(lam - lr).max() <= 1e-12 * np.abs(lr).max()
    assert np.abs(res - rr).max() <= 1e-10
    # Ritz values of a random subspace are simple: compare vectors up to sign
    sgn = np.sign(np.sum(X * Xr, axis=0))
    assert np.abs(X * sgn - Xr).max() <= 1e-9 * np.abs(Xr).max()
    # B_Q-orthonormality of the new basis
    assert np.abs(X.T @ X - np.eye(m0)).max() <= 1e-10
    S.close()


# ------------------------------------------------------------------ full Algorithm 2

def test_solve_lap2d_50_matches_closed_form_and_oracle(torch):
    wl = inputs.workload_lap2d_50()
    S = _solver(wl.A, wl.emin, wl.emax, wl.m0, nc=wl.nc, inner_iters=wl.inner_iters)
    rc = S.solve(wl.X0())
    assert rc == 0, rc
    lam, X, res = S.eigenpairs()
    st = S.stats()
    ref = np.loadtxt(os.path.join(GOLDEN, "lap2d_50x50_lowest11.txt"))[:10]
    assert lam.size == 10
    assert np.abs(lam - ref).max() / np.abs(ref).max() <= 1e-10
    assert res.max() <= 1e-10
    # independent FP64 CPU residual of the returned pairs
    As = wl.A.to_scipy()
    AX = As @ X
    r_cpu = np.linalg.norm(AX - X * lam, axis=0) / np.linalg.norm(AX, axis=0)
    assert r_cpu.max() <= 2e-10
    # eigenspace per cluster vs brute force (lambda_2 = lambda_3, ...)
    e, U = np.linalg.eigh(As.toarray())
    P = X @ X.T
    Pr = U[:, :10] @ U[:, :10].T
    assert np.abs(P - Pr).max() <= 1e-8
    # same iteration count as the oracle within one (rounding decides the last step)
    z, w = orc.contour_nodes("gl_half", wl.nc, wl.emin, wl.emax)
    out = orc.ifeast(As, wl.X0(), wl.emin, wl.emax, z, w, inner="gmres", k=10, max_outer=60)
    assert abs(out["iters"] - st["outer_iters"]) <= 1
    assert st["seq_matvecs"] == 10 * st["outer_iters"]
    # near convergence some x_j span an invariant Krylov space early (happy
    # breakdown) and stop before 10 steps, on both sides
    tot_oracle = sum(h["total_inner"] for h in out["history"])
    assert 0.9 * tot_oracle <= st["total_matvecs"] <= 10 * 160 * st["outer_iters"]
    S.close()


def test_solve_from_device_input_and_workspace_owned_by_library(torch):
    wl = inputs.workload_lap2d_50()
    S = _solver(wl.A, wl.emin, wl.emax, wl.m0, nc=wl.nc, torch_workspace=False)
    rc = S.solve(torch.as_tensor(wl.X0(), device="cuda"))
    assert rc == 0
    lam, X, res = S.eigenpairs(on_device=True)
    assert lam.is_cuda and X.shape == (wl.A.n, 10)
    ref = np.loadtxt(os.path.join(GOLDEN, "lap2d_50x50_lowest11.txt"))[:10]
    assert np.abs(lam.cpu().numpy() - ref).max() / ref.max() <= 1e-10
    # the three output paths give the same vectors: device block, host block of
    # exactly cnt columns, and a wider host block whose extra columns stay untouched
    lam_h, X_h, res_h = S.eigenpairs()
    assert (X.cpu().numpy() == X_h).all() and (res.cpu().numpy() == res_h).all()
    import ctypes as ct
    cap = 13
    wide = np.full((wl.A.n, cap), 7.5)
    m = ct.c_int(0)
    rc = S.lib.ifeast_eigenpairs(S.h, cap, ct.byref(m), None, wide.ctypes.data, None, 0)
    assert rc == 0 and m.value == 10
    assert (wide[:, :10] == X_h).all() and (wide[:, 10:] == 7.5).all()
    S.close()


def test_m0_too_small_and_no_eigenvalues(torch):
    from paper_1706_00692_gb300._lib import IFEAST_ERR_M0_TOO_SMALL, IFEAST_STATUS_NO_EIGENVALUES
    A = inputs.laplacian((12, 12))
    ev = orc.laplacian_closed_form_eigs((12, 12))
    # 12 eigenvalues inside, m0 = 8
    S = _solver(A, 0.0, 0.5 * (ev[11] + ev[12]), 8, nc=8, inner_iters=10, max_outer=8)
    assert S.solve(inputs.initial_subspace(A.n, 8, 0)) == IFEAST_ERR_M0_TOO_SMALL
    S.close()
    # interval in a gap below the spectrum
    S = _solver(A, -1.0, 0.5 * ev[0], 6, nc=8, inner_iters=10, max_outer=3)
    assert S.solve(inputs.initial_subspace(A.n, 6, 0)) == IFEAST_STATUS_NO_EIGENVALUES
    S.close()


def test_not_converged_keeps_last_iterate(torch):
    from paper_1706_00692_gb300._lib import IFEAST_ERR_NOT_CONVERGED
    wl = inputs.workload_lap2d_50()
    S = _solver(wl.A, wl.emin, wl.emax, wl.m0, nc=wl.nc, max_outer=3)
    assert S.solve(wl.X0()) == IFEAST_ERR_NOT_CONVERGED
    lam, X, res = S.eigenpairs()
    assert S.stats()["outer_iters"] == 3 and lam.size >= 1 and np.isfinite(res).all()
    S.close()


@pytest.mark.parametrize("m0,scaled", [(16, False), (20, True), (48, True), (80, True), (80, False),
                                       (96, False), (96, True)])
def test_rayleigh_ritz_update_fp64_accurate(torch, m0, scaled):
    """X = Q X_Q and the residuals computed by the library (on the tensor cores
    for m0 <= 80: exact BF16 digit products of 7-bit digit planes; in FP64
    otherwise) agree with the FP64 oracle's product of the library's own X_Q:
    each X entry to 1e-12 of its row's scale, and the residuals to the FP64
    rounding of the product (a ragged grid so that the last row tile is partial; rows of Q
    scaled over 3 and columns over 6 orders of magnitude, signs mixed)."""
    A = inputs.add_diagonal(inputs.laplacian((17, 13, 9)), inputs.random_potential(1989, 2))
    Q = inputs.initial_subspace(A.n, m0, 5)
    if scaled:
        g = np.random.default_rng(6)
        Q *= 10.0 ** g.uniform(-1.5, 1.5, size=(A.n, 1))
        Q *= 10.0 ** g.uniform(-3, 3, size=(1, m0))
    S = _solver(A, 0.0, 8.0, m0)
    X, lam, res = S.rayleigh_ritz(torch.as_tensor(Q, device="cuda"))
    X, lam, res = X.cpu().numpy(), lam.cpu().numpy(), res.cpu().numpy()
    S.close()
    As = A.to_scipy()
    # the library's X_Q, recovered from its X in FP64 (Q has full column rank);
    # X - Q X_Q then holds the part of the update's error outside span(Q)
    XQ = np.linalg.lstsq(Q, X, rcond=None)[0]
    Xr = Q @ XQ
    rowscale = np.abs(Q).max(axis=1, keepdims=True) * np.abs(XQ).max(axis=0, keepdims=True)
    assert (np.abs(X - Xr) / rowscale).max() <= 1e-12
    AX = As @ X
    nAX = np.linalg.norm(AX, axis=0)
    r = np.linalg.norm(AX - X * lam[None, :], axis=0) / nAX
    # the library forms A X as (A Q) X_Q, this check as A (Q X_Q): in FP64 the
    # two differ by rounding of the size eps |A| |Q| |X_Q| (columnwise), which
    # the scaled cases make far larger than eps ||A X||
    M = np.linalg.norm((abs(As) @ np.abs(Q)) @ np.abs(XQ), axis=0)
    assert (np.abs(res - r) <= 64 * np.finfo(float).eps * M / nAX + 1e-14).all()
    lr, _ = orc.rayleigh_ritz(Q, As @ Q)
    assert np.abs(lam - lr).max() <= 1e-9 * np.abs(lr).max()


@pytest.mark.parametrize("m0", [1, 5, 17, 31, 32, 47, 63, 64, 79, 80])
def test_rayleigh_ritz_tensor_core_shapes(torch, m0):
    """Every chunk shape of the tensor-core Gram (48- and 32-column chunks,
    8-row groups of the M = 128 operand) and update (32- and 16-column chunks)
    on n = 2,011 rows (a partial last 96-row slab and 128-row tile): eigenvalues
    as the oracle's to 1e-12 relative, X^T X = I to 1e-10, and the residuals as
    a CPU FP64 recomputation from the returned X and lambda."""
    A = inputs.add_diagonal(inputs.laplacian((2011,)), inputs.random_potential(2011, 8))
    Q = inputs.initial_subspace(A.n, m0, 31)
    S = _solver(A, 0.0, 2.0, m0)
    X, lam, res = S.rayleigh_ritz(torch.as_tensor(Q, device="cuda"))
    X, lam, res = X.cpu().numpy(), lam.cpu().numpy(), res.cpu().numpy()
    S.close()
    As = A.to_scipy()
    lr, XQ = orc.rayleigh_ritz(Q, As @ Q)
    assert np.abs(lam - lr).max() <= 1e-12 * np.abs(lr).max()
    assert np.abs(X.T @ X - np.eye(m0)).max() <= 1e-10
    assert np.abs(res - orc.eigen_residuals(As @ X, X, lam)).max() <= 1e-10


@pytest.mark.parametrize("m0", [23, 24, 25, 41, 57, 80, 150, 223, 256])
def test_reduced_eig_cluster_sizes(torch, m0):
    """The reduced eigenproblem for m0 >= 24 runs its Jacobi sweeps on an 8-CTA
    cluster (rows of C split ceil(m0 / 8) per CTA; 41 leaves the last CTA
    without rows, 57 with one); 23 stays on one CTA, 256 is the largest m0.
    Eigenvalues as the oracle's Rayleigh-Ritz to 1e-12 relative, X^T X = I to
    1e-10, residuals as a CPU FP64 recomputation from the returned X and lambda."""
    A = inputs.add_diagonal(inputs.laplacian((50, 50)), inputs.random_potential(2500, 12))
    Q = inputs.initial_subspace(A.n, m0, 41)
    S = _solver(A, 0.0, 8.0, m0)
    X, lam, res = S.rayleigh_ritz(torch.as_tensor(Q, device="cuda"))
    X, lam, res = X.cpu().numpy(), lam.cpu().numpy(), res.cpu().numpy()
    S.close()
    As = A.to_scipy()
    lr, _ = orc.rayleigh_ritz(Q, As @ Q)
    assert np.all(np.diff(lam) >= 0)
    assert np.abs(lam - lr).max() <= 1e-12 * np.abs(lr).max()
    assert np.abs(X.T @ X - np.eye(m0)).max() <= 1e-10
    assert np.abs(res - orc.eigen_residuals(As @ X, X, lam)).max() <= 1e-10
