"""Non-Hermitian extension on the CUDA path (real non-symmetric A; Galerkin
Rayleigh-Ritz with a general reduced eigensolver), against the oracle's
ifeast_nonsym / rayleigh_ritz_nonsym and closed-form or dense spectra.

Tolerances: the reduced problem is solved in FP64 by different algorithms
(LAPACK's in the oracle; Householder + complex shifted QR here), so Ritz
values agree to 1e-10 of the largest and residuals to 1e-9. Converged
eigenvalues are checked at the operator's eigenvector condition number
(at most 60 for the upwind operator) times the 1e-10 residual target."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import ifeast_oracle as orc
from paper_1706_00692_gb300 import inputs

pytestmark = pytest.mark.gpu


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
    return Solver(A, emin, emax, m0, nonsymmetric=True, **kw)


def _skew_laplacian(grid=(10, 8), skew=0.35):
    """2D Laplacian plus a skew-symmetric coupling along x: real,
    non-symmetric, with complex-conjugate eigenvalue pairs."""
    L = inputs.laplacian(grid).to_scipy()
    n = L.shape[0]
    off = np.full(n - 1, skew)
    M = (L + sp.diags(off, 1) - sp.diags(off, -1)).tocsr()
    M.sort_indices()
    return inputs.CSR(n, M.indptr.astype(np.int32), M.indices.astype(np.int32),
                      M.data.astype(np.float64))


def _order(theta):
    return np.lexsort((theta.imag, theta.real))


@pytest.mark.parametrize("case,m0", [("upwind", 12), ("upwind", 1), ("skew", 40), ("upwind", 64)])
def test_rayleigh_ritz_nonsym_matches_oracle(torch, case, m0):
    A = inputs.upwind_convection_diffusion((16, 12), 10.0) if case == "upwind" else _skew_laplacian()
    As = A.to_scipy()
    Q = inputs.initial_subspace(A.n, m0, 5)
    S = _solver(A, 0.0, 100.0, m0)
    X, theta, res = S.rayleigh_ritz_nonsym(torch.as_tensor(Q, device="cuda"))
    X, theta, res = X.cpu().numpy(), theta.cpu().numpy(), res.cpu().numpy()
    to, U, LiT = orc.rayleigh_ritz_nonsym(Q, As @ Q)
    Xo = Q @ LiT
    assert np.abs(X - Xo).max() <= 1e-11 * np.abs(Xo).max()
    assert np.abs(X.T @ X - np.eye(m0)).max() <= 1e-10
    # pair each Ritz value with the oracle's nearest one (conjugate pairs share
    # a real part up to rounding, so a sort would not pair them reliably)
    io = np.array([np.argmin(np.abs(to - t)) for t in theta])
    assert np.array_equal(np.sort(io), np.arange(m0))
    scale = np.abs(to).max()
    assert np.abs(theta - to[io]).max() <= 1e-10 * scale
    ro = orc.eigen_residuals(As @ Xo @ U, Xo @ U, to)
    assert np.abs(res - ro[io]).max() <= 1e-9
    S.close()


def test_solve_upwind_matches_closed_form_and_oracle(torch):
    grid, Pe, cnt, m0 = (16, 12), 10.0, 6, 12
    A = inputs.upwind_convection_diffusion(grid, Pe)
    cf = inputs.upwind_convection_diffusion_eigs(grid, Pe)
    emax = 0.5 * (cf[cnt - 1] + cf[cnt])
    X0 = inputs.initial_subspace(A.n, m0, 0)
    S = _solver(A, 0.0, emax, m0, nc=8, rule="trap_half", inner_iters=32, max_outer=40)
    rc = S.solve(X0)
    assert rc == 0, rc
    lam, X, res = S.eigenpairs_complex()
    assert lam.size == cnt
    assert np.abs(lam.real - cf[:cnt]).max() <= 60.0 * 1e-10 * cf[cnt - 1]
    assert np.abs(lam.imag).max() <= 60.0 * 1e-10 * cf[cnt - 1]
    assert res.max() <= 1e-10
    As = A.to_scipy()
    # independent residuals of the returned unit vectors
    assert np.abs(np.linalg.norm(X, axis=0) - 1.0).max() <= 1e-10
    r_cpu = np.linalg.norm(As @ X - X * lam, axis=0) / np.linalg.norm(As @ X, axis=0)
    assert r_cpu.max() <= 2e-10
    z, w = orc.contour_nodes("trap_half", 8, 0.0, emax)
    out = orc.ifeast_nonsym(As, X0, emax / 2, emax / 2, z, w, inner="gmres", k=32, max_outer=40)
    assert out["converged"]
    assert abs(S.stats()["outer_iters"] - out["iters"]) <= 1
    S.close()


def test_full_circle_rule_equals_half_rule(torch):
    grid, Pe, cnt, m0 = (16, 12), 10.0, 6, 12
    A = inputs.upwind_convection_diffusion(grid, Pe)
    cf = inputs.upwind_convection_diffusion_eigs(grid, Pe)
    emax = 0.5 * (cf[cnt - 1] + cf[cnt])
    X0 = inputs.initial_subspace(A.n, m0, 0)
    out = []
    for rule, nc in [("trap_half", 8), ("trap_full", 16)]:
        S = _solver(A, 0.0, emax, m0, nc=nc, rule=rule, inner_iters=32, max_outer=40)
        assert S.solve(X0) == 0
        out.append((S.eigenpairs_complex()[0], S.stats()["outer_iters"]))
        S.close()
    assert out[0][1] == out[1][1]
    assert np.array_equal(out[0][0], out[1][0])  # the same computation


def test_solve_complex_spectrum_matches_dense_eig(torch):
    A = _skew_laplacian()
    emin, emax, m0 = -0.3, 1.0, 11
    c, r = 0.5 * (emin + emax), 0.5 * (emax - emin)
    ev = np.linalg.eigvals(A.to_scipy().toarray())
    inside = ev[np.abs(ev - c) < r]
    inside = inside[_order(inside)]
    assert (np.abs(inside.imag) > 1e-3).sum() >= 2  # a conjugate pair inside
    S = _solver(A, emin, emax, m0, nc=8, rule="trap_half", inner_iters=32, max_outer=40)
    rc = S.solve(inputs.initial_subspace(A.n, m0, 0))
    assert rc == 0, rc
    lam, X, res = S.eigenpairs_complex()
    assert lam.size == inside.size
    assert np.abs(lam - inside).max() <= 1e-9 * np.abs(inside).max()
    assert res.max() <= 1e-10
    As = A.to_scipy()
    r_cpu = np.linalg.norm(As @ X - X * lam, axis=0) / np.linalg.norm(As @ X, axis=0)
    assert r_cpu.max() <= 2e-10
    S.close()


def test_symmetric_entry_points_refuse_nonsymmetric_handles(torch):
    from paper_1706_00692_gb300 import IFEASTError
    A = inputs.upwind_convection_diffusion((6, 5), 10.0)
    S = _solver(A, 0.0, 100.0, 4)
    with pytest.raises(IFEASTError):
        S.eigenpairs()
    S.close()


@pytest.mark.parametrize("grid,cnt,m0,max_iters", [((16, 12), 6, 12, 16), ((30, 24), 10, 20, 20)])
def test_block_correction_solve_matches_oracle(torch, grid, cnt, m0, max_iters):
    """Block correction of the non-symmetric iteration (nonsym_correction=1):
    from the second outer iteration on the systems (z_k I - A) E_k = A X - X C
    replace (z_k I - A) Y_k = X. On 30 x 24 the plain form stalls near 1e-4;
    solved for the correction both sizes reach 1e-10, the closed-form
    eigenvalues (the eigenvector condition number times the target), and the
    oracle's iteration count within one."""
    Pe = 10.0
    A = inputs.upwind_convection_diffusion(grid, Pe)
    cf = inputs.upwind_convection_diffusion_eigs(grid, Pe)
    emax = 0.5 * (cf[cnt - 1] + cf[cnt])
    X0 = inputs.initial_subspace(A.n, m0, 0)
    S = _solver(A, 0.0, emax, m0, nc=8, rule="trap_half", inner_iters=32, max_outer=40,
                nonsym_correction=True)
    rc = S.solve(X0)
    assert rc == 0, rc
    lam, X, res = S.eigenpairs_complex()
    iters = S.stats()["outer_iters"]
    S.close()
    assert lam.size == cnt and iters <= max_iters
    lr = np.sort(lam.real)
    assert np.abs(lr - cf[:cnt]).max() <= 1e4 * 1e-10 * cf[cnt - 1]
    assert np.abs(lam.imag).max() <= 1e4 * 1e-10 * cf[cnt - 1]
    assert res.max() <= 1e-10
    As = A.to_scipy()
    r_cpu = np.linalg.norm(As @ X - X * lam, axis=0) / np.linalg.norm(As @ X, axis=0)
    assert r_cpu.max() <= 2e-10
    z, w = orc.contour_nodes("trap_half", 8, 0.0, emax)
    out = orc.ifeast_nonsym(As, X0, emax / 2, emax / 2, z, w, inner="gmres", k=32, max_outer=40,
                            correction=True)
    assert out["converged"]
    assert abs(iters - out["iters"]) <= 1


def test_block_correction_node_chunks_equal_all_nodes(torch):
    """The block correction with the contour nodes solved two at a time
    (node_chunk=2: each pass adds its nodes' E_k M_k to Q, the first also
    X Re(sum_k w_k M_k)) gives the all-nodes iteration: the same iteration
    count and eigenvalues to rounding."""
    grid, Pe, cnt, m0 = (16, 12), 10.0, 6, 12
    A = inputs.upwind_convection_diffusion(grid, Pe)
    cf = inputs.upwind_convection_diffusion_eigs(grid, Pe)
    emax = 0.5 * (cf[cnt - 1] + cf[cnt])
    X0 = inputs.initial_subspace(A.n, m0, 0)
    out = []
    for chunk in (0, 2):
        S = _solver(A, 0.0, emax, m0, nc=8, rule="trap_half", inner_iters=32, max_outer=40,
                    nonsym_correction=True, node_chunk=chunk)
        assert S.solve(X0) == 0
        out.append((S.eigenpairs_complex()[0], S.stats()["outer_iters"]))
        S.close()
    assert out[0][1] == out[1][1]
    assert np.abs(np.sort(out[0][0].real) - np.sort(out[1][0].real)).max() <= 1e-12 * cf[cnt - 1]
