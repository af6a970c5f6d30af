"""Pins of the oracle's non-Hermitian extension (real non-symmetric A; the
paper states that the method extends, without steps). The test operator is
an upwind convection-diffusion discretisation with a closed-form real
spectrum; it is non-normal (its eigenvector matrix has condition number
(1 + Pe h)^(N/2), 60 at most here), so eigenvalue errors are checked at that
condition number times the residual target."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import ifeast_oracle as orc
from paper_1706_00692_gb300 import inputs


@pytest.mark.parametrize("grid,Pe", [((24, 20), 0.0), ((24, 20), 10.0), ((9, 7), 40.0)])
def test_upwind_closed_form_matches_dense_eig(grid, Pe):
    A = inputs.upwind_convection_diffusion(grid, Pe).to_scipy().toarray()
    if Pe > 0:
        assert np.abs(A - A.T).max() > 1.0  # non-symmetric
    ev = np.linalg.eigvals(A)
    assert np.abs(ev.imag).max() <= 1e-9 * np.abs(ev).max()
    cf = inputs.upwind_convection_diffusion_eigs(grid, Pe)
    assert np.abs(np.sort(ev.real) - cf).max() <= 1e-12 * cf.max()


def _problem(grid=(10, 8), Pe=10.0, cnt=5, m0=9, nc=6, rule="trap_half"):
    A = inputs.upwind_convection_diffusion(grid, Pe)
    cf = inputs.upwind_convection_diffusion_eigs(grid, Pe)
    emax = 0.5 * (cf[cnt - 1] + cf[cnt])
    z, w = orc.contour_nodes(rule, nc, 0.0, emax)
    X = inputs.initial_subspace(A.n, m0, 3)
    return A, cf, emax, z, w, X


def test_exact_filter_equals_spectral_definition():
    A, cf, emax, z, w, X = _problem()
    Ad = A.to_scipy().toarray()
    Q = orc._filtered_subspace_exact(Ad, X, z, w, True)
    Qs = orc.filter_step_spectral_nonsym(Ad, X, z, w, True)
    assert np.abs(Q - Qs).max() <= 1e-10 * np.abs(Qs).max()
    # the filter of a non-normal matrix is not the symmetric formula: U rho U^T X
    # with an orthonormal U would differ
    lam, U = np.linalg.eigh(0.5 * (Ad + Ad.T))
    Qwrong = U @ (orc.filter_rho(lam, z, w, True)[:, None] * (U.T @ X))
    assert np.abs(Q - Qwrong).max() > 1e-3 * np.abs(Q).max()


def test_full_circle_equals_half_rule_for_real_matrix():
    A, cf, emax, zh, wh, X = _problem(nc=6)
    zf, wf = orc.contour_nodes("trap_full", 12, 0.0, emax)
    Ad = A.to_scipy().toarray()
    Qf = orc._filtered_subspace_exact(Ad, X, zf, wf, False)
    Qh = orc._filtered_subspace_exact(Ad, X, zh, wh, True)
    assert np.abs(Qf.imag).max() <= 1e-12 * np.abs(Qf).max()
    assert np.abs(Qf.real - Qh).max() <= 1e-12 * np.abs(Qh).max()


def test_rayleigh_ritz_nonsym_recovers_invariant_subspace():
    A, cf, emax, z, w, X = _problem()
    Ad = A.to_scipy().toarray()
    lam, V = np.linalg.eig(Ad)
    idx = np.argsort(lam.real)[:6]
    g = np.random.default_rng(7)
    Q = V[:, idx].real @ g.standard_normal((6, 6))  # any basis of the invariant subspace
    theta, U, Linv_T = orc.rayleigh_ritz_nonsym(Q, Ad @ Q)
    assert np.abs(np.sort(theta.real) - cf[:6]).max() <= 1e-10 * cf[5]
    assert np.abs(theta.imag).max() <= 1e-10 * cf[5]
    Xb = Q @ Linv_T
    assert np.abs(Xb.T @ Xb - np.eye(6)).max() <= 1e-12
    Vr = Xb @ U
    assert orc.eigen_residuals(Ad @ Vr, Vr, theta).max() <= 1e-10
    # a planted mistake (dropping B_Q = Q^T Q, i.e. projecting on a
    # non-orthonormal basis as if it were orthonormal) is visible
    theta_bad = np.linalg.eigvals(Q.T @ Ad @ Q)
    assert np.abs(np.sort(theta_bad.real) - cf[:6]).max() > 1e-3 * cf[5]


def test_feast_nonsym_converges_to_closed_form():
    grid, Pe, cnt, m0 = (24, 20), 10.0, 8, 14
    A = inputs.upwind_convection_diffusion(grid, Pe)
    cf = inputs.upwind_convection_diffusion_eigs(grid, Pe)
    emax = 0.5 * (cf[cnt - 1] + cf[cnt])
    z, w = orc.contour_nodes("trap_half", 8, 0.0, emax)
    out = orc.ifeast_nonsym(A.to_scipy(), inputs.initial_subspace(A.n, m0, 0), emax / 2, emax / 2,
                            z, w, inner="exact", max_outer=20)
    assert out["converged"]
    th = out["theta"][out["inside"]]
    assert th.size == cnt
    kappa = 60.0
    assert np.abs(np.sort(th.real) - cf[:cnt]).max() <= kappa * 1e-10 * cf[cnt - 1]
    assert np.abs(th.imag).max() <= kappa * 1e-10 * cf[cnt - 1]
    assert out["res"][out["inside"]].max() <= 1e-10


def test_ifeast_nonsym_gmres_converges_to_closed_form():
    grid, Pe, cnt, m0 = (16, 12), 10.0, 6, 12
    A = inputs.upwind_convection_diffusion(grid, Pe)
    cf = inputs.upwind_convection_diffusion_eigs(grid, Pe)
    emax = 0.5 * (cf[cnt - 1] + cf[cnt])
    z, w = orc.contour_nodes("trap_half", 8, 0.0, emax)
    out = orc.ifeast_nonsym(A.to_scipy(), inputs.initial_subspace(A.n, m0, 0), emax / 2, emax / 2,
                            z, w, inner="gmres", k=32, max_outer=40)
    assert out["converged"]
    th = out["theta"][out["inside"]]
    assert th.size == cnt
    assert np.abs(np.sort(th.real) - cf[:cnt]).max() <= 60.0 * 1e-10 * cf[cnt - 1]


def _orthonormal_block(n, m0, seed):
    return np.linalg.qr(inputs.initial_subspace(n, m0, seed))[0]


@pytest.mark.parametrize("perturb", [0.0, 0.3])
def test_correction_filter_equals_exact_filter(perturb):
    """(zI - A)^{-1} X = [X + (zI - A)^{-1} R](zI - C)^{-1} with R = A X - X C
    holds for any C: with GMRES run to the full dimension the correction form
    reproduces the exact filter, for the Galerkin C = X^T A X and for a
    perturbed one."""
    A, cf, emax, z, w, _ = _problem()
    Ad = A.to_scipy().toarray()
    As = A.to_scipy()
    X = _orthonormal_block(A.n, 9, 4)
    C = X.T @ (As @ X)
    if perturb:
        C = C + perturb * np.random.default_rng(7).standard_normal(C.shape) * np.abs(C).max()
    stats = {"inner_steps": []}
    Q = orc._filtered_subspace_gmres_correction_nonsym(As, X, C, z, w, True, A.n, 0.0, stats)
    Qe = orc._filtered_subspace_exact(Ad, X, z, w, True)
    assert np.abs(Q - Qe).max() <= 1e-9 * np.abs(Qe).max()


def test_correction_filter_planted_mistakes_are_caught():
    """A residual with X and C in the wrong order, or (zI - C) applied instead
    of its inverse, moves the exactly solved filter away from the exact one."""
    A, cf, emax, z, w, _ = _problem()
    Ad = A.to_scipy().toarray()
    X = _orthonormal_block(A.n, 9, 4)
    C = X.T @ Ad @ X
    Qe = orc._filtered_subspace_exact(Ad, X, z, w, True)
    I = np.eye(A.n)
    bad1 = np.zeros(X.shape)
    bad2 = np.zeros(X.shape)
    for zk, wk in zip(z, w):
        Rw = Ad @ X - X @ C.T                                     # C transposed
        Ew = np.linalg.solve(zk * I - Ad, Rw.astype(complex))
        bad1 += (wk * np.linalg.solve((zk * np.eye(9) - C).T, (X + Ew).T).T).real
        E = np.linalg.solve(zk * I - Ad, (Ad @ X - X @ C).astype(complex))
        bad2 += (wk * (X + E) @ (zk * np.eye(9) - C)).real          # no inverse
    assert np.abs(bad1 - Qe).max() > 1e-3 * np.abs(Qe).max()
    assert np.abs(bad2 - Qe).max() > 1e-3 * np.abs(Qe).max()


def test_correction_form_converges_where_plain_form_stalls():
    """On the 30 x 24 upwind problem (Pe = 10, the 10 lowest eigenvalues, m0 =
    20, GMRES(32), 8 trapezoid nodes) the plain form's inner error, relative to
    ||x_j||, holds ||R_F|| near 1e-4; solved for the correction from the second
    iteration on, the iteration reaches 1e-10 and the closed-form eigenvalues."""
    grid, Pe, cnt, m0 = (30, 24), 10.0, 10, 20
    A = inputs.upwind_convection_diffusion(grid, Pe)
    cf = inputs.upwind_convection_diffusion_eigs(grid, Pe)
    emax = 0.5 * (cf[cnt - 1] + cf[cnt])
    z, w = orc.contour_nodes("trap_half", 8, 0.0, emax)
    X0 = inputs.initial_subspace(A.n, m0, 0)
    out = orc.ifeast_nonsym(A.to_scipy(), X0, emax / 2, emax / 2, z, w, k=32, max_outer=25,
                            correction=True)
    assert out["converged"] and out["iters"] <= 20
    th = np.sort(out["theta"][out["inside"]].real)
    assert th.size == cnt
    # eigenvector condition number (1 + Pe h)^(N/2) times the residual target
    assert np.abs(th - cf[:cnt]).max() <= 1e4 * 1e-10 * cf[cnt - 1]
