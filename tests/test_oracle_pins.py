"""Pins for the CPU oracle: each checks it against something other than itself
(closed forms, brute force, the spectral definition, library solvers)."""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import ifeast_oracle as orc
from paper_1706_00692_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- contour / filter

@pytest.mark.parametrize("N", [4, 8, 16])
@pytest.mark.parametrize("t", [0.0, 0.3, 0.9, 1.2, 2.0, -0.7, -1.5])
def test_trapezoid_filter_closed_form(N, t):
    """N offset trapezoid nodes on the full circle give rho(t) = 1/(1+t^N),
    t=(lambda-c)/r; the half-contour form with N/2 upper nodes is identical."""
    emin, emax = -1.0, 3.0
    c, r = 1.0, 2.0
    lam = c + t * r
    z, w = orc.contour_nodes(orc.TRAP_FULL, N, emin, emax)
    full = orc.filter_rho(np.array([lam]), z, w, half=False)[0]
    assert abs(full - 1.0 / (1.0 + t ** N)) < 1e-13
    zh, wh = orc.contour_nodes(orc.TRAP_HALF, N // 2, emin, emax)
    half = orc.filter_rho(np.array([lam]), zh, wh, half=True)[0]
    assert abs(half - 1.0 / (1.0 + t ** N)) < 1e-13


def test_trapezoid_value_16_nodes():
    z, w = orc.contour_nodes(orc.TRAP_HALF, 8, 0.0, 2.0)
    assert abs(orc.filter_rho(np.array([1.0 + 1.2]), z, w, True)[0] - 1 / (1 + 1.2 ** 16)) < 1e-14


@pytest.mark.parametrize("nc", [4, 8, 12])
def test_gl_half_centre_is_one(nc):
    """At the centre every term is w_k/(r e^{i theta_k}) = g_k/2 and the
    Gauss-Legendre weights sum to 2."""
    z, w = orc.contour_nodes(orc.GL_HALF, nc, 2.0, 5.0)
    assert abs(orc.filter_rho(np.array([3.5]), z, w, True)[0] - 1.0) < 1e-14


def test_gl_half_tends_to_indicator():
    """Exact contour integral of 1/(z-lambda) is 1 inside, 0 outside."""
    z, w = orc.contour_nodes(orc.GL_HALF, 48, -1.0, 1.0)
    inside = orc.filter_rho(np.linspace(-0.6, 0.6, 13), z, w, True)
    outside = orc.filter_rho(np.concatenate([np.linspace(-5, -1.6, 7), np.linspace(1.6, 5, 7)]), z, w, True)
    assert np.abs(inside - 1).max() < 1e-9
    assert np.abs(outside).max() < 1e-9


def test_half_contour_equals_full_circle_gl():
    """Half contour with its folded weights equals the full-circle Gauss-Legendre
    sum obtained by mirroring the nodes into the lower half plane."""
    z, w = orc.contour_nodes(orc.GL_HALF, 8, 0.5, 2.5)
    zf = np.concatenate([z, z.conj()])
    wf = np.concatenate([w, w.conj()]) / 2.0
    lam = np.linspace(-2, 5, 31)
    a = orc.filter_rho(lam, z, w, True)
    b = orc.filter_rho(lam, zf, wf, False)
    assert np.abs(b.imag).max() < 1e-13
    assert np.abs(a - b.real).max() < 1e-13


# ---------------------------------------------------------------- stencils

@pytest.mark.parametrize("grid", [(7,), (7, 5), (4, 5, 3)])
def test_laplacian_generator_closed_form(grid):
    A = inputs.laplacian(grid).to_scipy().toarray()
    assert np.allclose(A, A.T)
    ev = np.linalg.eigvalsh(A)
    assert np.abs(ev - orc.laplacian_closed_form_eigs(grid)).max() < 1e-12
    assert np.abs(ev - inputs.laplacian_eigs(grid)).max() < 1e-12


def test_golden_lap2d_50():
    vals = np.loadtxt(os.path.join(GOLDEN, "lap2d_50x50_lowest11.txt"))
    A = inputs.laplacian((50, 50)).to_scipy().toarray()
    ev = np.linalg.eigvalsh(A)[:11]
    assert np.abs(ev - vals).max() < 1e-12
    wl = inputs.workload_lap2d_50()
    assert abs(wl.emax - 0.5 * (vals[9] + vals[10])) < 1e-15


def test_potential_weyl_bounds():
    """lam_j(L) <= lam_j(L + diag(U[0,1))) <= lam_j(L) + 1."""
    L = inputs.laplacian((6, 5, 4))
    A = inputs.add_diagonal(L, inputs.random_potential(L.n, 3))
    el = np.linalg.eigvalsh(L.to_scipy().toarray())
    ea = np.linalg.eigvalsh(A.to_scipy().toarray())
    assert np.all(ea >= el - 1e-12) and np.all(ea <= el + 1 + 1e-12)
    B = inputs.add_diagonal_fast(L, inputs.random_potential(L.n, 3))
    assert np.array_equal(A.val, B.val)


# ---------------------------------------------------------------- GMRES

def _rand_complex_matrix(n, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal((n, n)) + 1j * g.standard_normal((n, n)) + 4 * np.eye(n)


def test_gmres_full_dimension_is_exact():
    n = 12
    M = _rand_complex_matrix(n, 1)
    b = np.random.default_rng(2).standard_normal(n)
    out = orc.gmres(lambda v: M @ v, b, n)
    assert np.abs(out["y"] - np.linalg.solve(M, b)).max() < 1e-10


@pytest.mark.parametrize("k", [1, 3, 6])
def test_gmres_minimal_residual_brute_force(k):
    """GMRES returns the minimiser of ||b - M y|| over K_k(M, b): compare with
    lstsq on an orthonormalised explicit Krylov matrix."""
    n = 15
    M = _rand_complex_matrix(n, 5)
    b = np.random.default_rng(6).standard_normal(n).astype(np.complex128)
    K = np.zeros((n, k), np.complex128)
    v = b.copy()
    for j in range(k):
        K[:, j] = v
        v = M @ v
    Qk, _ = np.linalg.qr(K)
    c = np.linalg.lstsq(M @ Qk, b, rcond=None)[0]
    y_bf = Qk @ c
    out = orc.gmres(lambda x: M @ x, b, k)
    assert out["steps"] == k
    assert np.abs(out["y"] - y_bf).max() < 1e-9 * np.abs(y_bf).max()
    true_res = np.linalg.norm(b - M @ out["y"])
    assert abs(out["res_est"] - true_res) < 1e-10 * np.linalg.norm(b)


def test_gmres_tolerance_stop_is_first_step_below():
    n = 30
    M = _rand_complex_matrix(n, 8)
    b = np.random.default_rng(9).standard_normal(n)
    full = [orc.gmres(lambda x: M @ x, b, s)["res_est"] for s in range(1, 20)]
    tol = 0.5 * (full[6] + full[7]) / np.linalg.norm(b)
    out = orc.gmres(lambda x: M @ x, b, 19, tol_rel=tol)
    first = next(i for i, r in enumerate(full) if r <= tol * np.linalg.norm(b)) + 1
    assert out["steps"] == first


def test_shifted_gmres_shared_basis_equals_per_shift():
    """Section 3: the Krylov basis of (zI - A) does not depend on z, so GMRES on
    the real basis of K(A, x) with the shifted Hessenberg gives the same y."""
    A = inputs.add_diagonal(inputs.laplacian((8, 7)), inputs.random_potential(56, 1)).to_scipy()
    x = np.random.default_rng(4).standard_normal(56)
    for z in [0.3 + 0.2j, 1.7 + 0.05j, 4.0 + 1.0j]:
        a = orc.gmres(lambda v: orc.shifted_apply(A, z, v), x, 10)
        b = orc.gmres_shared_basis(A, x, z, 10)
        assert np.abs(a["y"] - b["y"]).max() < 1e-10 * np.abs(a["y"]).max()
        assert abs(a["res_est"] - b["res_est"]) < 1e-10 * np.linalg.norm(x)


# ---------------------------------------------------------------- FEAST / IFEAST

def _small_problem():
    A = inputs.laplacian((12, 12))
    ev = orc.laplacian_closed_form_eigs((12, 12))
    emin, emax = 0.0, 0.5 * (ev[5] + ev[6])
    return A, ev, emin, emax


def test_exact_filter_step_matches_spectral_definition():
    """Alg. 1 steps 1-2 with dense LU equal U rho(Lambda) U^T X (Eq. rhoh)."""
    A, ev, emin, emax = _small_problem()
    Ad = A.to_scipy().toarray()
    z, w = orc.contour_nodes(orc.GL_HALF, 8, emin, emax)
    X = inputs.initial_subspace(A.n, 9, 0)
    Q_lu = orc._filtered_subspace_exact(Ad, X, z, w, True)
    Q_sp = orc.filter_step_spectral(Ad, X, z, w, True)
    assert np.abs(Q_lu - Q_sp).max() < 1e-11 * np.abs(Q_sp).max()


def test_feast_exact_matches_brute_force():
    A, ev, emin, emax = _small_problem()
    z, w = orc.contour_nodes(orc.GL_HALF, 8, emin, emax)
    out = orc.feast(A.to_scipy(), inputs.initial_subspace(A.n, 10, 1), emin, emax, z, w)
    assert out["converged"]
    lam = out["lam"][out["inside"]]
    assert lam.size == 6
    assert np.abs(lam - ev[:6]).max() < 1e-12
    # spectral projector of the wanted cluster
    Ad = A.to_scipy().toarray()
    e, U = np.linalg.eigh(Ad)
    P_ref = U[:, :6] @ U[:, :6].T
    Xi = out["X"][:, out["inside"]]
    P = Xi @ Xi.T
    assert np.abs(P - P_ref).max() < 1e-9


def test_ifeast_exact_inner_reproduces_feast():
    """Solving the shifted systems to full accuracy turns Algorithm 2 into
    Algorithm 1: compare Ritz values iterate by iterate."""
    A, ev, emin, emax = _small_problem()
    z, w = orc.contour_nodes(orc.GL_HALF, 6, emin, emax)
    X0 = inputs.initial_subspace(A.n, 9, 2)
    h1, h2 = [], []
    orc.ifeast(A.to_scipy(), X0, emin, emax, z, w, inner="exact", max_outer=3, tol=0.0,
               callback=lambda it, lam, X, res, ins: h1.append(lam.copy()))
    orc.ifeast(A.to_scipy(), X0, emin, emax, z, w, inner="gmres", k=A.n, max_outer=3, tol=0.0,
               callback=lambda it, lam, X, res, ins: h2.append(lam.copy()))
    assert len(h1) == len(h2) == 3
    for a, b in zip(h1, h2):
        # wanted Ritz values (inside the interval) to 1e-10; the unwanted ones,
        # which the filter damps, carry the rounding of the 144-step Krylov run
        ins = (a > emin) & (a < emax)
        assert np.abs(a[ins] - b[ins]).max() < 1e-10 * np.abs(a).max()
        assert np.abs(a - b).max() < 1e-7 * np.abs(a).max()


def test_rayleigh_ritz_recovers_exact_pairs():
    A, ev, emin, emax = _small_problem()
    Ad = A.to_scipy().toarray()
    e, U = np.linalg.eigh(Ad)
    g = np.random.default_rng(3)
    Msix = g.standard_normal((6, 6))
    Q = U[:, [0, 3, 7, 9, 20, 40]] @ Msix
    lam, XQ = orc.rayleigh_ritz(Q, Ad @ Q)
    assert np.abs(lam - e[[0, 3, 7, 9, 20, 40]]).max() < 1e-9  # cond(Msix) ~ 1e2
    Bq = Q.T @ Q
    assert np.abs(XQ.T @ Bq @ XQ - np.eye(6)).max() < 1e-10


def test_residual_definition():
    lam = np.array([1.0, 2.0])
    X = np.eye(3)[:, :2]
    AX = np.array([[1.0, 0.0], [0.0, 2.0], [0.0, 0.5]])
    r = orc.eigen_residuals(AX, X, lam)
    assert abs(r[0]) < 1e-16 and abs(r[1] - 0.5 / math.hypot(2.0, 0.5)) < 1e-15


@pytest.mark.slow
def test_ifeast_gmres10_lap2d_50_converges_to_closed_form():
    """The 50x50 workload: 8 Gauss-Legendre half-circle nodes, m0=20, GMRES
    fixed at 10 steps, converges to relative residual <= 1e-10 and the 10
    eigenvalues equal the closed form to 1e-10 relative."""
    wl = inputs.workload_lap2d_50()
    z, w = orc.contour_nodes(orc.GL_HALF, 8, wl.emin, wl.emax)
    out = orc.ifeast(wl.A.to_scipy(), wl.X0(), wl.emin, wl.emax, z, w, inner="gmres", k=10,
                     alpha=0.0, tol=1e-10, max_outer=60)
    assert out["converged"]
    lam = out["lam"][out["inside"]]
    ref = np.loadtxt(os.path.join(GOLDEN, "lap2d_50x50_lowest11.txt"))[:10]
    assert lam.size == 10
    assert np.abs(lam - ref).max() / np.abs(ref).max() < 1e-10
    assert out["res"][out["inside"]].max() <= 1e-10


def test_convergence_rate_bound_exact_solves():
    """With exact solves (alpha_j = 0) Eq. (upperbound) reduces to the subspace
    iteration rate |gamma_{m0+1}|/|gamma_j|: the error of the wanted subspace
    (sine of the largest principal angle) shrinks at least that fast."""
    A, ev, emin, emax = _small_problem()
    Ad = A.to_scipy().toarray()
    e, U = np.linalg.eigh(Ad)
    z, w = orc.contour_nodes(orc.GL_HALF, 4, emin, emax)
    m0 = 8
    gam = np.sort(np.abs(orc.filter_rho(e, z, w, True)))[::-1]
    rate = gam[m0] / gam[5]
    errs = []

    def cb(it, lam, X, res, ins):
        Xq, _ = np.linalg.qr(X)
        s = sla.subspace_angles(U[:, :6], Xq)
        errs.append(np.sin(s.max()))

    orc.ifeast(A.to_scipy(), inputs.initial_subspace(A.n, m0, 7), emin, emax, z, w, inner="exact",
               max_outer=4, tol=0.0, callback=cb)
    for a, b in zip(errs[:-1], errs[1:]):
        if a > 1e-12:
            assert b <= 1.5 * rate * a + 1e-13


def test_residual_form_identity_exact_solves():
    """(zI - A)^{-1} x = (x + (zI - A)^{-1}(A x - lam x)) / (z - lam) for any
    scalar lam: the right-hand side the shared-basis inner solver uses after
    the first outer iteration. Checked with dense LU on a random Ritz pair."""
    A = inputs.add_diagonal(inputs.laplacian((7, 6)), inputs.random_potential(42, 9))
    Ad = A.to_scipy().toarray()
    x = inputs.initial_subspace(42, 1, 3)[:, 0]
    lam = x @ Ad @ x / (x @ x)
    for z in [0.5 + 0.3j, 3.0 + 0.01j]:
        M = z * np.eye(42) - Ad
        lhs = np.linalg.solve(M, x)
        rhs = (x + np.linalg.solve(M, Ad @ x - lam * x)) / (z - lam)
        assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(lhs).max()


# ---------------------------------------------------------------- generalized problem A x = lam B x

@pytest.mark.parametrize("grid", [(9,), (7, 6), (4, 5, 3)])
def test_fem_generator_closed_form(grid):
    """Q1 stiffness/mass pencil: eigenvalues sum_d (6/h^2)(1 - cos t)/(2 + cos t)."""
    K, M = inputs.fem_q1(grid)
    Kd, Md = K.to_scipy().toarray(), M.to_scipy().toarray()
    assert np.allclose(Kd, Kd.T) and np.allclose(Md, Md.T)
    assert np.linalg.eigvalsh(Md).min() > 0
    ev = sla.eigh(Kd, Md, eigvals_only=True)
    ref = inputs.fem_q1_eigs(grid)
    assert np.abs(ev - ref).max() <= 1e-10 * ref.max()
    assert np.array_equal(K.rowptr, M.rowptr) and np.array_equal(K.colidx, M.colidx)


def _fem_problem():
    K, M = inputs.fem_q1((10, 9))
    ev = inputs.fem_q1_eigs((10, 9))
    return K, M, ev, 0.0, 0.5 * (ev[5] + ev[6])


def test_generalized_exact_filter_matches_spectral_definition():
    K, M, ev, emin, emax = _fem_problem()
    Kd, Md = K.to_scipy().toarray(), M.to_scipy().toarray()
    z, w = orc.contour_nodes(orc.GL_HALF, 8, emin, emax)
    X = inputs.initial_subspace(K.n, 9, 4)
    Q_lu = orc._filtered_subspace_exact(Kd, X, z, w, True, Md)
    Q_sp = orc.filter_step_spectral(Kd, X, z, w, True, Md)
    assert np.abs(Q_lu - Q_sp).max() < 1e-10 * np.abs(Q_sp).max()


def test_generalized_feast_matches_brute_force():
    K, M, ev, emin, emax = _fem_problem()
    z, w = orc.contour_nodes(orc.GL_HALF, 8, emin, emax)
    out = orc.feast(K.to_scipy(), inputs.initial_subspace(K.n, 10, 1), emin, emax, z, w,
                    B=M.to_scipy())
    assert out["converged"]
    lam = out["lam"][out["inside"]]
    assert lam.size == 6
    assert np.abs(lam - ev[:6]).max() <= 1e-11 * ev[5]
    X = out["X"][:, out["inside"]]
    Md = M.to_scipy().toarray()
    assert np.abs(X.T @ Md @ X - np.eye(6)).max() < 1e-9  # B-orthonormal Ritz vectors


def test_generalized_ifeast_exact_inner_reproduces_feast():
    K, M, ev, emin, emax = _fem_problem()
    z, w = orc.contour_nodes(orc.GL_HALF, 6, emin, emax)
    X0 = inputs.initial_subspace(K.n, 9, 2)
    h1, h2 = [], []
    orc.ifeast(K.to_scipy(), X0, emin, emax, z, w, inner="exact", max_outer=3, tol=0.0,
               B=M.to_scipy(), callback=lambda it, lam, X, res, ins: h1.append(lam.copy()))
    orc.ifeast(K.to_scipy(), X0, emin, emax, z, w, inner="gmres", k=K.n, max_outer=3, tol=0.0,
               B=M.to_scipy(), callback=lambda it, lam, X, res, ins: h2.append(lam.copy()))
    for a, b in zip(h1, h2):
        ins = (a > emin) & (a < emax)
        assert np.abs(a[ins] - b[ins]).max() < 1e-9 * np.abs(a).max()


# ---------------------------------------------------------------- residual form of the GMRES filter

def _correction_case(B_too):
    if B_too:
        A, B = inputs.fem_q1((6, 5))
        Bs = B.to_scipy()
    else:
        A, Bs = inputs.add_diagonal(inputs.laplacian((6, 5)), inputs.random_potential(30, 4)), None
    As = A.to_scipy()
    X = inputs.initial_subspace(30, 4, 8)
    lam = np.array([0.3, 1.7, 2.2, 9.0])  # any scalars off the contour
    return As, Bs, X, lam


@pytest.mark.parametrize("B_too", [False, True])
def test_gmres_correction_filter_equals_plain_filter_with_exact_solves(B_too):
    """With GMRES run to n steps (an exact solve), the residual-form filter
    sum_k w_k (x_j + (z_k B - A)^{-1} r_j) / (z_k - lam_j) equals the plain
    filter sum_k w_k (z_k B - A)^{-1} B x_j (dense LU) for every lam_j: the
    identity (z B - A)^{-1} B x = (x + (z B - A)^{-1}(A x - lam B x)) / (z - lam)."""
    As, Bs, X, lam = _correction_case(B_too)
    z, w = orc.contour_nodes("gl_half", 5, 0.0, 4.0 if not B_too else 400.0)
    ref = orc._filtered_subspace_exact(As.toarray(), X, z, w, True,
                                       None if Bs is None else Bs.toarray())
    got = orc._filtered_subspace_gmres_correction(As, X, lam, z, w, True, 30, 0.0,
                                                  {"inner_steps": []}, Bs)
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


def test_gmres_correction_filter_mutations_fail():
    """A dropped x_j term or a sign error in the residual is caught by the
    exact-solve identity."""
    As, Bs, X, lam = _correction_case(False)
    z, w = orc.contour_nodes("gl_half", 5, 0.0, 4.0)
    ref = orc._filtered_subspace_exact(As.toarray(), X, z, w, True)
    scale = np.abs(ref).max()
    # mutation 1: correction only (no x_j / (z - lam) term)
    Rres = As @ X - X * lam[None, :]
    Q1 = np.zeros(X.shape, np.complex128)
    Q2 = np.zeros(X.shape, np.complex128)
    for zk, wk in zip(z, w):
        M = zk * np.eye(30) - As.toarray()
        for j in range(4):
            e = np.linalg.solve(M, Rres[:, j])
            Q1[:, j] += wk * e / (zk - lam[j])
            e2 = np.linalg.solve(M, -Rres[:, j])  # mutation 2: residual sign
            Q2[:, j] += wk * (X[:, j] + e2) / (zk - lam[j])
    assert np.abs(Q1.real - ref).max() > 1e-3 * scale
    assert np.abs(Q2.real - ref).max() > 1e-3 * scale


def test_ifeast_correction_converges_to_closed_form_generalized():
    """IFEAST with the GMRES residual form on the Q1 FEM pencil reaches the
    closed-form eigenvalues; the plain form with the same k also converges
    (the two differ only in the inner solver's starting point)."""
    grid = (12, 10)
    K, M = inputs.fem_q1(grid)
    ev = inputs.fem_q1_eigs(grid)
    cnt = 5
    emin, emax = 0.0, 0.5 * (ev[cnt - 1] + ev[cnt])
    z, w = orc.contour_nodes("gl_half", 8, emin, emax)
    X0 = inputs.initial_subspace(K.n, 10, 0)
    for corr in (np.inf, 1e-3, None):
        out = orc.ifeast(K.to_scipy(), X0, emin, emax, z, w, inner="gmres", k=12, alpha=1e-2,
                         max_outer=40, B=M.to_scipy(), correction_rf=corr)
        assert out["converged"], corr
        lam = out["lam"][out["inside"]]
        assert lam.size == cnt
        assert np.abs(lam - ev[:cnt]).max() <= 1e-10 * ev[cnt - 1]


# ---------------------------------------------------------------- shared basis: plain and residual form

# Krylov steps allowed for an exact solve at n = 30: the MGS Arnoldi basis loses
# orthogonality near step n, so the invariant subspace is reached a step or two
# later (the breakdown test then ends the run)
KFULL = 40


def _shared_case():
    A = inputs.add_diagonal(inputs.laplacian((6, 5)), inputs.random_potential(30, 11))
    X = inputs.initial_subspace(30, 4, 12)
    lam = np.array([1.1, 2.9, 3.3, 6.5])  # any scalars off the contour
    z, w = orc.contour_nodes("trap_half", 6, 0.5, 4.0)
    return A.to_scipy(), X, lam, z, w


def test_shared_filter_full_dimension_equals_exact_filter():
    """At k >= n the shared-basis GMRES iterate of every node is the exact solve,
    so the filter equals dense LU (Alg. 1 steps 1-2) and U rho(Lambda) U^T X."""
    As, X, lam, z, w = _shared_case()
    got = orc._filtered_subspace_shared(As, X, z, w, True, KFULL, 0.0, {"inner_steps": []})
    ref = orc._filtered_subspace_exact(As.toarray(), X, z, w, True)
    spec = orc.filter_step_spectral(As.toarray(), X, z, w, True)
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()
    assert np.abs(got - spec).max() <= 1e-10 * np.abs(spec).max()


def test_shared_correction_filter_full_dimension_equals_exact_filter():
    """Residual form of the shared-basis filter (right-hand sides r_j = A x_j -
    lam_j x_j, Q_j = rho(lam_j) x_j + Re sum_k w_k y'_kj / (z_k - lam_j)): at k >= n
    it equals the exact filter for any lam_j (an identity of the shifted
    systems), half and full contour."""
    As, X, lam, z, w = _shared_case()
    got = orc._filtered_subspace_shared_correction(As, X, lam, z, w, True, KFULL, 0.0,
                                                   {"inner_steps": []})
    ref = orc._filtered_subspace_exact(As.toarray(), X, z, w, True)
    spec = orc.filter_step_spectral(As.toarray(), X, z, w, True)
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()
    assert np.abs(got - spec).max() <= 1e-10 * np.abs(spec).max()
    zf, wf = orc.contour_nodes("trap_full", 8, 0.5, 4.0)
    gotf = orc._filtered_subspace_shared_correction(As, X, lam, zf, wf, False, KFULL, 0.0,
                                                    {"inner_steps": []})
    reff = orc._filtered_subspace_exact(As.toarray(), X, zf, wf, False)
    assert np.abs(gotf - reff).max() <= 1e-10 * np.abs(reff).max()


def test_shared_correction_filter_mutations_fail():
    """Planted mistakes in the residual form are caught by the exact-solve
    identity: the rho(lam_j) x_j term dropped, the residual's sign flipped, the
    weights not divided by z_k - lam_j."""
    As, X, lam, z, w = _shared_case()
    ref = orc._filtered_subspace_exact(As.toarray(), X, z, w, True)
    scale = np.abs(ref).max()
    Rres = As @ X - X * lam[None, :]
    rho = orc.filter_rho(lam, z, w, True)
    q_nox = np.zeros(X.shape, np.complex128)
    q_sign = X * rho[None, :] + 0j
    q_wt = X * rho[None, :] + 0j
    for zk, wk in zip(z, w):
        for j in range(4):
            y = orc.gmres_shared_basis(As, Rres[:, j], zk, KFULL)["y"]
            ym = orc.gmres_shared_basis(As, -Rres[:, j], zk, KFULL)["y"]
            q_nox[:, j] += wk * y / (zk - lam[j])
            q_sign[:, j] += wk * ym / (zk - lam[j])
            q_wt[:, j] += wk * y
    for bad in (q_nox, q_sign, q_wt):
        assert np.abs(bad.real - ref).max() > 1e-3 * scale


def test_shared_correction_stop_bound_is_first_step_below():
    """The residual-form stop bound: a (node, column) pair stops at the first
    step whose least-squares residual of the correction system is within
    tol ||x_j|| |z_k - lam_j|, i.e. the original system's residual within
    tol ||x_j|| (Alg. 2 step 1). Brute force: the minimal residual over an
    explicitly orthonormalised Krylov space (Gram-Schmidt applied twice)."""
    As, X, lam, z, w = _shared_case()
    Ad = As.toarray()
    tol = 3e-2
    stats = {"inner_steps": []}
    orc._filtered_subspace_shared_correction(As, X, lam, z, w, True, 30, tol, stats)
    Rres = As @ X - X * lam[None, :]

    def min_res(M, r, d):
        Qb = np.zeros((30, d))
        q = r / np.linalg.norm(r)
        for i in range(d):
            Qb[:, i] = q
            v = Ad @ q
            for _ in range(2):
                v = v - Qb[:, :i + 1] @ (Qb[:, :i + 1].T @ v)
            q = v / np.linalg.norm(v)
        c = np.linalg.lstsq(M @ Qb, r + 0j, rcond=None)[0]
        return np.linalg.norm(r - M @ Qb @ c)

    steps = iter(stats["inner_steps"])
    for zk in z:
        M = zk * np.eye(30) - Ad
        for j in range(4):
            s = next(steps)
            assert 1 <= s <= 20
            bound = tol * np.linalg.norm(X[:, j]) * abs(zk - lam[j])
            assert min_res(M, Rres[:, j], s) <= bound * (1 + 1e-6)
            if s > 1:
                assert min_res(M, Rres[:, j], s - 1) > bound * (1 - 1e-6)


def test_shared_correction_ifeast_converges_to_brute_force():
    """IFEAST with the shared basis and the residual form from the second
    iteration on (the GPU solver's schedule) reaches the brute-force
    eigenvalues of an interior window."""
    A = inputs.add_diagonal(inputs.laplacian((6, 5, 4)), inputs.random_potential(120, 3))
    ev = np.linalg.eigvalsh(A.to_scipy().toarray())
    i0, cnt = 12, 4
    emin, emax = 0.5 * (ev[i0 - 1] + ev[i0]), 0.5 * (ev[i0 + cnt - 1] + ev[i0 + cnt])
    z, w = orc.contour_nodes("trap_half", 6, emin, emax)
    out = orc.ifeast(A.to_scipy(), inputs.initial_subspace(A.n, 8, 0), emin, emax, z, w,
                     inner="shared", k=40, alpha=1e-2, max_outer=30, correction_rf=np.inf)
    assert out["converged"]
    lam = out["lam"][out["inside"]]
    assert lam.size == cnt
    assert np.abs(lam - ev[i0:i0 + cnt]).max() <= 1e-10 * np.abs(ev).max()


# ---------------------------------------------------------------- step-level references

def test_ref_spmm_shift_matches_dense_shifted_matrix():
    """W[:, c] = (z_c I - A) V[:, c], checked against the dense shifted matrix
    built entry by entry, on complex columns; a flipped sign (A - z I) fails."""
    A = inputs.random_sparse_symmetric(40, 3, 2)
    Ad = A.to_scipy().toarray()
    g = np.random.default_rng(5)
    V = g.standard_normal((40, 6)) + 1j * g.standard_normal((40, 6))
    zcol = np.array([0.3 + 0.1j, 1.5 - 0.2j, 2.0, -0.7 + 2j, 0.0, 5.0 + 0.5j])
    got = orc.ref_spmm_shift(A.to_scipy(), V, zcol)
    for c in range(6):
        M = np.array([[(zcol[c] if i == j else 0.0) - Ad[i, j] for j in range(40)]
                      for i in range(40)])
        ref = M @ V[:, c]
        assert np.abs(got[:, c] - ref).max() <= 1e-13 * np.abs(ref).max()
        assert np.abs(-got[:, c] - ref).max() > 0.1 * np.abs(ref).max()


def test_convergence_bound_delta_matches_resolvent_norms():
    """Delta = sum_k ||w_k (z_k I - A)^{-1}||_2 (Eq. deltadef) over the full
    circle, from the dense resolvents' spectral norms: a half rule's weights
    hold the factor 2 of the mirrored lower-half node (w/2 at z and at conj z)."""
    A = inputs.add_diagonal(inputs.laplacian((5, 4)), inputs.random_potential(20, 2))
    Ad = A.to_scipy().toarray()
    ev = np.linalg.eigvalsh(Ad)
    z, w = orc.contour_nodes("gl_half", 5, 1.0, 3.0)
    ref = 0.0
    for zk, wk in zip(list(z) + list(z.conj()), list(w / 2) + list(w.conj() / 2)):
        ref += np.linalg.norm(wk * np.linalg.inv(zk * np.eye(20) - Ad), 2)
    assert abs(orc.convergence_bound_delta(ev, z, w, True) - ref) <= 1e-12 * ref


# ---------------------------------------------------------------- seeded initial subspace

def test_philox_known_answers():
    """Philox4x32-10 reproduces the generator's published known-answer vectors."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = orc.philox4x32_10([np.array([c]) for c in v[:4]], [np.array([k]) for k in v[4:6]])
        assert [int(o[0]) for o in out] == v[6:]


def test_seeded_normal_block_layout_and_distribution():
    """Pair p of the row-major block comes from counter p (so a larger block
    extends a smaller one), different seeds give different blocks, and the
    values are standard normal (Kolmogorov-Smirnov against the normal CDF,
    moments)."""
    from scipy import stats
    X = orc.seeded_normal_block(2001, 7, 123)
    Y = orc.seeded_normal_block(3001, 7, 123)
    assert np.array_equal(X.ravel(), Y.ravel()[: X.size])
    assert not np.allclose(X, orc.seeded_normal_block(2001, 7, 124))
    assert not np.allclose(X, orc.seeded_normal_block(2001, 7, 123 + (1 << 32)))
    x = Y.ravel()
    assert abs(x.mean()) < 4.0 / np.sqrt(x.size)
    assert abs(x.var() - 1.0) < 6.0 * np.sqrt(2.0 / x.size)
    assert stats.kstest(x, "norm").pvalue > 1e-3
    # the cosine and sine halves of Box-Muller are independent N(0,1)
    assert abs(np.corrcoef(x[0::2][:10000], x[1::2][:10000])[0, 1]) < 0.05


# ---------------------------------------------------------------- eigenvalues an interval holds

def test_eigenvalues_in_interval_matches_dense():
    """Shift-invert Lanczos around the interval centre returns exactly the
    dense eigvalsh eigenvalues inside the interval, with their neighbours
    outside, and raises when k does not reach both ends."""
    A = inputs.add_diagonal(inputs.laplacian((11, 10, 9)), inputs.random_potential(990, 4))
    ev = np.linalg.eigvalsh(A.to_scipy().toarray())
    emin, emax = 0.5 * (ev[99] + ev[100]), 0.5 * (ev[129] + ev[130])
    lam, res, below, above = orc.eigenvalues_in_interval(A.to_scipy(), emin, emax, 40)
    assert lam.size == 30
    assert np.abs(lam - ev[100:130]).max() <= 1e-12 * np.abs(ev).max()
    assert res.max() <= 1e-10
    assert below == pytest.approx(ev[99], abs=1e-12) and above == pytest.approx(ev[130], abs=1e-12)
    with pytest.raises(ValueError):
        orc.eigenvalues_in_interval(A.to_scipy(), emin, emax, 20)
    # a fill-reducing ordering changes the factorisation only
    perm = orc.grid_nested_dissection((11, 10, 9))
    assert np.array_equal(np.sort(perm), np.arange(990))
    lam2, res2, _, _ = orc.eigenvalues_in_interval(A.to_scipy(), emin, emax, 40, perm)
    assert np.abs(lam2 - ev[100:130]).max() <= 1e-12 * np.abs(ev).max()
