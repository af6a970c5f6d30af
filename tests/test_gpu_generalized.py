"""Generalized problem A x = lambda B x on the CUDA path (Section 2.2: the
shifted systems become (z_k B - A) Y_k = B X and the reduced problem
A_Q X_Q = B_Q X_Q Lambda with B_Q = Q^T B Q), against the oracle and the
closed-form spectrum of Q1 finite elements.

Tolerances as in the standard-problem parity tests: step outputs agree to
1e-11 of the block's largest entry (same FP64 formulas, other summation
order), converged eigenvalues to 1e-10 relative, residuals <= 1e-10."""
import numpy as np
import pytest

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


def _solver(A, B, emin, emax, m0, **kw):
    from paper_1706_00692_gb300 import Solver
    return Solver(A, emin, emax, m0, B=B, **kw)


def _pencil_with_other_pattern():
    # B with a pattern of its own (diagonal + one off-diagonal band) and a
    # ragged row count: exercises B's CSR independently of A's.
    A = inputs.add_diagonal(inputs.laplacian((13, 11, 7)), inputs.random_potential(1001, 5))
    n = A.n
    g = np.random.default_rng(9)
    d = 1.0 + g.random(n)
    off = 0.2 * g.random(n - 3)
    import scipy.sparse as sp
    Bs = (sp.diags(d) + sp.diags(off, 3) + sp.diags(off, -3)).tocsr()
    Bs.sort_indices()
    B = inputs.CSR(n, Bs.indptr.astype(np.int32), Bs.indices.astype(np.int32), Bs.data.copy())
    return A, B


@pytest.mark.parametrize("case", ["fem", "own_pattern"])
def test_spmm_shift_with_B(torch, case):
    if case == "fem":
        A, B = inputs.fem_q1((20, 17))
    else:
        A, B = _pencil_with_other_pattern()
    m0, nc = 5, 3
    S = _solver(A, B, 0.0, 1.0, m0, nc=nc)
    g = np.random.default_rng(2)
    V = g.standard_normal((A.n, m0 * nc)) + 1j * g.standard_normal((A.n, m0 * nc))
    z = g.standard_normal(nc) + 1j * g.standard_normal(nc)
    W = S.spmm_shift(torch.as_tensor(V, device="cuda"), z).cpu().numpy()
    ref = (B.to_scipy() @ V) * np.repeat(z, m0)[None, :] - A.to_scipy() @ V
    assert np.abs(W - ref).max() <= 1e-13 * np.abs(ref).max()
    S.close()


@pytest.mark.parametrize("case", ["fem", "own_pattern"])
@pytest.mark.parametrize("k,alpha", [(1, 0.0), (6, 0.0), (24, 0.05)])
def test_filter_matches_oracle(torch, case, k, alpha):
    if case == "fem":
        A, B = inputs.fem_q1((20, 17))
        ev = inputs.fem_q1_eigs((20, 17))
        emin, emax, m0, nc = 0.0, 0.5 * (ev[5] + ev[6]), 9, 8
    else:
        A, B = _pencil_with_other_pattern()
        emin, emax, m0, nc = 0.5, 1.0, 7, 5
    X = inputs.initial_subspace(A.n, m0, 13)
    S = _solver(A, B, emin, emax, m0, nc=nc, inner_iters=k, alpha=alpha)
    RF = 1.0
    Q, steps = S.apply_filter(torch.as_tensor(X, device="cuda"), RF=RF)
    z, w = orc.contour_nodes("gl_half", nc, emin, emax)
    stats = {"inner_steps": []}
    Qr = orc._filtered_subspace_gmres(A.to_scipy(), X, z, w, True, k, alpha * RF, stats,
                                      B=B.to_scipy())
    assert (steps.cpu().numpy() == np.array(stats["inner_steps"])).all()
    assert np.abs(Q.cpu().numpy() - Qr).max() <= 1e-11 * np.abs(Qr).max()
    S.close()


@pytest.mark.parametrize("m0", [1, 9, 40])
def test_rayleigh_ritz_matches_oracle(torch, m0):
    A, B = inputs.fem_q1((20, 17))
    Q = inputs.initial_subspace(A.n, m0, 4)
    S = _solver(A, B, 0.0, 100.0, m0)
    X, lam, res = S.rayleigh_ritz(torch.as_tensor(Q, device="cuda"))
    X, lam, res = X.cpu().numpy(), lam.cpu().numpy(), res.cpu().numpy()
    As, Bs = A.to_scipy(), B.to_scipy()
    lr, XQ = orc.rayleigh_ritz(Q, As @ Q, Bs @ Q)
    Xr = Q @ XQ
    rr = orc.eigen_residuals(As @ Xr, Xr, lr, Bs @ Xr)
    assert np.abs(lam - lr).max() <= 1e-12 * np.abs(lr).max()
    assert np.abs(res - rr).max() <= 1e-10
    sgn = np.sign(np.sum(X * Xr, axis=0))
    assert np.abs(X * sgn - Xr).max() <= 1e-9 * np.abs(Xr).max()
    # B-orthonormal Ritz vectors
    assert np.abs(X.T @ (Bs @ X) - np.eye(m0)).max() <= 1e-10
    S.close()


@pytest.mark.parametrize("k,alpha", [(32, 1e-2), (10, 0.0)])
def test_solve_fem_q1_matches_closed_form_and_oracle(torch, k, alpha):
    grid, cnt, m0 = (30, 25), 6, 12
    K, M = inputs.fem_q1(grid)
    ev = inputs.fem_q1_eigs(grid)
    emin, emax = 0.0, 0.5 * (ev[cnt - 1] + ev[cnt])
    X0 = inputs.initial_subspace(K.n, m0, 0)
    S = _solver(K, M, emin, emax, m0, nc=8, inner_iters=k, alpha=alpha, max_outer=40)
    rc = S.solve(X0)
    assert rc == 0, rc
    lam, X, res = S.eigenpairs()
    assert lam.size == cnt
    assert np.abs(lam - ev[:cnt]).max() <= 1e-10 * ev[cnt - 1]
    assert res.max() <= 1e-10
    Ks, Ms = K.to_scipy(), M.to_scipy()
    assert np.abs(X.T @ (Ms @ X) - np.eye(cnt)).max() <= 1e-9
    # the library's residuals are the oracle's formula on the returned vectors
    assert np.abs(res - orc.eigen_residuals(Ks @ X, X, lam, Ms @ X)).max() <= 1e-12
    z, w = orc.contour_nodes("gl_half", 8, emin, emax)
    out = orc.ifeast(Ks, X0, emin, emax, z, w, inner="gmres", k=k, alpha=alpha, max_outer=40,
                     B=Ms)
    assert out["converged"]
    # same iteration count within one (rounding decides the last step)
    assert abs(S.stats()["outer_iters"] - out["iters"]) <= 1
    assert np.abs(lam - out["lam"][out["inside"]]).max() <= 1e-10 * ev[cnt - 1]
    S.close()


def test_minres_with_B_is_refused(torch):
    from paper_1706_00692_gb300 import IFEASTError
    K, M = inputs.fem_q1((6, 5))
    with pytest.raises(IFEASTError):
        _solver(K, M, 0.0, 100.0, 4, inner="minres", inner_iters=50)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("chunk", [1, 2, 3])
def test_node_chunks_equal_the_all_nodes_filter(torch, precision, tol, chunk):
    """opts.node_chunk: the shifted systems run chunk nodes at a time and Q is
    summed over the passes. Every system's arithmetic is unchanged, so the
    step counts are identical and Q differs from the all-nodes filter only by
    the order of the sum over nodes (FP32 sums with the FP32 basis: 1e-5 of the
    block's largest entry); the oracle agrees (plain and residual form)."""
    A, B = inputs.fem_q1((14, 12))
    emin, emax, m0, nc = 0.0, 200.0, 6, 6
    X = inputs.initial_subspace(A.n, m0, 3)
    Xn = X / np.linalg.norm(X, axis=0)[None, :]
    lam = np.linspace(20.0, 260.0, m0)
    outs = []
    for nch in (0, chunk):
        S = _solver(A, B, emin, emax, m0, nc=nc, inner="gmres", inner_iters=12, alpha=0.3,
                    precision=precision, node_chunk=nch)
        Q, st = S.apply_filter(torch.as_tensor(X, device="cuda"), RF=0.5)
        outs.append((Q.cpu().numpy(), st.cpu().numpy()))
        if precision == "fp32":
            Qr, str_ = S.apply_filter_residual(torch.as_tensor(Xn, device="cuda"), lam, RF=0.5)
            outs[-1] += (Qr.cpu().numpy(), str_.cpu().numpy())
        S.close()
    assert np.array_equal(outs[0][1], outs[1][1])
    assert np.abs(outs[0][0] - outs[1][0]).max() <= tol * np.abs(outs[0][0]).max()
    if precision == "fp32":
        assert np.array_equal(outs[0][3], outs[1][3])
        assert np.abs(outs[0][2] - outs[1][2]).max() <= tol * np.abs(outs[0][2]).max()
    z, w = orc.contour_nodes("gl_half", nc, emin, emax)
    stats = {"inner_steps": []}
    ref = orc._filtered_subspace_gmres(A.to_scipy(), X, z, w, True, 12, 0.3 * 0.5, stats,
                                       B.to_scipy())
    ref_steps = np.array(stats["inner_steps"])
    assert (outs[1][1] == ref_steps).mean() >= 0.95
    if (outs[1][1] == ref_steps).all():
        assert np.abs(outs[1][0] - ref).max() <= (2e-5 if precision == "fp32" else 1e-11) * \
            np.abs(ref).max()


def test_node_chunked_solve_matches_closed_form(torch):
    """A full generalized solve with two nodes per pass reaches the closed-form
    Q1 FEM eigenvalues like the all-nodes solve."""
    grid = (30, 25)
    A, B = inputs.fem_q1(grid)
    ev = inputs.fem_q1_eigs(grid)
    cnt = 8
    emin, emax = 0.0, 0.5 * (ev[cnt - 1] + ev[cnt])
    S = _solver(A, B, emin, emax, 14, nc=8, inner="gmres", inner_iters=32, alpha=1e-2,
                precision="fp32", node_chunk=2)
    rc = S.solve(inputs.initial_subspace(A.n, 14, 0))
    assert rc == 0, rc
    lam, X, res = S.eigenpairs()
    S.close()
    assert lam.size == cnt
    assert np.abs(lam - ev[:cnt]).max() <= 1e-10 * ev[cnt - 1]
    assert res.max() <= 1e-10
