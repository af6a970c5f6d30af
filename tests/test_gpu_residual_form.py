"""The residual form of the shifted solves (the right-hand sides the solver
uses from its second outer iteration on), the seeded initial subspace, the
caller-given contour, the per-solve stream and the time limit, all through the
C ABI, against the oracle.

Residual form: with r_j = A x_j - lam_j x_j, (z I - A)^{-1} x_j =
(x_j + (z I - A)^{-1} r_j) / (z - lam_j), so the filter is
Q_j = rho(lam_j) x_j + Re sum_k w_k y'_kj / (z_k - lam_j) with y'_kj the inner
solver's iterate for (z_k I - A) y' = r_j (Section 3 shared basis, or per-node
GMRES). The oracle functions are _filtered_subspace_shared_correction and
_filtered_subspace_gmres_correction (pinned on the CPU at k >= n against dense
LU and the spectral definition)."""
import ctypes as ct

import numpy as np
import pytest

from oracle import ifeast_oracle as orc
from paper_1706_00692_gb300 import inputs

pytestmark = pytest.mark.gpu

# Largest entry error of the FP32 filter relative to the block's largest entry.
# The Lanczos vectors, the sparse products and the dots are FP32 (unit roundoff
# u = 6.0e-8); the three-term recurrence over k <= 10 steps and the FP64
# least-squares solves on FP32-rounded alpha, beta carry that rounding into the
# coefficients with a growth of a few units per step, and the block's largest
# entry bounds every term of the sum. A bound of ~300 u covers k = 10 with room
# for the conditioning of the shifted systems at the nodes nearest the real
# axis (Im z >= 0.05 r here); measured worst cases are recorded in the tests'
# assertion messages.
FP32_TOL = 2e-5
# 16-bit storage of the Lanczos vectors: every stored entry is rounded to
# u = 4.9e-4 (FP16) or 3.9e-3 (BF16) relative; over a few steps the block then
# differs from the FP64 oracle by a few u of its largest entry, more in the
# residual form, whose correction terms carry 1/|z_k - lam_j| (measured at
# k = 10: FP16 5.8e-3, BF16 7.4e-2). BF16 keeps 2^3 = 8 times FP16's rounding.
FP16_TOL = 1e-2
BF16_TOL = 8 * FP16_TOL + 2e-2


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1706_00692_gb300.build import build
    build()
    return t


def _problem():
    A = inputs.add_diagonal(inputs.laplacian((13, 11, 7)), inputs.random_potential(1001, 5))
    return A, 0.9, 1.4


def _pairs(n, m0, seed):
    """Unit columns and scalars inside and around the interval (the identity
    holds for any pairs; Ritz pairs are one case)."""
    X = inputs.initial_subspace(n, m0, seed)
    X /= np.linalg.norm(X, axis=0)[None, :]
    lam = np.linspace(0.8, 1.5, m0)
    return X, lam


@pytest.mark.parametrize("precision,m0,tol", [("fp64", 7, 1e-9), ("fp32", 7, FP32_TOL),
                                              ("fp32", 12, FP32_TOL), ("fp16", 12, FP16_TOL),
                                              ("bf16", 12, BF16_TOL)])
@pytest.mark.parametrize("k", [1, 4, 10])
def test_shared_basis_residual_form_matches_oracle(torch, precision, m0, tol, k):
    """m0 = 7: generic step kernel; m0 = 12: four-column (fixed-width row) kernel."""
    from paper_1706_00692_gb300 import Solver
    A, emin, emax = _problem()
    nc = 5
    X, lam = _pairs(A.n, m0, 41)
    S = Solver(A, emin, emax, m0, nc=nc, inner="minres", inner_iters=k, precision=precision)
    Q, steps = S.apply_filter_residual(torch.as_tensor(X, device="cuda"), lam)
    z, w = orc.contour_nodes("gl_half", nc, emin, emax)
    Qr = orc._filtered_subspace_shared_correction(A.to_scipy(), X, lam, z, w, True, k, 0.0,
                                                  {"inner_steps": []})
    err = np.abs(Q.cpu().numpy() - Qr).max() / np.abs(Qr).max()
    assert err <= tol, err
    assert (steps.cpu().numpy() == k).all()
    S.close()


def test_shared_basis_residual_form_stop_steps(torch):
    """Tolerance mode: each (node, column) pair stops at the first step whose
    residual is within alpha RF ||x_j|| |z_k - lam_j|; the stop decision is
    taken in FP64 on differently rounded least-squares problems, so a pair
    within rounding of the bound may stop one step apart. (Values are compared
    at fixed k <= 10 above: over the 20-60 steps taken here the three-term
    Lanczos basis loses orthogonality against the oracle's fully
    orthogonalised Arnoldi basis, so the two iterates differ by more than
    rounding while both meet the same residual bound.)"""
    from paper_1706_00692_gb300 import Solver
    A, emin, emax = _problem()
    m0, nc = 8, 4
    X, lam = _pairs(A.n, m0, 42)
    S = Solver(A, emin, emax, m0, nc=nc, inner="minres", inner_iters=60, alpha=0.5,
               precision="fp64")
    Q, steps = S.apply_filter_residual(torch.as_tensor(X, device="cuda"), lam, RF=0.02)
    z, w = orc.contour_nodes("gl_half", nc, emin, emax)
    stats = {"inner_steps": []}
    Qr = orc._filtered_subspace_shared_correction(A.to_scipy(), X, lam, z, w, True, 60, 0.01,
                                                  stats)
    st = steps.cpu().numpy()
    ref = np.array(stats["inner_steps"])
    assert np.abs(st - ref).max() <= 1
    assert (st == ref).mean() >= 0.9
    assert st.min() < st.max()  # the pairs stopped at different steps
    assert np.isfinite(Q.cpu().numpy()).all() and np.abs(Qr).max() > 0
    S.close()


@pytest.mark.parametrize("B_too", [False, True])
def test_gmres_fp32_residual_form_matches_oracle(torch, B_too):
    """Per-node GMRES with the FP32 basis in residual form, standard and
    generalized (r_j = A x_j - lam_j B x_j)."""
    from paper_1706_00692_gb300 import Solver
    if B_too:
        A, B = inputs.fem_q1((14, 12))
        emin, emax = 0.0, 200.0
    else:
        (A, emin, emax), B = _problem(), None
    m0, nc, k = 6, 4, 10
    X, lam = _pairs(A.n, m0, 43)
    if B_too:
        lam = np.linspace(20.0, 260.0, m0)
    S = Solver(A, emin, emax, m0, nc=nc, inner="gmres", inner_iters=k, precision="fp32", B=B)
    Q, steps = S.apply_filter_residual(torch.as_tensor(X, device="cuda"), lam)
    z, w = orc.contour_nodes("gl_half", nc, emin, emax)
    Qr = orc._filtered_subspace_gmres_correction(A.to_scipy(), X, lam, z, w, True, k, 0.0,
                                                 {"inner_steps": []},
                                                 None if B is None else B.to_scipy())
    err = np.abs(Q.cpu().numpy() - Qr).max() / np.abs(Qr).max()
    assert err <= FP32_TOL, err
    assert (steps.cpu().numpy() == k).all()
    S.close()


def test_residual_form_unsupported_for_fp64_gmres(torch):
    from paper_1706_00692_gb300 import IFEASTError, Solver
    A, emin, emax = _problem()
    S = Solver(A, emin, emax, 4, nc=4, inner="gmres", inner_iters=5, precision="fp64")
    X, lam = _pairs(A.n, 4, 44)
    with pytest.raises(IFEASTError):
        S.apply_filter_residual(torch.as_tensor(X, device="cuda"), lam)
    S.close()


@pytest.mark.parametrize("n,m0,seed", [(1001, 7, 0), (517, 8, 123456789),
                                       (3, 1, (7 << 32) + 5)])
def test_seeded_initial_subspace_matches_oracle(torch, n, m0, seed):
    """The device's Philox4x32-10 + Box-Muller block equals the oracle's
    (independent implementation from the published definition); the integer
    stream is the same, so only the math library's last bits of log, cos and
    sin may differ."""
    from paper_1706_00692_gb300 import initial_subspace
    X = initial_subspace(n, m0, seed).cpu().numpy()
    ref = orc.seeded_normal_block(n, m0, seed)
    assert np.abs(X - ref).max() <= 1e-14 * max(1.0, np.abs(ref).max())


def test_solve_from_seed_equals_solve_from_its_block(torch):
    """ifeast_solve(X0 = NULL, seed) starts from ifeast_initial_subspace(seed):
    both solves are bit-identical, and match the closed form."""
    from paper_1706_00692_gb300 import Solver, initial_subspace
    wl = inputs.workload_lap2d_50()
    out = []
    for mode in ("seed", "block"):
        S = Solver(wl.A, wl.emin, wl.emax, wl.m0, nc=wl.nc, inner="minres", inner_iters=200,
                   alpha=1e-2, precision="fp32")
        rc = S.solve(None, seed=77) if mode == "seed" else \
            S.solve(initial_subspace(wl.A.n, wl.m0, 77))
        assert rc == 0
        out.append(S.eigenpairs())
        S.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    ev = inputs.laplacian_eigs((50, 50))
    assert np.abs(out[0][0] - ev[:10]).max() <= 1e-10 * ev[9]


def test_user_contour_equals_builtin_rule(torch):
    """IFEAST_USER with the nodes and weights of the built-in GL rule gives the
    built-in rule's solve bit for bit; a full-circle trapezoid rule given as
    its upper-half nodes with doubled weights gives TRAP_FULL's."""
    from paper_1706_00692_gb300 import Solver, contour_nodes
    wl = inputs.workload_lap2d_50()
    X0 = wl.X0()
    res = {}
    for name, kw in [("gl", dict(rule="gl_half", nc=8)),
                     ("gl_user", dict(rule="user", user_nodes=contour_nodes("gl_half", 8, wl.emin,
                                                                             wl.emax))),
                     ("trap_full", dict(rule="trap_full", nc=16)),
                     ("trap_user", dict(rule="user", user_nodes=contour_nodes("trap_half", 8, wl.emin,
                                                                               wl.emax)))]:
        S = Solver(wl.A, wl.emin, wl.emax, wl.m0, inner="minres", inner_iters=200, alpha=1e-2,
                   precision="fp64", **kw)
        assert S.solve(X0) == 0
        res[name] = S.eigenpairs()
        S.close()
    for a, b in (("gl", "gl_user"), ("trap_full", "trap_user")):
        assert np.array_equal(res[a][0], res[b][0]) and np.array_equal(res[a][1], res[b][1])


def test_solve_on_a_given_stream(torch):
    """ifeast_solve on a stream other than the handle's gives the same pairs."""
    from paper_1706_00692_gb300 import Solver, _lib
    wl = inputs.workload_lap2d_50()
    S = Solver(wl.A, wl.emin, wl.emax, wl.m0, nc=wl.nc, inner="minres", inner_iters=200,
               alpha=1e-2, precision="fp32")
    X0 = torch.as_tensor(wl.X0(), device="cuda")
    assert S.solve(X0) == 0
    lam0, X0r, _ = S.eigenpairs()
    s2 = torch.cuda.Stream()
    torch.cuda.synchronize()
    rc = _lib.load().ifeast_solve(S.h, ct.c_void_p(X0.data_ptr()), 1, 0,
                                  ct.c_void_p(s2.cuda_stream))
    assert rc == 0
    lam1, X1r, _ = S.eigenpairs()
    assert np.array_equal(lam0, lam1) and np.array_equal(X0r, X1r)
    S.close()


def test_time_limit_stops_the_solve(torch):
    """A time limit far below one outer iteration cuts the Lanczos loop at its
    first lagged check: TIMEOUT after one outer iteration, the last iterate's
    pairs retrievable, and the handle usable for the next solve."""
    from paper_1706_00692_gb300 import Solver, _lib
    A = inputs.add_diagonal(inputs.laplacian((40, 40, 40)), inputs.random_potential(64000, 2))
    ev = inputs.laplacian_eigs((40, 40, 40))
    emin, emax = ev[300] + 0.5, ev[330] + 0.5
    S = Solver(A, emin, emax, 48, nc=8, rule="trap_half", inner="minres", inner_iters=3000,
               alpha=1e-6, precision="fp32", time_limit_ms=2.0)
    for _ in range(2):
        rc = S.solve(None, seed=3)
        assert rc == _lib.IFEAST_ERR_TIMEOUT, rc
        st = S.stats()
        assert st["outer_iters"] == 1
        assert st["max_inner"] < 3000
        lam, res = S.ritz_all()
        assert np.isfinite(lam).all() and np.isfinite(res).all()
    S.close()
