"""CPU oracle for FEAST / IFEAST (Gavin & Polizzi, arXiv 1706.00692).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` may import this module. The CUDA library and
its Python binding never call it, and it imports nothing from them.

Plain, slow, obviously-correct float64 numpy/scipy code. Library primitives
(sparse mat-vec, dense LU, Cholesky, symmetric eigensolver, least squares) are
used as single steps; nothing is blocked, fused or reordered beyond what the
cited definitions state.

Map to the paper:
  contour_nodes / filter_rho ......... Eq. (contour_int_quad), Eq. (rhoh), the
                                        half-contour symmetry of Section 4.1
  feast .............................. Algorithm 1 (direct shifted solves)
  ifeast ............................. Algorithm 2 (iterative shifted solves,
                                        stopping rule ||x-(zI-A)y|| <= alpha*||R_F||)
  gmres .............................. GMRES of Section 2.2 (zero initial guess,
                                        modified Gram-Schmidt Arnoldi, Givens)
  _filtered_subspace_gmres_correction  Alg. 2 step 1 solved for the correction of
  _filtered_subspace_shared_correction  the current Ritz pairs (an identity of the
                                        shifted systems; reading in its docstring)
  gmres_shared_basis ................. Section 3, Eqs. (yz)-(contint_krylov):
                                        the Krylov basis does not depend on z
  rayleigh_ritz ...................... Algorithm 1/2 step 3 (B_Q = Q^T B Q for A x = lam B x)
  eigen_residuals .................... Algorithm 1/2 step 4
  convergence_bound .................. Eq. (upperbound), Eq. (deltadef)
  ifeast_nonsym / rayleigh_ritz_nonsym  non-Hermitian extension (stated without
                                        steps in the paper; readings in the docstring)
  seeded_normal_block ................ the random X^(0) (Alg. 1 input), Philox4x32-10
                                        + Box-Muller from their published definitions
  eigenvalues_in_interval ............ the eigenvalues an interval holds (problem
                                        statement, Section 1) by shift-invert Lanczos
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

GL_HALF = "gl_half"
TRAP_HALF = "trap_half"
TRAP_FULL = "trap_full"


# ---------------------------------------------------------------------------
# Contour and quadrature (Eq. contour_int_quad; half-contour symmetry, Sec. 4.1)
# ---------------------------------------------------------------------------

def contour_nodes(rule: str, nc: int, emin: float, emax: float):
    """Quadrature nodes z_k and weights w_k for (1/2 pi i) \\oint (zI-A)^{-1} dz
    on the circle with centre c=(emin+emax)/2 and radius r=(emax-emin)/2.

    Parametrise z = c + r e^{i theta}; then dz/(2 pi i) = r e^{i theta} d theta/(2 pi).
    * TRAP_FULL: nc points theta_j = 2 pi (j - 1/2)/nc, w_j = r e^{i theta_j}/nc;
      the filter is the plain sum sum_j w_j/(z_j - lambda).
    * TRAP_HALF / GL_HALF (real symmetric A): the lower half of the circle
      contributes the complex conjugate of the upper half, so only nc nodes on
      the upper half are used and the filter is 2 Re of their sum. The factor 2
      is folded into the weights, so filter = Re sum_k w_k/(z_k - lambda):
        TRAP_HALF: theta_j = pi (j - 1/2)/nc, w_j = r e^{i theta_j}/nc
        GL_HALF:   Gauss-Legendre (x_e, g_e) on (-1,1), theta_e = (pi/2)(1 - x_e),
                   w_e = (g_e/2) r e^{i theta_e}
    Returns (z, w) as complex128 arrays of length nc.
    """
    c = 0.5 * (emin + emax)
    r = 0.5 * (emax - emin)
    if rule == TRAP_FULL:
        th = 2.0 * math.pi * (np.arange(1, nc + 1) - 0.5) / nc
        return c + r * np.exp(1j * th), r * np.exp(1j * th) / nc
    if rule == TRAP_HALF:
        th = math.pi * (np.arange(1, nc + 1) - 0.5) / nc
        return c + r * np.exp(1j * th), r * np.exp(1j * th) / nc
    if rule == GL_HALF:
        x, g = np.polynomial.legendre.leggauss(nc)
        th = 0.5 * math.pi * (1.0 - x)
        return c + r * np.exp(1j * th), 0.5 * g * r * np.exp(1j * th)
    raise ValueError(rule)


def is_half_rule(rule: str) -> bool:
    return rule in (GL_HALF, TRAP_HALF)


def filter_rho(lam, z, w, half: bool):
    """Rational filter rho_hat(lambda) = sum_k w_k (z_k - lambda)^{-1} (Eq. rhoh),
    taking the real part for a half contour."""
    lam = np.asarray(lam, dtype=np.float64)
    s = np.sum(w[None, :] / (z[None, :] - lam.reshape(-1, 1)), axis=1).reshape(lam.shape)
    return s.real if half else s


# ---------------------------------------------------------------------------
# Sparse operator (the method touches A only through products, Section 1.2)
# ---------------------------------------------------------------------------

def csr_to_scipy(rowptr, colidx, val, n):
    return sp.csr_matrix((np.asarray(val, np.float64), np.asarray(colidx), np.asarray(rowptr)),
                         shape=(n, n))


def shifted_apply(A, z, V):
    """W = (z I - A) V  (one column block of Algorithm 2 step 1's operator)."""
    return z * V - A @ V


# ---------------------------------------------------------------------------
# GMRES (Section 2.2): zero initial guess, MGS Arnoldi, Givens least squares
# ---------------------------------------------------------------------------

def givens_params(a, b):
    """Unitary rotation G = [[conj(c), conj(s)], [-s, c]] with G [a; b] = [rho; 0],
    rho = sqrt(|a|^2 + |b|^2) >= 0."""
    rho = math.hypot(abs(a), abs(b))
    if rho == 0.0:
        return 1.0 + 0j, 0j, 0.0
    return a / rho, b / rho, rho


def gmres(matvec, b, k, tol_rel=0.0, breakdown_rel=1e-14):
    """GMRES for M y = b with y_0 = 0, at most k Arnoldi steps, stopping as soon
    as the least-squares residual |g_{s+1}| <= tol_rel * ||b|| (tol_rel <= 0:
    run all k).

    Returns dict(y, steps, res_est, V, H) where V is (steps+1, n) and H the
    (steps+1) x steps Hessenberg matrix of the Arnoldi relation
    M V[:steps].T = V.T H (for inspection by tests)."""
    b = np.asarray(b, dtype=np.complex128)
    n = b.shape[0]
    beta = np.linalg.norm(b)
    V = np.zeros((k + 1, n), np.complex128)
    H = np.zeros((k + 1, k), np.complex128)
    R = np.zeros((k, k), np.complex128)
    cs = np.zeros(k, np.complex128)
    sn = np.zeros(k, np.complex128)
    g = np.zeros(k + 1, np.complex128)
    if beta == 0.0:
        return dict(y=np.zeros(n, np.complex128), steps=0, res_est=0.0, V=V[:1], H=H[:1, :0])
    V[0] = b / beta
    g[0] = beta
    steps = 0
    for s in range(k):
        w = matvec(V[s])
        for l in range(s + 1):                      # modified Gram-Schmidt
            H[l, s] = np.vdot(V[l], w)
            w = w - H[l, s] * V[l]
        H[s + 1, s] = np.linalg.norm(w)
        happy = H[s + 1, s].real <= breakdown_rel * beta
        if not happy:
            V[s + 1] = w / H[s + 1, s]
        col = H[: s + 2, s].copy()
        for l in range(s):                          # previous rotations
            a, bb = col[l], col[l + 1]
            col[l] = np.conj(cs[l]) * a + np.conj(sn[l]) * bb
            col[l + 1] = -sn[l] * a + cs[l] * bb
        cs[s], sn[s], rho = givens_params(col[s], col[s + 1])
        col[s], col[s + 1] = rho, 0.0
        R[: s + 1, s] = col[: s + 1]
        g[s + 1] = -sn[s] * g[s]
        g[s] = np.conj(cs[s]) * g[s]
        steps = s + 1
        if happy or (tol_rel > 0.0 and abs(g[s + 1]) <= tol_rel * beta):
            break
    y_small = sla.solve_triangular(R[:steps, :steps], g[:steps], lower=False)
    y = V[:steps].T @ y_small
    return dict(y=y, steps=steps, res_est=abs(g[steps]), V=V[: steps + 1], H=H[: steps + 1, :steps],
                y_small=y_small)


def arnoldi_real(A, x, k, breakdown_rel=1e-14):
    """Arnoldi on the real matrix A from x (MGS). Returns V (steps+1, n), the
    (steps+1) x steps Hessenberg H, beta = ||x||, steps."""
    n = x.shape[0]
    beta = np.linalg.norm(x)
    V = np.zeros((k + 1, n))
    H = np.zeros((k + 1, k))
    V[0] = x / beta
    steps = 0
    for s in range(k):
        w = A @ V[s]
        for l in range(s + 1):
            H[l, s] = V[l] @ w
            w = w - H[l, s] * V[l]
        H[s + 1, s] = np.linalg.norm(w)
        steps = s + 1
        if H[s + 1, s] <= breakdown_rel * beta:
            break
        V[s + 1] = w / H[s + 1, s]
    return V[: steps + 1], H[: steps + 1, :steps], beta, steps


def gmres_shared_basis(A, x, z, k, tol_rel=0.0):
    """GMRES for (z I - A) y = x using the basis of K(A, x) (Section 3: the
    Krylov basis V is the same for every shift z). With A V_s = V_{s+1} Hbar,
    (z I - A) V_s = V_{s+1} (z Ibar - Hbar); the small least-squares problem is
    min || beta e_1 - (z Ibar - Hbar) y ||, solved here with lstsq at every s
    until the residual drops to tol_rel * ||x|| (or all k steps)."""
    V, H, beta, steps = arnoldi_real(A, x, k)
    for s in range(1, steps + 1):
        Hz = -H[: s + 1, :s].astype(np.complex128)
        Hz[np.arange(s), np.arange(s)] += z
        rhs = np.zeros(s + 1, np.complex128)
        rhs[0] = beta
        ys = np.linalg.lstsq(Hz, rhs, rcond=None)[0]
        res = np.linalg.norm(rhs - Hz @ ys)
        if (tol_rel > 0.0 and res <= tol_rel * beta) or s == steps:
            return dict(y=V[:s].T @ ys, steps=s, res_est=res)
    raise AssertionError("unreachable")


# ---------------------------------------------------------------------------
# Rayleigh-Ritz and residuals (Algorithm 1/2 steps 3 and 4)
# ---------------------------------------------------------------------------

def cholesky_shifted(Bq):
    """Cholesky of the reduced Gram matrix; if it is not numerically positive
    definite, retry once with the shift 11 (n m0 + m0 (m0+1)) u ||B_Q||_2 of
    shifted CholeskyQR (Fukaya et al., 2020); n is taken as m0 here since only
    the m0 x m0 matrix is factored. Returns (L, shifted_flag)."""
    try:
        return np.linalg.cholesky(Bq), False
    except np.linalg.LinAlgError:
        m = Bq.shape[0]
        shift = 11.0 * (m * m + m * (m + 1)) * np.finfo(float).eps * np.linalg.norm(Bq, 2)
        return np.linalg.cholesky(Bq + shift * np.eye(m)), True


def rayleigh_ritz(Q, AQ, BQ=None):
    """Solve A_Q X_Q = B_Q X_Q Lambda with A_Q = Q^H A Q, B_Q = Q^H B Q (B = I
    when BQ is None) through B_Q = L L^H, C = L^{-1} A_Q L^{-H}, C = U Lambda
    U^H, X_Q = L^{-H} U. Returns (lam ascending, X_Q) with X_Q^H B_Q X_Q = I."""
    Aq = Q.conj().T @ AQ
    Bq = Q.conj().T @ (Q if BQ is None else BQ)
    Aq = 0.5 * (Aq + Aq.conj().T)
    Bq = 0.5 * (Bq + Bq.conj().T)
    L, _ = cholesky_shifted(Bq)
    Li_Aq = sla.solve_triangular(L, Aq, lower=True)
    C = sla.solve_triangular(L, Li_Aq.conj().T, lower=True).conj().T
    C = 0.5 * (C + C.conj().T)
    lam, U = np.linalg.eigh(C)
    XQ = sla.solve_triangular(L.conj().T, U, lower=False)
    return lam, XQ


def eigen_residuals(AX, X, lam, BX=None):
    """Relative eigenpair residuals ||A x_j - lam_j B x_j|| / ||A x_j|| (B = I
    when BX is None)."""
    num = np.linalg.norm(AX - (X if BX is None else BX) * lam[None, :], axis=0)
    den = np.linalg.norm(AX, axis=0)
    return num / np.where(den > 0, den, 1.0)


def in_interval(lam, emin, emax):
    return (lam > emin) & (lam < emax)


# ---------------------------------------------------------------------------
# FEAST (Algorithm 1) and IFEAST (Algorithm 2)
# ---------------------------------------------------------------------------

def _filtered_subspace_exact(A_dense, X, z, w, half, B_dense=None):
    """Sum_k w_k (z_k B - A)^{-1} B X by dense LU (Alg. 1 steps 1-2; the
    generalized systems of Eq. generalized_linsys when B is given)."""
    n = X.shape[0]
    Bd = np.eye(n) if B_dense is None else B_dense
    rhs = (Bd @ X).astype(np.complex128)
    Q = np.zeros(X.shape, np.complex128)
    for zk, wk in zip(z, w):
        lu = sla.lu_factor(zk * Bd - A_dense)
        Q += wk * sla.lu_solve(lu, rhs)
    return Q.real if half else Q


def _filtered_subspace_gmres(A, X, z, w, half, k, tol_rel, stats, B=None):
    """Per (node, column) GMRES on (z_k B - A) y = B x_j (Alg. 2 step 1;
    Eq. generalized_linsys when B is given)."""
    n, m0 = X.shape
    rhs = X if B is None else B @ X
    Q = np.zeros(X.shape, np.complex128)
    for zk, wk in zip(z, w):
        if B is None:
            op = lambda v, zk=zk: shifted_apply(A, zk, v)
        else:
            op = lambda v, zk=zk: zk * (B @ v) - A @ v
        for j in range(m0):
            out = gmres(op, rhs[:, j], k, tol_rel)
            stats["inner_steps"].append(out["steps"])
            Q[:, j] += wk * out["y"]
    return Q.real if half else Q


def _filtered_subspace_gmres_correction(A, X, lam, z, w, half, k, tol_rel, stats, B=None):
    """The same filter from the current Ritz pairs (lam_j, x_j): with the residual
    r_j = A x_j - lam_j B x_j the shifted solution is exactly
    (z_k B - A)^{-1} B x_j = (x_j + e_kj) / (z_k - lam_j), (z_k B - A) e_kj = r_j,
    so GMRES (zero initial guess) runs on the correction systems only. The stop
    bound is the one of Alg. 2 on the original system, whose residual is the
    correction's divided by |z_k - lam_j|: |g_{s+1}| <= tol_rel ||B x_j|| |z_k - lam_j|."""
    n, m0 = X.shape
    BX = X if B is None else B @ X
    Rres = A @ X - BX * lam[None, :]
    Q = np.zeros(X.shape, np.complex128)
    for zk, wk in zip(z, w):
        if B is None:
            op = lambda v, zk=zk: shifted_apply(A, zk, v)
        else:
            op = lambda v, zk=zk: zk * (B @ v) - A @ v
        for j in range(m0):
            rn = np.linalg.norm(Rres[:, j])
            tol_j = 0.0
            if tol_rel > 0.0 and rn > 0.0:
                tol_j = tol_rel * np.linalg.norm(BX[:, j]) * abs(zk - lam[j]) / rn
            out = gmres(op, Rres[:, j], k, tol_j)
            stats["inner_steps"].append(out["steps"])
            Q[:, j] += wk * (X[:, j] + out["y"]) / (zk - lam[j])
    return Q.real if half else Q


def _filtered_subspace_shared(A, X, z, w, half, k, tol_rel, stats):
    """Sum_k w_k y_kj with y_kj the GMRES iterate of (z_k I - A) y = x_j on the
    real Krylov basis of K(A, x_j), which every node shares (Section 3,
    Eqs. yz-contint_krylov); stop per (node, column) once the least-squares
    residual is <= tol_rel ||x_j|| (Alg. 2 step 1)."""
    n, m0 = X.shape
    Q = np.zeros(X.shape, np.complex128)
    for zk, wk in zip(z, w):
        for j in range(m0):
            out = gmres_shared_basis(A, X[:, j], zk, k, tol_rel)
            stats["inner_steps"].append(out["steps"])
            Q[:, j] += wk * out["y"]
    return Q.real if half else Q


def _filtered_subspace_shared_correction(A, X, lam, z, w, half, k, tol_rel, stats):
    """The shared-basis filter (Section 3) solved for the correction of the
    current Ritz pairs (lam_j, x_j), B = I. With r_j = A x_j - lam_j x_j the
    shifted solution is exactly
        (z_k I - A)^{-1} x_j = (x_j + y'_kj) / (z_k - lam_j),  (z_k I - A) y'_kj = r_j,
    so every node's system is solved on the one real basis of K(A, r_j) and
        Q_j = rho(lam_j) x_j + sum_k w_k y'_kj / (z_k - lam_j)
    (rho of Eq. rhoh; real part for a half contour). The stop test is Alg. 2's
    on the original system, whose residual is the correction's divided by
    |z_k - lam_j|: least-squares residual <= tol_rel ||x_j|| |z_k - lam_j|."""
    n, m0 = X.shape
    Rres = A @ X - X * lam[None, :]
    rho = filter_rho(lam, z, w, half)
    Q = X * rho[None, :] + 0j
    for zk, wk in zip(z, w):
        for j in range(m0):
            rn = np.linalg.norm(Rres[:, j])
            if rn == 0.0:
                stats["inner_steps"].append(0)
                continue
            tol_j = 0.0
            if tol_rel > 0.0:
                tol_j = tol_rel * np.linalg.norm(X[:, j]) * abs(zk - lam[j]) / rn
            out = gmres_shared_basis(A, Rres[:, j], zk, k, tol_j)
            stats["inner_steps"].append(out["steps"])
            Q[:, j] += wk * out["y"] / (zk - lam[j])
    return Q.real if half else Q


def ifeast(A, X0, emin, emax, z, w, *, half=True, inner="gmres", k=10, alpha=0.0,
           tol=1e-10, max_outer=100, callback=None, B=None, correction_rf=None):
    """Algorithm 2 (and, with inner="exact", Algorithm 1) for a real symmetric
    problem A x = lambda x, or A x = lambda B x with B symmetric positive
    definite (the generalized systems (z_k B - A) Y_k = B X of Section 2.2).

    inner: "exact" dense LU per node (Alg. 1 step 1),
           "gmres" per-node complex GMRES (Alg. 2 step 1),
           "shared" GMRES on the shift-independent Krylov basis (Section 3).
    k: maximum inner steps. alpha > 0: stop each inner solve once
    ||x_j - (z_k I - A) y|| <= alpha * ||R_F|| * ||x_j|| (Alg. 2 step 1 with the
    residual measured relative to the right-hand side, ||R_F|| = 1 at the
    start); alpha <= 0: run exactly k steps.
    correction_rf: None, or a bound: from the second iteration on, once the
    previous ||R_F|| <= correction_rf, inner="gmres" (and inner="shared")
    solves for the correction of the Ritz pairs of the previous iteration
    (_filtered_subspace_gmres_correction, _filtered_subspace_shared_correction;
    the same filter in exact arithmetic). correction_rf = inf: from the second
    iteration on, whatever ||R_F||.
    ||R_F|| is the largest relative residual ||A x_j - lam_j x_j||/||A x_j||
    over Ritz values strictly inside (emin, emax).

    Returns dict(lam, X, res, inside, iters, history, converged).
    """
    A = A.tocsr() if sp.issparse(A) else A
    if B is not None:
        B = B.tocsr() if sp.issparse(B) else B
        if inner == "shared":
            raise ValueError("the shift-independent basis needs B = I")
    X = np.asarray(X0, dtype=np.float64).copy()
    RF = 1.0
    history = []
    A_dense = None
    B_dense = None
    for it in range(1, max_outer + 1):
        stats = {"inner_steps": []}
        tol_rel = alpha * RF if alpha > 0 else 0.0
        if inner == "exact":
            if A_dense is None:
                A_dense = A.toarray() if sp.issparse(A) else np.asarray(A)
                if B is not None:
                    B_dense = B.toarray() if sp.issparse(B) else np.asarray(B)
            Q = _filtered_subspace_exact(A_dense, X, z, w, half, B_dense)
        elif inner == "gmres" and correction_rf is not None and it > 1 and RF <= correction_rf:
            Q = _filtered_subspace_gmres_correction(A, X, lam, z, w, half, k, tol_rel, stats, B)
        elif inner == "gmres":
            Q = _filtered_subspace_gmres(A, X, z, w, half, k, tol_rel, stats, B)
        elif inner == "shared" and correction_rf is not None and it > 1 and RF <= correction_rf:
            Q = _filtered_subspace_shared_correction(A, X, lam, z, w, half, k, tol_rel, stats)
        elif inner == "shared":
            Q = _filtered_subspace_shared(A, X, z, w, half, k, tol_rel, stats)
        else:
            raise ValueError(inner)
        AQ = A @ Q
        BQ = None if B is None else B @ Q
        lam, XQ = rayleigh_ritz(Q, AQ, BQ)
        X = Q @ XQ
        AX = AQ @ XQ
        res = eigen_residuals(AX, X, lam, None if B is None else BQ @ XQ)
        inside = in_interval(lam, emin, emax)
        RF = float(res[inside].max()) if inside.any() else 1.0
        history.append(dict(RF=RF, count=int(inside.sum()),
                            max_inner=max(stats["inner_steps"], default=0),
                            total_inner=int(sum(stats["inner_steps"]))))
        if callback is not None:
            callback(it, lam, X, res, inside)
        if inside.any() and RF <= tol:
            return dict(lam=lam, X=X, res=res, inside=inside, iters=it, history=history,
                        converged=True)
    return dict(lam=lam, X=X, res=res, inside=inside, iters=max_outer, history=history,
                converged=False)


def feast(A, X0, emin, emax, z, w, *, half=True, tol=1e-10, max_outer=100, B=None):
    """Algorithm 1: FEAST with direct (dense LU) shifted solves."""
    return ifeast(A, X0, emin, emax, z, w, half=half, inner="exact", tol=tol, max_outer=max_outer,
                  B=B)


# ---------------------------------------------------------------------------
# Non-Hermitian extension (the paper states that the method extends to
# non-Hermitian problems without giving the steps; readings below)
# ---------------------------------------------------------------------------

def rayleigh_ritz_nonsym(Q, AQ):
    """Galerkin projection onto span(Q) for a real non-symmetric A:
    B_Q = Q^T Q = L L^T, Xb = Q L^{-T} (orthonormal columns), C = Xb^T A Xb =
    L^{-1} Q^T A Q L^{-T}, C U = U diag(theta) with complex theta and unit
    columns u_j. The Ritz vectors are Xb u_j (unit norm). Returns (theta, U,
    Linv_T) with Linv_T = L^{-T}."""
    Bq = Q.T @ Q
    Bq = 0.5 * (Bq + Bq.T)
    L, _ = cholesky_shifted(Bq)
    Linv_T = sla.solve_triangular(L.T, np.eye(L.shape[0]), lower=False)
    C = Linv_T.T @ (Q.T @ AQ) @ Linv_T
    theta, U = sla.eig(C)
    U = U / np.linalg.norm(U, axis=0)[None, :]
    return theta, U, Linv_T


def in_circle(theta, c, r):
    return np.abs(theta - c) < r


def _filtered_subspace_gmres_correction_nonsym(A, X, C, z, w, half, k, tol_rel, stats):
    """The non-symmetric filter from a real basis X and a square C (the Galerkin
    matrix X^T A X of the previous Rayleigh-Ritz): with R = A X - X C,
        (z I - A)^{-1} X = [X + (z I - A)^{-1} R] (z I - C)^{-1}
    holds exactly for any X and any C with z I - C invertible, since
    (z I - A)^{-1} X (z I - C) = (z I - A)^{-1} ((z I - A) X + R). GMRES (zero
    initial guess, at most k steps) runs on (z_k I - A) e = r_j only, stopped
    at |g_{s+1}| <= tol_rel ||x_j|| (Alg. 2's bound with the correction's
    right-hand side), and
        Q = sum_k w_k (X + E_k) (z_k I - C)^{-1}
    (real part for a half rule). The inner error is then relative to ||R||,
    which falls with the outer iteration, not to ||X||."""
    n, m0 = X.shape
    R = A @ X - X @ C
    Q = np.zeros(X.shape, np.complex128)
    for zk, wk in zip(z, w):
        op = lambda v, zk=zk: shifted_apply(A, zk, v)
        E = np.zeros(X.shape, np.complex128)
        for j in range(m0):
            rn = np.linalg.norm(R[:, j])
            if rn == 0.0:
                stats["inner_steps"].append(0)
                continue
            tol_j = tol_rel * np.linalg.norm(X[:, j]) / rn if tol_rel > 0.0 else 0.0
            out = gmres(op, R[:, j], k, tol_j)
            stats["inner_steps"].append(out["steps"])
            E[:, j] = out["y"]
        Q += wk * np.linalg.solve((zk * np.eye(m0) - C).T, (X + E).T).T
    return Q.real if half else Q


def ifeast_nonsym(A, X0, c, r, z, w, *, half=True, inner="gmres", k=10, alpha=0.0,
                  tol=1e-10, max_outer=100, correction=False):
    """IFEAST (Algorithm 2; Algorithm 1 with inner="exact") for a real
    non-symmetric A, eigenvalues inside the circle |lambda - c| < r.

    Readings taken (the paper gives no steps for this case):
    * contour: the circle itself; for real A and a real block X the solutions
      at conjugate nodes are conjugate, so a half-contour rule with the Re-sum
      (half=True) equals the full-circle sum with twice the nodes;
    * the subspace carried between iterations is the real orthonormal basis
      X = Q L^{-T} of span(Q) (B_Q = Q^T Q = L L^T), not the complex Ritz
      vectors; the span, and hence the iteration, is the same;
    * Rayleigh-Ritz is the Galerkin projection C = X^T A X with a general
      eigensolver; residuals ||A x_j - theta_j x_j|| / ||A x_j|| of the unit
      Ritz vectors x_j = X u_j; ||R_F|| is their maximum over theta_j inside
      the circle;
    * inner stop ||x_j - (z_k I - A) y|| <= alpha ||R_F|| ||x_j|| (||x_j|| = 1);
    * correction=True: from the second outer iteration on the filter runs on
      the residual block R = A X - X C of the previous Rayleigh-Ritz
      (_filtered_subspace_gmres_correction_nonsym), whose inner error falls
      with ||R||; the first iteration is the plain form.

    Returns dict(theta, V (Ritz vectors, n x m0 complex), res, inside, iters,
    history, converged)."""
    A = A.tocsr() if sp.issparse(A) else A
    X = np.asarray(X0, dtype=np.float64).copy()
    RF = 1.0
    history = []
    A_dense = None
    C = None  # Galerkin matrix X^T A X of the last Rayleigh-Ritz
    for it in range(1, max_outer + 1):
        stats = {"inner_steps": []}
        tol_rel = alpha * RF if alpha > 0 else 0.0
        if correction and C is not None and inner == "gmres":
            Q = _filtered_subspace_gmres_correction_nonsym(A, X, C, z, w, half, k, tol_rel, stats)
        elif inner == "exact":
            if A_dense is None:
                A_dense = A.toarray() if sp.issparse(A) else np.asarray(A)
            Q = _filtered_subspace_exact(A_dense, X, z, w, half)
        elif inner == "gmres":
            Q = _filtered_subspace_gmres(A, X, z, w, half, k, tol_rel, stats)
        else:
            raise ValueError(inner)
        # a full-circle rule pairs conjugate nodes: for real A and X the sum is real
        Q = np.asarray(Q.real, dtype=np.float64)
        AQ = A @ Q
        theta, U, Linv_T = rayleigh_ritz_nonsym(Q, AQ)
        X = Q @ Linv_T
        AX = AQ @ Linv_T
        C = X.T @ AX
        V = X @ U
        res = eigen_residuals(AX @ U, V, theta)
        inside = in_circle(theta, c, r)
        RF = float(res[inside].max()) if inside.any() else 1.0
        history.append(dict(RF=RF, count=int(inside.sum()),
                            max_inner=max(stats["inner_steps"], default=0)))
        if inside.any() and RF <= tol:
            return dict(theta=theta, V=V, res=res, inside=inside, iters=it, history=history,
                        converged=True)
    return dict(theta=theta, V=V, res=res, inside=inside, iters=max_outer, history=history,
                converged=False)


def filter_step_spectral_nonsym(A_dense, X, z, w, half=True):
    """sum_k w_k (z_k I - A)^{-1} X = V rho(Lambda) V^{-1} X for a diagonalisable
    A = V Lambda V^{-1}, rho(lambda) = sum_k w_k / (z_k - lambda) (Eq. rhoh with
    the eigenvector basis in place of an orthonormal one); real part for a
    half rule."""
    lam, V = np.linalg.eig(A_dense)
    rho = np.sum(w[None, :] / (z[None, :] - lam[:, None]), axis=1)
    Y = V @ (rho[:, None] * np.linalg.solve(V, X.astype(np.complex128)))
    return Y.real if half else Y


# ---------------------------------------------------------------------------
# One filtering step from the spectral definition (Eq. rhoh), for pins
# ---------------------------------------------------------------------------

def filter_step_spectral(A_dense, X, z, w, half=True, B_dense=None):
    """rho_hat X = U rho_hat(Lambda) U^H B X with A U = B U Lambda, U^H B U = I
    (Eq. rhoh; B = I for the standard problem)."""
    if B_dense is None:
        lam, U = np.linalg.eigh(A_dense)
        BX = X
    else:
        lam, U = sla.eigh(A_dense, B_dense)
        BX = B_dense @ X
    r = filter_rho(lam, z, w, half)
    return U @ (r[:, None] * (U.conj().T @ BX))


def convergence_bound_delta(lam_all, z, w, half=True):
    """Delta = sum_k ||w_k (z_k I - A)^{-1}|| (Eq. deltadef) over the nodes of the
    whole contour, for normal A with spectrum lam_all, where the resolvent's
    2-norm is 1 / min |z_k - lambda|. A half rule's weights hold the factor 2
    of the mirrored lower-half node (weight w_k / 2 at z_k and at conj(z_k),
    whose resolvents have the same norm), so both rules sum |w_k| / min|z_k - lambda|
    over the given nodes."""
    d = 0.0
    for zk, wk in zip(z, w):
        d += abs(wk) / np.min(np.abs(zk - lam_all))
    return d


# ---------------------------------------------------------------------------
# Step-level references for kernel parity (same maths as the steps above)
# ---------------------------------------------------------------------------

def ref_spmm_shift(A, V, zcol):
    """W[:, c] = zcol[c] V[:, c] - A V[:, c] (Alg. 2 step 1 operator on a block)."""
    return V * zcol[None, :] - A @ V


# ---------------------------------------------------------------------------
# Seeded random initial subspace (Alg. 1/2 input X^(0), "random"): the
# counter-based generator Philox4x32-10 from its published definition
# (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
# SC'11) and the Box-Muller transform
# ---------------------------------------------------------------------------

_PHILOX_M0, _PHILOX_M1 = 0xD2511F53, 0xCD9E8D57      # round multipliers
_PHILOX_W0, _PHILOX_W1 = 0x9E3779B9, 0xBB67AE85      # key increments (Weyl sequence)


def philox4x32_10(counter, key):
    """Philox4x32 with 10 rounds on arrays of counters: counter (4, N) and key
    (2, N) unsigned 32-bit words; returns the (4, N) output words. One round:
    (hi0, lo0) = M0 * c0 and (hi1, lo1) = M1 * c2 as 64-bit products, then
    c = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key is bumped by
    (W0, W1) before every round but the first."""
    mask = np.uint64(0xFFFFFFFF)
    c = [np.asarray(counter[i], dtype=np.uint64) & mask for i in range(4)]
    k0 = np.asarray(key[0], dtype=np.uint64) & mask
    k1 = np.asarray(key[1], dtype=np.uint64) & mask
    for r in range(10):
        if r > 0:
            k0 = (k0 + np.uint64(_PHILOX_W0)) & mask
            k1 = (k1 + np.uint64(_PHILOX_W1)) & mask
        p0 = np.uint64(_PHILOX_M0) * c[0]   # < 2^64: exact in uint64
        p1 = np.uint64(_PHILOX_M1) * c[2]
        c = [(p1 >> np.uint64(32)) ^ c[1] ^ k0, p1 & mask,
             (p0 >> np.uint64(32)) ^ c[3] ^ k1, p0 & mask]
    return np.stack(c).astype(np.uint32)


def seeded_normal_block(n, m0, seed):
    """X^(0): n x m0 (row-major) i.i.d. N(0,1). Element pair e = 2p, 2p + 1
    takes the Philox4x32-10 block of counter (p mod 2^32, p div 2^32, 0, 0)
    under key (seed mod 2^32, seed div 2^32); its words x0..x3 make the 53-bit
    uniforms u1 = (2^26 (x0 >> 5) + (x1 >> 6) + 1) / 2^53 in (0, 1] and
    u2 = (2^26 (x2 >> 5) + (x3 >> 6)) / 2^53 in [0, 1), and Box-Muller gives
    sqrt(-2 ln u1) cos(2 pi u2) and sqrt(-2 ln u1) sin(2 pi u2)."""
    total = n * m0
    pairs = (total + 1) // 2
    p = np.arange(pairs, dtype=np.uint64)
    zero = np.zeros(pairs, dtype=np.uint64)
    ctr = [p & np.uint64(0xFFFFFFFF), p >> np.uint64(32), zero, zero]
    key = [np.full(pairs, seed & 0xFFFFFFFF, dtype=np.uint64),
           np.full(pairs, (seed >> 32) & 0xFFFFFFFF, dtype=np.uint64)]
    x = philox4x32_10(ctr, key).astype(np.uint64)
    a = (x[0] >> np.uint64(5)) * np.uint64(1 << 26) + (x[1] >> np.uint64(6))
    b = (x[2] >> np.uint64(5)) * np.uint64(1 << 26) + (x[3] >> np.uint64(6))
    u1 = (a.astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = b.astype(np.float64) * 2.0 ** -53
    rad = np.sqrt(-2.0 * np.log(u1))
    t = (2.0 * math.pi) * u2
    out = np.empty(2 * pairs)
    out[0::2] = rad * np.cos(t)
    out[1::2] = rad * np.sin(t)
    return out[:total].reshape(n, m0)


# ---------------------------------------------------------------------------
# Eigenpairs an interval holds, from the plain definition (the problem
# statement of Section 1): for checks at sizes a dense solver cannot reach
# ---------------------------------------------------------------------------

def grid_nested_dissection(shape):
    """A fill-reducing symmetric ordering of the unknowns of a grid (last
    index fastest) for the sparse LU below: geometric nested dissection,
    i.e. split the box at the middle plane of its longest side, order the two
    halves recursively and the separating plane last. Returns a permutation
    of range(prod(shape))."""
    idx = np.arange(int(np.prod(shape))).reshape(shape)
    out = []

    def rec(block):
        if block.size <= 64:
            out.append(block.ravel())
            return
        ax = int(np.argmax(block.shape))
        m = block.shape[ax] // 2
        rec(block.take(range(0, m), axis=ax))
        rec(block.take(range(m + 1, block.shape[ax]), axis=ax))
        out.append(block.take([m], axis=ax).ravel())

    rec(idx)
    return np.concatenate(out)


def eigenpairs_near(A, sigma, k, perm=None):
    """The k eigenpairs of the real symmetric sparse A whose eigenvalues lie
    closest to sigma, by shift-invert Lanczos (ARPACK through
    scipy.sparse.linalg.eigsh with a sparse LU of A - sigma I: eigenvalues nu
    of (A - sigma I)^{-1}, lambda = sigma + 1/nu), one library step. perm: an
    optional symmetric ordering applied before the LU (fill only; the
    operator is the same). Returns (lam ascending, X unit columns, res) with
    res_j = ||A x_j - lam_j x_j||; for symmetric A an exact eigenvalue lies
    within res_j of lam_j."""
    import scipy.sparse.linalg as spla
    A = sp.csr_matrix(A)
    n = A.shape[0]
    M = (A - sigma * sp.identity(n, format="csr")).tocsr()
    if perm is None:
        lu = spla.splu(M.tocsc(), permc_spec="MMD_AT_PLUS_A")
        solve = lu.solve
    else:
        perm = np.asarray(perm)
        lu = spla.splu(M[perm][:, perm].tocsc(), permc_spec="NATURAL", diag_pivot_thresh=0.1,
                       options=dict(SymmetricMode=True))

        def solve(b):
            y = np.empty_like(b)
            y[perm] = lu.solve(b[perm])
            return y
    op = spla.LinearOperator(A.shape, matvec=solve, dtype=np.float64)
    lam, X = spla.eigsh(A, k=k, sigma=sigma, which="LM", OPinv=op, tol=0.0)
    order = np.argsort(lam)
    lam, X = lam[order], X[:, order]
    X = X / np.linalg.norm(X, axis=0)[None, :]
    res = np.linalg.norm(A @ X - X * lam[None, :], axis=0)
    return lam, X, res


def eigenvalues_in_interval(A, emin, emax, k, perm=None):
    """All eigenvalues of the real symmetric A inside the open interval (emin,
    emax), with their residual bounds, from the k eigenvalues closest to the
    centre: the set is complete when the farthest of the k lies at or beyond
    the half-width on each side of the centre found (then no eigenvalue of
    the interval is left out); raises otherwise. Also returns the nearest
    eigenvalue found below emin and above emax (the gaps at the ends)."""
    c, r = 0.5 * (emin + emax), 0.5 * (emax - emin)
    lam, _, res = eigenpairs_near(A, c, k, perm)
    if not (lam.min() <= emin and lam.max() >= emax):
        raise ValueError("k too small: the eigenvalues found do not reach both interval ends")
    inside = (lam > emin) & (lam < emax)
    below = lam[lam <= emin].max()
    above = lam[lam >= emax].min()
    return lam[inside], res[inside], below, above


# ---------------------------------------------------------------------------
# Textbook closed form used as a pin (not part of the method)
# ---------------------------------------------------------------------------

def laplacian_closed_form_eigs(grid):
    """Eigenvalues of the unit-spacing Dirichlet finite-difference Laplacian on
    a d-dimensional grid: sum over dimensions of 2 - 2 cos(p pi/(N+1)),
    p = 1..N. Ascending."""
    ev = np.zeros(1)
    for N in grid:
        mu = 2.0 - 2.0 * np.cos(np.arange(1, N + 1) * math.pi / (N + 1))
        ev = (ev[:, None] + mu[None, :]).ravel()
    return np.sort(ev)
