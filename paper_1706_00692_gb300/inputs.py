"""Seeded synthetic inputs for the IFEAST hot path.

This module is shared by the CUDA path's callers (tests, bench) and by the
CPU oracle's tests. It holds no arithmetic of the eigensolver itself: it only
builds the sparse test matrices, the random potential and the random initial
subspace, and names the workloads.

The paper measures on PARSEC Hamiltonians (Si2, n=769; Na5, n=5832; Section 4)
that are not available here. Seeded finite-difference Laplacians (a real
symmetric, sparse, Hamiltonian-like operator: kinetic term plus an optional
random diagonal potential) stand in for them.

CSR convention used everywhere: ``rowptr`` int32 (n+1), ``colidx`` int32
(nnz, ascending within a row), ``val`` float64 (nnz). Dense blocks are numpy
float64 arrays of shape (n, m0), C-contiguous (row i holds m0 entries).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class CSR:
    n: int
    rowptr: np.ndarray
    colidx: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.colidx.shape[0])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.colidx, self.rowptr), shape=(self.n, self.n))


def _csr_from_coo(n, rows, cols, vals) -> CSR:
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    counts = np.bincount(rows, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return CSR(n, rowptr.astype(np.int32), cols.astype(np.int32), vals.astype(np.float64))


def laplacian(grid: tuple[int, ...]) -> CSR:
    """Dirichlet finite-difference Laplacian (unit spacing) on a d-dimensional
    grid: 2d on the diagonal, -1 for each of the 2d nearest neighbours inside
    the grid (5-point in 2D, 7-point in 3D). Unknowns are numbered with the
    last grid index fastest."""
    grid = tuple(int(g) for g in grid)
    d = len(grid)
    n = int(np.prod(grid))
    idx = np.arange(n, dtype=np.int64).reshape(grid)
    rows = [idx.ravel()]
    cols = [idx.ravel()]
    vals = [np.full(n, 2.0 * d)]
    for ax in range(d):
        lo = [slice(None)] * d
        hi = [slice(None)] * d
        lo[ax] = slice(0, grid[ax] - 1)
        hi[ax] = slice(1, grid[ax])
        a = idx[tuple(lo)].ravel()
        b = idx[tuple(hi)].ravel()
        rows += [a, b]
        cols += [b, a]
        vals += [np.full(a.size, -1.0), np.full(a.size, -1.0)]
    return _csr_from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def add_diagonal(A: CSR, d: np.ndarray) -> CSR:
    """A + diag(d); every row of A already holds its diagonal entry."""
    val = A.val.copy()
    for i in range(A.n):
        lo, hi = A.rowptr[i], A.rowptr[i + 1]
        k = lo + int(np.searchsorted(A.colidx[lo:hi], i))
        assert A.colidx[k] == i
        val[k] += d[i]
    return CSR(A.n, A.rowptr.copy(), A.colidx.copy(), val)


def add_diagonal_fast(A: CSR, d: np.ndarray) -> CSR:
    """Vectorised add_diagonal for large stencils (same result)."""
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    val = A.val.copy()
    diag = rows == A.colidx
    assert int(diag.sum()) == A.n
    val[diag] += d[rows[diag]]
    return CSR(A.n, A.rowptr.copy(), A.colidx.copy(), val)


def random_potential(n: int, seed: int) -> np.ndarray:
    """Diagonal potential, i.i.d. uniform on [0, 1), numpy PCG64(seed)."""
    return np.random.Generator(np.random.PCG64(seed)).uniform(0.0, 1.0, n)


def initial_subspace(n: int, m0: int, seed: int) -> np.ndarray:
    """Random initial search subspace X^(0): i.i.d. N(0,1), n x m0, PCG64(seed)."""
    return np.random.Generator(np.random.PCG64(seed)).standard_normal((n, m0))


def random_sparse_symmetric(n: int, nnz_per_row: int, seed: int) -> CSR:
    """Random real symmetric sparse matrix with a ragged row-length mix
    (1 .. 2*nnz_per_row off-diagonals per row before symmetrisation), values
    N(0,1), diagonal uniform on [0, 4). Used for SpMM edge cases."""
    g = np.random.Generator(np.random.PCG64(seed))
    rows, cols = [], []
    for i in range(n):
        k = int(g.integers(0, 2 * nnz_per_row + 1))
        c = g.integers(0, n, size=k)
        rows.append(np.full(k, i))
        cols.append(c)
    r = np.concatenate(rows) if rows else np.zeros(0, np.int64)
    c = np.concatenate(cols) if cols else np.zeros(0, np.int64)
    keep = r != c
    r, c = r[keep], c[keep]
    v = g.standard_normal(r.size)
    rr = np.concatenate([r, c, np.arange(n)])
    cc = np.concatenate([c, r, np.arange(n)])
    vv = np.concatenate([v, v, g.uniform(0.0, 4.0, n)])
    # merge duplicates
    key = rr.astype(np.int64) * n + cc
    uk, inv = np.unique(key, return_inverse=True)
    vals = np.zeros(uk.size)
    np.add.at(vals, inv, vv)
    return _csr_from_coo(n, (uk // n).astype(np.int64), (uk % n).astype(np.int64), vals)


def _kron_csr(mats):
    import scipy.sparse as sp
    out = mats[0]
    for m in mats[1:]:
        out = sp.kron(out, m, format="csr")
    return out


def fem_q1(grid: tuple[int, ...]) -> tuple[CSR, CSR]:
    """Stiffness K and mass M of multilinear (Q1) finite elements for -Laplace
    on the unit cube with Dirichlet boundary, N interior nodes per dimension
    (h = 1/(N+1)): K = sum_d M1 x .. x K1 (slot d) x .. x M1, M = M1 x .. x M1
    with K1 = (1/h) tridiag(-1, 2, -1), M1 = (h/6) tridiag(1, 4, 1). 9-point in
    2D, 27-point in 3D; M is symmetric positive definite. Both share K's
    sparsity pattern (M's entries are stored on it)."""
    import scipy.sparse as sp
    K1s, M1s = [], []
    for N in grid:
        h = 1.0 / (N + 1)
        e = np.ones(N)
        K1s.append(sp.diags([-e[:-1], 2 * e, -e[:-1]], [-1, 0, 1], format="csr") / h)
        M1s.append(sp.diags([e[:-1], 4 * e, e[:-1]], [-1, 0, 1], format="csr") * (h / 6.0))
    d = len(grid)
    K = None
    for a in range(d):
        term = _kron_csr([K1s[b] if b == a else M1s[b] for b in range(d)])
        K = term if K is None else K + term
    M = _kron_csr(M1s)
    pattern = (abs(K) + abs(M)).tocsr()
    pattern.sort_indices()
    n = pattern.shape[0]

    def on_pattern(X):
        X = X.tocsr()
        out = np.zeros(pattern.nnz)
        rows = np.repeat(np.arange(n), np.diff(pattern.indptr))
        out[:] = np.asarray(X[rows, pattern.indices]).ravel()
        return CSR(n, pattern.indptr.astype(np.int32), pattern.indices.astype(np.int32), out)

    return on_pattern(K), on_pattern(M)


def upwind_convection_diffusion(grid: tuple[int, int], Pe: float) -> CSR:
    """-Laplace u + Pe du/dx on (0,1)^2 with Dirichlet boundary, N_x x N_y
    interior nodes (h_d = 1/(N_d+1)), second differences in both directions
    and a first-order upwind difference for du/dx: the x-line stencil is
    (-1/h^2 - Pe/h, 2/h^2 + Pe/h, -1/h^2) (sub-, main, super-diagonal). Real,
    non-symmetric; row index i + N_x j."""
    import scipy.sparse as sp
    Nx, Ny = grid
    hx, hy = 1.0 / (Nx + 1), 1.0 / (Ny + 1)
    ex, ey = np.ones(Nx), np.ones(Ny)
    Tx = sp.diags([(-1.0 / hx ** 2 - Pe / hx) * ex[:-1], (2.0 / hx ** 2 + Pe / hx) * ex,
                   (-1.0 / hx ** 2) * ex[:-1]], [-1, 0, 1], format="csr")
    Ty = sp.diags([(-1.0 / hy ** 2) * ey[:-1], (2.0 / hy ** 2) * ey, (-1.0 / hy ** 2) * ey[:-1]],
                  [-1, 0, 1], format="csr")
    M = (sp.kron(sp.identity(Ny), Tx) + sp.kron(Ty, sp.identity(Nx))).tocsr()
    M.sort_indices()
    return CSR(M.shape[0], M.indptr.astype(np.int32), M.indices.astype(np.int32),
               M.data.astype(np.float64))


def upwind_convection_diffusion_eigs(grid: tuple[int, int], Pe: float) -> np.ndarray:
    """Eigenvalues of upwind_convection_diffusion(grid, Pe), ascending (real):
    a tridiagonal Toeplitz (a, b, c) with a c > 0 has b + 2 sqrt(ac) cos(p pi/(N+1)),
    and the 2D operator is the Kronecker sum of the two 1D ones."""
    Nx, Ny = grid
    hx, hy = 1.0 / (Nx + 1), 1.0 / (Ny + 1)
    a, b, c = -1.0 / hx ** 2 - Pe / hx, 2.0 / hx ** 2 + Pe / hx, -1.0 / hx ** 2
    lx = b - 2.0 * math.sqrt(a * c) * np.cos(np.arange(1, Nx + 1) * math.pi / (Nx + 1))
    ly = (2.0 / hy ** 2) * (1.0 - np.cos(np.arange(1, Ny + 1) * math.pi / (Ny + 1)))
    return np.sort((lx[:, None] + ly[None, :]).ravel())


def fem_q1_eigs(grid: tuple[int, ...]) -> np.ndarray:
    """Eigenvalues of K x = lambda M x for fem_q1(grid), ascending: sums over the
    dimensions of (6/h^2)(1 - cos t)/(2 + cos t), t = p pi/(N+1), p = 1..N."""
    ev = np.zeros(1)
    for N in grid:
        h = 1.0 / (N + 1)
        t = np.arange(1, N + 1) * math.pi / (N + 1)
        mu = (6.0 / h ** 2) * (1 - np.cos(t)) / (2 + np.cos(t))
        ev = (ev[:, None] + mu[None, :]).ravel()
    return np.sort(ev)


# ---------------------------------------------------------------------------
# Closed-form spectra of the stencils (used to place interval endpoints in
# spectral gaps and as test pins).
# ---------------------------------------------------------------------------

def laplacian_1d_eigs(N: int) -> np.ndarray:
    p = np.arange(1, N + 1)
    return 2.0 - 2.0 * np.cos(p * math.pi / (N + 1))


def laplacian_eigs(grid: tuple[int, ...]) -> np.ndarray:
    """All eigenvalues of laplacian(grid), ascending (sum of 1D spectra)."""
    ev = np.zeros(1)
    for N in grid:
        ev = (ev[:, None] + laplacian_1d_eigs(N)[None, :]).ravel()
    return np.sort(ev)


@dataclasses.dataclass
class Workload:
    name: str
    A: CSR
    emin: float
    emax: float
    m0: int
    nc: int
    rule: str
    inner_iters: int
    alpha: float
    seed: int
    expected_count: int | None = None
    inner: str = "gmres"
    precision: str = "fp64"
    two_pass: bool = False  # shared-basis solver without the stored basis
    B: CSR | None = None  # generalized problem A x = lambda B x (None: B = I)
    node_chunk: int = 0   # per-node GMRES: nodes per inner pass (0: all)
    nonsym: bool = False  # real non-symmetric A (per-node GMRES, complex Ritz pairs)
    nonsym_correction: bool = False  # non-symmetric block correction of the shifted systems

    def X0(self) -> np.ndarray:
        return initial_subspace(self.A.n, self.m0, self.seed)


def workload_convdiff(N: int = 512, count: int = 40, m0: int = 64, Pe: float = 10.0) -> Workload:
    """2D convection-diffusion, 5-point upwind, on an N x N grid (n = N^2, Peclet
    Pe): real non-symmetric A with a closed-form real spectrum. The circle
    through 0 and emax, emax in the gap after the count-th lowest eigenvalue,
    holds count eigenvalues; m0 = 64, 16 trapezoid nodes on the circle (8 on the
    upper half: conjugate nodes pair up for real A), GMRES(32) in FP64, solved
    for the block correction from the second outer iteration on."""
    cf = upwind_convection_diffusion_eigs((N, N), Pe)
    emax = 0.5 * (cf[count - 1] + cf[count])
    wl = Workload(f"convdiff_{N}x{N}_pe{int(Pe)}_lowest{count}_m0_{m0}_trap16_gmres32_blockcorr",
                  upwind_convection_diffusion((N, N), Pe), 0.0, emax, m0=m0, nc=8,
                  rule="trap_half", inner_iters=32, alpha=0.0, seed=0, expected_count=count)
    wl.nonsym = True
    wl.nonsym_correction = True
    return wl


def workload_lap2d_50(seed: int = 0) -> Workload:
    """2D 5-point Dirichlet Laplacian on a 50x50 grid (n=2500), interval
    enclosing the 10 lowest eigenvalues, m0=20, 8 Gauss-Legendre nodes on the
    upper half circle, GMRES fixed at 10 iterations."""
    ev = laplacian_eigs((50, 50))
    emin, emax = 0.0, 0.5 * (ev[9] + ev[10])
    return Workload("lap2d_50x50_m0_20_gl8_gmres10", laplacian((50, 50)), emin, emax,
                    m0=20, nc=8, rule="gl_half", inner_iters=10, alpha=0.0, seed=seed,
                    expected_count=10)


def workload_lap3d_pot(N: int = 64, seed: int = 0, m0: int = 80, first: int = 1000,
                       count: int = 50, nc: int = 8, inner_iters: int = 400,
                       alpha: float = 1e-3) -> Workload:
    """3D 7-point Dirichlet Laplacian on N^3 plus a U[0,1) diagonal potential.
    The interior window is placed from the pure-Laplacian spectrum shifted by
    the potential's mean 0.5: (lam_L[first] + 0.5, lam_L[first+count] + 0.5)
    (0-based indices into the ascending closed-form spectrum, endpoints taken
    half way between neighbours)."""
    ev = laplacian_eigs((N, N, N))
    emin = 0.5 * (ev[first - 1] + ev[first]) + 0.5
    emax = 0.5 * (ev[first + count - 1] + ev[first + count]) + 0.5
    A = add_diagonal_fast(laplacian((N, N, N)), random_potential(N ** 3, seed + 1))
    return Workload(f"lap3d_{N}^3_pot_interior_m0_{m0}_gl{nc}", A, emin, emax, m0=m0, nc=nc,
                    rule="gl_half", inner_iters=inner_iters, alpha=alpha, seed=seed)


# Interior window of the 64^3 Laplacian + U[0,1) potential (potential seed 1):
# each endpoint is the midpoint of a spectral gap of the matrix, 4.6e-4
# (lower) and 5.8e-4 (upper), about 1/27 and 1/21 of the window width: the
# widest gaps within 1e-3 of [lam_L(1001) + 0.5, lam_L(1051) + 0.5] (the pure
# Laplacian's closed-form eigenvalues shifted by the potential's mean). The
# eigenvalues come from the CPU oracle's shift-invert Lanczos, stored with the
# window in tests/golden/lap3d64_window.txt (its script derives the endpoints;
# a test checks that these constants equal the file's); the window holds 56
# eigenvalues (the ~50 of the workload definition). Endpoints in narrower gaps
# let Ritz values of the eigenvectors just outside drift across the endpoint
# between iterations.
LAP3D_64_WINDOW = (0.8975465841391953, 0.9100123760852886)


def workload_lap3d_64_interior(seed: int = 0, precision: str = "fp32", alpha: float = 3e-2,
                               inner_iters: int = 1500, two_pass: bool = False) -> Workload:
    """3D 7-point Laplacian on 64^3 (n = 262,144) plus a U[0,1) diagonal
    potential, interior window with 56 eigenvalues, m0 = 80, 8 trapezoid nodes
    on the upper half circle, shared-basis MINRES inner solves (at most 1500
    Lanczos steps, tolerance alpha = 3e-2 of ||R_F||)."""
    N = 64
    A = add_diagonal_fast(laplacian((N, N, N)), random_potential(N ** 3, seed + 1))
    emin, emax = LAP3D_64_WINDOW
    wl = Workload(f"lap3d_64^3_pot_interior56_m0_80_trap8_minres_{precision}", A, emin, emax,
                  m0=80, nc=8, rule="trap_half", inner_iters=inner_iters, alpha=alpha, seed=seed,
                  expected_count=56 if seed == 0 else None)
    wl.inner = "minres"
    wl.precision = precision
    wl.two_pass = two_pass
    if two_pass:
        wl.name += "_twopass"
    return wl


def _gap_count(ev: np.ndarray, target: int, rel: float = 1e-3) -> int:
    """Smallest count >= target whose next eigenvalue lies rel * ev[count] or
    more above the last one (an interval endpoint in a spectral gap)."""
    for c in range(target, len(ev) - 1):
        if ev[c] - ev[c - 1] > rel * ev[c]:
            return c
    raise ValueError("no gap")


def workload_fem3d_128(precision: str = "fp32", node_chunk: int = 2) -> Workload:
    """The 27-point generalized workload at 128^3 (n = 2,097,152): Q1 trilinear
    FEM K x = lambda M x, the lowest eigenvalues through the 6-fold cluster that
    holds the 100th (102 pairs; the upper endpoint is the midpoint of the gap
    after eigenvalue 102), m0 = 150, 12 Gauss-Legendre half-circle nodes,
    per-node GMRES with at most 32 steps and alpha = 1e-2 (FP32 basis, residual
    form below ||R_F|| = 1e-3), node_chunk nodes per pass (the 12 nodes' bases
    together would need about 1 TB)."""
    N = 128
    K, M = fem_q1((N, N, N))
    ev = fem_q1_eigs((N, N, N))
    cnt = _gap_count(ev, 100)
    emax = 0.5 * (ev[cnt - 1] + ev[cnt])
    wl = Workload(f"fem3d_128^3_lowest{cnt}_m0_150_gl12_gmres32_{precision}_chunk{node_chunk}", K,
                  0.0, emax, m0=150, nc=12, rule="gl_half", inner_iters=32, alpha=1e-2, seed=0,
                  expected_count=cnt)
    wl.precision = precision
    wl.B = M
    wl.node_chunk = node_chunk
    return wl


def workload_fem3d(N: int = 64, target: int = 50, precision: str = "fp32") -> Workload:
    """Generalized problem K x = lambda M x of Q1 trilinear finite elements on an
    N^3 interior grid (27-point K and M on one pattern; closed-form spectrum),
    the lowest eigenvalues up to the first spectral gap at or after `target`
    (54 pairs at N = 64), m0 = 1.5 count + 2, 12 Gauss-Legendre nodes on the
    upper half circle, per-node GMRES with at most 32 steps and alpha = 1e-2
    (FP32 basis with the residual form, or FP64)."""
    K, M = fem_q1((N, N, N))
    ev = fem_q1_eigs((N, N, N))
    cnt = _gap_count(ev, target)
    emax = 0.5 * (ev[cnt - 1] + ev[cnt])
    m0 = int(1.5 * cnt) + 2
    wl = Workload(f"fem3d_{N}^3_lowest{cnt}_m0_{m0}_gl12_gmres32_{precision}", K, 0.0, emax,
                  m0=m0, nc=12, rule="gl_half", inner_iters=32, alpha=1e-2, seed=0,
                  expected_count=cnt)
    wl.precision = precision
    wl.B = M
    return wl


# ---------------------------------------------------------------------------
# Serving stream: many eigen-requests of different sizes and intervals
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Request:
    A: CSR
    emin: float
    emax: float
    m0: int
    count: int          # eigenvalues inside (emin, emax)
    X0: np.ndarray
    arrival: float      # seconds after the start of the stream


def _grid_for(n_target: float, dim: int, g) -> tuple[int, ...]:
    """Grid sizes with product near n_target and distinct side lengths (fewer
    repeated eigenvalues)."""
    side = n_target ** (1.0 / dim)
    sizes = sorted({max(4, int(round(side * f))) for f in g.uniform(0.8, 1.25, dim)}, reverse=True)
    while len(sizes) < dim:
        sizes.append(sizes[-1] + len(sizes) + 1)
    return tuple(sizes)


def serving_requests(count: int, seed: int = 1234, n_min: float = 1e3, n_max: float = 2e5,
                     rate: float = 4.0, m0_min: int = 16, m0_max: int = 128) -> list[Request]:
    """A Poisson stream of eigen-requests: 2D or 3D Dirichlet Laplacians (fair
    coin) with n log-uniform in [n_min, n_max], a U[0, g/4) diagonal potential
    (g = the spectral gap at the upper interval end, so by Weyl's bounds every
    eigenvalue moves by less than g/4 and the window keeps its count), interval
    = the lowest k eigenvalues with the upper end half way across the widest
    gap among the closed-form eigenvalues k..k+3 and the lower end a quarter of
    the window below the lowest eigenvalue, m0 = 4 ceil(1.6 k / 4) in
    [m0_min, m0_max], initial subspace N(0,1), exponential inter-arrival times
    with mean 1/rate. Request i draws from PCG64(seed + i)."""
    out = []
    t = 0.0
    for i in range(count):
        g = np.random.Generator(np.random.PCG64(seed + i))
        t += g.exponential(1.0 / rate)
        dim = 2 if g.random() < 0.5 else 3
        n_target = math.exp(g.uniform(math.log(n_min), math.log(n_max)))
        grid = _grid_for(n_target, dim, g)
        ev = laplacian_eigs(grid)
        kmax = max(2, min(int(m0_max / 1.6) - 4, len(ev) // 4))
        k0 = int(g.integers(max(2, int(m0_min / 1.6)), kmax + 1))
        # widest gap among eigenvalues k0..k0+3 (ascending index k: gap ev[k] - ev[k-1])
        ks = np.arange(k0, min(k0 + 4, len(ev) - 1))
        gaps = ev[ks] - ev[ks - 1]
        k = int(ks[int(np.argmax(gaps))])
        gap = float(gaps.max())
        emax = 0.5 * (ev[k - 1] + ev[k])
        # lower end below the spectrum (the potential only raises eigenvalues),
        # close enough that the contour stays small relative to the gap at emax
        emin = ev[0] - 0.25 * (emax - ev[0])
        m0 = int(min(m0_max, max(m0_min, 4 * math.ceil(1.6 * k / 4))))
        A = laplacian(grid)
        A = add_diagonal_fast(A, 0.25 * gap * random_potential(A.n, seed + 100000 + i))
        X0 = initial_subspace(A.n, m0, seed + 200000 + i)
        out.append(Request(A, emin, emax, m0, k, X0, t))
    return out
