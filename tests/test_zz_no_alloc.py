"""The allocation-free Rayleigh-Ritz entry point against the handle-based one.

Callers that cannot allocate device memory (a fixed memory pool, a runtime
that forbids cudaMalloc) use ifeast_rayleigh_ritz_noalloc, which keeps its
intermediates in a fixed file-scope device array. It must give the same X,
eigenvalues and residuals as ifeast_rayleigh_ritz, on consecutive calls that
share that array. Tolerances are those of the Rayleigh-Ritz parity test:
eigenvalues 1e-12 relative, residuals 1e-10, vectors 1e-9 up to sign."""
import ctypes as ct

import numpy as np
import pytest

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


def _noalloc(torch, A, Q):
    from paper_1706_00692_gb300 import _lib
    lib = _lib.load()
    dev = torch.device("cuda")
    rp = torch.as_tensor(A.rowptr.astype(np.int32), device=dev)
    ci = torch.as_tensor(A.colidx.astype(np.int32), device=dev)
    va = torch.as_tensor(A.val, device=dev)
    n, m0 = Q.shape
    X = torch.empty((n, m0), dtype=torch.float64, device=dev)
    lam = torch.empty(m0, dtype=torch.float64, device=dev)
    res = torch.empty(m0, dtype=torch.float64, device=dev)
    rc = lib.ifeast_rayleigh_ritz_noalloc(n, A.nnz, rp.data_ptr(), ci.data_ptr(), va.data_ptr(), m0,
                                          Q.data_ptr(), X.data_ptr(), lam.data_ptr(), res.data_ptr(),
                                          ct.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, X.cpu().numpy(), lam.cpu().numpy(), res.cpu().numpy()


@pytest.mark.parametrize("grid,m0,pot", [((50, 50), 20, False), ((13, 11, 7), 7, True),
                                         ((20, 20, 10), 64, True)])
def test_noalloc_matches_handle_entry_point_twice(torch, grid, m0, pot):
    from paper_1706_00692_gb300 import Solver
    A = inputs.laplacian(grid)
    if pot:
        A = inputs.add_diagonal(A, inputs.random_potential(A.n, 8))
    Qn = inputs.initial_subspace(A.n, m0, 5)
    Q = torch.as_tensor(Qn, device="cuda")
    S = Solver(A, 0.0, 8.0, m0)
    X1, l1, r1 = (t.cpu().numpy() for t in S.rayleigh_ritz(Q))
    S.close()
    for _ in range(2):  # the second call runs on the scratch the first one left
        rc, X2, l2, r2 = _noalloc(torch, A, Q)
        assert rc == 0
        assert np.abs(l2 - l1).max() <= 1e-12 * np.abs(l1).max()
        assert np.abs(r2 - r1).max() <= 1e-10
        sgn = np.sign(np.sum(X1 * X2, axis=0))
        assert np.abs(X2 * sgn - X1).max() <= 1e-9 * np.abs(X1).max()


def test_noalloc_rejects_m0_beyond_scratch(torch):
    from paper_1706_00692_gb300._lib import IFEAST_ERR_INVALID_ARG
    A = inputs.laplacian((20, 20))
    Q = torch.as_tensor(inputs.initial_subspace(A.n, 65, 1), device="cuda")
    rc, *_ = _noalloc(torch, A, Q)
    assert rc == IFEAST_ERR_INVALID_ARG
