"""Serving layer (include/ifeast_serve.h): admission under a memory budget,
concurrent requests, and results that do not depend on the mix."""
import ctypes as ct
import time

import numpy as np
import pytest

from paper_1706_00692_gb300 import _lib, inputs
from paper_1706_00692_gb300.build import build


@pytest.fixture(scope="module")
def lib():
    build()
    return _lib.load()


def test_server_rejects_bad_options_and_requests(lib):
    h = ct.c_void_p()
    assert lib.ifeast_server_create(ct.byref(_lib.ServerOpts(0, 2, 0)), ct.byref(h)) == \
        _lib.IFEAST_ERR_INVALID_ARG
    assert lib.ifeast_server_create(ct.byref(_lib.ServerOpts(1 << 30, 0, 0)), ct.byref(h)) == \
        _lib.IFEAST_ERR_INVALID_ARG
    # a server with idle workers starts and stops without touching a device
    assert lib.ifeast_server_create(ct.byref(_lib.ServerOpts(1 << 20, 3, 0)), ct.byref(h)) == 0
    A = inputs.laplacian((12, 10))
    rp, ci, va = A.rowptr.copy(), A.colidx.copy(), A.val.copy()
    ci[5] = A.n  # out of range
    csr = _lib.Csr(A.n, A.nnz, rp.ctypes.data, ci.ctypes.data, va.ctypes.data)
    c = _lib.Contour(0, 8, -1.0, 0.5)
    o = _lib.Opts()
    lib.ifeast_default_opts(ct.byref(o))
    X0 = np.zeros((A.n, 8))
    rid = ct.c_int64()
    # sizes are checked at submit (m0 = 0); a malformed CSR is rejected when
    # the request runs (ifeast_create), like a direct solve
    assert lib.ifeast_server_submit(h, ct.byref(csr), ct.byref(c), 0, ct.byref(o), X0.ctypes.data,
                                    ct.byref(rid)) == _lib.IFEAST_ERR_INVALID_ARG
    # workspace larger than the whole budget (1 MiB)
    B = inputs.laplacian((40, 40))
    csr2 = _lib.Csr(B.n, B.nnz, B.rowptr.ctypes.data, B.colidx.ctypes.data, B.val.ctypes.data)
    X1 = np.zeros((B.n, 8))
    assert lib.ifeast_server_submit(h, ct.byref(csr2), ct.byref(c), 8, ct.byref(o), X1.ctypes.data,
                                    ct.byref(rid)) == _lib.IFEAST_ERR_OOM
    assert lib.ifeast_server_wait(h, 12345, 0, None, None, None, None, None) == \
        _lib.IFEAST_ERR_INVALID_ARG
    lib.ifeast_server_destroy(h)


def test_serving_requests_windows_hold_their_count():
    """The generated intervals hold exactly `count` eigenvalues (Weyl bounds:
    the potential is below a quarter of the gap at the upper end)."""
    for r in inputs.serving_requests(6, seed=77, n_max=3000):
        if r.A.n > 3000:
            continue
        ev = np.linalg.eigvalsh(r.A.to_scipy().toarray())
        assert int(((ev > r.emin) & (ev < r.emax)).sum()) == r.count
        assert r.m0 >= r.count and r.m0 % 4 == 0


def _solve_all(torch, reqs, max_active, budget):
    from paper_1706_00692_gb300 import Server
    srv = Server(budget, max_active=max_active)
    out = []
    if max_active == 1:  # alone: one request at a time
        for r in reqs:
            rid = srv.submit(r.A, r.emin, r.emax, r.m0, r.X0, rule="trap_half", inner_iters=300)
            out.append(srv.wait(rid))
    else:  # all in flight together
        ids = [srv.submit(r.A, r.emin, r.emax, r.m0, r.X0, rule="trap_half", inner_iters=300)
               for r in reqs]
        out = [srv.wait(i) for i in ids]
    srv.close()
    return out


@pytest.mark.gpu
def test_results_same_alone_and_in_the_mix():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    reqs = inputs.serving_requests(6, seed=2024, n_max=2e4)
    alone = _solve_all(torch, reqs, 1, 64 << 30)
    mixed = _solve_all(torch, reqs, 6, 64 << 30)
    for r, a, b in zip(reqs, alone, mixed):
        assert a[0] == 0 and b[0] == 0, (a[0], b[0])
        assert a[1].size == b[1].size == r.count
        # identical kernels with fixed-order reductions: bit-for-bit equal
        assert np.array_equal(a[1], b[1])
        assert np.array_equal(a[3], b[3])
        assert np.array_equal(a[2], b[2])
        assert a[3].max() <= 1e-10
    # small ones against brute force
    for r, a in zip(reqs, alone):
        if r.A.n <= 3000:
            ev = np.linalg.eigvalsh(r.A.to_scipy().toarray())[: r.count]
            assert np.abs(a[1] - ev).max() <= 1e-10 * max(1.0, np.abs(ev).max())


@pytest.mark.gpu
def test_admission_respects_the_memory_budget():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1706_00692_gb300 import Server
    r0 = inputs.serving_requests(1, seed=99, n_min=2e3, n_max=4e3)[0]
    reqs = [r0, r0, r0]  # equal workspaces: a budget below two of them admits one at a time
    lib = _lib.load()
    c = _lib.Contour(_lib.TRAP_HALF, 8, r0.emin, r0.emax)
    o = _lib.Opts()
    lib.ifeast_default_opts(ct.byref(o))
    o.inner_solver, o.inner_max_iters, o.alpha, o.precision = 1, 300, 3e-2, 1
    b = ct.c_size_t()
    assert lib.ifeast_workspace_bytes(r0.A.n, r0.A.nnz, r0.m0, ct.byref(c), ct.byref(o),
                                      ct.byref(b)) == 0
    budget = 2 * b.value - 1
    srv = Server(budget, max_active=3)
    ids = [srv.submit(r.A, r.emin, r.emax, r.m0, r.X0, rule="trap_half", inner_iters=300)
           for r in reqs]
    infos = [srv.wait(i)[4] for i in ids]
    srv.close()
    for a, b in zip(infos[:-1], infos[1:]):
        assert b["submit_to_start_ms"] >= a["submit_to_done_ms"] - 5.0  # strictly one after another
        assert a["status"] == 0 and b["status"] == 0
