"""C ABI checks that need no GPU: the library loads, exports every function
declared in include/*.h, computes the contour like the oracle, and rejects
malformed input on the host before touching a device."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

from oracle import ifeast_oracle as orc
from paper_1706_00692_gb300 import _lib, inputs
from paper_1706_00692_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build()
    return _lib.load()


def _declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(inc, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(ifeast_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 12
    for nm in names:
        assert hasattr(lib, nm), nm
        assert nm in _lib.SIGNATURES, f"{nm} has no ctypes signature"


@pytest.mark.parametrize("rule,nc,emin,emax", [("gl_half", 8, 0.0, 0.066), ("gl_half", 1, -2.0, 3.0),
                                                ("gl_half", 24, 0.8968, 0.9104),
                                                ("trap_half", 4, 1.0, 5.0), ("trap_full", 16, 0.0, 629.7)])
def test_contour_nodes_match_oracle(lib, rule, nc, emin, emax):
    c = _lib.Contour(_lib.RULES[rule], nc, emin, emax)
    zw = np.zeros(4 * nc)
    assert lib.ifeast_contour_nodes(ct.byref(c), zw.ctypes.data) == 0
    zw = zw.reshape(nc, 4)
    z, w = orc.contour_nodes(rule, nc, emin, emax)
    scale = max(abs(emin), abs(emax), emax - emin)
    assert np.abs(zw[:, 0] + 1j * zw[:, 1] - z).max() <= 4e-16 * scale * 4
    assert np.abs(zw[:, 2] + 1j * zw[:, 3] - w).max() <= 4e-16 * (emax - emin) * 4


def test_contour_rejects_bad_interval(lib):
    zw = np.zeros(8)
    for c in [_lib.Contour(0, 2, 1.0, 1.0), _lib.Contour(0, 0, 0.0, 1.0), _lib.Contour(7, 2, 0.0, 1.0)]:
        assert lib.ifeast_contour_nodes(ct.byref(c), zw.ctypes.data) == _lib.IFEAST_ERR_INVALID_ARG


def _opts(lib, **kw):
    o = _lib.Opts()
    lib.ifeast_default_opts(ct.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def test_default_opts(lib):
    o = _opts(lib)
    assert (o.inner_solver, o.inner_max_iters, o.alpha, o.max_outer, o.tol, o.precision,
            o.verbose, o.nonsymmetric, o.minres_two_pass, o.correction_rf) == \
        (0, 10, 0.0, 100, 1e-10, 0, 0, 0, 0, 1e-3)


def test_fp32_gmres_workspace(lib):
    """The FP32 GMRES basis and work vector take half the bytes of the FP64 ones
    (plus FP32 copies of A, FP32 weights and the residual-form block)."""
    c = _lib.Contour(0, 8, 0.0, 1.0)
    n, nnz, m0, K = 4096, 20480, 16, 20
    b64, b32 = ct.c_size_t(), ct.c_size_t()
    assert lib.ifeast_workspace_bytes(n, nnz, m0, ct.byref(c), ct.byref(
        _opts(lib, inner_max_iters=K)), ct.byref(b64)) == 0
    assert lib.ifeast_workspace_bytes(n, nnz, m0, ct.byref(c), ct.byref(
        _opts(lib, inner_max_iters=K, precision=1)), ct.byref(b32)) == 0
    basis64 = (K + 2) * n * 8 * m0 * 16
    extra32 = nnz * 4 + K * 8 * m0 * 8 + n * m0 * 8 + 2 * m0 * 8
    assert abs((b64.value - b32.value) - (basis64 // 2 - extra32)) <= 16 * 256


def test_workspace_bytes_grows_with_basis(lib):
    c = _lib.Contour(0, 8, 0.0, 1.0)
    b1, b2 = ct.c_size_t(), ct.c_size_t()
    assert lib.ifeast_workspace_bytes(2500, 12300, 20, ct.byref(c), ct.byref(_opts(lib)), ct.byref(b1)) == 0
    assert lib.ifeast_workspace_bytes(2500, 12300, 20, ct.byref(c),
                                      ct.byref(_opts(lib, inner_max_iters=20)), ct.byref(b2)) == 0
    # the (k+1) x n x C complex basis dominates: 10 more vectors of 2500 x 160 x 16 bytes
    assert b2.value - b1.value >= 10 * 2500 * 160 * 16


def _create(lib, A, m0=4, opts=None, contour=None, B=None):
    rp = np.ascontiguousarray(A.rowptr, np.int32)
    ci = np.ascontiguousarray(A.colidx, np.int32)
    v = np.ascontiguousarray(A.val, np.float64)
    csr = _lib.Csr(A.n, A.nnz, rp.ctypes.data, ci.ctypes.data, v.ctypes.data)
    h = ct.c_void_p()
    c = contour or _lib.Contour(0, 4, 0.0, 1.0)
    rc = lib.ifeast_create(ct.byref(csr), B, ct.byref(c), m0, ct.byref(opts or _opts(lib)), None, 0,
                           None, ct.byref(h))
    return rc, h


def test_create_rejects_malformed_csr(lib):
    A = inputs.laplacian((5, 4))
    bad_col = inputs.CSR(A.n, A.rowptr.copy(), A.colidx.copy(), A.val.copy())
    bad_col.colidx[3] = A.n
    assert _create(lib, bad_col)[0] == _lib.IFEAST_ERR_INVALID_ARG
    bad_ptr = inputs.CSR(A.n, A.rowptr.copy(), A.colidx.copy(), A.val.copy())
    bad_ptr.rowptr[5], bad_ptr.rowptr[6] = bad_ptr.rowptr[6], bad_ptr.rowptr[5]
    assert _create(lib, bad_ptr)[0] == _lib.IFEAST_ERR_INVALID_ARG
    nan_val = inputs.CSR(A.n, A.rowptr.copy(), A.colidx.copy(), A.val.copy())
    nan_val.val[0] = np.nan
    assert _create(lib, nan_val)[0] == _lib.IFEAST_ERR_INVALID_ARG


def test_create_rejects_bad_options(lib):
    A = inputs.laplacian((5, 4))
    assert _create(lib, A, m0=0)[0] == _lib.IFEAST_ERR_INVALID_ARG
    assert _create(lib, A, m0=A.n + 1)[0] == _lib.IFEAST_ERR_INVALID_ARG
    assert _create(lib, A, opts=_opts(lib, inner_max_iters=0))[0] == _lib.IFEAST_ERR_INVALID_ARG
    assert _create(lib, A, opts=_opts(lib, inner_max_iters=33))[0] == _lib.IFEAST_ERR_INVALID_ARG
    assert _create(lib, A, opts=_opts(lib, max_outer=0))[0] == _lib.IFEAST_ERR_INVALID_ARG
    assert _create(lib, A, opts=_opts(lib, inner_solver=9))[0] == _lib.IFEAST_ERR_UNSUPPORTED
    # per-node GMRES: FP64 or FP32 basis (FP16 storage is the shared-basis solver's)
    assert _create(lib, A, opts=_opts(lib, precision=2))[0] == _lib.IFEAST_ERR_UNSUPPORTED
    # the FP32 GMRES basis needs the residual form, i.e. real Ritz pairs
    assert _create(lib, A, opts=_opts(lib, precision=1, nonsymmetric=1))[0] == \
        _lib.IFEAST_ERR_UNSUPPORTED
    for bad in (-1.0, float("nan")):
        assert _create(lib, A, opts=_opts(lib, correction_rf=bad))[0] == _lib.IFEAST_ERR_INVALID_ARG
    # FP16 storage needs the four-column kernels (m0 % 4 == 0)
    assert _create(lib, A, m0=7, opts=_opts(lib, inner_solver=1, inner_max_iters=8,
                                            precision=2))[0] == _lib.IFEAST_ERR_UNSUPPORTED
    assert _create(lib, A, opts=_opts(lib, precision=3))[0] == _lib.IFEAST_ERR_UNSUPPORTED
    assert _create(lib, A, opts=_opts(lib, inner_solver=1, inner_max_iters=5000))[0] == \
        _lib.IFEAST_ERR_INVALID_ARG
    assert _create(lib, A, contour=_lib.Contour(0, 4, 1.0, 0.5))[0] == _lib.IFEAST_ERR_INVALID_ARG
    # a full-circle rule needs an even node count (it runs as the half rule on nc/2)
    assert _create(lib, A, contour=_lib.Contour(2, 5, 0.0, 0.5))[0] == _lib.IFEAST_ERR_INVALID_ARG
    # the non-symmetric extension: GMRES inner solves, m0 <= 64, flag 0 or 1
    assert _create(lib, A, opts=_opts(lib, nonsymmetric=1, inner_solver=1,
                                      inner_max_iters=8))[0] == _lib.IFEAST_ERR_UNSUPPORTED
    big = inputs.laplacian((10, 10))
    assert _create(lib, big, m0=65, opts=_opts(lib, nonsymmetric=1))[0] == _lib.IFEAST_ERR_UNSUPPORTED
    assert _create(lib, A, opts=_opts(lib, nonsymmetric=2))[0] == _lib.IFEAST_ERR_INVALID_ARG
    # the two-pass mode: shared-basis solver with FP32 or FP16 vectors, m0 % 4 == 0
    assert _create(lib, A, opts=_opts(lib, minres_two_pass=1))[0] == _lib.IFEAST_ERR_UNSUPPORTED
    assert _create(lib, A, opts=_opts(lib, minres_two_pass=1, inner_solver=1, inner_max_iters=8))[0] \
        == _lib.IFEAST_ERR_UNSUPPORTED
    assert _create(lib, A, m0=6, opts=_opts(lib, minres_two_pass=1, inner_solver=1,
                                            inner_max_iters=8, precision=1))[0] == \
        _lib.IFEAST_ERR_UNSUPPORTED
    assert _create(lib, A, opts=_opts(lib, minres_two_pass=2))[0] == _lib.IFEAST_ERR_INVALID_ARG


def _csr_ref(M, keep):
    arrs = (np.ascontiguousarray(M.rowptr, np.int32), np.ascontiguousarray(M.colidx, np.int32),
            np.ascontiguousarray(M.val, np.float64))
    keep.append(arrs)
    return ct.byref(_lib.Csr(M.n, M.nnz, *(a.ctypes.data for a in arrs)))


def test_create_checks_B(lib):
    K, M = inputs.fem_q1((5, 4))
    keep = []
    # B of another size, malformed B, and B with the shared-basis inner solver
    # (its Krylov basis is only z-independent for B = I) are refused on the host.
    assert _create(lib, K, B=_csr_ref(inputs.laplacian((4, 4)), keep))[0] == \
        _lib.IFEAST_ERR_INVALID_ARG
    bad = inputs.CSR(M.n, M.rowptr.copy(), M.colidx.copy(), M.val.copy())
    bad.colidx[0] = -1
    assert _create(lib, K, B=_csr_ref(bad, keep))[0] == _lib.IFEAST_ERR_INVALID_ARG
    assert _create(lib, K, B=_csr_ref(M, keep), opts=_opts(lib, inner_solver=1))[0] == \
        _lib.IFEAST_ERR_UNSUPPORTED
    c = _lib.Contour(0, 8, 0.0, 1.0)
    b0, b1 = ct.c_size_t(), ct.c_size_t()
    assert lib.ifeast_workspace_bytes(K.n, K.nnz, 4, ct.byref(c), ct.byref(_opts(lib)),
                                      ct.byref(b0)) == 0
    assert lib.ifeast_workspace_bytes_generalized(K.n, K.nnz, M.nnz, 4, ct.byref(c),
                                                  ct.byref(_opts(lib)), ct.byref(b1)) == 0
    # B's CSR plus the n x m0 blocks B Q and B X
    assert b1.value - b0.value >= 4 * (K.n + 1) + 12 * M.nnz + 2 * 8 * K.n * 4


def test_strerror_and_null_handles(lib):
    for code in range(11):
        assert lib.ifeast_strerror(code)
    assert lib.ifeast_solve(None, None, 0, 0, None) == _lib.IFEAST_ERR_INVALID_ARG
    assert lib.ifeast_stats(None, None) == _lib.IFEAST_ERR_INVALID_ARG
    assert lib.ifeast_apply_filter_residual(None, None, None, None, 1.0, None) == \
        _lib.IFEAST_ERR_INVALID_ARG
    assert lib.ifeast_initial_subspace(0, 4, 1, None, None) == _lib.IFEAST_ERR_INVALID_ARG
    assert lib.ifeast_initial_subspace(10, 4, 1, None, None) == _lib.IFEAST_ERR_INVALID_ARG
    assert lib.ifeast_set_profiling(None, 1) == _lib.IFEAST_ERR_INVALID_ARG
    assert lib.ifeast_kernel_times(None, 4, None, None, 0) == _lib.IFEAST_ERR_INVALID_ARG
    assert lib.ifeast_kernel_launches(None, 4, None, 0) == _lib.IFEAST_ERR_INVALID_ARG
    lib.ifeast_destroy(None)


def test_kernel_class_names(lib):
    """22 kernel classes with distinct names; the profiler's sampled classes exist."""
    names = [lib.ifeast_kernel_name(k).decode() for k in range(22)]
    assert len(set(names)) == 22 and "unknown" not in names
    assert {"lanczos_step", "lanczos_reduce", "lanczos_givens", "gmres_spmm_dot"} <= set(names)
    assert lib.ifeast_kernel_name(22).decode() == "unknown"


def test_product_path_has_no_oracle_import():
    pkg = os.path.join(ROOT, "paper_1706_00692_gb300")
    for dp, _, fs in os.walk(pkg):
        for f in fs:
            if f.endswith((".py", ".cu", ".h", ".cuh")):
                text = open(os.path.join(dp, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", text, re.M), os.path.join(dp, f)
                assert "ifeast_oracle" not in text, os.path.join(dp, f)


def test_two_pass_workspace_drops_the_basis(lib):
    c = _lib.Contour(1, 8, 0.0, 1.0)
    n, nnz, m0, K = 100000, 700000, 80, 1000
    b1, b2 = ct.c_size_t(), ct.c_size_t()
    o1 = _opts(lib, inner_solver=1, inner_max_iters=K, precision=1)
    o2 = _opts(lib, inner_solver=1, inner_max_iters=K, precision=1, minres_two_pass=1)
    assert lib.ifeast_workspace_bytes(n, nnz, m0, ct.byref(c), ct.byref(o1), ct.byref(b1)) == 0
    assert lib.ifeast_workspace_bytes(n, nnz, m0, ct.byref(c), ct.byref(o2), ct.byref(b2)) == 0
    # K + 1 FP32 basis vectors become three slots plus one FP32 accumulator
    assert b1.value - b2.value >= (K + 1 - 4) * n * m0 * 4


def test_user_contour_nodes_and_validation(lib):
    """IFEAST_USER: the given nodes come back unchanged; a missing array, a
    non-finite entry or a node on the real axis is rejected."""
    z, w = orc.contour_nodes("gl_half", 6, 0.2, 1.4)
    zw = np.ascontiguousarray(np.stack([z.real, z.imag, w.real, w.imag], axis=1))
    c = _lib.Contour(_lib.USER, 6, 0.2, 1.4, zw.ctypes.data)
    out = np.zeros(24)
    assert lib.ifeast_contour_nodes(ct.byref(c), out.ctypes.data) == 0
    assert np.array_equal(out.reshape(6, 4), zw)
    for bad in (None, "nan", "real"):
        zb = zw.copy()
        if bad == "nan":
            zb[2, 2] = np.nan
        elif bad == "real":
            zb[4, 1] = 0.0
        cb = _lib.Contour(_lib.USER, 6, 0.2, 1.4, None if bad is None else zb.ctypes.data)
        assert lib.ifeast_contour_nodes(ct.byref(cb), out.ctypes.data) == _lib.IFEAST_ERR_INVALID_ARG
    # the workspace query validates the same way
    nb = ct.c_size_t()
    cb = _lib.Contour(_lib.USER, 6, 0.2, 1.4, None)
    assert lib.ifeast_workspace_bytes(100, 300, 4, ct.byref(cb), ct.byref(_opts(lib)),
                                      ct.byref(nb)) == _lib.IFEAST_ERR_INVALID_ARG
    assert lib.ifeast_workspace_bytes(100, 300, 4, ct.byref(c), ct.byref(_opts(lib)),
                                      ct.byref(nb)) == 0


def test_bf16_and_time_limit_options(lib):
    """BF16 storage exists for the shared-basis solver (m0 % 4 == 0) only; a NaN
    time limit is invalid."""
    c = _lib.Contour(1, 8, 0.0, 1.0)
    nb = ct.c_size_t()
    ok = _opts(lib, inner_solver=1, inner_max_iters=100, precision=_lib.BF16)
    assert lib.ifeast_workspace_bytes(1000, 7000, 8, ct.byref(c), ct.byref(ok), ct.byref(nb)) == 0
    f32 = ct.c_size_t()
    o32 = _opts(lib, inner_solver=1, inner_max_iters=100, precision=_lib.FP32)
    assert lib.ifeast_workspace_bytes(1000, 7000, 8, ct.byref(c), ct.byref(o32), ct.byref(f32)) == 0
    assert f32.value - nb.value >= 2 * 101 * 1000 * 8  # half the basis bytes
    assert lib.ifeast_workspace_bytes(1000, 7000, 6, ct.byref(c), ct.byref(ok), ct.byref(nb)) == \
        _lib.IFEAST_ERR_UNSUPPORTED
    gm = _opts(lib, precision=_lib.BF16)
    assert lib.ifeast_workspace_bytes(1000, 7000, 8, ct.byref(c), ct.byref(gm), ct.byref(nb)) == \
        _lib.IFEAST_ERR_UNSUPPORTED
    bad = _opts(lib, time_limit_ms=float("nan"))
    assert lib.ifeast_workspace_bytes(1000, 7000, 8, ct.byref(c), ct.byref(bad), ct.byref(nb)) == \
        _lib.IFEAST_ERR_INVALID_ARG


def test_noalloc_rejects_overlapping_x_and_q(lib):
    """X = Q X_Q is not formed in place: an X range overlapping Q's returns
    INVALID_ARG before any device work (the pointers are never dereferenced)."""
    n, m0 = 1000, 8
    rp = ct.c_void_p(0x10000)
    base = 0x7f0000000000
    nbytes = n * m0 * 8
    for off in (0, 8, nbytes - 8, -(nbytes - 8)):
        rc = lib.ifeast_rayleigh_ritz_noalloc(n, 3000, rp, rp, rp, m0, ct.c_void_p(base),
                                              ct.c_void_p(base + off), rp, rp, None)
        assert rc == _lib.IFEAST_ERR_INVALID_ARG, off


def test_node_chunk_option(lib):
    """node_chunk: per-node GMRES only, a divisor of the node count; the
    workspace holds one chunk's Krylov bases."""
    c = _lib.Contour(0, 12, 0.0, 1.0)
    n, nnz, m0 = 20000, 140000, 16
    full, part = ct.c_size_t(), ct.c_size_t()
    assert lib.ifeast_workspace_bytes(n, nnz, m0, ct.byref(c), ct.byref(_opts(lib, inner_max_iters=20)),
                                      ct.byref(full)) == 0
    assert lib.ifeast_workspace_bytes(n, nnz, m0, ct.byref(c),
                                      ct.byref(_opts(lib, inner_max_iters=20, node_chunk=3)),
                                      ct.byref(part)) == 0
    # the (K + 1) x n x C complex FP64 basis shrinks from 12 to 3 nodes' columns
    assert full.value - part.value >= 21 * n * 9 * m0 * 16
    assert lib.ifeast_workspace_bytes(n, nnz, m0, ct.byref(c),
                                      ct.byref(_opts(lib, node_chunk=5)),
                                      ct.byref(part)) == _lib.IFEAST_ERR_INVALID_ARG
    assert lib.ifeast_workspace_bytes(n, nnz, m0, ct.byref(c),
                                      ct.byref(_opts(lib, node_chunk=-1)),
                                      ct.byref(part)) == _lib.IFEAST_ERR_INVALID_ARG
    assert lib.ifeast_workspace_bytes(n, nnz, m0, ct.byref(c),
                                      ct.byref(_opts(lib, inner_solver=1, inner_max_iters=50,
                                                     precision=1, node_chunk=2)),
                                      ct.byref(part)) == _lib.IFEAST_ERR_UNSUPPORTED


def test_plain_loads_option(lib):
    """plain_loads: 0 (default, TMA-streamed FP32 GMRES basis) or 1; anything
    else is rejected; it does not change the workspace."""
    o = _lib.Opts()
    lib.ifeast_default_opts(ct.byref(o))
    assert o.plain_loads == 0
    c = _lib.Contour(0, 8, 0.0, 1.0)
    a, b = ct.c_size_t(), ct.c_size_t()
    assert lib.ifeast_workspace_bytes(5000, 30000, 12, ct.byref(c),
                                      ct.byref(_opts(lib, precision=1, inner_max_iters=20)),
                                      ct.byref(a)) == 0
    assert lib.ifeast_workspace_bytes(5000, 30000, 12, ct.byref(c),
                                      ct.byref(_opts(lib, precision=1, inner_max_iters=20,
                                                     plain_loads=1)),
                                      ct.byref(b)) == 0
    assert a.value == b.value
    assert lib.ifeast_workspace_bytes(5000, 30000, 12, ct.byref(c),
                                      ct.byref(_opts(lib, plain_loads=2)),
                                      ct.byref(b)) == _lib.IFEAST_ERR_INVALID_ARG


def test_nonsym_correction_option(lib):
    """nonsym_correction: 0 (default, the plain form) or 1 (block correction of
    the non-symmetric iteration); anything else is rejected."""
    o = _lib.Opts()
    lib.ifeast_default_opts(ct.byref(o))
    assert o.nonsym_correction == 0
    c = _lib.Contour(0, 8, 0.0, 1.0)
    b = ct.c_size_t()
    assert lib.ifeast_workspace_bytes(5000, 30000, 12, ct.byref(c),
                                      ct.byref(_opts(lib, nonsymmetric=1, nonsym_correction=1)),
                                      ct.byref(b)) == 0
    assert lib.ifeast_workspace_bytes(5000, 30000, 12, ct.byref(c),
                                      ct.byref(_opts(lib, nonsym_correction=2)),
                                      ct.byref(b)) == _lib.IFEAST_ERR_INVALID_ARG
