"""Python binding of libifeast: argument marshalling over the C ABI only.

Device memory (the handle's workspace, inputs and outputs) comes from PyTorch
tensors and kernels run on the current PyTorch CUDA stream; every step of
the computation runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as ct

import numpy as np

from . import _lib
from .inputs import CSR


class IFEASTError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = _lib.load().ifeast_strerror(code).decode()
        super().__init__(f"{where}: {msg} (status {code})")


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libifeast needs a CUDA device; none is available")
    return torch


def contour_nodes(rule: str, nc: int, emin: float, emax: float):
    """Nodes z_k and weights w_k computed by the library (complex numpy arrays)."""
    lib = _lib.load()
    c = _lib.Contour(_lib.RULES[rule], nc, emin, emax)
    zw = np.zeros(4 * nc)
    rc = lib.ifeast_contour_nodes(ct.byref(c), zw.ctypes.data)
    if rc:
        raise IFEASTError(rc, "ifeast_contour_nodes")
    zw = zw.reshape(nc, 4)
    return zw[:, 0] + 1j * zw[:, 1], zw[:, 2] + 1j * zw[:, 3]


def initial_subspace(n: int, m0: int, seed: int, device="cuda"):
    """The library's seeded random subspace (i.i.d. N(0,1), Philox4x32-10 +
    Box-Muller, drawn on the device) as a CUDA float64 (n, m0) tensor."""
    torch = _torch()
    lib = _lib.load()
    X = torch.empty((n, m0), dtype=torch.float64, device=device)
    rc = lib.ifeast_initial_subspace(n, m0, seed, X.data_ptr(),
                                     ct.c_void_p(torch.cuda.current_stream(X.device).cuda_stream))
    if rc:
        raise IFEASTError(rc, "ifeast_initial_subspace")
    return X


def _user_zw(nodes):
    """(z, w) complex arrays -> the nc x 4 float64 array of IFEAST_USER."""
    z, w = (np.asarray(a, dtype=np.complex128).ravel() for a in nodes)
    return np.ascontiguousarray(np.stack([z.real, z.imag, w.real, w.imag], axis=1))


class Solver:
    """One IFEAST problem (A, optional SPD B, interval, m0, contour, options)
    bound to a handle. rule="user" takes the nodes and weights from
    user_nodes=(z, w) (filter Re sum_k w_k / (z_k - lambda))."""

    def __init__(self, A: CSR, emin: float, emax: float, m0: int, *, nc: int = 8,
                 rule: str = "gl_half", inner: str = "gmres", inner_iters: int = 10,
                 alpha: float = 0.0, max_outer: int = 100, tol: float = 1e-10,
                 precision: str = "fp64", device: str | int = "cuda",
                 torch_workspace: bool = True, verbose: bool = False, B: CSR | None = None,
                 nonsymmetric: bool = False, two_pass: bool = False,
                 correction_rf: float | None = None, user_nodes=None,
                 time_limit_ms: float = 0.0, node_chunk: int = 0, plain_loads: bool = False,
                 nonsym_correction: bool = False):
        torch = _torch()
        self.lib = _lib.load()
        self.torch = torch
        self.device = torch.device(device)
        self.n, self.m0 = int(A.n), int(m0)
        self.emin, self.emax = float(emin), float(emax)
        self._zw = None
        if rule == "user":
            self._zw = _user_zw(user_nodes)
            nc = self._zw.shape[0]
        self.nc = int(nc)
        self.contour = _lib.Contour(_lib.RULES[rule], nc, emin, emax,
                                    None if self._zw is None else self._zw.ctypes.data)
        self.opts = _lib.Opts()
        self.lib.ifeast_default_opts(ct.byref(self.opts))
        self.opts.inner_max_iters = inner_iters
        self.opts.alpha = alpha
        self.opts.max_outer = max_outer
        self.opts.tol = tol
        self.opts.inner_solver = _lib.INNERS[inner]
        self.opts.precision = _lib.PRECISIONS[precision]
        self.opts.verbose = 1 if verbose else 0
        self.opts.nonsymmetric = 1 if nonsymmetric else 0
        self.opts.minres_two_pass = 1 if two_pass else 0
        if correction_rf is not None:
            self.opts.correction_rf = correction_rf
        self.opts.time_limit_ms = float(time_limit_ms)
        self.opts.node_chunk = int(node_chunk)
        self.opts.plain_loads = 1 if plain_loads else 0
        self.opts.nonsym_correction = 1 if nonsym_correction else 0
        nbytes = ct.c_size_t(0)
        rc = self.lib.ifeast_workspace_bytes_generalized(
            self.n, A.nnz, -1 if B is None else B.nnz, self.m0, ct.byref(self.contour),
            ct.byref(self.opts), ct.byref(nbytes))
        if rc:
            raise IFEASTError(rc, "ifeast_workspace_bytes_generalized")
        self.workspace_bytes = int(nbytes.value)
        with torch.cuda.device(self.device):
            self.stream = torch.cuda.current_stream(self.device)
            if torch_workspace:
                self._ws = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=self.device)
                ws_ptr, ws_len = self._ws.data_ptr(), self.workspace_bytes
            else:
                self._ws, ws_ptr, ws_len = None, None, 0
            self._rowptr = np.ascontiguousarray(A.rowptr, dtype=np.int32)
            self._colidx = np.ascontiguousarray(A.colidx, dtype=np.int32)
            self._val = np.ascontiguousarray(A.val, dtype=np.float64)
            csr = _lib.Csr(self.n, A.nnz, self._rowptr.ctypes.data, self._colidx.ctypes.data,
                           self._val.ctypes.data)
            bref = None
            if B is not None:
                self._B = (np.ascontiguousarray(B.rowptr, dtype=np.int32),
                           np.ascontiguousarray(B.colidx, dtype=np.int32),
                           np.ascontiguousarray(B.val, dtype=np.float64))
                bref = ct.byref(_lib.Csr(int(B.n), B.nnz, *(a.ctypes.data for a in self._B)))
            h = ct.c_void_p()
            rc = self.lib.ifeast_create(ct.byref(csr), bref, ct.byref(self.contour), self.m0,
                                        ct.byref(self.opts), ws_ptr, ws_len,
                                        ct.c_void_p(self.stream.cuda_stream), ct.byref(h))
            if rc:
                raise IFEASTError(rc, "ifeast_create")
            self.h = h

    # ------------------------------------------------------------------ full solve
    def solve(self, X0=None, seed: int = 0) -> int:
        """Algorithm 2 from X0 (numpy (n, m0) float64 on the host, or a CUDA
        float64 tensor; None: the library's seeded random subspace from seed).
        Returns the library status (0 = converged)."""
        torch = self.torch
        if X0 is None:
            return int(self.lib.ifeast_solve(self.h, None, 0, int(seed), None))
        if isinstance(X0, np.ndarray):
            x = np.ascontiguousarray(X0, dtype=np.float64)
            assert x.shape == (self.n, self.m0)
            return int(self.lib.ifeast_solve(self.h, x.ctypes.data, 0, 0, None))
        assert X0.is_cuda and X0.dtype == torch.float64 and X0.shape == (self.n, self.m0)
        X0 = X0.contiguous()
        return int(self.lib.ifeast_solve(self.h, X0.data_ptr(), 1, 0, None))

    def eigenpairs(self, on_device: bool = False):
        """(lam, X, res) for the Ritz pairs inside the interval, ascending."""
        torch = self.torch
        m = ct.c_int(0)
        rc = self.lib.ifeast_eigenpairs(self.h, 0, ct.byref(m), None, None, None, 0)
        if rc:
            raise IFEASTError(rc, "ifeast_eigenpairs")
        cnt = m.value
        if on_device:
            lam = torch.empty(cnt, dtype=torch.float64, device=self.device)
            X = torch.empty((self.n, cnt), dtype=torch.float64, device=self.device)
            res = torch.empty(cnt, dtype=torch.float64, device=self.device)
            ptrs = (lam.data_ptr(), X.data_ptr(), res.data_ptr()) if cnt else (None, None, None)
        else:
            lam, X, res = np.zeros(cnt), np.zeros((self.n, cnt)), np.zeros(cnt)
            ptrs = (lam.ctypes.data, X.ctypes.data, res.ctypes.data) if cnt else (None, None, None)
        rc = self.lib.ifeast_eigenpairs(self.h, cnt, ct.byref(m), *ptrs, 1 if on_device else 0)
        if rc:
            raise IFEASTError(rc, "ifeast_eigenpairs")
        return lam, X, res

    def eigenpairs_complex(self):
        """Non-symmetric handles: (lam complex, X complex (n, m), res) for the
        Ritz pairs inside the contour's circle, ordered by real, then imaginary
        part."""
        m = ct.c_int(0)
        rc = self.lib.ifeast_eigenpairs_complex(self.h, 0, ct.byref(m), None, None, None, 0)
        if rc:
            raise IFEASTError(rc, "ifeast_eigenpairs_complex")
        cnt = m.value
        lam = np.zeros(cnt, np.complex128)
        X = np.zeros((self.n, cnt), np.complex128)
        res = np.zeros(cnt)
        ptrs = (lam.ctypes.data, X.ctypes.data, res.ctypes.data) if cnt else (None, None, None)
        rc = self.lib.ifeast_eigenpairs_complex(self.h, cnt, ct.byref(m), *ptrs, 0)
        if rc:
            raise IFEASTError(rc, "ifeast_eigenpairs_complex")
        return lam, X, res

    def rayleigh_ritz_nonsym(self, Q):
        """Galerkin Rayleigh-Ritz on a CUDA float64 (n, m0) tensor: returns
        (X orthonormal basis, theta complex (m0,) unordered, res)."""
        torch = self.torch
        Q = Q.contiguous()
        X = torch.empty_like(Q)
        theta = torch.empty(self.m0, dtype=torch.complex128, device=self.device)
        res = torch.empty(self.m0, dtype=torch.float64, device=self.device)
        rc = self.lib.ifeast_rayleigh_ritz_nonsym(self.h, Q.data_ptr(), X.data_ptr(),
                                                  theta.data_ptr(), res.data_ptr())
        if rc:
            raise IFEASTError(rc, "ifeast_rayleigh_ritz_nonsym")
        return X, theta, res

    def ritz_all(self):
        lam, res = np.zeros(self.m0), np.zeros(self.m0)
        rc = self.lib.ifeast_ritz_all(self.h, lam.ctypes.data, res.ctypes.data, 0)
        if rc:
            raise IFEASTError(rc, "ifeast_ritz_all")
        return lam, res

    def stats(self) -> dict:
        s = _lib.Stats()
        rc = self.lib.ifeast_stats(self.h, ct.byref(s))
        if rc:
            raise IFEASTError(rc, "ifeast_stats")
        return {f: getattr(s, f) for f, _ in _lib.Stats._fields_}

    # ------------------------------------------------------------------ steps
    def apply_filter(self, X, RF: float = 1.0):
        """Alg. 2 steps 1-2 on a CUDA float64 (n, m0) tensor: returns (Q, steps)."""
        torch = self.torch
        X = X.contiguous()
        Q = torch.empty_like(X)
        steps = torch.empty(self.nc * self.m0, dtype=torch.int32, device=self.device)
        rc = self.lib.ifeast_apply_filter(self.h, X.data_ptr(), Q.data_ptr(), float(RF),
                                          steps.data_ptr())
        if rc:
            raise IFEASTError(rc, "ifeast_apply_filter")
        return Q, steps

    def apply_filter_residual(self, X, lam, RF: float = 1.0):
        """Alg. 2 steps 1-2 in residual form for the pairs (lam_j, x_j): X a CUDA
        float64 (n, m0) tensor, lam (m0,). Returns (Q, steps)."""
        torch = self.torch
        X = X.contiguous()
        lam = torch.as_tensor(lam, dtype=torch.float64, device=self.device).contiguous()
        Q = torch.empty_like(X)
        steps = torch.empty(self.nc * self.m0, dtype=torch.int32, device=self.device)
        rc = self.lib.ifeast_apply_filter_residual(self.h, X.data_ptr(), lam.data_ptr(),
                                                   Q.data_ptr(), float(RF), steps.data_ptr())
        if rc:
            raise IFEASTError(rc, "ifeast_apply_filter_residual")
        return Q, steps

    def rayleigh_ritz(self, Q):
        """Alg. 2 steps 3-4 on a CUDA float64 (n, m0) tensor: returns (X, lam, res)."""
        torch = self.torch
        Q = Q.contiguous()
        X = torch.empty_like(Q)
        lam = torch.empty(self.m0, dtype=torch.float64, device=self.device)
        res = torch.empty(self.m0, dtype=torch.float64, device=self.device)
        rc = self.lib.ifeast_rayleigh_ritz(self.h, Q.data_ptr(), X.data_ptr(), lam.data_ptr(),
                                           res.data_ptr())
        if rc:
            raise IFEASTError(rc, "ifeast_rayleigh_ritz")
        return X, lam, res

    def spmm_shift(self, V, z):
        """W[:, c] = z[c // m0] B V[:, c] - A V[:, c] (B = I unless given) for a CUDA
        complex128 (n, C) V."""
        torch = self.torch
        V = V.contiguous()
        assert V.dtype == torch.complex128 and V.shape[0] == self.n
        C = V.shape[1]
        zt = torch.as_tensor(np.asarray(z, dtype=np.complex128), device=self.device)
        W = torch.empty_like(V)
        rc = self.lib.ifeast_spmm_shift(self.h, V.data_ptr(), W.data_ptr(), C, C // zt.numel(),
                                        zt.data_ptr())
        if rc:
            raise IFEASTError(rc, "ifeast_spmm_shift")
        return W

    # ------------------------------------------------------------------ timing
    def set_profiling(self, on: bool | int = True):
        """True/1: time every launch; N >= 2: time every N-th launch of the
        Lanczos step and Givens kernels (and every other launch); False: off."""
        rc = self.lib.ifeast_set_profiling(self.h, int(on))
        if rc:
            raise IFEASTError(rc, "ifeast_set_profiling")

    def kernel_times(self, reset: bool = False) -> dict:
        """{kernel class: (timed launches, their total ms)} measured with CUDA events."""
        ms = np.zeros(32)
        cnt = np.zeros(32, dtype=np.int64)
        k = self.lib.ifeast_kernel_times(self.h, 32, ms.ctypes.data, cnt.ctypes.data,
                                         1 if reset else 0)
        return {self.lib.ifeast_kernel_name(i).decode(): (int(cnt[i]), float(ms[i]))
                for i in range(k) if cnt[i] > 0}

    def kernel_launches(self, reset: bool = False) -> dict:
        """{kernel class: launches} since profiling was switched on (timed or not)."""
        cnt = np.zeros(32, dtype=np.int64)
        k = self.lib.ifeast_kernel_launches(self.h, 32, cnt.ctypes.data, 1 if reset else 0)
        return {self.lib.ifeast_kernel_name(i).decode(): int(cnt[i])
                for i in range(k) if cnt[i] > 0}

    def close(self):
        if getattr(self, "h", None):
            self.lib.ifeast_destroy(self.h)
            self.h = None
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous serving of many solves on one GPU (include/ifeast_serve.h).

    Requests are admitted in arrival order as their device workspace fits in
    ``mem_budget_bytes``; up to ``max_active`` run at once, each on its own
    stream and worker thread inside the library."""

    def __init__(self, mem_budget_bytes: int, max_active: int = 8, device: int = 0):
        self.lib = _lib.load()
        o = _lib.ServerOpts(int(mem_budget_bytes), int(max_active), int(device))
        h = ct.c_void_p()
        rc = self.lib.ifeast_server_create(ct.byref(o), ct.byref(h))
        if rc:
            raise IFEASTError(rc, "ifeast_server_create")
        self.h = h
        self._meta = {}

    def submit(self, A: CSR, emin: float, emax: float, m0: int, X0: np.ndarray, *, nc: int = 8,
               rule: str = "gl_half", inner: str = "minres", inner_iters: int = 300,
               alpha: float = 3e-2, max_outer: int = 100, tol: float = 1e-10,
               precision: str = "fp32", two_pass: bool = False, user_nodes=None) -> int:
        zw = _user_zw(user_nodes) if rule == "user" else None
        if zw is not None:
            nc = zw.shape[0]
        c = _lib.Contour(_lib.RULES[rule], nc, emin, emax, None if zw is None else zw.ctypes.data)
        o = _lib.Opts()
        self.lib.ifeast_default_opts(ct.byref(o))
        o.inner_solver = _lib.INNERS[inner]
        o.inner_max_iters = inner_iters
        o.alpha = alpha
        o.max_outer = max_outer
        o.tol = tol
        o.precision = _lib.PRECISIONS[precision]
        o.minres_two_pass = 1 if two_pass else 0
        rp = np.ascontiguousarray(A.rowptr, dtype=np.int32)
        ci = np.ascontiguousarray(A.colidx, dtype=np.int32)
        va = np.ascontiguousarray(A.val, dtype=np.float64)
        x = np.ascontiguousarray(X0, dtype=np.float64)
        assert x.shape == (A.n, m0)
        csr = _lib.Csr(A.n, A.nnz, rp.ctypes.data, ci.ctypes.data, va.ctypes.data)
        rid = ct.c_int64()
        rc = self.lib.ifeast_server_submit(self.h, ct.byref(csr), ct.byref(c), m0, ct.byref(o),
                                           x.ctypes.data, ct.byref(rid))
        if rc:
            raise IFEASTError(rc, "ifeast_server_submit")
        self._meta[rid.value] = (A.n, m0)
        return rid.value

    def wait(self, rid: int):
        """(status, lam, X, res, info dict) of request rid (blocks until done)."""
        n, m0 = self._meta.pop(rid)
        lam, X, res = np.zeros(m0), np.zeros((n, m0)), np.zeros(m0)
        m = ct.c_int()
        info = _lib.RequestInfo()
        rc = self.lib.ifeast_server_wait(self.h, rid, m0, ct.byref(m), lam.ctypes.data,
                                         X.ctypes.data, res.ctypes.data, ct.byref(info))
        k = min(m.value, m0)
        d = {f: getattr(info, f) for f, _ in _lib.RequestInfo._fields_}
        return rc, lam[:k], X[:, :k], res[:k], d

    def close(self):
        if getattr(self, "h", None):
            self.lib.ifeast_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
