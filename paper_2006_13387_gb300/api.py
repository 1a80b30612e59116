"""Python front end of libtopsolve: argument marshalling for the C ABI.

Device mode passes torch CUDA tensors (FP64) and the current torch stream;
host mode passes NumPy arrays.  All arithmetic runs in the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import weakref

import numpy as np

from . import _native as N


class TopSolveError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{N.STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(ctx_ptr, st, allow=(N.TS_OK,)):
    if st not in allow:
        msg = N.lib().ts_last_error(ctx_ptr)
        raise TopSolveError(st, msg.decode() if msg else "")
    return st


def _ptr(a):
    """Device pointer of a torch tensor or host pointer of a NumPy array."""
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


class Context:
    """Binds the library to the current CUDA device and a stream (default: the
    current torch stream)."""

    def __init__(self, stream=None):
        L = N.lib()
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream
            except Exception:
                stream = 0
        self._p = C.c_void_p()
        self._designs = weakref.WeakSet()
        self._pending = {}
        st = L.ts_ctx_create(C.c_void_p(stream), C.byref(self._p))
        if st != N.TS_OK:
            raise TopSolveError(st, "ts_ctx_create failed")

    # -- request loop (ts_submit / ts_poll) ------------------------------------
    def set_slots(self, n):
        """Concurrent requests of the request loop (before the first submit)."""
        _check(self._p, N.lib().ts_ctx_set_slots(self._p, int(n)))

    def submit(self, design, f, u=None, rtol=1e-8, rho=None):
        """Queues a solve of `design` (after rebuilding it for `rho`, if given)
        and returns a ticket at once.  The arrays are kept alive here until the
        request has been polled to completion."""
        L = N.lib()
        f, u = design._vectors(f, u)
        keep_rho = None
        if rho is not None:
            keep_rho = design._rho_buffer(rho)
        t = C.c_int64()
        if keep_rho is None:
            st = L.ts_submit(self._p, design._h, _ptr(f), _ptr(u), f.shape[0], rtol, C.byref(t))
        else:
            st = L.ts_submit_update(self._p, design._h, _ptr(keep_rho), _ptr(f), _ptr(u), f.shape[0], rtol,
                                    C.byref(t))
        _check(self._p, st)
        self._pending[t.value] = (design, f, u, keep_rho)
        return t.value

    def poll(self, ticket, allow_not_converged=True):
        """None while the request is queued or running; then (u, stats)."""
        nrhs = self._pending[ticket][1].shape[0]
        stats = (N.TsStats * nrhs)()
        st = N.lib().ts_poll(self._p, ticket, stats)
        if st == N.TS_PENDING:
            return None
        design, f, u, rho = self._pending.pop(ticket)
        if rho is not None:
            design._keep = rho
            design.coarse_dim = int(N.lib().ts_coarse_dim(design._h))
        allow = (N.TS_OK, N.TS_NOT_CONVERGED) if allow_not_converged else (N.TS_OK,)
        _check(self._p, st, allow)
        return u, [s.as_dict() for s in stats]

    def wait(self, ticket, **kw):
        """Polls until the request has finished; returns (u, stats)."""
        import time
        while True:
            r = self.poll(ticket, **kw)
            if r is not None:
                return r
            time.sleep(0.0002)

    def drain(self):
        """Waits for every outstanding request (results discarded)."""
        for t in list(self._pending):
            try:
                self.wait(t)
            except TopSolveError:
                pass

    def kernel_launches(self):
        """Kernels launched by this context so far (graph kernel nodes included)."""
        return int(N.lib().ts_ctx_kernel_launches(self._p))

    def close(self):
        """Destroys every design made on this context, then the context (a
        handle must never outlive its context)."""
        if self._p:
            self.drain()
            for d in list(self._designs):
                d.close()
            N.lib().ts_ctx_destroy(self._p)
            self._p = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Design:
    """One design rho: preconditioner built by ts_setup, solves by ts_solve."""

    def __init__(self, ctx, *, dim, nx, ny, nz=0, blk, overlap, rho, E0, Emin, p, nu, dirichlet,
                 precision="fp64", tau_scale=2.0, max_modes=16, rotations=True, coarse=True, max_iter=5000,
                 energy_tol=-1.0, warm_start=False, refine=0, coarse_layout="auto", coarse_method="eig",
                 snapshots=15, rebuild="policy", rebuild_factor=1.5, device=True):
        L = N.lib()
        self.ctx = ctx
        self.device = device
        blk = tuple(blk) if not np.isscalar(blk) else (blk,) * dim
        mesh = N.TsMesh(dim, nx, ny, nz, blk[0], blk[1], blk[2] if dim == 3 else 1, overlap)
        d = np.ascontiguousarray(np.asarray(dirichlet, dtype=np.int64))
        bcs = N.TsBcs(d.size, d.ctypes.data_as(C.POINTER(C.c_int64)))
        o = N.TsOptions()
        L.ts_options_default(C.byref(o))
        o.precision = {"fp64": N.TS_FP64, "mixed": N.TS_MIXED_FP32, "fp32": N.TS_MIXED_FP32, "tf32": N.TS_MIXED_TF32,
                       "3xtf32": N.TS_MIXED_3XTF32}[precision]
        o.tau_scale = tau_scale
        o.max_modes = max_modes
        # eigenvalue slots per problem of coarse_info: 48 for the M_EE space
        self.max_modes = 48 if coarse_method == "elastic" else int(max_modes)
        o.rotations = 1 if rotations else 0
        o.coarse = 1 if coarse else 0
        o.max_iter = max_iter
        o.energy_tol = energy_tol
        o.warm_start = 1 if warm_start else 0
        o.refine = refine
        o.coarse_layout = {"auto": 0, "dense": 1, "blockline": 2, "nd": 3}[coarse_layout]
        o.coarse_method = {"eig": 0, "rand": 1, "elastic": 2}[coarse_method]
        o.rand_snapshots = int(snapshots)
        o.rebuild_policy = {"always": 0, "policy": 1}[rebuild]
        o.rebuild_factor = float(rebuild_factor)
        o.mem_is_device = 1 if device else 0
        if device:
            import torch
            rho_t = rho if isinstance(rho, torch.Tensor) else torch.as_tensor(np.asarray(rho, np.float64))
            rho_t = rho_t.to(device="cuda", dtype=torch.float64).contiguous()
            self._keep = rho_t
            rp = _ptr(rho_t)
        else:
            rho_a = np.ascontiguousarray(np.asarray(rho, dtype=np.float64))
            self._keep = rho_a
            rp = _ptr(rho_a)
        self._h = C.c_void_p()
        if not ctx._p:
            raise TopSolveError(N.TS_ERR_INVALID, "context is closed")
        _check(ctx._p, L.ts_setup(ctx._p, C.byref(mesh), rp, E0, Emin, p, nu, C.byref(bcs), C.byref(o),
                                  C.byref(self._h)))
        ctx._designs.add(self)
        self.ndof = int(L.ts_ndof(self._h))
        self.n_el = nx * ny * (nz if dim == 3 else 1)
        self.coarse_dim = int(L.ts_coarse_dim(self._h))

    # -- solves ---------------------------------------------------------------
    def _vectors(self, f, u):
        if self.device:
            import torch
            f = f.to(device="cuda", dtype=torch.float64).contiguous()
            if f.dim() == 1:
                f = f.unsqueeze(0)
            if u is None:
                u = torch.zeros_like(f)
        else:
            f = np.ascontiguousarray(np.atleast_2d(np.asarray(f, dtype=np.float64)))
            if u is None:
                u = np.zeros_like(f)
        return f, u

    def _rho_buffer(self, rho):
        if self.device:
            import torch
            r = rho if isinstance(rho, torch.Tensor) else torch.as_tensor(np.asarray(rho, np.float64))
            return r.to(device="cuda", dtype=torch.float64).contiguous()
        return np.ascontiguousarray(np.asarray(rho, dtype=np.float64))

    def update_density(self, rho):
        """Moves the design to new densities by its rebuild policy
        (ts_update_density)."""
        r = self._rho_buffer(rho)
        _check(self.ctx._p, N.lib().ts_update_density(self._h, _ptr(r)))
        self._keep = r
        self.coarse_dim = int(N.lib().ts_coarse_dim(self._h))

    def solve(self, f, u=None, rtol=1e-8, allow_not_converged=True):
        """f: [nrhs, ndof] (torch CUDA FP64 in device mode, NumPy otherwise).
        Returns (u, list of stats dicts)."""
        L = N.lib()
        f, u = self._vectors(f, u)
        nrhs = f.shape[0]
        stats = (N.TsStats * nrhs)()
        st = L.ts_solve(self._h, _ptr(f), _ptr(u), nrhs, rtol, stats)
        allow = (N.TS_OK, N.TS_NOT_CONVERGED) if allow_not_converged else (N.TS_OK,)
        _check(self.ctx._p, st, allow)
        return u, [s.as_dict() for s in stats]

    def apply_K(self, x):
        import torch
        y = torch.empty_like(x)
        _check(self.ctx._p, N.lib().ts_apply_K(self._h, _ptr(x), _ptr(y)))
        return y

    def sensitivity(self, u):
        """Compliance sensitivities of Eq. 1003 for displacements u (torch CUDA
        FP64, ndof): returns (dc [n_el] torch CUDA FP64, compliance float)."""
        import torch
        u = u.reshape(-1).contiguous()
        dc = torch.empty(self.n_el, dtype=torch.float64, device=u.device)
        c = C.c_double()
        _check(self.ctx._p, N.lib().ts_sensitivity(self._h, _ptr(u), _ptr(dc), C.byref(c)))
        return dc, c.value

    def oc_update(self, dc, volfrac, move=0.2):
        """Optimality-criteria update of this design's densities (ts_oc_update):
        returns the new densities (torch CUDA FP64, n_el)."""
        import torch
        dc = dc.contiguous()
        out = torch.empty_like(dc)
        _check(self.ctx._p, N.lib().ts_oc_update(self._h, _ptr(dc), float(volfrac), float(move), _ptr(out)))
        return out

    def apply_M(self, r):
        import torch
        z = torch.empty_like(r)
        _check(self.ctx._p, N.lib().ts_apply_M(self._h, _ptr(r), _ptr(z)))
        return z

    def apply_M_parts(self, r):
        import torch
        zl = torch.empty_like(r)
        zc = torch.empty_like(r)
        _check(self.ctx._p, N.lib().ts_apply_M_parts(self._h, _ptr(r), _ptr(zl), _ptr(zc)))
        return zl, zc

    def apply_M_block(self, r, which=3):
        """z = M^{-1} r on up to 8 columns (torch CUDA FP64 [nrhs, ndof])
        through the block path's kernels: which 1 level 1, 2 coarse, 3 both."""
        import torch
        r = r.contiguous()
        z = torch.empty_like(r)
        _check(self.ctx._p, N.lib().ts_apply_M_block(self._h, _ptr(r), _ptr(z), int(r.shape[0]), int(which)))
        return z

    def time_kernel(self, kernel, reps=20):
        """(ms per launch, algorithmic FLOPs, algorithmic bytes) of one kernel,
        timed with CUDA events on the library's stream."""
        ms, fl, by = C.c_double(), C.c_double(), C.c_double()
        _check(self.ctx._p, N.lib().ts_time_kernel(self._h, kernel.encode(), reps, C.byref(ms), C.byref(fl),
                                                   C.byref(by)))
        return ms.value, fl.value, by.value

    def level1_info(self):
        ns, fe, lu = C.c_int(), C.c_int64(), C.c_int64()
        _check(self.ctx._p, N.lib().ts_level1_info(self._h, C.byref(ns), C.byref(fe), C.byref(lu)))
        return dict(n_sub=ns.value, factor_entries=fe.value, local_unknowns=lu.value)

    def coarse_info(self):
        """Per heat eigenproblem: coarse node, component, count below tau,
        modes selected and the selected eigenvalues ([n][max_modes], NaN
        padded; sized by this design's own max_modes)."""
        max_modes = self.max_modes
        L = N.lib()
        n = int(L.ts_coarse_problems(self._h))
        out = dict(node=np.zeros(n, np.int32), comp=np.zeros(n, np.int32), below=np.zeros(n, np.int32),
                   selected=np.zeros(n, np.int32), eig=np.full((n, max_modes), np.nan))
        if n:
            _check(self.ctx._p, L.ts_coarse_info(self._h, _ptr(out["node"]), _ptr(out["comp"]), _ptr(out["below"]),
                                                 _ptr(out["selected"]), _ptr(out["eig"])))
        return out

    def close(self):
        if self._h:
            N.lib().ts_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def design_from_problem(ctx, prob, **kw):
    """Convenience: build a Design from any object with the fields of a
    problem description (dim, nx, ny, nz, blk, overlap, rho, E0, Emin, p, nu,
    dirichlet)."""
    return Design(ctx, dim=prob.dim, nx=prob.nx, ny=prob.ny, nz=prob.nz, blk=prob.blk, overlap=prob.overlap,
                  rho=prob.rho, E0=prob.E0, Emin=prob.Emin, p=prob.p, nu=prob.nu, dirichlet=prob.dirichlet, **kw)
