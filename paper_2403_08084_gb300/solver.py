"""Python face of the C ABI: one object per (mesh, tableau, dt, options).

Each method forwards to the ``irk_*`` entry point of the same name in
libirk.so; arguments are marshalled to raw pointers (device tensors are passed
through, host arrays are copied by the library inside the call).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L


def _current_stream():
    try:
        import torch

        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:  # pragma: no cover - torch is part of the environment
        pass
    return None


class Solver:
    """Stage-coupled RK solver for the Q1 heat equation on an N x N mesh of the unit square.

    Vectors use the full (N+1)^2 node grid, x fastest; stage vectors hold the s
    values of a node contiguously.  See include/irk.h.
    """

    def __init__(self, n_cells: int, tableau, dt: float, *, kappa=None, levels: int = 1, dim: int = 2,
                 precond: str = "lower", vcycle: str = "fp64", nu_pre: int = 2, nu_post: int = 2,
                 omega: float = 2.0 / 3.0, rtol: float = 1e-10, restart: int = 50, maxit: int = 500,
                 orth: str = "cgs2", solver: str = "fgmres", splitting: str = "ai", warm_start: bool = False,
                 stream=None):
        A = np.ascontiguousarray(tableau.A, dtype=np.float64)
        self.s = int(A.shape[0])
        self.N, self.dim, self.dt = int(n_cells), int(dim), float(dt)
        self.n_nodes = (self.N + 1) ** self.dim
        self.n_cells = self.N**self.dim
        self._A = L.dbl_array(A.reshape(-1))
        self._b = L.dbl_array(tableau.b)
        self._c = L.dbl_array(tableau.c)
        tab = L.irk_tableau(self.s, self._A, self._b, self._c)
        if kappa is not None:
            kap = np.ascontiguousarray(np.asarray(kappa, dtype=np.float64).reshape(-1))
            if kap.size != self.n_cells:
                raise ValueError(f"kappa needs {self.n_cells} values, got {kap.size}")
            self._kappa = L.dbl_array(kap)
            kptr = C.cast(self._kappa, C.POINTER(C.c_double))
        else:
            kptr = None
        mesh = L.irk_mesh(self.dim, self.N, int(levels), kptr)
        opt = L.irk_options()
        L.lib.irk_default_options(C.byref(opt))
        opt.precond = L.PC[precond]
        opt.vcycle_prec = L.PREC[vcycle]
        opt.nu_pre, opt.nu_post, opt.omega = int(nu_pre), int(nu_post), float(omega)
        opt.rtol, opt.restart, opt.maxit = float(rtol), int(restart), int(maxit)
        opt.orth = L.ORTH[orth]
        opt.solver = L.SOLVER[solver]
        opt.splitting = L.SPLIT[splitting]
        opt.warm_start = int(bool(warm_start))
        self.options = opt
        self.stream = stream if stream is not None else _current_stream()
        h = C.c_void_p()
        L.check(L.lib.irk_create(C.byref(h), C.byref(mesh), C.byref(tab), self.dt, C.byref(opt), self.stream))
        self._h = h
        self.last_stats: dict = {}

    # -- lifetime -------------------------------------------------------
    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            L.lib.irk_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- entry points ---------------------------------------------------
    def _stats(self, st: L.irk_stats, rc: int, allow_noconv: bool) -> dict:
        self.last_stats = st.as_dict()
        if rc == L.IRK_ENOCONV and allow_noconv:
            return self.last_stats
        L.check(rc)
        return self.last_stats

    def irk_step(self, u_n, u_np1, *, f_space=None, f_coef=None, f_stages=None, stages_out=None,
                 allow_noconv: bool = False) -> dict:
        nn, ns = self.n_nodes, self.n_nodes * self.s
        coef = L.dbl_array(f_coef) if f_coef is not None else None
        st = L.irk_stats()
        rc = L.lib.irk_step(self._h, L.ptr(u_n, count=nn), L.ptr(f_space, count=nn),
                            C.cast(coef, C.c_void_p) if coef is not None else None, L.ptr(f_stages, count=ns),
                            L.ptr(u_np1, count=nn), L.ptr(stages_out, count=ns), C.byref(st))
        return self._stats(st, rc, allow_noconv)

    step = irk_step

    def irk_step_dirichlet(self, u_n, g_stages, u_np1, *, f_space=None, f_coef=None, f_stages=None,
                           stages_out=None, allow_noconv: bool = False) -> dict:
        """One step with DAE-type Dirichlet data (Sec. 2.1): g_stages[p * s + i] = g(t_n + c_i dt) at
        boundary node p; u_n's boundary entries are the current boundary values."""
        nn, ns = self.n_nodes, self.n_nodes * self.s
        coef = L.dbl_array(f_coef) if f_coef is not None else None
        st = L.irk_stats()
        rc = L.lib.irk_step_dirichlet(self._h, L.ptr(u_n, count=nn), L.ptr(g_stages, count=ns),
                                      L.ptr(f_space, count=nn),
                                      C.cast(coef, C.c_void_p) if coef is not None else None,
                                      L.ptr(f_stages, count=ns), L.ptr(u_np1, count=nn),
                                      L.ptr(stages_out, count=ns), C.byref(st))
        return self._stats(st, rc, allow_noconv)

    step_dirichlet = irk_step_dirichlet

    def irk_solve(self, r, k, allow_noconv: bool = False) -> dict:
        ns = self.n_nodes * self.s
        st = L.irk_stats()
        rc = L.lib.irk_solve(self._h, L.ptr(r, count=ns), L.ptr(k, count=ns), C.byref(st))
        return self._stats(st, rc, allow_noconv)

    solve = irk_solve

    def irk_apply_operator(self, x, y, transpose: bool = False) -> None:
        ns = self.n_nodes * self.s
        L.check(L.lib.irk_apply_operator(self._h, L.ptr(x, count=ns), L.ptr(y, count=ns), int(transpose)))

    apply_operator = irk_apply_operator

    def irk_apply_mass(self, x, y) -> None:
        nn = self.n_nodes
        L.check(L.lib.irk_apply_mass(self._h, L.ptr(x, count=nn), L.ptr(y, count=nn)))

    apply_mass = irk_apply_mass

    def irk_apply_preconditioner(self, v, z, transpose: bool = False) -> None:
        ns = self.n_nodes * self.s
        L.check(L.lib.irk_apply_preconditioner(self._h, L.ptr(v, count=ns), L.ptr(z, count=ns), int(transpose)))

    apply_preconditioner = irk_apply_preconditioner

    def irk_step_adjoint(self, u_n, stages, lam_np1, lam_n, grad_accum=None, allow_noconv: bool = False) -> dict:
        nn, ns = self.n_nodes, self.n_nodes * self.s
        st = L.irk_stats()
        rc = L.lib.irk_step_adjoint(self._h, L.ptr(u_n, count=nn), L.ptr(stages, count=ns),
                                    L.ptr(lam_np1, count=nn), L.ptr(lam_n, count=nn),
                                    L.ptr(grad_accum, count=self.n_cells), C.byref(st))
        return self._stats(st, rc, allow_noconv)

    step_adjoint = irk_step_adjoint

    def irk_perf_select(self, classes=()) -> None:
        """Reset the instrumentation counters and time the named kernel classes."""
        mask = 0
        for c in classes:
            mask |= 1 << L.K_CLASSES.index(c)
        L.check(L.lib.irk_perf_select(self._h, mask))

    perf_select = irk_perf_select

    def irk_perf_read(self) -> dict:
        p = L.irk_perf()
        L.check(L.lib.irk_perf_read(self._h, C.byref(p)))
        return p.as_dict()

    perf_read = irk_perf_read

    def irk_set_kappa(self, kappa) -> None:
        kap = np.ascontiguousarray(np.asarray(kappa, dtype=np.float64).reshape(-1))
        if kap.size != self.n_cells:
            raise ValueError(f"kappa needs {self.n_cells} values, got {kap.size}")
        L.check(L.lib.irk_set_kappa(self._h, C.c_void_p(kap.ctypes.data)))

    set_kappa = irk_set_kappa

    def irk_reset_initial_guess(self) -> None:
        """The next step starts FGMRES from zero (with ``warm_start``; a no-op otherwise)."""
        L.check(L.lib.irk_reset_initial_guess(self._h))

    reset_initial_guess = irk_reset_initial_guess
