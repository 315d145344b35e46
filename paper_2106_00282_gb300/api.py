"""Thin Python binding of libdim (names follow include/dim.h).

PyTorch provides device memory and the stream; every computation runs in the
CUDA kernels behind the C ABI.  There is no CPU fallback: without a CUDA device
or without libdim.so the calls raise.

    s = Solver(params, nx, ny, dx, dy)
    U = s.from_primitive(prim)          # prim: (5, ny, nx) float64 alpha_2, p, T, u, v
    dt = s.step(U, nsteps=10)           # U: (8, ny, nx) float64 on the device, in place

Gradients (FP64): ``Solver.grad`` is the adjoint of nsteps steps (dim_grad);
``steps`` and ``from_primitive`` are the same maps as torch.autograd functions,
differentiable with respect to the state, the primitive fields and the
parameter vector (k0_1, k0_2, mu_1, mu_2, I_1, I_2).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import check


def _dev_ptr(t: torch.Tensor, shape=None) -> int:
    if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError("expected a contiguous float64 CUDA tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {tuple(t.shape)}")
    return t.data_ptr()


class Solver:
    """One grid, one parameter set, one CUDA stream (a dim_ctx)."""

    def __init__(self, params, nx: int, ny: int, dx: float, dy: float, stream: torch.cuda.Stream | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("libdim needs a CUDA device")
        self.L = _lib.load()
        self.params, self.nx, self.ny, self.dx, self.dy = params, nx, ny, dx, dy
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._p = _lib.make_params(params)
        self._ctx = C.c_void_p()
        check(self.L.dim_init(C.byref(self._ctx), C.byref(self._p), nx, ny, dx, dy,
                              C.c_void_p(self.stream.cuda_stream)), "dim_init")

    @property
    def state_shape(self):
        return (8, self.ny, self.nx)

    def close(self):
        if self._ctx:
            self.L.dim_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def from_primitive(self, prim: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        U = out if out is not None else torch.empty(self.state_shape, dtype=torch.float64, device=prim.device)
        check(self.L.dim_from_primitive(self._ctx, _dev_ptr(prim, (5, self.ny, self.nx)),
                                        _dev_ptr(U, self.state_shape)), "dim_from_primitive")
        return U

    def cfl_dt(self, U: torch.Tensor) -> float:
        dt = C.c_double(0.0)
        check(self.L.dim_cfl_dt(self._ctx, _dev_ptr(U, self.state_shape), C.byref(dt)), "dim_cfl_dt")
        return dt.value

    def step(self, U: torch.Tensor, nsteps: int = 1, sync: bool = True):
        """nsteps split steps in place; with sync returns dt of the last step
        and raises on an inadmissible end-of-step state."""
        if sync:
            dt = C.c_double(0.0)
            check(self.L.dim_step(self._ctx, _dev_ptr(U, self.state_shape), nsteps, C.byref(dt)), "dim_step")
            return dt.value
        check(self.L.dim_step(self._ctx, _dev_ptr(U, self.state_shape), nsteps, None), "dim_step")
        return None

    def step_host(self, U_host: torch.Tensor, nsteps: int = 1) -> float:
        """The same on a host (ideally pinned) float64 tensor: H2D, steps, D2H."""
        if U_host.is_cuda or U_host.dtype != torch.float64 or not U_host.is_contiguous():
            raise ValueError("expected a contiguous float64 host tensor")
        dt = C.c_double(0.0)
        check(self.L.dim_step_host(self._ctx, U_host.data_ptr(), nsteps, C.byref(dt)), "dim_step_host")
        return dt.value

    def hllc_sweep(self, U: torch.Tensor, axis: int, dt: float, relax: bool = True):
        check(self.L.dim_hllc_sweep(self._ctx, _dev_ptr(U, self.state_shape), axis, dt, int(relax)),
              "dim_hllc_sweep")

    def relax(self, U: torch.Tensor, which: int):
        check(self.L.dim_relax(self._ctx, _dev_ptr(U, self.state_shape), which), "dim_relax")

    def cheb_parabolic(self, U: torch.Tensor, kind: int, dt: float) -> int:
        P = C.c_int(0)
        check(self.L.dim_cheb_parabolic(self._ctx, _dev_ptr(U, self.state_shape), kind, dt, C.byref(P)),
              "dim_cheb_parabolic")
        return P.value

    def status(self, reset: bool = False) -> int:
        f = C.c_uint(0)
        check(self.L.dim_status(self._ctx, C.byref(f), int(reset)), "dim_status")
        return f.value

    def wait_selftest(self, seconds: float = 0.2) -> int:
        """Failure-detection self-test of the bounded waits (dim_wait_selftest):
        returns the DIM_* code, DIM_ETIMEOUT when the wait ran out as designed."""
        return int(self.L.dim_wait_selftest(self._ctx, float(seconds)))

    def step_sched(self, U: torch.Tensor, nsteps: int, sched: torch.Tensor | None = None) -> torch.Tensor:
        """nsteps steps (FP64) in place.  sched None: the schedule (CFL maximum S
        and every LIM lambda_max, per step) is recorded and returned as a
        (nsteps, 11) device tensor; a given sched is replayed (the map with time
        steps and Chebyshev parameters held fixed)."""
        replay = sched is not None
        if sched is None:
            sched = torch.zeros((nsteps, _lib.SCHED), dtype=torch.float64, device=U.device)
        check(self.L.dim_step_sched(self._ctx, _dev_ptr(U, self.state_shape), nsteps,
                                    _dev_ptr(sched, (nsteps, _lib.SCHED)), int(replay)), "dim_step_sched")
        return sched

    def grad(self, U0: torch.Tensor, nsteps: int, dJ_dUT: torch.Tensor, ckpt_every: int = 20):
        """Adjoint of nsteps steps from U0 (dim_grad): returns (dJ/dU0 device
        tensor, dJ/d(k0_1, k0_2, mu_1, mu_2, I_1, I_2) numpy array)."""
        out = torch.empty_like(U0)
        gp = (C.c_double * _lib.GRAD_NPARAMS)()
        check(self.L.dim_grad(self._ctx, _dev_ptr(U0, self.state_shape), nsteps, ckpt_every,
                              _dev_ptr(dJ_dUT, self.state_shape), _dev_ptr(out, self.state_shape), gp), "dim_grad")
        return out, np.array(list(gp))

    def from_primitive_vjp(self, prim: torch.Tensor, Ubar: torch.Tensor) -> torch.Tensor:
        """(dU/dprim)^T Ubar of from_primitive at prim (dim_from_primitive_vjp)."""
        out = torch.empty_like(prim)
        check(self.L.dim_from_primitive_vjp(self._ctx, _dev_ptr(prim, (5, self.ny, self.nx)),
                                            _dev_ptr(Ubar, self.state_shape), _dev_ptr(out, (5, self.ny, self.nx))),
              "dim_from_primitive_vjp")
        return out

    def profile(self, enable: bool = True, reset: bool = True):
        check(self.L.dim_profile(self._ctx, int(enable), int(reset)), "dim_profile")

    def kernel_time(self, name: str):
        n = C.c_int(0)
        ms = C.c_double(0.0)
        check(self.L.dim_kernel_time(self._ctx, name.encode(), C.byref(n), C.byref(ms)), "dim_kernel_time")
        return n.value, ms.value


def param_vector(params) -> torch.Tensor:
    """(k0_1, k0_2, mu_1, mu_2, I_1, I_2) of a parameter set, float64 on the CPU."""
    return torch.tensor([params.k0[0], params.k0[1], params.mu[0], params.mu[1], params.src[0], params.src[1]],
                        dtype=torch.float64)


class _Steps(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U0, pvec, solver, nsteps, ckpt_every):
        ref = param_vector(solver.params)
        if not torch.equal(pvec.detach().cpu().to(torch.float64), ref):
            raise ValueError("pvec must hold the solver's (k0_1, k0_2, mu_1, mu_2, I_1, I_2)")
        UT = U0.detach().clone()
        solver.step(UT, nsteps)
        ctx.solver, ctx.nsteps, ctx.ckpt = solver, nsteps, ckpt_every
        ctx.pdev, ctx.pdtype = pvec.device, pvec.dtype
        ctx.save_for_backward(U0.detach())
        return UT

    @staticmethod
    def backward(ctx, gUT):
        (U0,) = ctx.saved_tensors
        gU0, gp = ctx.solver.grad(U0, ctx.nsteps, gUT.contiguous(), ctx.ckpt)
        return gU0, torch.tensor(gp, dtype=ctx.pdtype, device=ctx.pdev), None, None, None


class _FromPrimitive(torch.autograd.Function):
    @staticmethod
    def forward(ctx, prim, solver):
        p = prim.detach().contiguous()
        ctx.solver = solver
        ctx.save_for_backward(p)
        return solver.from_primitive(p)

    @staticmethod
    def backward(ctx, gU):
        (p,) = ctx.saved_tensors
        return ctx.solver.from_primitive_vjp(p, gU.contiguous()), None


def steps(U0: torch.Tensor, solver: "Solver", nsteps: int, ckpt_every: int = 20, pvec: torch.Tensor | None = None):
    """U_T = nsteps split steps of U0 (FP64), as a torch.autograd function.
    Backward calls dim_grad (adjoint with the run's schedule and branches held
    fixed, checkpoints every ckpt_every steps) and returns the gradients with
    respect to U0 and pvec = (k0_1, k0_2, mu_1, mu_2, I_1, I_2), which must be
    the solver's own values (param_vector(solver.params))."""
    if pvec is None:
        pvec = param_vector(solver.params)
    return _Steps.apply(U0, pvec, solver, nsteps, ckpt_every)


def from_primitive(prim: torch.Tensor, solver: "Solver") -> torch.Tensor:
    """dim_from_primitive as a torch.autograd function (backward:
    dim_from_primitive_vjp)."""
    return _FromPrimitive.apply(prim, solver)


class Batch:
    """Many independent grids (same parameters, FP32 bulk) advanced together:
    one persistent launch per step, replayed from a CUDA graph (a dim_batch)."""

    def __init__(self, params, grids, stream: torch.cuda.Stream | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("libdim needs a CUDA device")
        self.L = _lib.load()
        self.params = params
        self.grids = list(grids)
        n = len(self.grids)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._p = _lib.make_params(params)
        nx = (C.c_int * n)(*[g[0] for g in self.grids])
        ny = (C.c_int * n)(*[g[1] for g in self.grids])
        dx = (C.c_double * n)(*[g[2] for g in self.grids])
        dy = (C.c_double * n)(*[g[3] for g in self.grids])
        self._b = C.c_void_p()
        check(self.L.dim_batch_init(C.byref(self._b), C.byref(self._p), n, nx, ny, dx, dy,
                                    C.c_void_p(self.stream.cuda_stream)), "dim_batch_init")
        off = (C.c_longlong * (n + 1))()
        check(self.L.dim_batch_layout(self._b, off), "dim_batch_layout")
        self.offsets = list(off)
        self.ncell = self.offsets[-1]

    def close(self):
        if self._b:
            self.L.dim_batch_destroy(self._b)
            self._b = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def pack_primitive(self, prims) -> torch.Tensor:
        """Primitive arrays (5, ny, nx) per instance -> one packed device buffer."""
        buf = torch.empty(5 * self.ncell, dtype=torch.float64)
        for i, pr in enumerate(prims):
            o, n = self.offsets[i], self.offsets[i + 1] - self.offsets[i]
            buf[5 * o:5 * o + 5 * n] = torch.from_numpy(pr.reshape(-1))
        return buf.cuda()

    def from_primitive(self, prim_packed: torch.Tensor) -> torch.Tensor:
        U = torch.empty(8 * self.ncell, dtype=torch.float64, device=prim_packed.device)
        check(self.L.dim_batch_from_primitive(self._b, _dev_ptr(prim_packed), _dev_ptr(U)), "dim_batch_from_primitive")
        return U

    def state(self, U: torch.Tensor, i: int) -> torch.Tensor:
        """View of instance i as (8, ny, nx)."""
        nx, ny = self.grids[i][0], self.grids[i][1]
        o = self.offsets[i]
        return U[8 * o:8 * o + 8 * nx * ny].view(8, ny, nx)

    def step(self, U: torch.Tensor, nsteps: int = 1):
        check(self.L.dim_batch_step(self._b, _dev_ptr(U), nsteps), "dim_batch_step")

    def autotune(self, U: torch.Tensor):
        cfg = (C.c_int * 6)()
        check(self.L.dim_batch_autotune(self._b, _dev_ptr(U), cfg), "dim_batch_autotune")
        return list(cfg)

    def status(self):
        n = len(self.grids)
        flags = (C.c_uint * n)()
        anyf = C.c_uint(0)
        check(self.L.dim_batch_status(self._b, flags, C.byref(anyf)), "dim_batch_status")
        return list(flags), anyf.value
