"""ctypes binding of the FP64 CPU oracle (``dim_oracle.cc``).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
CPU-baseline / reference leg of the benchmark.  The product path never loads
this module.  Arrays are numpy float64, state shape (8, ny, nx).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dim_oracle.cc")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


SCHED = 11  # doubles per step in a schedule record: S, lambda_max heat x8, viscous x, viscous y


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (no FMA contraction)."""
    out = _LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", out, _SRC, "-lm"]
        subprocess.check_call(cmd)
    return out


class _Params(C.Structure):
    _fields_ = [
        ("gamma", C.c_double * 2), ("pinf", C.c_double * 2), ("cv", C.c_double * 2),
        ("k0", C.c_double * 2), ("k_exp", C.c_double), ("T_ref", C.c_double),
        ("mu", C.c_double * 2), ("cfl", C.c_double),
        ("limiter", C.c_int), ("bc", C.c_int * 2), ("trelax", C.c_int), ("n_outer", C.c_int),
        ("p_policy", C.c_int), ("p_fixed", C.c_int), ("p_min", C.c_int), ("p_max", C.c_int),
        ("precision", C.c_int), ("src", C.c_double * 2),
        ("heat_alpha", C.c_int), ("trelax_iters", C.c_int),
    ]


def _params(p) -> _Params:
    s = _Params()
    s.gamma[:] = list(p.gamma)
    s.pinf[:] = list(p.pinf)
    s.cv[:] = list(p.cv)
    s.k0[:] = list(p.k0)
    s.k_exp = p.k_exp
    s.T_ref = p.T_ref
    s.mu[:] = list(p.mu)
    s.cfl = p.cfl
    s.limiter = p.limiter
    s.bc[:] = list(p.bc)
    s.trelax = p.trelax
    s.n_outer = p.n_outer
    s.p_policy = p.p_policy
    s.p_fixed = p.p_fixed
    s.p_min = p.p_min
    s.p_max = p.p_max
    s.precision = 0
    s.src[:] = list(getattr(p, "src", (0.0, 0.0)))
    s.heat_alpha = getattr(p, "heat_alpha", 0)
    s.trelax_iters = getattr(p, "trelax_iters", 20)
    return s


_D = C.POINTER(C.c_double)


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        P = C.POINTER(_Params)
        i, d, u = C.c_int, C.c_double, C.c_uint
        L.orc_from_primitive.argtypes = [P, i, i, _D, _D]; L.orc_from_primitive.restype = u
        L.orc_dt.argtypes = [P, i, i, d, d, _D]; L.orc_dt.restype = d
        L.orc_sweep.argtypes = [P, i, i, d, d, i, d, _D]; L.orc_sweep.restype = u
        L.orc_prelax.argtypes = [P, i, _D]; L.orc_prelax.restype = u
        L.orc_trelax.argtypes = [P, i, _D]; L.orc_trelax.restype = u
        L.orc_heat.argtypes = [P, i, i, d, d, d, _D, C.POINTER(i)]; L.orc_heat.restype = u
        L.orc_viscous.argtypes = [P, i, i, d, d, i, d, _D, C.POINTER(i)]; L.orc_viscous.restype = u
        L.orc_step.argtypes = [P, i, i, d, d, _D, i, d, _D, C.POINTER(i)]; L.orc_step.restype = u
        L.orc_step_sched.argtypes = [P, i, i, d, d, _D, i, _D, i]; L.orc_step_sched.restype = u
        L.orc_count_ops.argtypes = [P, i, i, d, d, _D, i, d, C.POINTER(C.c_ulonglong)]
        L.orc_count_ops.restype = i
        L.orc_step_frozen.argtypes = [P, i, i, d, d, _D, i, _D, C.c_void_p, C.c_size_t, i, C.POINTER(C.c_size_t)]
        L.orc_step_frozen.restype = u
        L.orc_step_tangent.argtypes = [P, _D, i, i, d, d, _D, _D, i, _D]; L.orc_step_tangent.restype = u
        L.orc_step_tangent_ext.argtypes = [P, _D, i, i, d, d, _D, _D, i, _D, C.c_void_p, C.c_size_t]
        L.orc_step_tangent_ext.restype = u
        L.orc_cheb_P.argtypes = [P, d, d]; L.orc_cheb_P.restype = i
        L.orc_cheb_schedule.argtypes = [i, d, _D]; L.orc_cheb_schedule.restype = None
        L.orc_lim_solve.argtypes = [P, i, i, d, d, d, _D, _D, _D, _D, _D]; L.orc_lim_solve.restype = i
        L.orc_diagnostics.argtypes = [P, i, _D, _D]; L.orc_diagnostics.restype = None
        L.orc_heat_coeffs.argtypes = [P, i, _D, _D]; L.orc_heat_coeffs.restype = None
        L.orc_equilibrium.argtypes = [P, d, d, d, _D, _D]; L.orc_equilibrium.restype = u
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _state(U: np.ndarray) -> np.ndarray:
    U = np.ascontiguousarray(U, dtype=np.float64)
    assert U.shape[0] == 8
    return U


def from_primitive(params, prim: np.ndarray) -> np.ndarray:
    prim = np.ascontiguousarray(prim, dtype=np.float64)
    _, ny, nx = prim.shape
    U = np.empty((8, ny, nx))
    st = lib().orc_from_primitive(C.byref(_params(params)), nx, ny, _ptr(prim), _ptr(U))
    if st:
        raise ValueError(f"non-physical initial data (status {st})")
    return U


def dt(params, U, dx, dy) -> float:
    U = _state(U)
    return lib().orc_dt(C.byref(_params(params)), U.shape[2], U.shape[1], dx, dy, _ptr(U))


def sweep(params, U, dx, dy, axis, dt_):
    U = _state(U).copy()
    st = lib().orc_sweep(C.byref(_params(params)), U.shape[2], U.shape[1], dx, dy, axis, dt_, _ptr(U))
    return U, st


def prelax(params, U):
    U = _state(U).copy()
    st = lib().orc_prelax(C.byref(_params(params)), U.shape[1] * U.shape[2], _ptr(U))
    return U, st


def trelax(params, U):
    U = _state(U).copy()
    st = lib().orc_trelax(C.byref(_params(params)), U.shape[1] * U.shape[2], _ptr(U))
    return U, st


def heat(params, U, dx, dy, tau):
    U = _state(U).copy()
    pu = C.c_int(0)
    st = lib().orc_heat(C.byref(_params(params)), U.shape[2], U.shape[1], dx, dy, tau, _ptr(U), C.byref(pu))
    return U, st, pu.value


def viscous(params, U, dx, dy, axis, tau):
    U = _state(U).copy()
    pu = C.c_int(0)
    st = lib().orc_viscous(C.byref(_params(params)), U.shape[2], U.shape[1], dx, dy, axis, tau, _ptr(U),
                           C.byref(pu))
    return U, st, pu.value


def step(params, U, dx, dy, nsteps=1, dt_fixed=0.0):
    """nsteps full split steps; returns (U, status, dt_last, P_heat)."""
    U = _state(U).copy()
    dtl = C.c_double(0.0)
    ph = C.c_int(0)
    st = lib().orc_step(C.byref(_params(params)), U.shape[2], U.shape[1], dx, dy, _ptr(U), nsteps, dt_fixed,
                        C.byref(dtl), C.byref(ph))
    return U, st, dtl.value, ph.value


def step_sched(params, U, dx, dy, nsteps, sched=None):
    """nsteps steps; with sched=None the schedule (S and every lambda_max, per
    step) is recorded and returned, with a given sched it is replayed.
    Returns (U, status, sched)."""
    U = _state(U).copy()
    replay = sched is not None
    if sched is None:
        sched = np.zeros((nsteps, SCHED))
    sched = np.ascontiguousarray(sched, dtype=np.float64)
    assert sched.shape == (nsteps, SCHED)
    st = lib().orc_step_sched(C.byref(_params(params)), U.shape[2], U.shape[1], dx, dy, _ptr(U), nsteps,
                              _ptr(sched), int(replay))
    return U, st, sched


def step_frozen(params, U, dx, dy, nsteps, frozen=None):
    """nsteps steps.  frozen=None: record the schedule and every branch of the
    sweeps (limiter operand, Davis bounds, HLLC region) and return them;
    frozen=(sched, tape): replay them, so the run follows the recorded
    branches (the branch-frozen map).  Returns (U, status, (sched, tape))."""
    U = _state(U).copy()
    lib_ = lib()
    if frozen is None:
        sched = np.zeros((nsteps, SCHED))
        cap = 1 << 16
        while True:
            tape = np.zeros(cap, dtype=np.uint8)
            used = C.c_size_t(0)
            Ur = U.copy()
            st = lib_.orc_step_frozen(C.byref(_params(params)), U.shape[2], U.shape[1], dx, dy, _ptr(Ur), nsteps,
                                      _ptr(sched), tape.ctypes.data, cap, 0, C.byref(used))
            if used.value <= cap:
                return Ur, st, (sched, tape[:used.value].copy())
            cap = used.value
    sched, tape = frozen
    sched = np.ascontiguousarray(sched, dtype=np.float64).copy()
    tape = np.ascontiguousarray(tape, dtype=np.uint8)
    used = C.c_size_t(0)
    st = lib_.orc_step_frozen(C.byref(_params(params)), U.shape[2], U.shape[1], dx, dy, _ptr(U), nsteps, _ptr(sched),
                              tape.ctypes.data, tape.size, 1, C.byref(used))
    if used.value != tape.size:
        raise ValueError(f"branch record of {tape.size} decisions replayed by a run taking {used.value}")
    return U, st, (sched, tape)


def step_tangent(params, U, dU, dx, dy, nsteps, dparams=None):
    """Tangent-linear map of nsteps steps with the schedule frozen at the run's
    own values: returns (U_T, dU_T, status, sched).  dparams: tangents of
    (k0_1, k0_2, mu_1, mu_2, I_1, I_2) or None."""
    U = _state(U).copy()
    dU = _state(dU).copy()
    assert dU.shape == U.shape
    sched = np.zeros((nsteps, SCHED))
    dp = None if dparams is None else np.ascontiguousarray(dparams, dtype=np.float64)
    st = lib().orc_step_tangent(C.byref(_params(params)), None if dp is None else _ptr(dp), U.shape[2], U.shape[1],
                                dx, dy, _ptr(U), _ptr(dU), nsteps, _ptr(sched))
    return U, dU, st, sched


def step_tangent_ext(params, U, dU, dx, dy, nsteps, frozen, dparams=None):
    """The tangent in long double following the double run's schedule and
    branches (frozen = (sched, tape) from step_frozen): a reference for the
    rounding error of the double tangent.  Returns (U_T, dU_T, status)."""
    U = _state(U).copy()
    dU = _state(dU).copy()
    sched, tape = frozen
    sched = np.ascontiguousarray(sched, dtype=np.float64).copy()
    tape = np.ascontiguousarray(tape, dtype=np.uint8)
    dp = None if dparams is None else np.ascontiguousarray(dparams, dtype=np.float64)
    st = lib().orc_step_tangent_ext(C.byref(_params(params)), None if dp is None else _ptr(dp), U.shape[2],
                                    U.shape[1], dx, dy, _ptr(U), _ptr(dU), nsteps, _ptr(sched), tape.ctypes.data,
                                    tape.size)
    if st & 64:
        raise ValueError("branch record does not match the extended run")
    return U, dU, st


COUNT_STAGES = {"wave_max": 0, "sweep_x": 1, "sweep_y": 2, "prelax": 3, "trelax": 4, "heat": 5, "viscous_x": 6,
                "viscous_y": 7}


def count_ops(params, U, dx, dy, stage, tau=0.0):
    """Floating-point operations one stage applies to state-dependent values:
    dict(add, mul, div, sqrt, pow, total, P)."""
    U = _state(U)
    out = (C.c_ulonglong * 5)()
    Pn = lib().orc_count_ops(C.byref(_params(params)), U.shape[2], U.shape[1], dx, dy, _ptr(U), COUNT_STAGES[stage],
                             tau, out)
    c = dict(zip(("add", "mul", "div", "sqrt", "pow"), (int(x) for x in out)))
    c["total"] = sum(c[k] for k in ("add", "mul", "div", "sqrt", "pow"))
    c["P"] = Pn
    return c


def cheb_P(params, tau, lam_max) -> int:
    return lib().orc_cheb_P(C.byref(_params(params)), tau, lam_max)


def cheb_schedule(P: int, lam: float) -> np.ndarray:
    b = np.zeros(2 * P - 1)
    lib().orc_cheb_schedule(P, lam, _ptr(b))
    return b


def lim_solve(params, lam, V, v0, dx, dy, tau):
    """One full LIM solve of dv/dt = V L_h v; arrays of shape (ny, nx)."""
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    V = np.ascontiguousarray(V, dtype=np.float64)
    v0 = np.ascontiguousarray(v0, dtype=np.float64)
    ny, nx = v0.shape
    v1 = np.empty_like(v0)
    lm = C.c_double(0.0)
    Pn = lib().orc_lim_solve(C.byref(_params(params)), nx, ny, dx, dy, tau, _ptr(lam), _ptr(V), _ptr(v0),
                             _ptr(v1), C.byref(lm))
    return v1, Pn, lm.value


def diagnostics(params, U):
    """(p1, p2, T1, T2, u, v), each shaped like one plane."""
    U = _state(U)
    out = np.empty((6,) + U.shape[1:])
    lib().orc_diagnostics(C.byref(_params(params)), U.shape[1] * U.shape[2], _ptr(U), _ptr(out))
    return out


def heat_coeffs(params, U):
    """(T, V, U_alpha, Lam) at each cell."""
    U = _state(U)
    out = np.empty((4,) + U.shape[1:])
    lib().orc_heat_coeffs(C.byref(_params(params)), U.shape[1] * U.shape[2], _ptr(U), _ptr(out))
    return out


def equilibrium(params, m1, m2, rhoe):
    T = C.c_double(0.0)
    a = C.c_double(0.0)
    st = lib().orc_equilibrium(C.byref(_params(params)), m1, m2, rhoe, C.byref(T), C.byref(a))
    return T.value, a.value, st
