"""ctypes declarations of the C ABI in include/dim.h (libdim.so).

Argument marshalling only: every step of the method runs in the CUDA kernels
of libdim.so.  Importing this module does not touch the GPU; ``load()`` fails
loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdim.so")

# return codes and status bits (include/dim.h)
DIM_OK, DIM_EINVAL, DIM_ECUDA, DIM_ENONPHYS, DIM_ENOROOT, DIM_ETIMEOUT, DIM_ENOTIMPL = 0, -1, -2, -3, -4, -5, -6
DIM_ETOOLARGE = -7
NOALLOC_MAX_CELLS = 65536
ST_NONPHYS, ST_NAN, ST_NOROOT, ST_TRANSIENT, ST_PCAP, ST_TIMEOUT = 1, 2, 4, 8, 16, 32
RELAX_PRESSURE, RELAX_TEMPERATURE = 0, 1
PRECISION_FP64, PRECISION_FP32_BULK = 0, 1
PARABOLIC_HEAT, PARABOLIC_VISCOUS_X, PARABOLIC_VISCOUS_Y = 0, 1, 2
SCHED = 11          # doubles per step of a schedule record (DIM_SCHED)
GRAD_NPARAMS = 6    # k0_1, k0_2, mu_1, mu_2, I_1, I_2 (DIM_GRAD_NPARAMS)

# every entry point the header declares
SYMBOLS = ["dim_init", "dim_destroy", "dim_from_primitive", "dim_cfl_dt", "dim_step", "dim_step_host",
           "dim_hllc_sweep", "dim_relax", "dim_cheb_parabolic", "dim_grad", "dim_status", "dim_profile",
           "dim_kernel_time", "dim_strerror", "dim_hllc_sweep_noalloc", "dim_batch_init", "dim_batch_destroy",
           "dim_batch_layout", "dim_batch_from_primitive", "dim_batch_step", "dim_batch_autotune",
           "dim_batch_status", "dim_step_sched", "dim_from_primitive_vjp", "dim_wait_selftest"]
# measurement and self-check entry points (include/dim_probe.h)
PROBE_SYMBOLS = ["dim_probe_rate", "dim_probe_ff_roundtrip"]
PROBE_DFMA, PROBE_DADDMUL, PROBE_DDIV, PROBE_DSQRT, PROBE_FFMA = 0, 1, 2, 3, 4


class DimParams(C.Structure):
    _fields_ = [
        ("gamma", C.c_double * 2), ("pinf", C.c_double * 2), ("cv", C.c_double * 2),
        ("k0", C.c_double * 2), ("k_exp", C.c_double), ("T_ref", C.c_double),
        ("mu", C.c_double * 2), ("cfl", C.c_double),
        ("limiter", C.c_int), ("bc", C.c_int * 2), ("trelax", C.c_int), ("n_outer", C.c_int),
        ("p_policy", C.c_int), ("p_fixed", C.c_int), ("p_min", C.c_int), ("p_max", C.c_int),
        ("precision", C.c_int), ("src", C.c_double * 2),
        ("heat_alpha", C.c_int), ("trelax_iters", C.c_int),
    ]


def make_params(p) -> DimParams:
    s = DimParams()
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
    s.precision = getattr(p, "precision", 0)
    s.src[:] = list(getattr(p, "src", (0.0, 0.0)))
    s.heat_alpha = getattr(p, "heat_alpha", 0)
    s.trelax_iters = getattr(p, "trelax_iters", 20)
    return s


_lib = None


def load(path: str = LIB_PATH):
    """Load libdim.so and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    L = C.CDLL(path)
    vp, i, d, u = C.c_void_p, C.c_int, C.c_double, C.c_uint
    pd = C.POINTER(C.c_double)
    L.dim_init.argtypes = [C.POINTER(vp), C.POINTER(DimParams), i, i, d, d, vp]
    L.dim_destroy.argtypes = [vp]
    L.dim_destroy.restype = None
    L.dim_from_primitive.argtypes = [vp, vp, vp]
    L.dim_cfl_dt.argtypes = [vp, vp, pd]
    L.dim_step.argtypes = [vp, vp, i, pd]
    L.dim_step_host.argtypes = [vp, vp, i, pd]
    L.dim_hllc_sweep.argtypes = [vp, vp, i, d, i]
    L.dim_relax.argtypes = [vp, vp, i]
    L.dim_cheb_parabolic.argtypes = [vp, vp, i, d, C.POINTER(i)]
    L.dim_grad.argtypes = [vp, vp, i, i, vp, vp, pd]
    L.dim_step_sched.argtypes = [vp, vp, i, vp, i]
    L.dim_from_primitive_vjp.argtypes = [vp, vp, vp, vp]
    L.dim_wait_selftest.argtypes = [vp, d]
    L.dim_status.argtypes = [vp, C.POINTER(u), i]
    L.dim_profile.argtypes = [vp, i, i]
    L.dim_kernel_time.argtypes = [vp, C.c_char_p, C.POINTER(i), pd]
    L.dim_hllc_sweep_noalloc.argtypes = [C.POINTER(DimParams), i, i, d, d, vp, i, d, i, vp]
    L.dim_strerror.argtypes = [i]
    L.dim_probe_rate.argtypes = [i, i, i, vp, pd, pd]
    L.dim_probe_rate.restype = i
    L.dim_probe_ff_roundtrip.argtypes = [vp, vp, i, vp]
    L.dim_probe_ff_roundtrip.restype = i
    L.dim_strerror.restype = C.c_char_p
    for name in SYMBOLS:
        if name not in ("dim_destroy", "dim_strerror") and not name.startswith("dim_batch"):
            getattr(L, name).restype = i
    declare_batch(L)
    _lib = L
    return L


class DimError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = load().dim_strerror(code).decode()
        super().__init__(f"{where}: {msg} ({code})")
        self.code = code


def check(code: int, where: str) -> int:
    if code != DIM_OK:
        raise DimError(code, where)
    return code


def declare_batch(L):
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    L.dim_batch_init.argtypes = [C.POINTER(vp), C.POINTER(DimParams), i, C.POINTER(i), C.POINTER(i),
                                 C.POINTER(d), C.POINTER(d), vp]
    L.dim_batch_destroy.argtypes = [vp]
    L.dim_batch_destroy.restype = None
    L.dim_batch_layout.argtypes = [vp, C.POINTER(C.c_longlong)]
    L.dim_batch_from_primitive.argtypes = [vp, vp, vp]
    L.dim_batch_step.argtypes = [vp, vp, i]
    L.dim_batch_autotune.argtypes = [vp, vp, C.POINTER(i)]
    L.dim_batch_status.argtypes = [vp, C.POINTER(C.c_uint), C.POINTER(C.c_uint)]
    for n in ("dim_batch_init", "dim_batch_layout", "dim_batch_from_primitive", "dim_batch_step",
              "dim_batch_autotune", "dim_batch_status"):
        getattr(L, n).restype = i
