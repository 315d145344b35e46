"""The C-ABI library builds, loads and exports every entry point include/dim.h
declares; argument validation needs no GPU (no compute call is made here)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header="dim.h"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dim_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2106_00282_gb300 import _lib, build

    build.build()
    return _lib.load()


def test_header_symbols_exported(lib):
    from paper_2106_00282_gb300 import _lib

    names = _declared()
    assert "dim_step" in names and "dim_cheb_parabolic" in names
    assert sorted(_lib.SYMBOLS) == names
    for n in names:
        assert getattr(lib, n) is not None, n
    probes = _declared("dim_probe.h")
    assert sorted(_lib.PROBE_SYMBOLS) == probes
    for n in probes:
        assert getattr(lib, n) is not None, n


def test_every_header_checked():
    assert sorted(os.listdir(os.path.join(ROOT, "include"))) == ["dim.h", "dim_probe.h"]


def test_strerror(lib):
    assert lib.dim_strerror(0) == b"ok"
    assert b"non-physical" in lib.dim_strerror(-3)


def test_init_rejects_bad_arguments(lib):
    """Validation happens before any CUDA call."""
    from paper_2106_00282_gb300 import _lib, inputs

    good = inputs.shock_tube().params
    ctx = C.c_void_p()
    cases = [
        (good, 0, 1, 1e-3, 1e-3),
        (good, 16385, 8192, 1e-3, 1e-3),  # above 2^27 cells
        (good, 1, 1, 1e-3, 1e-3),
        (good, 10, 1, -1.0, 1e-3),
        (good.replace(gamma=(1.0, 1.4)), 10, 1, 1e-3, 1e-3),
        (good.replace(cfl=0.0), 10, 1, 1e-3, 1e-3),
        (good.replace(limiter=7), 10, 1, 1e-3, 1e-3),
        (good.replace(p_max=65), 10, 1, 1e-3, 1e-3),
        (good.replace(p_policy=1, p_fixed=0), 10, 1, 1e-3, 1e-3),
        (good.replace(n_outer=0), 10, 1, 1e-3, 1e-3),
        (good.replace(bc=(0, 5)), 10, 1, 1e-3, 1e-3),
        (good.replace(trelax=3), 10, 1, 1e-3, 1e-3),
        (good.replace(trelax=inputs.TRELAX_MIDPOINT, trelax_iters=0), 10, 1, 1e-3, 1e-3),
        (good.replace(trelax=inputs.TRELAX_MIDPOINT, trelax_iters=1001), 10, 1, 1e-3, 1e-3),
        (good.replace(heat_alpha=2), 10, 1, 1e-3, 1e-3),
        # the paper's variants are FP64 kernels only
        (good.replace(trelax=inputs.TRELAX_MIDPOINT, precision=inputs.PRECISION_FP32_BULK), 10, 1, 1e-3, 1e-3),
        (good.replace(heat_alpha=inputs.HEAT_ALPHA_LINEAR, precision=inputs.PRECISION_FP32_BULK), 10, 1, 1e-3,
         1e-3),
    ]
    for p, nx, ny, dx, dy in cases:
        s = _lib.make_params(p)
        assert lib.dim_init(C.byref(ctx), C.byref(s), nx, ny, dx, dy, None) == _lib.DIM_EINVAL
    assert lib.dim_step(None, None, 1, None) == _lib.DIM_EINVAL
    assert lib.dim_grad(None, None, 1, 1, None, None, None) == _lib.DIM_EINVAL
    assert lib.dim_step_sched(None, None, 1, None, 0) == _lib.DIM_EINVAL
    assert lib.dim_from_primitive_vjp(None, None, None, None) == _lib.DIM_EINVAL
    assert lib.dim_wait_selftest(None, 0.1) == _lib.DIM_EINVAL
    ms, ops = C.c_double(), C.c_double()
    assert lib.dim_probe_rate(5, 0, 10, None, C.byref(ms), C.byref(ops)) == _lib.DIM_EINVAL
    assert lib.dim_probe_rate(0, 0, 0, None, C.byref(ms), C.byref(ops)) == _lib.DIM_EINVAL
    assert lib.dim_probe_ff_roundtrip(None, None, 4, None) == _lib.DIM_EINVAL
