"""dim_hllc_sweep_noalloc: the sweep for callers that cannot let a library
allocate device memory (an application pool allocator that owns all device
memory, a device-memory budget fixed at load time, loops that cannot take the
device-wide synchronization of cudaMalloc).  Its scratch is a fixed array in
the library, so it needs no context.  Checked against the context-based
dim_hllc_sweep through the C ABI, on two calls in a row (the second call runs
on the array the first one left behind), within the parity tolerance of the
other GPU tests.  This file is collected last and works alone in a fresh
process as well as after the other tests."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-11


def _rel_l1(a, b):
    num = np.abs(a - b).reshape(8, -1).sum(axis=1)
    den = np.abs(b).reshape(8, -1).sum(axis=1)
    return num / np.maximum(den, 1e-300)


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_sweep_matches_context_sweep(precision):
    """precision 0: the FP64 sweep; 1: the FP32-bulk sweep (the parameters pick
    the kernel on both paths)."""
    import torch

    from paper_2106_00282_gb300 import _lib, build, inputs as I
    from paper_2106_00282_gb300.api import Solver

    assert torch.cuda.is_available()
    build.build()
    L = _lib.load()
    wl = I.impact(240, 200)  # 48,000 cells: several tiles per axis and ragged tails
    wl.params = wl.params.replace(precision=precision)
    assert wl.nx * wl.ny <= _lib.NOALLOC_MAX_CELLS
    s = Solver(wl.params, wl.nx, wl.ny, wl.dx, wl.dy)
    U = s.from_primitive(torch.from_numpy(wl.prim).cuda())
    s.step(U, 5)  # a developed flow
    ref = U.clone()
    dt = s.cfl_dt(U)
    p = _lib.make_params(wl.params)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, axis in enumerate((0, 1)):
        s.hllc_sweep(ref, axis, dt, True)
        rc = L.dim_hllc_sweep_noalloc(C.byref(p), wl.nx, wl.ny, wl.dx, wl.dy, C.c_void_p(U.data_ptr()), axis, dt, 1,
                                      stream)
        assert rc == _lib.DIM_OK, L.dim_strerror(rc)
        torch.cuda.synchronize()
        e = _rel_l1(U.cpu().numpy(), ref.cpu().numpy())
        assert np.all(e <= TOL), (call, e)
    s.close()


def test_noalloc_rejects_oversized_grid():
    from paper_2106_00282_gb300 import _lib, inputs as I

    L = _lib.load()
    wl = I.impact(512, 256)  # 131,072 cells > DIM_NOALLOC_MAX_CELLS
    p = _lib.make_params(wl.params)
    rc = L.dim_hllc_sweep_noalloc(C.byref(p), wl.nx, wl.ny, wl.dx, wl.dy, C.c_void_p(1 << 20), 0, 1e-7, 1, None)
    assert rc == _lib.DIM_ETOOLARGE
    assert b"fixed scratch" in L.dim_strerror(rc)
