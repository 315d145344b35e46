"""The measurement and self-check entry points of include/dim_probe.h on the
GPU: the pipe-rate probes return plausible rates, and the FP32-bulk form's
conversion of the FP64 state to float-float pairs and back keeps the leading
46 bits of every value a state holds."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_pipe_rate_probes_run():
    """dim_probe_rate measures each kind on the GPU and returns a plausible rate."""
    import torch

    from paper_2106_00282_gb300 import _lib, build

    build.build()
    L = _lib.load()
    rates = {}
    for kind in range(5):
        ms, ops = C.c_double(), C.c_double()
        rc = L.dim_probe_rate(kind, 0, 2000, C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(ms),
                              C.byref(ops))
        assert rc == _lib.DIM_OK
        assert ms.value > 0 and ops.value > 0
        rates[kind] = ops.value / (ms.value * 1e-3)
    # FP32 FMA far above FP64 FMA; an FP64 division costs several FP64 issue slots
    assert rates[_lib.PROBE_FFMA] > 10 * rates[_lib.PROBE_DFMA]
    assert rates[_lib.PROBE_DDIV] < rates[_lib.PROBE_DFMA] / 2


def test_float_float_state_conversion_round_trip():
    """The FP32-bulk form carries the state as float pairs converted from and to
    FP64 with integer operations (dim_probe_ff_roundtrip): on values over the
    ranges a state holds (2^-80 .. 1e25, both signs) the round trip keeps the
    leading 46 bits; below 2^-80 the low float is dropped (23 bits kept); zeros
    stay signed zeros."""
    import torch

    from paper_2106_00282_gb300 import _lib, build

    build.build()
    L = _lib.load()
    rng = np.random.default_rng(5)
    x = np.exp(rng.uniform(np.log(1e-25), np.log(1e25), 1 << 20)) * rng.choice([-1.0, 1.0], 1 << 20)
    x = np.concatenate([x, [0.0, -0.0, 1.0, -1.0, 1e-6, 1 - 1e-6, 1 - 1e-12, 6e8, 3.42e10, 2.0 ** -80, 2.0 ** 100]])
    X = torch.from_numpy(x).cuda()
    Y = torch.empty_like(X)
    rc = L.dim_probe_ff_roundtrip(C.c_void_p(X.data_ptr()), C.c_void_p(Y.data_ptr()), x.size,
                                  C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == _lib.DIM_OK
    torch.cuda.synchronize()
    y = Y.cpu().numpy()
    nz = x != 0
    rel = np.abs(y[nz] - x[nz]) / np.abs(x[nz])
    big = np.abs(x[nz]) >= 2.0 ** -80
    assert rel[big].max() <= 2.0 ** -46, rel[big].max()
    assert rel[~big].max() <= 2.0 ** -23, rel[~big].max()
    assert np.all(np.signbit(y) == np.signbit(x))
    assert np.all(y[~nz] == 0)
    # the complement of a fraction near 1 keeps 46 bits of absolute precision:
    # 1 - (1 - 1e-6) to ~1e-8 of itself, 1 - (1 - 1e-12) to ~1e-2 of itself
    for d in (1e-6, 1e-12):
        i = int(np.argmin(np.abs(x - (1 - d))))
        assert abs((1.0 - y[i]) - (1.0 - x[i])) <= 2.0 ** -46
