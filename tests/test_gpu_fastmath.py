"""The FP64 division and square root of the FP32-bulk kernels (refined
hardware approximations with an IEEE fallback outside their domain) against
IEEE-754 division and square root (numpy on the host), through the C ABI
(dim_probe_fastmath): within one ulp on random normal operands over
1e-300..1e300, and exactly equal -- value, sign of zero, infinity, NaN -- on
zeros, subnormals, operands whose reciprocal is subnormal, infinities, NaN,
negative square-root arguments and quotients that overflow or underflow."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _run(a: np.ndarray, b: np.ndarray):
    import torch

    from paper_2106_00282_gb300 import _lib, build

    build.build()
    L = _lib.load()
    A = torch.from_numpy(a).cuda()
    B = torch.from_numpy(b).cuda()
    Q = torch.empty_like(A)
    R = torch.empty_like(A)
    rc = L.dim_probe_fastmath(C.c_void_p(A.data_ptr()), C.c_void_p(B.data_ptr()), C.c_void_p(Q.data_ptr()),
                              C.c_void_p(R.data_ptr()), a.size, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == _lib.DIM_OK
    torch.cuda.synchronize()
    return Q.cpu().numpy(), R.cpu().numpy()


def _ulp_distance(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Distance in units in the last place between finite doubles of one sign."""
    xi = x.view(np.int64).astype(np.float64)
    yi = y.view(np.int64).astype(np.float64)
    return np.abs(xi - yi)


def _same(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Bitwise equal, or both NaN."""
    return (x.view(np.int64) == y.view(np.int64)) | (np.isnan(x) & np.isnan(y))


def test_fast_div_sqrt_random_normal_operands():
    rng = np.random.default_rng(11)
    n = 1 << 22
    a = np.exp(rng.uniform(np.log(1e-300), np.log(1e300), n)) * rng.choice([-1.0, 1.0], n)
    b = np.exp(rng.uniform(np.log(1e-300), np.log(1e300), n)) * rng.choice([-1.0, 1.0], n)
    with np.errstate(all="ignore"):
        q_ref = a / b
        r_ref = np.sqrt(np.abs(a))
    q, _ = _run(a, b)
    _, r = _run(np.abs(a), b)
    # quotients in the normal range: within one ulp; the rest (over/underflow) exact
    normal = np.isfinite(q_ref) & (np.abs(q_ref) >= np.finfo(np.float64).tiny)
    d = _ulp_distance(q[normal], q_ref[normal])
    assert d.max() <= 1, d.max()
    assert np.mean(d == 0) > 0.999
    assert np.all(_same(q[~normal], q_ref[~normal]))
    dr = _ulp_distance(r, r_ref)
    assert dr.max() <= 1, dr.max()
    assert np.mean(dr == 0) > 0.999


def test_fast_div_sqrt_edge_operands():
    tiny = np.finfo(np.float64).tiny
    sub = [5e-324, 1e-310, 2.2e-308, tiny, tiny * (1 - 2 ** -52) * 1.0]
    big = [2.0 ** 1022, 1.5 * 2.0 ** 1022, np.finfo(np.float64).max, 2.0 ** 1021]
    special = [0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -1.0, 3.0, 1e300, 1e-300]
    vals = np.array(sub + [-x for x in sub] + big + [-x for x in big] + special, dtype=np.float64)
    a = np.repeat(vals, vals.size)
    b = np.tile(vals, vals.size)
    with np.errstate(all="ignore"):
        q_ref = a / b
        r_ref = np.sqrt(a)
    q, r = _run(a, b)
    ok = _same(q, q_ref)
    # a normal quotient computed on the fast path may differ by one ulp
    fast = np.isfinite(q_ref) & (np.abs(q_ref) >= tiny) & ~ok
    assert np.all(_ulp_distance(q[fast], q_ref[fast]) <= 1)
    assert np.all(ok | fast), list(zip(a[~(ok | fast)][:8], b[~(ok | fast)][:8], q[~(ok | fast)][:8]))
    assert np.all(_same(r, r_ref) | (np.isfinite(r_ref) & (_ulp_distance(r, r_ref) <= 1))), \
        list(zip(a[~_same(r, r_ref)][:8], r[~_same(r, r_ref)][:8]))
    # the zeros, infinities and NaN of IEEE division and square root, bit for bit
    edge = (a == 0) | (b == 0) | ~np.isfinite(a) | ~np.isfinite(b) | (np.abs(b) < tiny) | (np.abs(a) < tiny)
    assert np.all(_same(q[edge & ~np.isfinite(q_ref)], q_ref[edge & ~np.isfinite(q_ref)]))
    zero = q_ref == 0
    assert np.all(np.signbit(q[zero]) == np.signbit(q_ref[zero]))
    assert np.all(_same(r[(a <= 0) | ~np.isfinite(a)], r_ref[(a <= 0) | ~np.isfinite(a)]))


def test_pipe_rate_probes_run():
    """dim_probe_rate measures each kind on the GPU and returns a plausible rate."""
    import torch

    from paper_2106_00282_gb300 import _lib, build

    build.build()
    L = _lib.load()
    rates = {}
    for kind in range(6):
        ms, ops = C.c_double(), C.c_double()
        rc = L.dim_probe_rate(kind, 0, 2000, C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(ms),
                              C.byref(ops))
        assert rc == _lib.DIM_OK
        assert ms.value > 0 and ops.value > 0
        rates[kind] = ops.value / (ms.value * 1e-3)
    # FP32 FMA far above FP64 FMA; an FP64 division costs several FP64 issue slots
    assert rates[_lib.PROBE_FFMA] > 10 * rates[_lib.PROBE_DFMA]
    assert rates[_lib.PROBE_DDIV] < rates[_lib.PROBE_DFMA] / 2
