"""FP32-bulk form of the CUDA path (no FP64 arithmetic inside a step: the state
as float-float pairs holding the accumulation, the phase pressures' cancellation
against the cold energy, the volume fraction and a Newton correction of each
relaxation root; flux, relaxation and stencil arithmetic in FP32) against the
FP64 oracle.

Tolerance: relative L1 per conserved field <= 2e-5 after 100 steps.  The
momentum of a flow at rest up to thermal expansion (the conduction disc) is
roundoff noise -- a one-ulp change of the FP64 input already moves it by 1e-4
relative -- so a momentum plane is measured against the acoustic momentum
scale sum(rho) * (the largest wave speed) whenever its own L1 norm is below
1e-3 of that scale."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL32 = 2e-5


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2106_00282_gb300 import build

    build.build()
    return torch


def rel_l1_32(a, b, O, wl, params):
    num = np.abs(a - b).reshape(8, -1).sum(axis=1)
    den = np.abs(b).reshape(8, -1).sum(axis=1)
    rho = (b[0] + b[1]).sum()
    h = min(wl.dx if wl.nx > 1 else np.inf, wl.dy if wl.ny > 1 else np.inf)
    smax = params.cfl * h / O.dt(params, b, wl.dx, wl.dy)
    acoustic = rho * smax
    for q in (2, 3):
        den[q] = max(den[q], 1e-3 * acoustic)
    return num / np.maximum(den, 1e-300)


def _run(torch, O, wl, nsteps):
    from paper_2106_00282_gb300.api import Solver

    p32 = wl.params.replace(precision=1)
    s = Solver(p32, wl.nx, wl.ny, wl.dx, wl.dy)
    U = s.from_primitive(torch.from_numpy(np.ascontiguousarray(wl.prim)).cuda())
    s.step(U, nsteps, sync=False)
    st = s.status()
    Uo, sto, dto, ph = O.step(wl.params, O.from_primitive(wl.params, wl.prim), wl.dx, wl.dy, nsteps)
    return U.cpu().numpy(), Uo, st, sto


CASES = {
    "shock_tube_1000": lambda I: I.shock_tube(n=1000),
    "impact_160x80": lambda I: I.impact(160, 80),
    "conduction_96": lambda I: I.conduction_disc(n=96),
    "mixture_shock": lambda I: I.mixture_shock(n=400),
    "pvt_periodic": lambda I: I.pvt_translation(n=150, k=(0.6, 0.026)),
    "viscous_shock": lambda I: I.shock_tube(n=400, k=(1e6, 1e6), mu=(500.0, 1.0), p_policy=0),
    "ragged_131x37": lambda I: I.impact(131, 37),
    "shock_tube_column": lambda I: I.shock_tube(n=300, axis=1),
    "overbee_shock": lambda I: I.shock_tube(n=400, limiter=I.LIMITER_OVERBEE),
    "overbee_impact": lambda I: _with(I.impact(160, 80), limiter=I.LIMITER_OVERBEE),
    "heat_source": lambda I: _with(I.shock_tube(n=400), src=(1e12, 1e10)),
    "spitzer_like": lambda I: I.conduction_disc(n=96, k_exp=2.5),
    # the heat stage's blocked rounds with thread loads: periodic walls, and rows
    # not a multiple of 4 floats (the transmissive 2D cases above load by TMA)
    "conduction_periodic_96": lambda I: _with(I.conduction_disc(n=96), bc=(I.BC_PERIODIC, I.BC_PERIODIC)),
    "conduction_98": lambda I: I.conduction_disc(n=98),
    # TMA rounds on a grid lower than one region (most of each box beyond the
    # walls), with P fixed so that the blocked sweeps run
    "thin_tma_128x12": lambda I: _with(I.smooth_mixture(128, 12, bc=(I.BC_TRANSMISSIVE, I.BC_TRANSMISSIVE)),
                                       p_policy=I.P_FIXED, p_fixed=4),
}


def _with(wl, **kw):
    wl.params = wl.params.replace(**kw)
    return wl


# The Overbee limiter sits on the boundary of the TVD region and turns rounding
# noise into staircases: on the 2D impact the FP64 oracle itself moves by 1.3e-5
# under a 1e-7 relative change of its input, and FP32 rounding enters at every
# step, so this one case is held to 1e-3 (measured 5e-4); the Overbee shock tube
# meets the standard bound.
TOL_CASE = {"overbee_impact": 1e-3}


@pytest.mark.parametrize("case", list(CASES))
def test_fp32_bulk_100_steps(torch_cuda, O, I, case):
    from paper_2106_00282_gb300 import _lib

    wl = CASES[case](I)
    G, Uo, st, sto = _run(torch_cuda, O, wl, 100)
    e = rel_l1_32(G, Uo, O, wl, wl.params)
    print(f"[fp32] {case}: rel L1 per field {np.array2string(e, precision=2)}")
    assert np.all(e <= TOL_CASE.get(case, TOL32)), e
    assert not np.isnan(G).any()
    assert st & (_lib.ST_NONPHYS | _lib.ST_NAN | _lib.ST_TIMEOUT) == 0


def test_fp32_bulk_pvt(torch_cuda, O, I):
    """Sec. 4.1 translation in FP32 bulk: u and T stay uniform to 1e-5 (the
    consistent reconstruction of alpha and alpha rho; the cold energy of the
    stiff phase carried by the FP64 volume-fraction flux).  The pressure of the
    stiff phase is resolved only to the FP32 rounding of the total-energy flux:
    at 1000 m/s water carries rho u^2/2 = 5e8 J/m^3 against a thermal energy of
    3e4 J/m^3, so 6e-8 of the former moves p by ~1e-3 of itself."""
    wl = I.pvt_translation(n=200, k=(0.6, 0.026))
    G, Uo, st, sto = _run(torch_cuda, O, wl, 60)
    d = O.diagnostics(wl.params, G)
    assert np.max(np.abs(d[4] - 1000.0)) / 1000.0 < 1e-5
    assert np.max(np.abs(d[1] - 1e5)) / 1e5 < 1e-2
    assert np.max(np.abs(d[3] - 300.0)) / 300.0 < 1e-5


@pytest.mark.parametrize("which", ["impact", "conduction"])
def test_fp32_bulk_full_size(torch_cuda, O, I, oracle_full_size, which):
    """The benchmark sizes, in the benchmark's launch configuration: 100 steps of
    the 1024 x 512 impact, 20 steps of the 2048^2 conduction disc, against the
    FP64 oracle's run of the same steps."""
    from conftest import FULL_SIZE_STEPS

    from paper_2106_00282_gb300.api import Solver

    wl, Uo, sto = oracle_full_size(which)
    p32 = wl.params.replace(precision=1)
    s = Solver(p32, wl.nx, wl.ny, wl.dx, wl.dy)
    U = s.from_primitive(torch_cuda.from_numpy(np.ascontiguousarray(wl.prim)).cuda())
    s.step(U, FULL_SIZE_STEPS[which])
    st = s.status()
    G = U.cpu().numpy()
    s.close()
    assert st & 3 == 0 and sto & 3 == 0
    e = rel_l1_32(G, Uo, O, wl, wl.params)
    print(f"[fp32] full {which}, {FULL_SIZE_STEPS[which]} steps: rel L1 per field {np.array2string(e, precision=2)}")
    assert np.all(e <= TOL32), e


def test_fp32_bulk_stage_calls(torch_cuda, O, I):
    """The per-stage entry points in FP32-bulk precision (each converts the FP64
    state to float-float planes, runs the stage, converts back) against the
    FP64 oracle's stages on the same input: the hyperbolic sweep along x and y
    with and without the pressure relaxation, both relaxations on states out of
    equilibrium, the heat-conduction solve and the viscous solves along x and
    y.  One stage in FP32 bulk stays within 2e-6 relative L1 per field."""
    from test_oracle_relax import _nonequilibrium_state

    from paper_2106_00282_gb300 import _lib
    from paper_2106_00282_gb300.api import Solver

    tol = 2e-6

    def solver(wl):
        p32 = wl.params.replace(precision=1)
        return Solver(p32, wl.nx, wl.ny, wl.dx, wl.dy)

    def dev(a):
        return torch_cuda.from_numpy(np.ascontiguousarray(a)).cuda()

    # sweeps on a developed impact flow
    wl = I.impact(203, 77)
    Uo = O.step(wl.params, O.from_primitive(wl.params, wl.prim), wl.dx, wl.dy, 3)[0]
    s = solver(wl)
    dt = O.dt(wl.params, Uo, wl.dx, wl.dy)
    for axis in (0, 1):
        for relax in (False, True):
            U = dev(Uo)
            s.hllc_sweep(U, axis, dt, relax)
            ref, st = O.sweep(wl.params, Uo, wl.dx, wl.dy, axis, dt)
            if relax:
                ref, st = O.prelax(wl.params, ref)
            e = rel_l1_32(U.cpu().numpy(), ref, O, wl, wl.params)
            print(f"[fp32] sweep axis {axis} relax {relax}: {e.max():.2e}")
            assert np.all(e <= tol), (axis, relax, e)
    s.close()
    # relaxations
    for params in (I.impact(8, 8).params, I.shock_tube().params):
        U0 = _nonequilibrium_state(I, params, 5000, 21, dT=0.3, dp=0.3, dE=1e-3)
        wl = I.Workload("r", 5000, 1, 1.0, 1.0, params, None)
        s = solver(wl)
        for which, fn in ((_lib.RELAX_PRESSURE, O.prelax), (_lib.RELAX_TEMPERATURE, O.trelax)):
            U = dev(U0)
            s.relax(U, which)
            ref, st = fn(params, U0)
            G = U.cpu().numpy()
            e = np.abs(G - ref).reshape(8, -1).sum(1) / np.maximum(np.abs(ref).reshape(8, -1).sum(1), 1e-300)
            print(f"[fp32] relax {which}: {e.max():.2e}")
            assert np.all(e <= tol), (which, e)
        s.close()
    # heat conduction and viscous solves
    wl = I.conduction_disc(n=131, p_min=4, p_max=12)
    U0 = O.from_primitive(wl.params, wl.prim)
    s = solver(wl)
    U = dev(U0)
    P = s.cheb_parabolic(U, _lib.PARABOLIC_HEAT, 2e-5)
    ref, st, Po = O.heat(wl.params, U0, wl.dx, wl.dy, 2e-5)
    assert P == Po
    e = rel_l1_32(U.cpu().numpy(), ref, O, wl, wl.params)
    print(f"[fp32] heat P={P}: {e.max():.2e}")
    assert np.all(e <= tol), e
    s.close()
    wl = I.impact(150, 70)
    wl.params = wl.params.replace(mu=(50.0, 2.0))
    U0 = O.step(wl.params, O.from_primitive(wl.params, wl.prim), wl.dx, wl.dy, 4)[0]
    s = solver(wl)
    for axis in (0, 1):
        U = dev(U0)
        P = s.cheb_parabolic(U, _lib.PARABOLIC_VISCOUS_X if axis == 0 else _lib.PARABOLIC_VISCOUS_Y, 2e-7)
        ref, st, Po = O.viscous(wl.params, U0, wl.dx, wl.dy, axis, 2e-7)
        assert P == Po
        e = rel_l1_32(U.cpu().numpy(), ref, O, wl, wl.params)
        print(f"[fp32] viscous axis {axis} P={P}: {e.max():.2e}")
        assert np.all(e <= tol), (axis, e)
    s.close()
