"""Pins of the method variants: the Overbee interface-sharpening limiter
(Sec. 3.6, 4.1) and the external heat source I_k = alpha_k I_k (Eq. I)."""
import numpy as np


def _interface_cells(U):
    a = U[7]
    return int(np.sum((a > 0.01) & (a < 0.99)))


def test_overbee_consistent_keeps_pvt_and_sharpens(O, I):
    """Sec. 3.6: a homogeneous limiter applied to both alpha and alpha_k rho_k
    keeps rho_k* = rho_k, so u, p, T stay uniform; the Overbee limiter smears the
    translated interface over fewer cells than minmod."""
    res = {}
    for lim in (I.LIMITER_MINMOD, I.LIMITER_OVERBEE):
        wl = I.pvt_translation(n=200, k=(0.6, 0.026), limiter=lim)
        U = O.from_primitive(wl.params, wl.prim)
        U1, st, dt, _ = O.step(wl.params, U, wl.dx, wl.dy, 100)
        d = O.diagnostics(wl.params, U1)
        assert np.max(np.abs(d[4] - 1000.0)) / 1000.0 < 1e-10
        assert np.max(np.abs(d[3] - 300.0)) / 300.0 < 1e-9
        res[lim] = _interface_cells(U1)
    assert res[I.LIMITER_OVERBEE] < res[I.LIMITER_MINMOD]


def test_overbee_on_alpha_only_breaks_pvt(O, I):
    """Sec. 4.1 (reconstruction test): Overbee for the volume fraction with
    minmod for the phase densities fails to keep the phase densities and
    produces temperature spikes at the interface."""
    wl = I.pvt_translation(n=200, k=(0.0, 0.0), limiter=I.LIMITER_OVERBEE_ALPHA_ONLY)
    U = O.from_primitive(wl.params, wl.prim)
    U1, st, dt, _ = O.step(wl.params.replace(trelax=0), U, wl.dx, wl.dy, 50)
    d = O.diagnostics(wl.params, U1)
    # phase temperatures away from the uniform 300 K in the interface cells
    a = U1[7, 0]
    mixed = (a > 0.05) & (a < 0.95)
    assert mixed.any()
    spike = max(np.max(np.abs(d[2, 0][mixed] - 300.0)), np.max(np.abs(d[3, 0][mixed] - 300.0)))
    assert spike > 1.0


def test_heat_source_deposits_energy(O, I):
    """Without conduction (lambda = 0) a uniform state gains exactly
    tau (alpha_1 I_1 + alpha_2 I_2) of energy per unit volume in one heat stage,
    masses and momentum untouched, and stays in p,T equilibrium."""
    params = I.shock_tube().params.replace(k0=(0.0, 0.0), src=(3e9, 7e8))
    pr = I.random_states(300, 5, params, p_range=(1e5, 1e8), T_range=(250.0, 900.0))
    U = O.from_primitive(params, pr)
    tau = 1e-6
    U1, st, P = O.heat(params, U, 1.0, 1.0, tau)
    a2 = U[7]
    expect = tau * ((1 - a2) * 3e9 + a2 * 7e8)
    dE = U1[6] - U[6]
    assert np.max(np.abs(dE - expect) / expect) < 1e-6
    assert np.max(np.abs((U1[4] + U1[5]) - (U[4] + U[5]) - expect) / expect) < 1e-5
    assert np.array_equal(U1[[0, 1, 2, 3]], U[[0, 1, 2, 3]])
    d = O.diagnostics(params, U1)
    assert np.max(np.abs(d[2] - d[3]) / d[3]) < 1e-8


def test_heat_source_ideal_gas_temperature(O, I):
    """Ideal gases (V = 1/C): a uniform source raises T by tau I / (rho Cv)
    exactly, with conduction on (no gradient, no flux)."""
    params = I.Params(gamma=(1.4, 1.4), pinf=(0.0, 0.0), cv=(714.0, 714.0), k0=(0.1, 0.1), src=(2e6, 2e6))
    prim = np.zeros((5, 1, 16))
    prim[0] = 0.5
    prim[1] = 1e5
    prim[2] = 300.0
    U = O.from_primitive(params, prim)
    tau = 1e-4
    U1, st, P = O.heat(params, U, 0.01, 0.01, tau)
    rho = U[0] + U[1]
    T1 = O.heat_coeffs(params, U1)[0]
    assert np.max(np.abs(T1 - (300.0 + tau * 2e6 / (rho * 714.0)))) < 1e-9
