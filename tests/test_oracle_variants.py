"""Pins of the method variants: the Overbee interface-sharpening limiter
(Sec. 3.6, 4.1), the external heat source I_k = alpha_k I_k (Eq. I), the
paper's own implicit midpoint temperature relaxation (Sec. 3.4.1, Eqs.
ht_eq2_TR_dis, ht_eq3_TR_dis) and the linear (T, alpha) update of the heat
stage (Eqs. ht_eq2_ht, ht_eq3_ht)."""
import numpy as np

from test_oracle_relax import _nonequilibrium_state


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


# ---------------------------------------------------------------------------
# temperature relaxation by the paper's implicit midpoint scheme
# ---------------------------------------------------------------------------
def _midpoint(I, params, iters):
    return params.replace(trelax=I.TRELAX_MIDPOINT, trelax_iters=iters)


def _phase_T(params, U):
    """T_k = (E_k - alpha_k pinf_k) / (m_k Cv_k) (Eq. eos_stiffened)"""
    a2 = U[7]
    T1 = (U[4] - (1 - a2) * params.pinf[0]) / (U[0] * params.cv[0])
    T2 = (U[5] - a2 * params.pinf[1]) / (U[1] * params.cv[1])
    return T1, T2


def test_trelax_midpoint_equal_pinf_is_Taverage(O, I):
    """With pinf_1 = pinf_2 (B1 = 0) Eq. ht_eq3_TR_dis gives the mass-heat-capacity
    average of Eq. Taverage whatever B2 is, so after any number of iterations
    both phases sit at T' = (C1 T1 + C2 T2) / (C1 + C2)."""
    params = I.Params(gamma=(4.4, 1.4), pinf=(3e8, 3e8), cv=(1606.0, 714.0))
    U = _nonequilibrium_state(I, params, 200, 11, dT=0.3)
    T1, T2 = _phase_T(params, U)
    C1, C2 = U[0] * params.cv[0], U[1] * params.cv[1]
    Tav = (C1 * T1 + C2 * T2) / (C1 + C2)
    for iters in (1, 3, 20):
        U1, st = O.trelax(_midpoint(I, params, iters), U)
        assert st == 0
        T1n, T2n = _phase_T(params, U1)
        assert np.max(np.abs(T1n - Tav) / Tav) < 1e-9
        assert np.max(np.abs(T2n - Tav) / Tav) < 1e-9


def test_trelax_midpoint_conserves_energy(O, I):
    """Each iterate solves both discrete equations for its own B2, so
    C1 (T' - T1) + C2 (T' - T2) - B1 (alpha' - alpha) = 0: the internal energy
    E1 + E2 is conserved to roundoff after any iteration count; masses,
    momentum and the total energy are not touched."""
    for params in (I.impact(8, 8).params, I.shock_tube().params):
        U = _nonequilibrium_state(I, params, 300, 12, dT=0.2)
        for iters in (1, 2, 20):
            U1, st = O.trelax(_midpoint(I, params, iters), U)
            assert np.array_equal(U1[[0, 1, 2, 3, 6]], U[[0, 1, 2, 3, 6]])
            # the energy formula C T + pinf_1 - B1 alpha carries pinf_1: roundoff is relative to it
            scale = np.abs(U[4]) + np.abs(U[5]) + params.pinf[0]
            assert np.max(np.abs((U1[4] + U1[5]) - (U[4] + U[5])) / scale) < 1e-14
            T1n, T2n = _phase_T(params, U1)
            assert np.max(np.abs(T1n - T2n) / T2n) < 1e-8


def test_trelax_midpoint_third_order_to_equilibrium(O, I):
    """The midpoint scheme integrates the relaxation path (along which p1 = p2
    and the energy are kept and which ends at T1 = T2, i.e. at the exact
    equilibrium) with B2 at the averages: a one-step midpoint rule, so its
    volume fraction approaches the exact-equilibrium one like the cube of the
    initial temperature gap (ratio 8 per halving).  A wrong term or sign in
    B2 leaves an error of first order in the gap or worse."""
    params = I.impact(8, 8).params
    g, pi, cv = params.gamma, params.pinf, params.cv
    for a2 in (0.3, 1e-3):
        diffs = []
        for dT in (40.0, 20.0, 10.0, 5.0):
            p, T1, T2 = 2e8, 600.0, 600.0 + dT
            r1 = (p + pi[0]) / ((g[0] - 1) * cv[0] * T1)
            r2 = (p + pi[1]) / ((g[1] - 1) * cv[1] * T2)
            U = np.zeros((8, 1, 1))
            U[0], U[1] = (1 - a2) * r1, a2 * r2
            U[4] = (1 - a2) * (p + g[0] * pi[0]) / (g[0] - 1)
            U[5] = a2 * (p + g[1] * pi[1]) / (g[1] - 1)
            U[6] = U[4] + U[5]
            U[7] = a2
            Ue, st = O.trelax(params, U)
            Um, stm = O.trelax(_midpoint(I, params, 20), U)
            assert st == 0 and stm == 0
            Tm, Te = _phase_T(params, Um)[0][0, 0], _phase_T(params, Ue)[0][0, 0]
            assert abs(Tm - Te) < 1e-3 * dT
            diffs.append(abs(Um[7, 0, 0] - Ue[7, 0, 0]) / a2)
        diffs = np.array(diffs)
        assert np.all(diffs[:-1] / diffs[1:] > 6.0), diffs
        assert diffs[0] < 1e-4


def test_trelax_midpoint_iteration_converges(O, I):
    """The simple iteration settles: 20 iterations agree with 200 to a small
    fraction of the first iterate's distance, down to alpha ~ 1e-6."""
    params = I.impact(8, 8).params
    U = _nonequilibrium_state(I, params, 300, 13, dT=0.05)
    U1 = O.trelax(_midpoint(I, params, 1), U)[0]
    U20 = O.trelax(_midpoint(I, params, 20), U)[0]
    U200 = O.trelax(_midpoint(I, params, 200), U)[0]
    far = np.abs(U1[7] - U200[7])
    assert np.all(np.abs(U20[7] - U200[7]) <= 1e-3 * far + 1e-15 * U200[7])


# ---------------------------------------------------------------------------
# the heat stage's linear (T, alpha) update
# ---------------------------------------------------------------------------
def _source_states(I):
    params = I.shock_tube().params.replace(k0=(0.0, 0.0), src=(3e9, 7e8))
    pr = I.random_states(300, 5, params, p_range=(1e5, 1e8), T_range=(250.0, 900.0))
    return params, pr


def test_heat_linear_update_conserves_energy(O, I):
    """T += tau V q, alpha += tau U q with q = I1 + I2 (no gradient): the internal
    energy C T + pinf_1 - B1 alpha gains tau q (C V - B1 U) = tau q, since
    V = 1/(C + B1^2/K) and U = -B1 V/K; without the alpha term it would gain
    only tau q C V."""
    params, pr = _source_states(I)
    U = O.from_primitive(params, pr)
    lin = params.replace(heat_alpha=I.HEAT_ALPHA_LINEAR)
    for tau in (1e-3, 1e-5):
        U1, st, P = O.heat(lin, U, 1.0, 1.0, tau)
        assert st == 0
        a2 = U[7]
        expect = tau * ((1 - a2) * 3e9 + a2 * 7e8)
        de = (U1[4] + U1[5]) - (U[4] + U[5])
        assert np.max(np.abs(de - expect) / np.abs(U[4] + U[5])) < 1e-12
        assert np.max(np.abs((U1[6] - U[6]) - expect) / expect) < 1e-9
        assert np.array_equal(U1[[0, 1, 2, 3]], U[[0, 1, 2, 3]])


def test_heat_linear_update_is_first_order_projection(O, I):
    """V and U are the derivatives of the equilibrium projection along the
    manifold (Eqs. ht_eq2_ht, ht_eq3_ht), so the linear update and the
    projection differ at second order in the energy deposited: their gap,
    relative to the change of alpha, halves with tau."""
    params, pr = _source_states(I)
    U = O.from_primitive(params, pr)
    lin = params.replace(heat_alpha=I.HEAT_ALPHA_LINEAR)
    def gap(tau):
        Up = O.heat(params, U, 1.0, 1.0, tau)[0]
        Ul = O.heat(lin, U, 1.0, 1.0, tau)[0]
        return np.abs(Ul[7] - Up[7]) / np.abs(Up[7] - U[7])

    r0, r1 = np.median(gap(1e-4)), np.median(gap(5e-5))
    assert r0 < 1e-4
    assert 1.8 < r0 / r1 < 2.2
    # every cell, down to alpha ~ 1e-6, once the deposit is small
    assert np.max(gap(1e-7)) < 0.02


def test_heat_linear_equals_projection_without_B1(O, I):
    """Ideal gases (B1 = 0): U = 0 and V = 1/C, so alpha stays and
    T = T^n + tau q / C, which is also the equilibrium of the updated energy:
    both updates agree to roundoff on a conducting periodic field, also over
    several outer iterations of Algorithm 1 with a temperature-dependent
    conductivity (each iteration restarts from T^n with refreshed
    coefficients)."""
    n = 48
    x = (np.arange(n) + 0.5) / n
    prim = np.zeros((5, n, n))
    prim[0] = 0.4
    prim[1] = 1e5
    prim[2] = 300.0 + 80.0 * np.sin(2 * np.pi * x)[None, :] * np.cos(2 * np.pi * x)[:, None]
    for n_outer in (1, 3):
        params = I.Params(gamma=(1.4, 1.67), pinf=(0.0, 0.0), cv=(714.0, 3116.0), k0=(0.3, 0.1), k_exp=2.5,
                          bc=(1, 1), p_policy=I.P_CLAMP, p_min=3, p_max=12, n_outer=n_outer)
        U = O.from_primitive(params, prim)
        Up, st, P = O.heat(params, U, 1.0 / n, 1.0 / n, 2.0)
        Ul, st2, P2 = O.heat(params.replace(heat_alpha=I.HEAT_ALPHA_LINEAR), U, 1.0 / n, 1.0 / n, 2.0)
        assert st == 0 and st2 == 0 and P == P2 and P > 1
        assert np.max(np.abs(Ul[7] - Up[7])) < 1e-15
        den = np.maximum(np.abs(Up).reshape(8, -1).sum(1), 1e-300)
        assert np.max(np.abs(Ul - Up).reshape(8, -1).sum(1) / den) < 1e-14
        assert np.array_equal(Ul[7], U[7])
