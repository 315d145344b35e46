"""Pins of the oracle's viscous stage (Sec. 3.2) against the decay of viscous
waves and conservation."""
import math

import numpy as np


def _state(O, I, n, un_amp, ut_amp, mu=(0.5, 0.5)):
    params = I.Params(gamma=(1.4, 1.4), pinf=(0.0, 0.0), cv=(714.0, 714.0), mu=mu, bc=(1, 1),
                      p_policy=I.P_FORMULA, p_max=24)
    x = (np.arange(n) + 0.5) / n
    prim = np.zeros((5, 1, n))
    prim[0] = 0.5
    prim[1] = 1e5
    prim[2] = 300.0
    prim[3, 0] = un_amp * np.sin(2 * np.pi * x)
    prim[4, 0] = ut_amp * np.sin(2 * np.pi * x)
    return params, O.from_primitive(params, prim), x


def test_viscous_wave_decay(O, I):
    """rho du/dt = d/dx(4/3 mu du/dx), rho dv/dt = d/dx(mu dv/dx): a sine mode of
    wavenumber k decays as exp(-4/3 mu k^2 t / rho) (normal) and exp(-mu k^2 t /
    rho) (tangential); the LIM reproduces both rates."""
    n = 200
    params, U, x = _state(O, I, n, 1.0, 1.0)
    rho = U[0, 0, 0] + U[1, 0, 0]
    k = 2 * np.pi
    nu = 0.5 / rho
    tau = 0.02 / (nu * k * k)
    nst = 10
    for _ in range(nst):
        U, st, Pn = O.viscous(params, U, 1.0 / n, 1.0 / n, 0, tau)
    t = nst * tau
    u = U[2, 0] / (U[0, 0] + U[1, 0])
    v = U[3, 0] / (U[0, 0] + U[1, 0])
    gu = np.dot(u, np.sin(k * x)) / np.dot(np.sin(k * x), np.sin(k * x))
    gv = np.dot(v, np.sin(k * x)) / np.dot(np.sin(k * x), np.sin(k * x))
    # discrete symbol: k^2 -> (2 sin(k h / 2) / h)^2
    h = 1.0 / n
    kk = (2 * math.sin(k * h / 2) / h) ** 2
    assert abs(gu - math.exp(-4.0 / 3.0 * nu * kk * t)) < 2e-3
    assert abs(gv - math.exp(-nu * kk * t)) < 2e-3
    assert abs(math.log(gu) / math.log(gv) - 4.0 / 3.0) < 2e-2


def test_viscous_conservation_and_dissipation(O, I):
    """Momentum and total energy are conserved (flux form of the last sweep and
    of the energy update, Sec. 3.2); kinetic energy is dissipated and the
    internal energy sum_k E_k rises by the same amount to first order."""
    n = 128
    params, U, x = _state(O, I, n, 30.0, 20.0, mu=(2.0, 0.5))
    U1, st, Pn = O.viscous(params, U, 1.0 / n, 1.0 / n, 0, 2e-6)
    for q in (0, 1, 2, 3, 6):
        assert abs(U1[q].sum() - U[q].sum()) <= 1e-13 * np.abs(U[q]).sum() + 1e-12, q
    ke = lambda W: 0.5 * (W[2] ** 2 + W[3] ** 2) / (W[0] + W[1])
    dke = (ke(U1) - ke(U)).sum()
    de = ((U1[4] + U1[5]) - (U[4] + U[5])).sum()
    assert dke < 0
    assert abs(de + dke) < 0.05 * abs(dke)


def _sg_params(I, mu=(2.0, 0.5), p_max=24):
    """Water and air, stiffened gas (Sec. 4.2 constants), periodic walls."""
    return I.Params(gamma=(4.4, 1.4), pinf=(6e8, 0.0), cv=(1606.0, 714.0), mu=mu, bc=(1, 1),
                    p_policy=I.P_FORMULA, p_max=p_max)


def test_viscous_phase_split_uniform_alpha(O, I):
    """Sec. 3.2 internal-energy update: with alpha_k the same in every cell the
    face weights alpha_{k,i+1/2} equal alpha_k, so both phase increments are
    alpha_k times one common bracket, (E_k' - E_k) / alpha_k equal for k = 1, 2
    (here alpha_1 : alpha_2 = 0.7 : 0.3, two different stiffened gases, normal
    and tangential shear waves, several Chebyshev sweeps)."""
    n = 64
    params = _sg_params(I)
    x = (np.arange(n) + 0.5) / n
    prim = np.zeros((5, 1, n))
    prim[0] = 0.3
    prim[1] = 1e5
    prim[2] = 300.0
    prim[3, 0] = 30.0 * np.sin(2 * np.pi * x)
    prim[4, 0] = 20.0 * np.cos(4 * np.pi * x)
    U = O.from_primitive(params, prim)
    U1, st, Pn = O.viscous(params, U, 1.0 / n, 1.0 / n, 0, 0.05)
    assert Pn == 3
    d1 = (U1[4] - U[4]) / 0.7
    d2 = (U1[5] - U[5]) / 0.3
    scale = np.abs(d1).max()
    assert scale > 0
    # the increments (~1e3 J/m^3) are differences of stored energies ~5e8, so
    # they carry an absolute rounding of a few 1e-8: the bound is 1e-9 of the
    # increment, while a swapped weight would change d1/d2 by (0.3/0.7)^2
    assert np.max(np.abs(d1 - d2)) < 1e-9 * scale
    # and the common bracket carries the whole internal-energy change
    assert np.max(np.abs((U1[4] - U[4]) + (U1[5] - U[5]) - d1)) < 1e-9 * scale


def test_viscous_update_by_hand_with_alpha_gradient(O, I):
    """One Chebyshev parameter (P = 1: no predictor sweep, u_hat = u^n, the
    single sweep is the conservative one) on a 4-cell periodic line with a
    different volume fraction in every cell: every field of the Sec. 3.2
    update written out here in the paper's order -- face viscosity the mean of
    the cell mixture viscosities, F_vis = 4/3 mu_f du/dx (normal) and mu_f dv/dx
    (tangential), the face velocity and the face alpha_k the two-cell means,
    (rho u) += tau dF/dx, (rho E) += tau d(u_f F)/dx, and
    E_k += tau d(alpha_k,f u_f F)/dx - tau u_i d(alpha_k,f F)/dx."""
    params = _sg_params(I, p_max=1)
    a2 = np.array([0.1, 0.4, 0.8, 0.3])
    u = np.array([10.0, -5.0, 20.0, 3.0])
    w = np.array([2.0, 7.0, -4.0, 1.0])
    prim = np.zeros((5, 1, 4))
    prim[0, 0] = a2
    prim[1, 0] = [1e5, 2e5, 1.5e5, 3e5]
    prim[2, 0] = [300.0, 320.0, 290.0, 310.0]
    prim[3, 0] = u
    prim[4, 0] = w
    U = O.from_primitive(params, prim)
    dx, tau = 0.01, 3e-7
    U1, st, Pn = O.viscous(params, U, dx, dx, 0, tau)
    assert Pn == 1
    rho = U[0, 0] + U[1, 0]
    un, ut = U[2, 0] / rho, U[3, 0] / rho
    a1 = 1.0 - a2
    mu = a1 * params.mu[0] + a2 * params.mu[1]
    nxt = np.roll(np.arange(4), -1)  # face i+1/2 joins cells i and i+1 (periodic)
    mu_f = 0.5 * (mu + mu[nxt])
    Fn = 4.0 / 3.0 * mu_f * (un[nxt] - un) / dx
    Ft = mu_f * (ut[nxt] - ut) / dx
    Wf = 0.5 * (un + un[nxt]) * Fn + 0.5 * (ut + ut[nxt]) * Ft
    a_f = [0.5 * (a1 + a1[nxt]), 0.5 * (a2 + a2[nxt])]
    prv = np.roll(np.arange(4), 1)  # face i-1/2 has the index of cell i-1

    def d(face):  # difference across the cell: face i+1/2 minus face i-1/2
        return face - face[prv]

    expect = U[:, 0].copy()
    expect[2] += tau * d(Fn) / dx
    expect[3] += tau * d(Ft) / dx
    expect[6] += tau * d(Wf) / dx
    for k in range(2):
        expect[4 + k] += tau * d(a_f[k] * Wf) / dx - tau * (un * d(a_f[k] * Fn) + ut * d(a_f[k] * Ft)) / dx
    for q in range(8):
        ref = np.abs(expect[q] - U[q, 0]).max() + 1e-300
        assert np.max(np.abs(U1[q, 0] - expect[q])) <= 1e-12 * max(ref, 1e-12 * np.abs(U[q, 0]).max()), q
    # the phase increments differ from alpha-weighted shares of their sum
    # (the face weights are not the cell fractions)
    dE = U1[4, 0] - U[4, 0] + U1[5, 0] - U[5, 0]
    assert np.max(np.abs((U1[5, 0] - U[5, 0]) - a2 * dE)) > 1e-3 * np.abs(dE).max()


def _visc_P(O, params, U, dx, dy, axis, tau):
    return O.viscous(params, U, dx, dy, axis, tau)[2]


def test_viscous_P1_certificate_bound(O, I):
    """The FP32-bulk step skips the exact viscous lambda_max pass when a bound
    proves P = 1.  The mixture viscosity a_1 mu_1 + a_2 mu_2 is at most max mu_k,
    so every face coefficient is at most 4/3 of it, and the Gershgorin bound of
    the viscous operator (Sec. 3.2) gives lambda_max <= 16/3 max(mu_k) / rho_min
    max(1/h^2).  With P = ceil(pi/4 sqrt(tau lambda + 1)), P = 1 exactly when
    tau lambda <= (4/pi)^2 - 1.  The oracle's own choice of P pins the bound: at
    the time step where twice the bound meets that limit, the oracle chooses
    P = 1 on heterogeneous states along either axis.  A uniform state, where the
    bound is attained, shows it is tight: P = 2 once tau lambda_bound passes
    the limit."""
    lim = (4.0 / math.pi) ** 2 - 1.0
    rng = np.random.default_rng(7)
    nx, ny = 24, 16
    dx, dy = 1.0 / nx, 0.5 / ny
    ih2 = max(1.0 / dx ** 2, 1.0 / dy ** 2)
    for mu in ((1e-3, 1.8e-5), (500.0, 1.0), (0.2, 3.0)):
        params = I.Params(gamma=(4.4, 1.4), pinf=(6e8, 0.0), cv=(950.0, 718.0), mu=mu, bc=(0, 1),
                          p_policy=I.P_FORMULA, p_max=24)
        prim = np.zeros((5, ny, nx))
        prim[0] = rng.uniform(1e-6, 1.0 - 1e-6, size=(ny, nx))
        prim[1] = rng.uniform(5e4, 5e5, size=(ny, nx))
        prim[2] = rng.uniform(250.0, 3000.0, size=(ny, nx))
        prim[3] = rng.uniform(-50.0, 50.0, size=(ny, nx))
        prim[4] = rng.uniform(-50.0, 50.0, size=(ny, nx))
        U = O.from_primitive(params, prim)
        rho = U[0] + U[1]
        lam_b = 16.0 / 3.0 * max(mu) / rho.min() * ih2
        tau = lim / (2.0 * lam_b)
        for axis in (0, 1):
            assert _visc_P(O, params, U, dx, dy, axis, tau) == 1, (mu, axis)
    # uniform state, periodic x: every face coefficient is 4/3 mu, lambda_max equals the bound
    params = I.Params(gamma=(1.4, 1.4), pinf=(0.0, 0.0), cv=(714.0, 714.0), mu=(0.5, 0.5), bc=(1, 1),
                      p_policy=I.P_FORMULA, p_max=24)
    prim = np.zeros((5, 1, 64))
    prim[0] = 0.5
    prim[1] = 1e5
    prim[2] = 300.0
    U = O.from_primitive(params, prim)
    rho = U[0, 0, 0] + U[1, 0, 0]
    h = 1.0 / 64
    lam_b = 16.0 / 3.0 * 0.5 / rho / h ** 2
    assert _visc_P(O, params, U, h, h, 0, 0.99 * lim / lam_b) == 1
    assert _visc_P(O, params, U, h, h, 0, 1.01 * lim / lam_b) == 2
