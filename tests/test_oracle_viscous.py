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
