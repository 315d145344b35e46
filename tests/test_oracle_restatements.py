"""Plain forms of the formulas the oracle evaluates in an algebraically
restated order, written here as the paper states them and compared with the
oracle on well-conditioned states (the shock tube, the PVT translation and the
mixture shock of Sec. 4, after a few full steps).  The restatements -- the
constant reciprocals 1/(gamma_k - 1), 1/dx, 1/h^2 and 1/T_ref formed once and
multiplied, the mixture sound speed through A_k = rho_k c_k^2 (Eq. AK), the
prefactor 1/(1 + tau b_m) of Eq. (LIM) formed once per sweep -- change only
the rounding, so the two forms agree to ~1e-14 relative.  (The dense-matrix
check of the LIM sweeps in test_oracle_heat.py uses the division form of
Eq. LIM and the 1/h^2 of Eq. qk_dis per face.)"""
import numpy as np
import pytest


def _families(I):
    return {
        "shock_tube": I.shock_tube(n=200),
        "pvt": I.pvt_translation(n=120, k=(0.6, 0.026)),
        "mixture": I.mixture_shock(n=200),
    }


@pytest.fixture(scope="module")
def states(O, I):
    out = {}
    for name, wl in _families(I).items():
        U = O.from_primitive(wl.params, wl.prim)
        U = O.step(wl.params, U, wl.dx, wl.dy, 5)[0]
        out[name] = (wl, U)
    return out


def _plain_phase(params, U):
    """rho_k = m_k / alpha_k, p_k = (gamma_k - 1) E_k / alpha_k - gamma_k pinf_k."""
    a = [1.0 - U[7], U[7]]
    rho = [U[0] / a[0], U[1] / a[1]]
    p = [(params.gamma[k] - 1.0) * U[4 + k] / a[k] - params.gamma[k] * params.pinf[k] for k in range(2)]
    return a, rho, p


@pytest.mark.parametrize("name", ["shock_tube", "pvt", "mixture"])
def test_cfl_time_step_plain_form(O, states, name):
    """Sec. 3.1: c^2 = Y1 c1^2 + Y2 c2^2 with c_k^2 = gamma_k (p_k + pinf_k)/rho_k
    and Y_k = alpha_k rho_k / rho; dt = cfl / max (|u| + c)/dx."""
    wl, U = states[name]
    pr = wl.params
    a, rho_k, p = _plain_phase(pr, U)
    rho = U[0] + U[1]
    c2 = sum((a[k] * rho_k[k] / rho) * (pr.gamma[k] * (p[k] + pr.pinf[k]) / rho_k[k]) for k in range(2))
    s = (np.abs(U[2] / rho) + np.sqrt(c2)) / wl.dx
    dt_plain = pr.cfl / s.max()
    assert abs(O.dt(pr, U, wl.dx, wl.dy) / dt_plain - 1.0) < 1e-14


@pytest.mark.parametrize("name", ["shock_tube", "pvt", "mixture"])
def test_phase_energy_plain_form(O, states, name):
    """Eq. eos_stiffened: E_k = alpha_k (p + gamma_k pinf_k)/(gamma_k - 1), the
    conversion of the initial primitive fields."""
    wl, _ = states[name]
    pr = wl.params
    U = O.from_primitive(pr, wl.prim)
    a = [1.0 - wl.prim[0], wl.prim[0]]
    for k in range(2):
        plain = a[k] * (wl.prim[1] + pr.gamma[k] * pr.pinf[k]) / (pr.gamma[k] - 1.0)
        assert np.max(np.abs(U[4 + k] - plain) / np.abs(plain)) < 1e-15


@pytest.mark.parametrize("name", ["shock_tube", "pvt", "mixture"])
def test_pressure_relaxation_energy_plain_form(O, states, name):
    """Sec. 3.3 steps (2)-(3): with the relaxed fractions alpha_k', the pressure
    p = (rho e - sum alpha_k' gamma_k pinf_k/(gamma_k - 1)) / sum alpha_k'/(gamma_k - 1)
    and E_k = alpha_k' (p + gamma_k pinf_k)/(gamma_k - 1), rho e = rho E - rho|u|^2/2."""
    wl, U = states[name]
    pr = wl.params
    # move the phase pressures apart first: a sweep without relaxation
    Us, _ = O.sweep(pr, U, wl.dx, wl.dy, 0, O.dt(pr, U, wl.dx, wl.dy))
    Ur, _ = O.prelax(pr, Us)
    a = [1.0 - Ur[7], Ur[7]]
    rho = Us[0] + Us[1]
    rhoe = Us[6] - 0.5 * (Us[2] ** 2 + Us[3] ** 2) / rho
    g, pi = pr.gamma, pr.pinf
    num = rhoe - sum(a[k] * g[k] * pi[k] / (g[k] - 1.0) for k in range(2))
    den = sum(a[k] / (g[k] - 1.0) for k in range(2))
    p = num / den
    for k in range(2):
        plain = a[k] * (p + g[k] * pi[k]) / (g[k] - 1.0)
        assert np.max(np.abs(Ur[4 + k] - plain)) <= 1e-13 * np.abs(Us[6]).max(), k


def test_conductivity_law_plain_form(O, I, states):
    """lambda = alpha_1 k0_1 (T/T_ref)^a + alpha_2 k0_2 (T/T_ref)^a with the
    division by T_ref as written (a = 2, the conduction-disc law, and a = 2.5)."""
    wl, U = states["mixture"]
    for kexp in (2.0, 2.5):
        pr = wl.params.replace(k0=(0.6, 0.026), k_exp=kexp, T_ref=300.0)
        co = O.heat_coeffs(pr, U)
        T = co[0]
        a2 = U[7]
        plain = (1.0 - a2) * 0.6 * (T / 300.0) ** kexp + a2 * 0.026 * (T / 300.0) ** kexp
        assert np.max(np.abs(co[3] - plain) / plain) < 1e-14
