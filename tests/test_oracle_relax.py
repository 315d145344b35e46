"""Pins of the oracle's pressure and temperature relaxations (Sec. 3.3, 3.4.1)
against independent solutions of the defining equations."""
import numpy as np
import pytest
from scipy.optimize import brentq


def _nonequilibrium_state(I, params, n, seed, dT=0.0, dp=0.0, dE=0.0):
    """Cells with both phases at independent (p_k, T_k): p_k = p (1 +/- dp),
    T_k = T (1 +/- dT); the mixture energy rho E carries an extra fraction dE of
    the internal energy (the mismatch a hyperbolic sweep leaves behind)."""
    rng = np.random.default_rng(seed)
    pr = I.random_states(n, seed, params, p_range=(1e5, 1e9), T_range=(250.0, 1500.0))
    a2 = pr[0, 0]
    a1 = 1 - a2
    g, pi, cv = np.array(params.gamma), np.array(params.pinf), np.array(params.cv)
    p1 = pr[1, 0] * (1 + dp * rng.uniform(-1, 1, n))
    p2 = pr[1, 0] * (1 + dp * rng.uniform(-1, 1, n))
    T1 = pr[2, 0] * (1 + dT * rng.uniform(-1, 1, n))
    T2 = pr[2, 0] * (1 + dT * rng.uniform(-1, 1, n))
    r1 = (p1 + pi[0]) / ((g[0] - 1) * cv[0] * T1)
    r2 = (p2 + pi[1]) / ((g[1] - 1) * cv[1] * T2)
    U = np.zeros((8, 1, n))
    U[0, 0] = a1 * r1
    U[1, 0] = a2 * r2
    rho = U[0, 0] + U[1, 0]
    U[2, 0] = rho * pr[3, 0]
    U[3, 0] = rho * pr[4, 0]
    U[4, 0] = a1 * (p1 + g[0] * pi[0]) / (g[0] - 1)
    U[5, 0] = a2 * (p2 + g[1] * pi[1]) / (g[1] - 1)
    kin = 0.5 * (U[2, 0] ** 2 + U[3, 0] ** 2) / rho
    U[6, 0] = (U[4, 0] + U[5, 0]) * (1 + dE) + kin
    U[7, 0] = a2
    return U


def _step1_reference(params, E0, a0):
    """Step (1) of Sec. 3.3 solved from its definition: for a trial p, each phase
    obeys E_k^1 + p a_k^1 = E_k^0 + p a_k^0 (dE_k = -p_I da_k with p_I = p) and
    E_k^1 = a_k^1 (p + g_k pinf_k)/(g_k - 1) (Eq. eos_stiffened); a 2x2 linear
    solve per phase, then bracketing of a_1(p) + a_2(p) = 1."""
    g, pi = params.gamma, params.pinf

    def alphas(p):
        out = []
        for k in range(2):
            M = np.array([[1.0, p], [1.0, -(p + g[k] * pi[k]) / (g[k] - 1)]])
            rhs = np.array([E0[k] + p * a0[k], 0.0])
            out.append(np.linalg.solve(M, rhs)[1])
        return out

    lo = -min(pi) + 1e-9 * (1 + max(pi))
    f = lambda p: sum(alphas(p)) - 1.0
    # the sum decreases monotonically on (-min pinf, inf): exactly one root
    grid = lo + np.logspace(-6, 13, 400)
    vals = np.array([f(p) for p in grid])
    assert np.sum(np.sign(vals[1:]) != np.sign(vals[:-1])) == 1
    k = int(np.nonzero(np.sign(vals[1:]) != np.sign(vals[:-1]))[0][0])
    p = brentq(f, grid[k], grid[k + 1], xtol=1e-15 * abs(grid[k + 1]), rtol=1e-15, maxiter=300)
    return p, alphas(p)


@pytest.mark.parametrize("eos", ["water_air", "solid_air"])
def test_prelax_against_definition(O, I, eos):
    params = I.shock_tube().params if eos == "water_air" else I.impact(8, 8).params
    U = _nonequilibrium_state(I, params, 300, 7, dp=0.3, dE=1e-3)
    U1, st = O.prelax(params, U)
    assert st == 0
    g, pi = params.gamma, params.pinf
    for c in range(U.shape[2]):
        a2 = U[7, 0, c]
        p, (a1r, a2r) = _step1_reference(params, (U[4, 0, c], U[5, 0, c]), (1 - a2, a2))
        assert abs(U1[7, 0, c] - a2r) <= 1e-9 * min(a2r, 1 - a2r) + 1e-15
    d = O.diagnostics(params, U1)
    # step (3): one pressure in both phases, the one of the conservative energy
    scale = np.abs(d[1]) + pi[0]
    assert np.max(np.abs(d[0] - d[1]) / scale) < 1e-9
    rho = U[0] + U[1]
    rhoe = U[6] - 0.5 * (U[2] ** 2 + U[3] ** 2) / rho
    assert np.max(np.abs(U1[4] + U1[5] - rhoe) / np.abs(rhoe)) < 1e-13
    # masses and momenta untouched
    assert np.array_equal(U1[[0, 1, 2, 3, 6]], U[[0, 1, 2, 3, 6]])


def test_prelax_idempotent(O, I):
    params = I.impact(8, 8).params
    U = _nonequilibrium_state(I, params, 500, 3, dp=0.5, dE=1e-4)
    U1, _ = O.prelax(params, U)
    U2, _ = O.prelax(params, U1)
    for q in range(8):
        assert np.max(np.abs(U2[q] - U1[q]) / (np.abs(U1[q]) + 1e-300)) < 1e-9, q


def _entropy(params, U):
    """Mixture entropy rho s = sum_k m_k s_k with the SG phase entropy
    s_k = Cv_k ln((p_k + pinf_k) / rho_k^gamma_k) (Gibbs relation + EOS)."""
    g, pi, cv = np.array(params.gamma), np.array(params.pinf), np.array(params.cv)
    a2 = U[7]
    a = (1 - a2, a2)
    tot = 0.0
    for k in range(2):
        m, E = U[k], U[4 + k]
        p = (g[k] - 1) * E / a[k] - g[k] * pi[k]
        rho = m / a[k]
        tot = tot + m * cv[k] * (np.log(p + pi[k]) - g[k] * np.log(rho))
    return tot


def test_trelax_closed_forms_ideal(O, I):
    """Equal pinf (here two ideal gases): T' = (C1 T1 + C2 T2)/(C1 + C2)
    (Eq. Taverage, Sec. 3.5) and alpha' = G2 C2 / (G1 C1 + G2 C2)."""
    params = I.Params(gamma=(1.4, 1.67), pinf=(0.0, 0.0), cv=(714.0, 3116.0))
    U = _nonequilibrium_state(I, params, 400, 5, dT=0.5)
    U1, st = O.trelax(params, U)
    assert st == 0
    d0 = O.diagnostics(params, U)
    C1, C2 = U[0] * params.cv[0], U[1] * params.cv[1]
    Tav = (C1 * d0[2] + C2 * d0[3]) / (C1 + C2)
    d1 = O.diagnostics(params, U1)
    assert np.max(np.abs(d1[2] - Tav) / Tav) < 1e-12
    assert np.max(np.abs(d1[3] - Tav) / Tav) < 1e-12
    aex = 0.67 * C2 / (0.4 * C1 + 0.67 * C2)
    assert np.max(np.abs(U1[7] - aex) / np.minimum(aex, 1 - aex)) < 1e-9


@pytest.mark.parametrize("eos", ["water_air", "solid_air"])
def test_trelax_equilibrium_and_entropy(O, I, eos):
    """After the relaxation T1 = T2 and p1 = p2 (the state Eqs. ht_eq2_TR,
    ht_eq3_TR drive to), energy is conserved and the mixture entropy does not
    decrease (Sec. 2.3 thermal-relaxation entropy balance)."""
    params = I.shock_tube().params if eos == "water_air" else I.impact(8, 8).params
    U = _nonequilibrium_state(I, params, 400, 11, dT=0.3)
    U1, st = O.trelax(params, U)
    assert st == 0
    d = O.diagnostics(params, U1)
    assert np.max(np.abs(d[2] - d[3]) / d[3]) < 1e-8
    assert np.max(np.abs(d[0] - d[1]) / (np.abs(d[1]) + params.pinf[0])) < 1e-9
    # the equilibrium is solved in E = rho e - pinf_1, so energy is kept to
    # roundoff of (rho e + |pinf_1 - pinf_2|)
    scale = U[4] + U[5] + abs(params.pinf[0] - params.pinf[1])
    assert np.max(np.abs((U1[4] + U1[5]) - (U[4] + U[5])) / scale) < 1e-14
    s0, s1 = _entropy(params, U), _entropy(params, U1)
    assert np.all(s1 - s0 >= -1e-9 * np.abs(s0))


def test_trelax_equilibrium_fixed_point(O, I):
    """A state already in p,T equilibrium is left unchanged (Sec. 3.5)."""
    params = I.impact(8, 8).params
    pr = I.random_states(500, 2, params)
    U = O.from_primitive(params, pr)
    U1, _ = O.trelax(params, U)
    for q in (4, 5, 7):
        assert np.max(np.abs(U1[q] - U[q]) / np.abs(U[q])) < 1e-9, q


def _paper_midpoint(params, m1, m2, T1, T2, a2, iters=200):
    """The paper's implicit discretization, Eqs. (ht_eq2_TR_dis), (ht_eq3_TR_dis),
    with B2 = pinf_2 - p/r0 (the sign that keeps dp1 = dp2; r0 from Eq. r0 and
    A_k = g_k (p + pinf_k) from Eq. AK) evaluated at the averages, solved by simple
    iteration as the paper does."""
    g, pi, cv = params.gamma, params.pinf, params.cv
    C1, C2 = m1 * cv[0], m2 * cv[1]
    B1 = pi[0] - pi[1]
    Tn, an = T2, a2
    for _ in range(iters):
        T1a, T2a, aa = 0.5 * (T1 + Tn), 0.5 * (T2 + Tn), 0.5 * (a2 + an)
        a1a = 1 - aa
        # phase-2 pressure at the average state
        p = (g[1] - 1) * C2 * T2a / aa - pi[1]
        A1, A2 = g[0] * (p + pi[0]), g[1] * (p + pi[1])
        s = (g[0] - 1) / a1a + (g[1] - 1) / aa
        r0 = s / ((A1 / a1a + A2 / aa) / p - s)
        B2 = pi[1] - p / r0
        # linear 2x2 system in (T', alpha')
        Tn = (B2 * C1 * T1 + (B1 + B2) * C2 * T2) / (B2 * C1 + (B1 + B2) * C2)
        an = a2 - C2 * (Tn - T2) / B2
    return Tn, an


def test_trelax_limit_of_paper_scheme(O, I):
    """As the phase-temperature gap shrinks the paper's own discrete relaxation
    and the exact-equilibrium reading converge to each other faster than the
    gap (both end on p1 = p2, T1 = T2 to leading order)."""
    params = I.impact(8, 8).params
    g, pi, cv = params.gamma, params.pinf, params.cv
    diffs = []
    for dT in (40.0, 20.0, 10.0, 5.0):
        # both phases at p = 2e8 Pa, alpha_2 = 0.3; phase 1 at 600 K, phase 2 hotter
        a2, p, T1, T2 = 0.3, 2e8, 600.0, 600.0 + dT
        r1 = (p + pi[0]) / ((g[0] - 1) * cv[0] * T1)
        r2 = (p + pi[1]) / ((g[1] - 1) * cv[1] * T2)
        U = np.zeros((8, 1, 1))
        U[0], U[1] = (1 - a2) * r1, a2 * r2
        U[4] = (1 - a2) * (p + g[0] * pi[0]) / (g[0] - 1)
        U[5] = a2 * (p + g[1] * pi[1]) / (g[1] - 1)
        U[6] = U[4] + U[5]
        U[7] = a2
        U1, st = O.trelax(params, U)
        assert st == 0
        Tm, am = _paper_midpoint(params, U[0, 0, 0], U[1, 0, 0], T1, T2, a2)
        d = O.diagnostics(params, U1)
        diffs.append(abs(U1[7, 0, 0] - am) / a2)
        assert T1 < d[3, 0, 0] < T2
        assert abs(d[3, 0, 0] - Tm) / Tm < 1e-3
    diffs = np.array(diffs)
    assert np.all(diffs[1:] < 0.3 * diffs[:-1])
