"""Pins of the oracle's heat-conduction stage and Chebyshev local-iteration
method (Sec. 3.2 LIM, Sec. 3.4.2, Algorithm 1) against linear algebra, the
heat kernel and finite differences of the equilibrium manifold."""
import math

import numpy as np
import pytest
from scipy.linalg import expm


def _dense_operator(lam, V, dx, dy, bc):
    """The finite-volume diffusion operator V div(Lam grad .) of Eq. (qk_dis)
    assembled as a dense matrix, face coefficient = two-cell mean; transmissive
    walls carry no flux, periodic axes wrap."""
    ny, nx = lam.shape
    n = nx * ny
    A = np.zeros((n, n))
    idx = lambda i, j: j * nx + i
    for j in range(ny):
        for i in range(nx):
            c = idx(i, j)
            for (di, dj, h, ax) in ((1, 0, dx, 0), (-1, 0, dx, 0), (0, 1, dy, 1), (0, -1, dy, 1)):
                ext = nx if ax == 0 else ny
                if ext < 2:
                    continue
                ii, jj = i + di, j + dj
                if not (0 <= ii < nx and 0 <= jj < ny):
                    if bc[ax] != 1:
                        continue
                    ii %= nx
                    jj %= ny
                nb = idx(ii, jj)
                lf = 0.5 * (lam[j, i] + lam[jj, ii])
                A[c, nb] += lf / h ** 2
                A[c, c] -= lf / h ** 2
    return V.reshape(-1)[:, None] * A


def _params(I, **kw):
    return I.Params(**kw)


def test_cheb_schedule_properties(O):
    """b_{2P-1} = 0 (Eq. LIM_last), every b_m in [0, lambda_max), the first P-1
    and the last P entries are (a_P..a_2) and (a_P..a_1)."""
    for P in (1, 2, 4, 8, 16, 32):
        b = O.cheb_schedule(P, 7.0)
        assert b.size == 2 * P - 1
        assert b[-1] == 0.0
        assert np.all(b >= 0.0) and np.all(b < 7.0)
        assert np.array_equal(b[:P - 1], b[P - 1:2 * P - 2])
        assert np.all(np.diff(b[P - 1:]) < 0)


@pytest.mark.parametrize("P_policy", ["formula", "fixed8"])
def test_lim_fourier_modes(O, I, P_policy):
    """Periodic constant-coefficient grid: every Fourier mode is an eigenvector
    of one LIM solve (translation invariance of the stencil) and its gain is
    the stability function R(z), z = tau * eigenvalue: |R| <= 1 over the whole
    spectrum (the stability claim of Sec. 3.2) and R ~ exp(-z) for small z."""
    n = 64
    h = 1.0 / n
    p = _params(I, bc=(1, 1), p_policy=I.P_FORMULA if P_policy == "formula" else I.P_FIXED, p_fixed=8)
    lam = np.full((1, n), 2.0)
    V = np.full((1, n), 0.5)
    tau = 3e-3  # tau * lambda_max = 3e-3 * 4 * 0.5 * 2 / h^2 ~ 49 -> P = 6 by formula
    x = np.arange(n) * h
    gains = []
    for k in range(n // 2 + 1):
        v0 = np.cos(2 * np.pi * k * x)[None, :]
        v1, Pn, lm = O.lim_solve(p, lam, V, v0, h, h, tau)
        g = v1[0, 0]
        assert np.allclose(v1, g * v0, atol=1e-12 * max(1.0, abs(g)))
        z = tau * 4 * 0.5 * 2.0 / h ** 2 * math.sin(math.pi * k / n) ** 2
        gains.append((z, g))
    assert Pn == (6 if P_policy == "formula" else 8)
    for z, g in gains:
        assert abs(g) <= 1.0 + 1e-12
        if z < 0.05:
            assert abs(g - math.exp(-z)) < 2 * z * z + 1e-14


def test_lim_against_dense_solves(O, I):
    """Variable V and Lam on a small 2D grid (transmissive walls).  The 2P-2
    predictor sweeps iterate towards the implicit-Euler solution, so one LIM
    solve tends to the dense implicit solve (I - tau V L_h)^-1 v0 as P grows --
    the LIM-vs-implicit agreement of Sec. 4.2 -- and both approximate the exact
    exp(tau V L_h) v0 to first order (error / 4 when tau / 2)."""
    rng = np.random.default_rng(4)
    nx, ny = 9, 7
    dx, dy = 0.1, 0.13
    lam = rng.uniform(0.5, 2.0, (ny, nx))
    V = rng.uniform(0.5, 1.5, (ny, nx))
    v0 = rng.uniform(-1, 1, (ny, nx))
    A = _dense_operator(lam, V, dx, dy, (0, 0))
    tau = 4e-4  # tau lambda_max ~ 0.5
    imp = np.linalg.solve(np.eye(nx * ny) - tau * A, v0.reshape(-1))
    gaps = []
    for P in (2, 3, 4, 5):
        v1, Pn, lm = O.lim_solve(_params(I, p_policy=I.P_FIXED, p_fixed=P), lam, V, v0, dx, dy, tau)
        gaps.append(np.max(np.abs(v1.reshape(-1) - imp)))
        # Gershgorin: lambda_max bounds the spectrum of -A
        assert lm >= np.max(np.abs(np.linalg.eigvals(A))) * (1 - 1e-12)
    gaps = np.array(gaps)
    assert np.all(gaps[1:] < 0.05 * gaps[:-1]) and gaps[-1] < 1e-9
    errs = []
    for t in (4e-4, 2e-4, 1e-4):
        v1, Pn, lm = O.lim_solve(_params(I, p_policy=I.P_FIXED, p_fixed=4), lam, V, v0, dx, dy, t)
        errs.append(np.max(np.abs(v1.reshape(-1) - expm(t * A) @ v0.reshape(-1))))
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0


@pytest.mark.parametrize("tau,P", [(2e-3, 8), (1e-2, 16), (2e-2, 23)])
def test_lim_maximum_principle(O, I, tau, P):
    """Monotonicity of the LIM (Sec. 3.2): a step profile stays within its
    bounds for large tau lambda_max (up to 800, P = 23 sweeps pairs) and the
    conservative last sweep keeps its sum."""
    n = 100
    p = _params(I, p_policy=I.P_FORMULA, p_max=64)
    lam = np.ones((1, n))
    V = np.ones((1, n))
    v0 = np.where(np.arange(n) < 50, 1.0, 0.0)[None, :]
    v1, Pn, lm = O.lim_solve(p, lam, V, v0, 0.01, 0.01, tau)
    assert Pn == P
    assert v1.min() >= -1e-12 and v1.max() <= 1 + 1e-12
    assert abs(v1.sum() - v0.sum()) < 1e-10


def _cheb_b(P, lam):
    """Eq. LIM parameters: beta_m = cos((2m - 1) pi / (2P)) in decreasing order
    (reading of the ordering), a_m = lam (beta_1 - beta_m)/(1 + beta_1),
    b = (a_P, ..., a_2, a_P, ..., a_1)."""
    beta = [math.cos((2 * m - 1) * math.pi / (2 * P)) for m in range(1, P + 1)]
    a = [lam * (beta[0] - beta[m - 1]) / (1.0 + beta[0]) for m in range(1, P + 1)]
    return [a[m - 1] for m in range(P, 1, -1)] + [a[m - 1] for m in range(P, 0, -1)]


def test_lim_matches_dense_polynomial(O, I):
    """The 2P-1 sweeps equal the same recurrence carried out with the dense
    matrix of the operator (checks the stencil, the face means and the walls):
    Eq. LIM as printed, v <- (v^n + tau b_m v + tau A v) / (1 + tau b_m), with
    the 1/h^2 of Eq. qk_dis per face and the parameters b_m computed here."""
    rng = np.random.default_rng(9)
    nx, ny = 6, 5
    lam = rng.uniform(0.5, 2.0, (ny, nx))
    V = rng.uniform(0.5, 1.5, (ny, nx))
    v0 = rng.uniform(-1, 1, (ny, nx))
    for bc in ((0, 0), (1, 1), (1, 0)):
        p = _params(I, bc=bc, p_policy=I.P_FIXED, p_fixed=5)
        tau = 0.02
        v1, Pn, lm = O.lim_solve(p, lam, V, v0, 0.1, 0.1, tau)
        A = _dense_operator(lam, V, 0.1, 0.1, bc)
        b = _cheb_b(Pn, lm)
        assert np.allclose(b, O.cheb_schedule(Pn, lm), rtol=1e-14, atol=1e-14 * lm)
        v = v0.reshape(-1).copy()
        u0 = v.copy()
        for m in range(2 * Pn - 1):
            v = (u0 + tau * b[m] * v + tau * (A @ v)) / (1 + tau * b[m])
        assert np.max(np.abs(v - v1.reshape(-1))) < 1e-12


def _ideal_uniform_density(I, n, T, rho=1.0, a2=0.5):
    """Two identical ideal gases (B1 = 0): V = 1/C, U = 0, and with uniform
    density the conduction equation is linear with constant diffusivity."""
    params = I.Params(gamma=(1.4, 1.4), pinf=(0.0, 0.0), cv=(714.0, 714.0), k0=(0.05, 0.05),
                      p_policy=I.P_FORMULA, p_max=64)
    prim = np.zeros((5,) + T.shape)
    prim[0] = a2
    prim[1] = rho * 0.4 * 714.0 * T
    prim[2] = T
    return params, prim


def test_heat_kernel(O, I):
    """Single material, constant conductivity and density: the heat stage solves
    dT/dt = D T_xx, D = lambda/(rho Cv); a Gaussian pulse spreads as the heat
    kernel, error O(h^2 + tau)."""
    n = 400
    L = 1.0
    h = L / n
    x = (np.arange(n) + 0.5) * h - 0.5
    D = 0.05 / (1.0 * 714.0)
    t0 = 0.002 / D
    T = 300.0 + 50.0 * np.exp(-x ** 2 / (4 * D * t0))
    params, prim = _ideal_uniform_density(I, n, T[None, :])
    U = O.from_primitive(params, prim)
    tau = 0.05 * t0
    nst = 10
    for _ in range(nst):
        U, st, Pn = O.heat(params, U, h, h, tau)
        assert st == 0
    t1 = t0 + nst * tau
    Tex = 300.0 + 50.0 * math.sqrt(t0 / t1) * np.exp(-x ** 2 / (4 * D * t1))
    Tn = O.heat_coeffs(params, U)[0, 0]
    err = np.max(np.abs(Tn - Tex)) / 50.0
    assert err < 0.01
    assert Pn > 1


def test_heat_coefficients_are_manifold_derivatives(O, I):
    """V = dT/d(rho e) and U_alpha = d alpha/d(rho e) along the p,T-equilibrium
    manifold (the coefficients of Eqs. ht_eq2_ht, ht_eq3_ht), against central
    differences of the equilibrium projection (Richardson-extrapolated; the step
    moves T by 1e-5 and the smaller volume fraction by at most 1e-3 of itself)."""
    for params in (I.impact(8, 8).params, I.shock_tube().params):
        pr = I.random_states(50, 8, params, p_range=(1e5, 1e8))
        U = O.from_primitive(params, pr)
        co = O.heat_coeffs(params, U)
        for c in range(50):
            m1, m2 = U[0, 0, c], U[1, 0, c]
            rhoe = U[4, 0, c] + U[5, 0, c]
            T, V, Ua = co[0, 0, c], co[1, 0, c], co[2, 0, c]
            a2 = U[7, 0, c]
            d = 1e-5 * T / V
            if Ua != 0.0:
                d = min(d, 1e-3 * min(a2, 1 - a2) / abs(Ua))

            def cd(h):
                Tp, ap, _ = O.equilibrium(params, m1, m2, rhoe + h)
                Tm, am, _ = O.equilibrium(params, m1, m2, rhoe - h)
                return (Tp - Tm) / (2 * h), (ap - am) / (2 * h)

            (v1, u1), (v2, u2) = cd(d), cd(0.5 * d)
            V_fd, U_fd = (4 * v2 - v1) / 3, (4 * u2 - u1) / 3
            assert abs(V_fd - V) / abs(V) < 2e-5
            assert abs(U_fd - Ua) <= 2e-5 * abs(Ua) + 1e-12 * abs(V)


def test_heat_coefficients_ideal(O, I):
    """Ideal gases (pinf = 0): U_alpha = 0 and V = 1/C."""
    params = I.Params(gamma=(1.4, 1.67), pinf=(0.0, 0.0), cv=(714.0, 3116.0), k0=(1.0, 1.0))
    pr = I.random_states(100, 3, params)
    U = O.from_primitive(params, pr)
    co = O.heat_coeffs(params, U)
    C = U[0] * 714.0 + U[1] * 3116.0
    assert np.max(np.abs(co[1] * C - 1)) < 1e-14
    assert np.all(co[2] == 0.0)


def test_heat_conserves_energy_and_produces_entropy(O, I):
    """Periodic water/air box with a temperature field: the conservative last
    sweep keeps sum(rho E) to roundoff; the mixture entropy sum m_k s_k does not
    decrease (Sec. 2.3 heat-conduction stage, Eq. ent_neq1 integrated)."""
    wl = I.conduction_disc(n=40, p_min=4, p_max=8)
    p = wl.params.replace(bc=(1, 1))
    U = O.from_primitive(p, wl.prim)
    from test_oracle_relax import _entropy

    s0 = _entropy(p, U).sum()
    e0 = U[6].sum()
    for _ in range(5):
        U, st, Pn = O.heat(p, U, wl.dx, wl.dy, 2e-4)
        assert st == 0
    assert abs(U[6].sum() - e0) / np.abs(U[6]).sum() < 1e-14
    assert _entropy(p, U).sum() > s0
    d = O.diagnostics(p, U)
    assert np.max(np.abs(d[2] - d[3]) / d[3]) < 1e-8
    assert np.max(np.abs(d[0] - d[1]) / (np.abs(d[1]) + p.pinf[0])) < 1e-9
