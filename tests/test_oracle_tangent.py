"""Pins of the oracle's tangent-linear step (forward-mode dual numbers over the
same templated arithmetic as the oracle).

The step is piecewise smooth: the limiter operand, the Davis bounds and the
HLLC wave region switch with the state, and dt and every Chebyshev lambda_max
are frozen (Sec. 3.1 CFL bound, Sec. 3.2 parameters).  The tangent is the
derivative of the map with these branches and this schedule held fixed, so it
is checked against central differences of the oracle run with the nominal
run's branches and schedule replayed (the branch-frozen map), cell by cell;
with the limiter off the branch-free parts agree without freezing too."""
import numpy as np
import pytest


def direction(U0, params, seed, smooth=False):
    """A perturbation in physical units: 1e-3 of the phase masses, 1 m/s of
    momentum, 1 kPa of phase pressure in E_k, 1e-3 alpha_1 alpha_2 of the
    volume fraction; white noise or one smooth Fourier mode per field."""
    rng = np.random.default_rng(seed)
    ny, nx = U0.shape[1:]
    if smooth:
        x = (np.arange(nx) + 0.5) / nx
        y = (np.arange(ny) + 0.5) / ny
        X, Y = np.meshgrid(x, y)

        def g():
            return np.sin(2 * np.pi * X + rng.uniform(0, 6.3)) * np.cos(2 * np.pi * Y * (ny > 1) + rng.uniform(0, 6.3))
    else:
        def g():
            return rng.standard_normal((ny, nx))
    a2 = U0[7]
    a1 = 1.0 - a2
    rho = U0[0] + U0[1]
    d = np.zeros_like(U0)
    d[0] = 1e-3 * U0[0] * g()
    d[1] = 1e-3 * U0[1] * g()
    d[2] = rho * g()
    d[3] = rho * g() * (ny > 1)
    d[4] = a1 * 1e3 / (params.gamma[0] - 1.0) * g()
    d[5] = a2 * 1e3 / (params.gamma[1] - 1.0) * g()
    d[6] = d[4] + d[5] + rho * g()
    d[7] = 1e-3 * a1 * a2 * g()
    return d


def _shift(params, dp, eps):
    return params.replace(k0=(params.k0[0] + eps * dp[0], params.k0[1] + eps * dp[1]),
                          mu=(params.mu[0] + eps * dp[2], params.mu[1] + eps * dp[3]),
                          src=(params.src[0] + eps * dp[4], params.src[1] + eps * dp[5]))


def _cellwise(O, wl, nsteps, dU, h, dparams=None):
    p = wl.params
    U0 = O.from_primitive(p, wl.prim)
    Ut, dUt, st, sched = O.step_tangent(p, U0, dU, wl.dx, wl.dy, nsteps, dparams)
    U1, st1, fr = O.step_frozen(p, U0, wl.dx, wl.dy, nsteps)
    dp = np.zeros(6) if dparams is None else dparams
    fp = O.step_frozen(_shift(p, dp, h), U0 + h * dU, wl.dx, wl.dy, nsteps, fr)[0]
    fm = O.step_frozen(_shift(p, dp, -h), U0 - h * dU, wl.dx, wl.dy, nsteps, fr)[0]
    fd = (fp - fm) / (2 * h)
    sc = np.abs(dUt).reshape(8, -1).max(1)[:, None] + 1e-300
    return (np.abs(fd - dUt).reshape(8, -1) / sc).max(), Ut, U1, sched, fr


def test_tangent_value_is_the_oracle(O, I):
    """The value part of a tangent run is the oracle's run bit for bit, and so
    is its recorded schedule; replaying a record reproduces the run."""
    wl = I.smooth_mixture(24, 16, seed=2)
    p = wl.params
    U0 = O.from_primitive(p, wl.prim)
    dU = direction(U0, p, 1)
    Ut, dUt, st, sched = O.step_tangent(p, U0, dU, wl.dx, wl.dy, 4)
    Uo, sto, dto, _ = O.step(p, U0, wl.dx, wl.dy, 4)
    assert np.array_equal(Ut, Uo) and st == sto
    Us, sts, sch = O.step_sched(p, U0, wl.dx, wl.dy, 4)
    assert np.array_equal(sch, sched) and np.array_equal(Us, Uo)
    assert np.all(sched[:, 0] > 0) and np.all(sched[:, 9] > 0) and np.all(sched[:, 10] > 0) and np.all(sched[:, 1] > 0)
    assert p.cfl / sched[-1, 0] == dto
    Ur = O.step_sched(p, U0, wl.dx, wl.dy, 4, sched)[0]
    Uf, _, fr = O.step_frozen(p, U0, wl.dx, wl.dy, 4)
    Ufr = O.step_frozen(p, U0, wl.dx, wl.dy, 4, fr)[0]
    assert np.array_equal(Ur, Uo) and np.array_equal(Uf, Uo) and np.array_equal(Ufr, Uo)


def test_tangent_is_linear(O, I):
    wl = I.smooth_mixture(32, 1, seed=4)
    p = wl.params
    U0 = O.from_primitive(p, wl.prim)
    d1, d2 = direction(U0, p, 1), direction(U0, p, 2)
    t1 = O.step_tangent(p, U0, d1, wl.dx, wl.dy, 3)[1]
    t2 = O.step_tangent(p, U0, d2, wl.dx, wl.dy, 3)[1]
    t12 = O.step_tangent(p, U0, 2.0 * d1 - 3.0 * d2, wl.dx, wl.dy, 3)[1]
    sc = np.abs(t12).reshape(8, -1).max(1)[:, None] + 1e-300
    assert (np.abs(t12 - (2.0 * t1 - 3.0 * t2)).reshape(8, -1) / sc).max() < 1e-12


@pytest.mark.parametrize("case", ["lim0_1d", "minmod_1d", "overbee_1d", "minmod_2d", "overbee_transmissive_src_2d",
                                  "n_outer2_2d", "shock_tube", "conduction_disc", "impact"])
def test_tangent_matches_branch_frozen_differences(O, I, case):
    """Every stage (sweeps, pressure relaxation, viscous LIM, temperature
    relaxation, heat LIM with its equilibrium projection) on white-noise
    directions: the tangent equals the branch-frozen central difference in
    every cell and field."""
    steps, h, tol = 5, 1e-3, 1e-6
    if case == "lim0_1d":
        wl = I.smooth_mixture(64, 1, seed=1, limiter=I.LIMITER_NONE)
    elif case == "minmod_1d":
        wl = I.smooth_mixture(64, 1, seed=1)
    elif case == "overbee_1d":
        wl = I.smooth_mixture(64, 1, seed=1, limiter=I.LIMITER_OVERBEE)
    elif case == "minmod_2d":
        wl = I.smooth_mixture(24, 16, seed=2)
    elif case == "overbee_transmissive_src_2d":
        wl = I.smooth_mixture(24, 16, seed=2, bc=(0, 0), limiter=I.LIMITER_OVERBEE)
        wl.params = wl.params.replace(src=(1e9, 1e8))
    elif case == "n_outer2_2d":
        wl = I.smooth_mixture(24, 16, seed=2)
        wl.params = wl.params.replace(n_outer=2)
        steps = 3
    elif case == "shock_tube":
        wl = I.shock_tube(n=100)
        steps, h, tol = 10, 1e-4, 1e-5
    elif case == "conduction_disc":
        wl = I.conduction_disc(40)
        steps, h, tol = 4, 1e-4, 1e-5
    else:
        wl = I.impact(40, 20)
        steps, h, tol = 3, 1e-4, 1e-3
    U0 = O.from_primitive(wl.params, wl.prim)
    err = _cellwise(O, wl, steps, direction(U0, wl.params, 3), h)[0]
    print(f"[tangent] {case}: max cell relative error {err:.2e}")
    assert err < tol


def test_tangent_parameter_directions(O, I):
    """Tangents with respect to (k0_1, k0_2, mu_1, mu_2, I_1, I_2) against
    branch-frozen central differences of a scalar objective J = <w, U_T>."""
    # conduction and viscosity strong enough to move the state within 5 steps
    wl = I.smooth_mixture(24, 16, seed=2, k=(2e4, 2e3), mu=(5.0, 0.5))
    wl.params = wl.params.replace(src=(1e9, 1e8))
    p = wl.params
    U0 = O.from_primitive(p, wl.prim)
    rng = np.random.default_rng(7)
    w = rng.standard_normal(U0.shape) / (np.abs(U0).reshape(8, -1).mean(1)[:, None, None] + 1e-30)
    U1, st1, fr = O.step_frozen(p, U0, wl.dx, wl.dy, 5)
    base = np.array([2e4, 2e3, 5.0, 0.5, 1e9, 1e8])
    for k in range(6):
        dp = np.zeros(6)
        dp[k] = base[k]
        t = np.sum(w * O.step_tangent(p, U0, np.zeros_like(U0), wl.dx, wl.dy, 5, dp)[1])
        h = 1e-2
        jp = np.sum(w * O.step_frozen(_shift(p, dp, h), U0, wl.dx, wl.dy, 5, fr)[0])
        jm = np.sum(w * O.step_frozen(_shift(p, dp, -h), U0, wl.dx, wl.dy, 5, fr)[0])
        fd = (jp - jm) / (2 * h)
        print(f"[tangent] parameter {k}: dJ {t:+.6e} FD {fd:+.6e}")
        # roundoff floor of the difference quotient: a few ulps of sum |w U| over 2h
        assert abs(fd - t) <= 1e-6 * abs(t) + 1e-14 * np.sum(np.abs(w * U1)) / h


def test_branch_record_changes_nothing_without_perturbation(O, I):
    """A replayed branch record on a perturbed state really freezes the
    branches: the replayed run of a large perturbation differs from the free
    run of the same state (some branch switched), and the replay of the
    nominal state is the nominal run."""
    wl = I.smooth_mixture(64, 1, seed=1)
    p = wl.params
    U0 = O.from_primitive(p, wl.prim)
    U1, _, fr = O.step_frozen(p, U0, wl.dx, wl.dy, 5)
    dU = direction(U0, p, 3)
    Ufree = O.step_sched(p, U0 + 0.5 * dU, wl.dx, wl.dy, 5, fr[0])[0]
    Ufrozen = O.step_frozen(p, U0 + 0.5 * dU, wl.dx, wl.dy, 5, fr)[0]
    assert not np.array_equal(Ufree, Ufrozen)
    assert np.array_equal(O.step_frozen(p, U0, wl.dx, wl.dy, 5, fr)[0], U1)


def test_extended_tangent_agrees_on_well_conditioned_flows(O, I):
    """The long-double tangent, replaying the double run's schedule and
    branches, agrees with the double tangent where the flow is well
    conditioned (it is the rounding reference of the adjoint comparisons)."""
    for wl, steps in [(I.smooth_mixture(24, 16, seed=2), 4), (I.shock_tube(n=100), 6), (I.conduction_disc(40), 4)]:
        p = wl.params
        U0 = O.from_primitive(p, wl.prim)
        fr = O.step_frozen(p, U0, wl.dx, wl.dy, steps)[2]
        d = direction(U0, p, 5)
        dp = np.array([0.1, 0.01, 1e-4, 1e-6, 1e6, 1e5])
        t = O.step_tangent(p, U0, d, wl.dx, wl.dy, steps, dp)[1]
        te = O.step_tangent_ext(p, U0, d, wl.dx, wl.dy, steps, fr, dp)[1]
        sc = np.abs(te).reshape(8, -1).max(1)[:, None] + 1e-300
        err = (np.abs(t - te).reshape(8, -1) / sc).max()
        print(f"[tangent] double vs long-double tangent ({wl.name}): {err:.1e}")
        assert err < 1e-10

