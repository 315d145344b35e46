"""Seeded synthetic workloads for the split step of the two-temperature model.

This module holds parameters and geometry only: it returns, per cell, the
volume fraction alpha_2, pressure p, temperature T and velocity (u, v) of a
workload, plus the phase/EOS parameters and flags.  It contains none of the
method's arithmetic -- the conversion to conserved variables is done by the
consumer (the CUDA library or the oracle) with its own stiffened-gas EOS.

Workloads (paper Sec. 4 and the benchmark configurations):
  * ``shock_tube``      water/air shock tube, Sec. 4.2 (interface x = 0.7,
                        left p = 1e9 Pa, T = 293.02 K; right p = 1e5 Pa,
                        T = 7.02 K; gamma = 4.4/1.4, pinf = 6e8/0, Cv =
                        1606/714).  With k = (0.6, 0.026) W/m/K and P = 4
                        (8 stencil passes per step) this is the 1000-cell,
                        200-step, CFL 0.5 configuration.
  * ``pvt_translation`` interface translation, Sec. 4.1 (u = 1000 m/s,
                        p = 1e5 Pa, T = 300 K, interface at x = 0.2).
  * ``mixture_shock``   water-gas mixture shock tube, Sec. 4.3 (alpha = 0.5).
  * ``impact``          2D projectile impact, 1024 x 512 cells on 2 x 1 m.
  * ``conduction_disc`` 2D hot air disc in cold water with a seeded
                        sinusoidal interface perturbation, 2048^2 cells.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field

import numpy as np

# flag values shared by both consumers' parameter structs
LIMITER_NONE, LIMITER_MINMOD, LIMITER_OVERBEE = 0, 1, 2
LIMITER_OVERBEE_ALPHA_ONLY = 3  # the inconsistent combination (oracle only)
BC_TRANSMISSIVE, BC_PERIODIC = 0, 1
TRELAX_OFF, TRELAX_EQUILIBRIUM, TRELAX_MIDPOINT = 0, 1, 2
HEAT_ALPHA_PROJECTION, HEAT_ALPHA_LINEAR = 0, 1
P_FORMULA, P_FIXED, P_CLAMP = 0, 1, 2
PRECISION_FP64, PRECISION_FP32_BULK = 0, 1

ALPHA_FLOOR = 1e-6  # minor-phase volume fraction of a "pure" cell


@dataclass
class Params:
    """Phase parameters (phase 1 dense, phase 2 gas) and solver flags."""

    gamma: tuple = (4.4, 1.4)
    pinf: tuple = (6e8, 0.0)
    cv: tuple = (1606.0, 714.0)
    k0: tuple = (0.0, 0.0)          # lambda_k(T) = k0_k (T / T_ref)^k_exp
    k_exp: float = 0.0
    T_ref: float = 300.0
    mu: tuple = (0.0, 0.0)
    cfl: float = 0.5
    limiter: int = LIMITER_MINMOD
    bc: tuple = (BC_TRANSMISSIVE, BC_TRANSMISSIVE)
    trelax: int = TRELAX_EQUILIBRIUM
    n_outer: int = 1
    p_policy: int = P_FORMULA
    p_fixed: int = 1
    p_min: int = 1
    p_max: int = 24
    precision: int = PRECISION_FP64  # read by the CUDA library only; the oracle is FP64
    src: tuple = (0.0, 0.0)          # external heat source intensities I_k (W/m^3 of phase k)
    heat_alpha: int = HEAT_ALPHA_PROJECTION  # heat-stage (T, alpha) update
    trelax_iters: int = 20           # simple iterations of the midpoint temperature relaxation

    def replace(self, **kw) -> "Params":
        return dataclasses.replace(self, **kw)


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    dx: float
    dy: float
    params: Params
    prim: np.ndarray            # (5, ny, nx) float64: alpha_2, p, T, u, v
    steps: int = 1
    meta: dict = field(default_factory=dict)

    @property
    def ncell(self) -> int:
        return self.nx * self.ny


def _prim(ny: int, nx: int) -> np.ndarray:
    return np.zeros((5, ny, nx), dtype=np.float64)


def _centers(n: int, length: float) -> np.ndarray:
    h = length / n
    return (np.arange(n, dtype=np.float64) + 0.5) * h


# ---------------------------------------------------------------------------
# 1D workloads of Sec. 4
# ---------------------------------------------------------------------------
WATER = dict(gamma=4.4, pinf=6e8, cv=1606.0)
AIR = dict(gamma=1.4, pinf=0.0, cv=714.0)


def shock_tube(n: int = 1000, k=(0.6, 0.026), mu=(0.0, 0.0), p_policy=P_FIXED, p_fixed=4,
               trelax=TRELAX_EQUILIBRIUM, limiter=LIMITER_MINMOD, steps=200, axis=0) -> Workload:
    """Water/air shock tube of Sec. 4.2 on [0, 1] m, interface at x = 0.7."""
    params = Params(gamma=(WATER["gamma"], AIR["gamma"]), pinf=(WATER["pinf"], AIR["pinf"]),
                    cv=(WATER["cv"], AIR["cv"]), k0=tuple(k), mu=tuple(mu), cfl=0.5,
                    limiter=limiter, trelax=trelax, p_policy=p_policy, p_fixed=p_fixed)
    x = _centers(n, 1.0)
    left = x < 0.7
    pr = _prim(1, n)
    pr[0, 0] = np.where(left, ALPHA_FLOOR, 1.0 - ALPHA_FLOOR)
    pr[1, 0] = np.where(left, 1e9, 1e5)
    pr[2, 0] = np.where(left, 293.02, 7.02)
    wl = Workload("shock_tube", n, 1, 1.0 / n, 1.0 / n, params, pr, steps)
    return transpose(wl) if axis == 1 else wl


def pvt_translation(n: int = 200, k=(0.0, 0.0), steps=50, bc=BC_PERIODIC, limiter=LIMITER_MINMOD,
                    axis=0) -> Workload:
    """Interface translation of Sec. 4.1: u = 1000 m/s, p = 1e5 Pa, T = 300 K,
    left material gamma = 4.4, Cv = 500, pinf = 6e8, right gamma = 1.4, Cv = 200;
    interface at x = 0.2 (a second one at x = 0.6 closes the periodic box)."""
    params = Params(gamma=(4.4, 1.4), pinf=(6e8, 0.0), cv=(500.0, 200.0), k0=tuple(k), cfl=0.5,
                    limiter=limiter, bc=(bc, bc), p_policy=P_FORMULA)
    x = _centers(n, 1.0)
    left = (x < 0.2) | (x >= 0.6) if bc == BC_PERIODIC else x < 0.2
    pr = _prim(1, n)
    pr[0, 0] = np.where(left, ALPHA_FLOOR, 1.0 - ALPHA_FLOOR)
    pr[1, 0] = 1e5
    pr[2, 0] = 300.0
    pr[3, 0] = 1000.0
    wl = Workload("pvt_translation", n, 1, 1.0 / n, 1.0 / n, params, pr, steps)
    return transpose(wl) if axis == 1 else wl


def mixture_shock(n: int = 1000, k=(1e5, 1e7), steps=100) -> Workload:
    """Water-gas mixture shock of Sec. 4.3: alpha = 0.5 everywhere, left 1e9 Pa
    and 1000 K, right 1e5 Pa and 300 K, conductivities water 1e5, gas 1e7."""
    params = Params(gamma=(WATER["gamma"], AIR["gamma"]), pinf=(WATER["pinf"], AIR["pinf"]),
                    cv=(WATER["cv"], AIR["cv"]), k0=tuple(k), cfl=0.5, p_policy=P_FORMULA, p_max=64)
    x = _centers(n, 1.0)
    left = x < 0.5
    pr = _prim(1, n)
    pr[0, 0] = 0.5
    pr[1, 0] = np.where(left, 1e9, 1e5)
    pr[2, 0] = np.where(left, 1000.0, 300.0)
    return Workload("mixture_shock", n, 1, 1.0 / n, 1.0 / n, params, pr, steps)


def transpose(wl: Workload) -> Workload:
    """The same workload laid out along y (u becomes v)."""
    pr = np.ascontiguousarray(np.transpose(wl.prim, (0, 2, 1)))
    pr[[3, 4]] = pr[[4, 3]]
    p = wl.params.replace(bc=(wl.params.bc[1], wl.params.bc[0]))
    return Workload(wl.name + "_y", wl.ny, wl.nx, wl.dy, wl.dx, p, pr, wl.steps, dict(wl.meta))


# ---------------------------------------------------------------------------
# 2D workloads
# ---------------------------------------------------------------------------
# Solid projectile/target: gamma = 4.22, pinf = 3.42e10 with rho = 8900 kg/m^3 at
# 1e5 Pa and 300 K, i.e. Cv = (p + pinf) / ((gamma - 1) rho T) = 3978.2 J/kg/K.
SOLID = dict(gamma=4.22, pinf=3.42e10, cv=3978.2)


def impact(nx: int = 1024, ny: int = 512, steps=500, p_policy=P_FORMULA) -> Workload:
    """2D multiphase impact on [0,2] x [0,1] m: a 0.2 x 0.1 m solid projectile
    at [0.3,0.5] x [0.45,0.55] moving at u = +500 m/s touches a solid slab at
    x in [0.5, 0.7] (full height); air elsewhere; everything at 1e5 Pa, 300 K.
    k = (400, 0.026) W/m/K, mu = (1e-3, 1.8e-5) Pa s."""
    params = Params(gamma=(SOLID["gamma"], AIR["gamma"]), pinf=(SOLID["pinf"], AIR["pinf"]),
                    cv=(SOLID["cv"], AIR["cv"]), k0=(400.0, 0.026), mu=(1e-3, 1.8e-5), cfl=0.5,
                    p_policy=p_policy)
    x = _centers(nx, 2.0)[None, :]
    y = _centers(ny, 1.0)[:, None]
    proj = (x >= 0.3) & (x < 0.5) & (y >= 0.45) & (y < 0.55)
    slab = (x >= 0.5) & (x < 0.7) & (y >= 0.0 * y)
    solid = proj | slab
    pr = _prim(ny, nx)
    pr[0] = np.where(solid, ALPHA_FLOOR, 1.0 - ALPHA_FLOOR)
    pr[1] = 1e5
    pr[2] = 300.0
    pr[3] = np.where(proj, 500.0, 0.0)
    return Workload("impact", nx, ny, 2.0 / nx, 1.0 / ny, params, pr, steps)


def conduction_disc(n: int = 2048, seed: int = 3, steps=300, p_min=8, p_max=16, modes=(4, 16),
                    k_exp=2.0) -> Workload:
    """Hot air disc (T = 3000 K, r0 = 0.2, centre (0.5, 0.5)) in water at 300 K on
    [0,1]^2, p = 1e5 Pa, lambda_k = k0_k (T/300)^2 with k0 = (0.6, 0.026),
    mu = (1e-3, 1.8e-5).  Interface r(theta) = r0 + sum_m a_m cos(m theta + phi_m)
    for m in [modes], a_m ~ U[-1,1] * 0.01 r0, phi_m ~ U[0, 2 pi) from ``seed``;
    alpha_2 is a tanh profile of width 1.5 dx with the 1e-6 floor, and T mixes
    the two temperatures by alpha_2.  P = clamp(formula, p_min, p_max)."""
    rng = np.random.default_rng(seed)
    ms = np.arange(modes[0], modes[1] + 1)
    amp = rng.uniform(-1.0, 1.0, size=ms.size) * 0.01 * 0.2
    phase = rng.uniform(0.0, 2.0 * math.pi, size=ms.size)
    params = Params(gamma=(WATER["gamma"], AIR["gamma"]), pinf=(WATER["pinf"], AIR["pinf"]),
                    cv=(WATER["cv"], AIR["cv"]), k0=(0.6, 0.026), k_exp=k_exp, T_ref=300.0,
                    mu=(1e-3, 1.8e-5), cfl=0.5, p_policy=P_CLAMP, p_min=p_min, p_max=p_max)
    h = 1.0 / n
    x = _centers(n, 1.0)[None, :] - 0.5
    y = _centers(n, 1.0)[:, None] - 0.5
    r = np.hypot(x, y)
    th = np.arctan2(y, x)
    R = 0.2 + np.sum(amp[:, None, None] * np.cos(ms[:, None, None] * th[None] + phase[:, None, None]), axis=0)
    w = 1.5 * h
    s = 0.5 * (1.0 + np.tanh((R - r) / w))
    pr = _prim(n, n)
    pr[0] = ALPHA_FLOOR + (1.0 - 2.0 * ALPHA_FLOOR) * s
    pr[1] = 1e5
    pr[2] = 300.0 + (3000.0 - 300.0) * s
    return Workload("conduction_disc", n, n, h, h, params, pr, steps,
                    dict(seed=seed, modes=ms.tolist(), amp=amp.tolist(), phase=phase.tolist()))


def smooth_mixture(nx: int = 64, ny: int = 1, seed: int = 0, k=(0.6, 0.026), mu=(1e-3, 1.8e-5),
                   limiter=LIMITER_MINMOD, bc=(BC_PERIODIC, BC_PERIODIC), u_amp=20.0) -> Workload:
    """A smooth water/air mixture on the periodic unit square (or segment):
    alpha_2 = 0.5 + 0.3 f_1, p = 1e5 (1 + 0.05 f_2), T = 300 (1 + 0.05 f_3),
    u = u_amp f_4, v = u_amp f_5, each f_i a seeded sum of two low Fourier modes
    with |f_i| <= 1.  No cell pair has equal states, so slopes, wave-speed
    bounds and limiter branches are generic: the workload of the derivative
    checks (the step is piecewise smooth; at exactly uniform states the limiter
    is not differentiable)."""
    rng = np.random.default_rng(seed)
    hx, hy = 1.0 / nx, 1.0 / ny
    x = _centers(nx, 1.0)[None, :]
    y = _centers(ny, 1.0)[:, None] if ny > 1 else np.zeros((1, 1))

    def f():
        kx = rng.integers(1, 3, size=2)
        ky = rng.integers(1, 3, size=2) if ny > 1 else np.zeros(2, dtype=int)
        ph = rng.uniform(0.0, 2.0 * math.pi, size=2)
        g = (0.6 * np.sin(2.0 * math.pi * (kx[0] * x + ky[0] * y) + ph[0]) +
             0.4 * np.cos(2.0 * math.pi * (kx[1] * x - ky[1] * y) + ph[1]))
        return np.broadcast_to(g, (ny, nx))

    params = Params(gamma=(WATER["gamma"], AIR["gamma"]), pinf=(WATER["pinf"], AIR["pinf"]),
                    cv=(WATER["cv"], AIR["cv"]), k0=tuple(k), k_exp=2.0, T_ref=300.0, mu=tuple(mu), cfl=0.5,
                    limiter=limiter, bc=tuple(bc), p_policy=P_FORMULA)
    pr = _prim(ny, nx)
    pr[0] = 0.5 + 0.3 * f()
    pr[1] = 1e5 * (1.0 + 0.05 * f())
    pr[2] = 300.0 * (1.0 + 0.05 * f())
    pr[3] = u_amp * f()
    pr[4] = u_amp * f() if ny > 1 else 0.0
    dy = hy if ny > 1 else hx
    return Workload("smooth_mixture", nx, ny, hx, dy, params, pr, 10, dict(seed=seed))


def disc_interface(n: int, amp: np.ndarray, phase: np.ndarray, modes=(4, 19), r0: float = 0.2):
    """The interface indicator s in [0, 1] of the perturbed disc of
    `conduction_disc` (tanh profile of width 1.5 h), for given amplitudes."""
    ms = np.arange(modes[0], modes[1] + 1)
    h = 1.0 / n
    x = _centers(n, 1.0)[None, :] - 0.5
    y = _centers(n, 1.0)[:, None] - 0.5
    r = np.hypot(x, y)
    th = np.arctan2(y, x)
    R = r0 + np.sum(np.asarray(amp)[:, None, None] * np.cos(ms[:, None, None] * th[None] +
                                                          np.asarray(phase)[:, None, None]), axis=0)
    return 0.5 * (1.0 + np.tanh((R - r) / (1.5 * h))), r, th, ms


def disc_gradient(n: int = 512, seed: int = 3, steps: int = 200, ckpt: int = 20) -> Workload:
    """Gradient problem on the conduction disc: 512^2 cells, FP64, 200 steps,
    checkpoints every 20; 16 interface modes m = 4..19 with amplitudes
    a_m ~ U[-1,1] 0.01 r0 and phases phi_m ~ U[0, 2 pi) from ``seed``; the
    objective is the alpha(1-alpha)-weighted mean interface temperature, the
    parameters of interest (k0_1, k0_2, mu_1, mu_2) and the 16 amplitudes."""
    rng = np.random.default_rng(seed)
    ms = np.arange(4, 20)
    amp = rng.uniform(-1.0, 1.0, size=ms.size) * 0.01 * 0.2
    phase = rng.uniform(0.0, 2.0 * math.pi, size=ms.size)
    params = Params(gamma=(WATER["gamma"], AIR["gamma"]), pinf=(WATER["pinf"], AIR["pinf"]),
                    cv=(WATER["cv"], AIR["cv"]), k0=(0.6, 0.026), k_exp=2.0, T_ref=300.0,
                    mu=(1e-3, 1.8e-5), cfl=0.5, p_policy=P_CLAMP, p_min=8, p_max=16)
    s = disc_interface(n, amp, phase)[0]
    pr = _prim(n, n)
    pr[0] = ALPHA_FLOOR + (1.0 - 2.0 * ALPHA_FLOOR) * s
    pr[1] = 1e5
    pr[2] = 300.0 + (3000.0 - 300.0) * s
    h = 1.0 / n
    return Workload("disc_gradient", n, n, h, h, params, pr, steps,
                    dict(seed=seed, modes=ms.tolist(), amp=amp.tolist(), phase=phase.tolist(), ckpt=ckpt))


def random_states(ncell: int, seed: int, params: Params, p_range=(1e5, 1e9), T_range=(200.0, 2000.0),
                  a_range=(1e-6, 1 - 1e-6), u_range=(-300.0, 300.0)) -> np.ndarray:
    """Random per-cell (alpha_2, p, T, u, v) for pointwise tests, shape (5, 1, ncell)."""
    rng = np.random.default_rng(seed)
    pr = _prim(1, ncell)
    la, lb = math.log(a_range[0]), math.log(a_range[1])
    # volume fractions spread over (1e-6, 1-1e-6), half of them near each end
    a = np.exp(rng.uniform(la, 0.0, size=ncell))
    flip = rng.random(ncell) < 0.5
    pr[0, 0] = np.clip(np.where(flip, 1.0 - a, a), a_range[0], a_range[1])
    pr[1, 0] = np.exp(rng.uniform(math.log(p_range[0]), math.log(p_range[1]), size=ncell))
    pr[2, 0] = rng.uniform(T_range[0], T_range[1], size=ncell)
    pr[3, 0] = rng.uniform(*u_range, size=ncell)
    pr[4, 0] = rng.uniform(*u_range, size=ncell)
    del lb
    return pr


def bench_workload(name: str = "impact") -> Workload:
    """The workload the benchmark times at one GPU."""
    if name == "impact":
        return impact()
    if name == "conduction_disc":
        return conduction_disc()
    if name == "shock_tube":
        return shock_tube()
    raise ValueError(name)


# ---------------------------------------------------------------------------
# batches of independent problems
# ---------------------------------------------------------------------------
def batch_instance(nx: int, ny: int, rng: np.random.Generator, kind: str | None = None) -> np.ndarray:
    """Primitive fields (5, ny, nx) of one water/air problem on a unit-height
    domain of square cells (width nx/ny): a 'riemann' setup (water at
    ratio * 1e5 Pa left of x = W/2, air at 1e5 Pa right) or a 'bubble' setup
    (an air bubble of radius R in water at 1e5 Pa, hit by water at ratio * 1e5
    Pa from x < W/4); ratio log-uniform in [10, 1e4], R uniform in [0.05, 0.3],
    everything at 300 K and at rest."""
    kind = kind or ("riemann" if rng.random() < 0.5 else "bubble")
    ratio = math.exp(rng.uniform(math.log(10.0), math.log(1e4)))
    R = rng.uniform(0.05, 0.3)
    h = 1.0 / ny
    W = nx * h
    x = (np.arange(nx) + 0.5)[None, :] * h
    y = (np.arange(ny) + 0.5)[:, None] * h
    pr = _prim(ny, nx)
    pr[2] = 300.0
    if kind == "riemann":
        left = (x < 0.5 * W) & (y >= 0.0 * y)
        pr[0] = np.where(left, ALPHA_FLOOR, 1.0 - ALPHA_FLOOR)
        pr[1] = np.where(left, 1e5 * ratio, 1e5)
    else:
        bubble = (x - 0.5 * W) ** 2 + (y - 0.5) ** 2 < R * R
        pr[0] = np.where(bubble, 1.0 - ALPHA_FLOOR, ALPHA_FLOOR)
        pr[1] = np.where((x < 0.25 * W) & (y >= 0.0 * y), 1e5 * ratio, 1e5)
    return pr


def batch_params() -> Params:
    """Water/air, heat conduction with the conduction-disc law, no viscosity,
    FP32 bulk, P by formula."""
    return Params(gamma=(WATER["gamma"], AIR["gamma"]), pinf=(WATER["pinf"], AIR["pinf"]),
                  cv=(WATER["cv"], AIR["cv"]), k0=(0.6, 0.026), k_exp=2.0, T_ref=300.0, mu=(0.0, 0.0),
                  cfl=0.5, p_policy=P_FORMULA, precision=PRECISION_FP32_BULK)


def batch(ninst: int = 256, seed: int = 4, sizes=(128, 256, 512, 1024)):
    """ninst instances with nx, ny drawn independently and uniformly from
    `sizes`; returns (params, list of (nx, ny, dx, dy), list of primitive arrays)."""
    rng = np.random.default_rng(seed)
    grids, prims = [], []
    for _ in range(ninst):
        nx = int(rng.choice(sizes))
        ny = int(rng.choice(sizes))
        h = 1.0 / ny
        grids.append((nx, ny, h, h))
        prims.append(batch_instance(nx, ny, rng))
    return batch_params(), grids, prims
