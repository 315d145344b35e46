"""Algorithmic FP64 operation counts per cell for each kernel of the step.

Counted from the formulas the kernels evaluate (one + - * / or sqrt = one
operation; comparisons, min/max and selects are free).  Face quantities are
counted once per face (one face per cell and axis); halo recomputation inside a
tile is not algorithmic work and is not counted.

hyperbolic sweep (one axis), per cell:
  primitives (alpha_1, rho, u_n, u_t, p_1, p_2)                          10
  minmod slopes (2 differences x 7) + face values (2 sides x 7 x 2)       42
  face states, 2 sides x (E_k, p, c^2 = (a1 A1 + a2 A2)/rho, rho u, rho E) 58
  HLLC: S_L, S_R, S*, star state, flux                                    53
  Godunov update with the R term                                          37
  pressure relaxation (quadratic, alpha, p from rho E, E_k)               65
                                                                  total  265
CFL wave-speed maximum, per cell                                          24
heat stage (temperature relaxation fused), per cell:
  equilibrium 28 + energies 10 + temperature 10 + coefficients 28 = 76 (A)
  Gershgorin bound 13 (B); per predictor sweep 19 (C, 2P - 2 of them);
  conservative last sweep + projection + check 63 (D)     total 152 + 19 (2P - 2)
viscous stage (one axis), per cell:
  velocities 4, bound 13, per predictor sweep 24 (two fields), fluxes 18,
  conservative update 48, + 65 when the pressure relaxation is fused
                                                 total 83 (+65) + 24 (2P - 2)
"""
from __future__ import annotations

SWEEP = 265
WAVE = 24
HEAT_BASE, HEAT_SWEEP = 152, 19
VISC_BASE, VISC_SWEEP, PRELAX = 83, 24, 65


def per_cell(kernel: str, params, P: int = 1) -> float:
    if kernel in ("sweep_x", "sweep_y"):
        return float(SWEEP)
    if kernel == "wave_max":
        return float(WAVE)
    if kernel == "heat":
        return float(HEAT_BASE + HEAT_SWEEP * (2 * P - 2))
    if kernel == "viscous_x":
        return float(VISC_BASE + VISC_SWEEP * (2 * P - 2))
    if kernel == "viscous_y":
        return float(VISC_BASE + PRELAX + VISC_SWEEP * (2 * P - 2))
    if kernel == "relax":
        return float(PRELAX)
    raise ValueError(kernel)
