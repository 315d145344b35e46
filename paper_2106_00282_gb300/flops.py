"""Algorithmic work per cell for each kernel of the step: FP64 operations
(FLOP) and state bytes (BYTES).

The algorithmic work of a stage is what the plain FP64 statement of the method
performs: the oracle run once on an operation-counting scalar type, counting
+ - * / sqrt and powers on state-dependent values (comparisons, min/max, abs
and selects are free; operations on constants are not counted), per cell in
the limit of a large grid (ghost cells of the sweeps and boundary faces
excluded).  tests/test_flops.py checks every entry below against that count.

per cell                                   1D      2D
  sweep, one axis (no limiter / minmod / Overbee)   186 / 200 / 203
  pressure relaxation (Sec. 3.3)                    62
  temperature relaxation (Sec. 3.4.1)               36
  CFL maximum                              21      24
  heat stage (Sec. 3.4.2), P = 1           96      105   (+4 with a power-law conductivity)
  heat, per Chebyshev predictor sweep      16      24
  viscous stage, one axis, P = 1                    104
  viscous, per Chebyshev predictor sweep            30   (two velocity fields)

The kernels fuse stages: a sweep kernel applies the pressure relaxation to
its output, the heat kernel starts with the temperature relaxation, the
viscous kernel of the last axis ends with the pressure relaxation.

Algorithmic state bytes of one launch, per cell: the conserved planes the
stage reads once and the planes it changes written once, 8 bytes per value
(a double, or the pair of floats of the FP32-bulk form); scratch planes and
re-reads are not algorithmic.  The whole step reads and writes the 8-plane
state once: 128 B.
  CFL maximum      reads m1, m2, rho u, rho v, E1, E2, alpha_2      56
  sweep            reads 8 planes, writes 8                         128
  viscous, x       reads 8, writes rho u, rho v, E1, E2, rho E      104
  viscous, y       as x, and alpha_2 (pressure relaxation)          112
  heat             reads 8, writes E1, E2, rho E, alpha_2            96
"""
from __future__ import annotations

SWEEP = {0: 186, 1: 200, 2: 203}   # by limiter: none, minmod, Overbee
PRELAX = 62
TRELAX = 36
WAVE = {1: 21, 2: 24}              # by number of active axes
HEAT_BASE = {1: 96, 2: 105}
HEAT_POWER_LAW = 4
HEAT_SWEEP = {1: 16, 2: 24}
VISC_BASE = 104
VISC_SWEEP = 30


def per_cell(kernel: str, params, P: int = 1, ndim: int = 2) -> float:
    """Algorithmic FP64 operations per cell of one launch of `kernel` (the
    names bench.py and dim_kernel_time use) with P Chebyshev parameters."""
    lim = params.limiter if params.limiter in SWEEP else 1
    if kernel in ("sweep_x", "sweep_y"):
        return float(SWEEP[lim] + PRELAX)
    if kernel == "wave_max":
        return float(WAVE[ndim])
    if kernel == "heat":
        law = HEAT_POWER_LAW if params.k_exp != 0.0 else 0
        return float(TRELAX + HEAT_BASE[ndim] + law + HEAT_SWEEP[ndim] * (2 * P - 2))
    if kernel == "viscous_x":
        return float(VISC_BASE + VISC_SWEEP * (2 * P - 2) + (PRELAX if ndim == 1 else 0))
    if kernel == "viscous_y":
        return float(VISC_BASE + VISC_SWEEP * (2 * P - 2) + PRELAX)
    if kernel == "relax":
        return float(PRELAX)
    raise ValueError(kernel)


BYTES = {"wave_max": 56, "sweep_x": 128, "sweep_y": 128, "viscous_x": 104, "viscous_y": 112, "heat": 96,
         "relax": 96}


def bytes_per_cell(kernel: str) -> float:
    """Algorithmic state bytes per cell of one launch of `kernel`."""
    return float(BYTES[kernel])
