"""The algorithmic operation counts of flops.py against the oracle run on an
operation-counting scalar type: per cell, in the limit of a large grid (two
extents along the sweep axis differenced to remove the ghost cells),
periodic walls, for 1D and 2D, the three limiters, constant and power-law
conductivity and P = 1, 2, 3."""
import itertools

import pytest


def _per_cell(O, I, stage, params, nx, ny, axis):
    res = []
    for scale in (1, 2):
        gx, gy = (nx * scale, ny) if axis == 0 else (nx, ny * scale)
        wl = I.smooth_mixture(gx, gy, seed=1)
        U = O.from_primitive(params, wl.prim)
        dt = O.dt(params, U, wl.dx, wl.dy)
        c = O.count_ops(params, U, wl.dx, wl.dy, stage, dt)
        res.append((gx * gy, c["total"], c["P"]))
    (n1, c1, P1), (n2, c2, P2) = res
    assert P1 == P2
    return (c2 - c1) / (n2 - n1), P2


@pytest.mark.parametrize("ndim", [1, 2])
def test_flop_counts_match_the_instrumented_oracle(O, I, ndim):
    from paper_2106_00282_gb300 import flops

    ny = 1 if ndim == 1 else 16
    base = I.smooth_mixture(8, 8, seed=1).params
    for lim, kexp in itertools.product((0, 1, 2), (0.0, 2.0)):
        p = base.replace(limiter=lim, k_exp=kexp)
        sweep = _per_cell(O, I, "sweep_x", p, 32, ny, 0)[0]
        prelax = _per_cell(O, I, "prelax", p, 32, ny, 0)[0]
        trelax = _per_cell(O, I, "trelax", p, 32, ny, 0)[0]
        wave = _per_cell(O, I, "wave_max", p, 32, ny, 0)[0]
        assert sweep + prelax == flops.per_cell("sweep_x", p, ndim=ndim)
        assert wave == flops.per_cell("wave_max", p, ndim=ndim)
        if ndim == 2:
            assert _per_cell(O, I, "sweep_y", p, 16, 32, 1)[0] + prelax == flops.per_cell("sweep_y", p, ndim=ndim)
        for P in (1, 2, 3):
            ph = p.replace(p_policy=1, p_fixed=P)
            heat, Ph = _per_cell(O, I, "heat", ph, 32, ny, 0)
            assert Ph == P
            # the 2D operator has ny + 1 rows of y faces, so the count per cell
            # is a + b / ny: take the large-ny limit a from ny = 16 and 64
            if ndim == 2:
                heat64 = _per_cell(O, I, "heat", ph, 32, 64, 0)[0]
                heat = heat64 + (heat64 - heat) * 16 / 48
            assert round(heat + trelax, 6) == flops.per_cell("heat", ph, P, ndim=ndim), (lim, kexp, P, heat)
            pv = p.replace(mu=(1e12, 1e11), p_max=P)
            visc, Pv = _per_cell(O, I, "viscous_x", pv, 32, ny, 0)
            assert Pv == P
            expect_x = visc + (prelax if ndim == 1 else 0.0)
            assert expect_x == flops.per_cell("viscous_x", pv, P, ndim=ndim)
            if ndim == 2:
                assert _per_cell(O, I, "viscous_y", pv, 16, 32, 1)[0] + prelax == flops.per_cell(
                    "viscous_y", pv, P, ndim=ndim)
