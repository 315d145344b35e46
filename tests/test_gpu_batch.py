"""Batches (dim_batch_*): many independent grids of uneven sizes advanced by
one persistent launch per step, replayed from a CUDA graph.

- every instance of the batch equals the same instance advanced alone by the
  single-grid FP32-bulk path (the same per-cell arithmetic);
- every instance is within the FP32-bulk tolerance of the FP64 oracle;
- the tile-shape variant the autotuner picks changes the work distribution,
  not the results."""
import numpy as np
import pytest

from test_gpu_fp32 import TOL32, rel_l1_32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch

    assert torch.cuda.is_available()
    from paper_2106_00282_gb300 import build, inputs as I

    build.build()
    params, grids, prims = I.batch(ninst=7, seed=7, sizes=(16, 24, 40, 64))
    return torch, I, params, grids, prims


def _rel(a, b):
    return np.abs(a - b).reshape(8, -1).sum(1) / np.maximum(np.abs(b).reshape(8, -1).sum(1), 1e-300)


def test_batch_equals_single_grids(setup, O):
    torch, I, params, grids, prims = setup
    from paper_2106_00282_gb300.api import Batch, Solver

    B = Batch(params, grids)
    U = B.from_primitive(B.pack_primitive(prims))
    B.step(U, 30)
    flags, anyf = B.status()
    assert anyf & 3 == 0, flags
    for i, (nx, ny, dx, dy) in enumerate(grids):
        s = Solver(params, nx, ny, dx, dy)
        Ui = s.from_primitive(torch.from_numpy(prims[i]).cuda())
        s.step(Ui, 30)
        e = _rel(B.state(U, i).cpu().numpy(), Ui.cpu().numpy())
        print(f"[batch] instance {i} {nx}x{ny}: batched vs alone {e.max():.2e}")
        assert np.all(e <= 1e-12), (i, e)
        s.close()
    B.close()


def test_batch_against_oracle(setup, O):
    torch, I, params, grids, prims = setup
    from paper_2106_00282_gb300.api import Batch

    B = Batch(params, grids)
    U = B.from_primitive(B.pack_primitive(prims))
    B.step(U, 40)
    for i, (nx, ny, dx, dy) in enumerate(grids):
        wl = I.Workload("b", nx, ny, dx, dy, params, prims[i])
        Uo = O.step(params, O.from_primitive(params, prims[i]), dx, dy, 40)[0]
        e = rel_l1_32(B.state(U, i).cpu().numpy(), Uo, O, wl, params)
        print(f"[batch] instance {i} {nx}x{ny}: vs FP64 oracle {e.max():.2e}")
        assert np.all(e <= TOL32), (i, e)
    B.close()


def test_batch_autotune_keeps_results(setup):
    torch, I, params, grids, prims = setup
    from paper_2106_00282_gb300.api import Batch

    B = Batch(params, grids)
    P = B.pack_primitive(prims)
    U0 = B.from_primitive(P)
    U1 = U0.clone()
    B.step(U0, 12)
    cfg = B.autotune(U1)
    assert len(cfg) == 6 and cfg[1] > 0 and cfg[2] * cfg[3] == 256 and cfg[4] * cfg[5] == 256
    B.step(U1, 12)
    torch.cuda.synchronize()
    assert torch.equal(U0, U1), cfg
    B.close()
