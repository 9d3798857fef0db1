"""Failure detection on the GPU without faulting it (host-made failures only).

  * a beam with one non-finite weight: the non-finite value reaches the field solve, the
    kernels flag it in the grid's device status word and hq_sync returns HQ_ERR_NUMERIC;
    a new grid then runs a clean sweep;
  * HQ_FAULT_BARRIER=1 makes the first grid barrier of the tensor-core solve wait for one
    CTA more than the launch has: the bounded wait runs out after about two seconds, every
    CTA leaves (nothing is in flight at that barrier: each CTA has drained its TMA loads
    and MMAs), hq_sync returns HQ_ERR_TIMEOUT, and a solve on another grid afterwards is
    correct, so the context stayed usable.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2109_10277_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hq():
    from paper_2109_10277_gb300 import hq as _hq
    _hq.load()
    torch.cuda.set_device(0)
    return _hq


def small_grid():
    return dict(nx=32, ny=32, nzeta=16, xmin=-4.0, xmax=4.0, ymin=-4.0, ymax=4.0, zeta_min=-3.0, zeta_max=3.0,
                shape_order=1, n_pc_iter=2, pc_mix=0.05, psi_guard=0.02)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_nonfinite_beam_weight_is_reported(hq, precision):
    g = small_grid()
    b = I.random_beam(2000, 0.5, 0.5, 0.8, 0.2)
    b["w"] = np.array(b["w"])
    b["w"][123] = float("nan")
    grid = hq.Grid(g, precision=precision)
    out = grid.alloc_out(("ez",))
    grid.sweep([hq.Beam(b)], out=out)
    with pytest.raises(hq.HQError) as e:
        grid.sync()
    assert e.value.status == 4, str(e.value)   # HQ_ERR_NUMERIC
    grid.sync()                                  # the flag was cleared by the report
    grid.close()
    b["w"][123] = b["w"][0]
    grid = hq.Grid(g, precision=precision)
    out = grid.alloc_out(("ez",))
    grid.sweep([hq.Beam(b)], out=out)
    grid.sync()
    assert torch.isfinite(out["ez"]).all() and float(out["ez"].abs().max()) > 0
    grid.close()


def test_solve_barrier_timeout_is_reported(hq, monkeypatch):
    g = dict(nx=128, ny=128, nzeta=4, xmin=-4.0, xmax=4.0, ymin=-4.0, ymax=4.0, zeta_min=0.0, zeta_max=1.0)
    gen = torch.Generator(device="cuda").manual_seed(5)
    src = torch.randn(2, 128, 128, dtype=torch.float32, device="cuda", generator=gen)
    monkeypatch.setenv("HQ_FAULT_BARRIER", "1")
    bad = hq.Grid(g, precision="fp32")
    monkeypatch.delenv("HQ_FAULT_BARRIER")
    bad.poisson_solve(src)
    with pytest.raises(hq.HQError) as e:
        bad.sync()
    assert e.value.status == 5, str(e.value)    # HQ_ERR_TIMEOUT
    bad.close()
    good = hq.Grid(g, precision="fp32")
    got = good.poisson_solve(src)
    good.sync()
    sp = O.GridSpec(**dict(g, nzeta=4))
    for r in range(2):
        ref = O.poisson_solve(sp, src[r].double().cpu())
        err = float(torch.linalg.norm(got[r].double().cpu() - ref) / torch.linalg.norm(ref))
        assert err <= 3e-5, err
    good.close()
