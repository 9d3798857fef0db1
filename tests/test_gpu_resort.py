"""Plasma re-sort by cell (Sec. 3.1: particle data kept sorted; a stable counting sort of the
plasma slice by cell every m slices, hq_grid_desc.resort_every).

The re-sort only permutes the plasma slice, so a sweep with it must meet the oracle (which never
sorts) at the bars of the unsorted sweeps: FP64 every field and slice within 10x the oracle's
own rounding floor and the plasma state, put back in initial order through `origin`, within
30x; FP32 the reduced blowout's on-axis Ez <= 1e-4 over the first period and Ez <= 1e-3 over the
bucket, with the same removed-particle count as without the re-sort.  Also checked: the stored
order is sorted by cell, stably, `origin` is a permutation, and the adjoint refuses the re-sort.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2109_10277_gb300 import inputs as I
from test_gpu_parity import assert_fp64_sweep, plasma_perm, reordered, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hq():
    from paper_2109_10277_gb300 import hq as _hq
    _hq.load()
    torch.cuda.set_device(0)
    return _hq


def sweep_gpu(hq, g, beams, precision, fields):
    grid = hq.Grid(g, precision=precision)
    out = grid.alloc_out(fields)
    grid.sweep([hq.Beam(b) for b in beams], out=out)
    removed = grid.sync()
    st = grid.plasma_state()
    raw = grid.plasma_state(initial_order=False)
    grid.close()
    return out, st, raw, removed


def cells(g, st):
    dx = (g["xmax"] - g["xmin"]) / g["nx"]
    dy = (g["ymax"] - g["ymin"]) / g["ny"]
    # the library's arithmetic: (x - xmin) times the reciprocal cell size, floored
    ix = torch.clamp(torch.floor((st["x"].cpu() - g["xmin"]) * (1.0 / dx)), 0, g["nx"] - 1)
    iy = torch.clamp(torch.floor((st["y"].cpu() - g["ymin"]) * (1.0 / dy)), 0, g["ny"] - 1)
    return (iy * g["nx"] + ix).to(torch.int64)


@pytest.mark.parametrize("m", [1, 5])
def test_resort_fp64_matches_oracle(hq, m):
    g = dict(I.grid_params("linear64"), shape_order=2, resort_every=m)
    # n_b = 2: hundreds of plasma particles change cell from slice 25 on (up to 5 cells)
    beams = [I.random_beam(100_000, 0.5, 0.5, 1.0, 2.0, energy_spread=1e-3)]
    sp = O.GridSpec(**{k: v for k, v in g.items() if k != "resort_every"})
    ref = O.sweep(sp, [O.as_beam(b) for b in beams])
    ref_perm = O.sweep(sp, [O.as_beam(b) for b in reordered(beams)], plasma_perm=plasma_perm(g),
                       reverse_ion_order=True, deposit_noise=2.0 ** -52)
    out, st, raw, removed = sweep_gpu(hq, g, beams, "fp64", O.FIELD_NAMES)
    assert_fp64_sweep(out, ref, ref_perm, O.FIELD_NAMES, spec=sp)
    for k in ("x", "y", "psi", "ux", "uy"):
        d = float((st[k].double().cpu() - ref.plasma[k]).abs().max())
        f = float((ref_perm.plasma[k] - ref.plasma[k]).abs().max())
        assert d <= max(1e-12, 30 * f), (k, d, f)
    assert removed == ref.removed
    # the stored order is a permutation of the initial placement, and not the identity
    org = raw["origin"].cpu()
    assert torch.equal(torch.sort(org).values, torch.arange(org.numel()))
    assert not torch.equal(org, torch.arange(org.numel()))


def test_resort_orders_by_cell(hq):
    """Right after a re-sort (hq_advance_slice(i) with i % m == 0) the stored plasma is ordered
    by cell; between re-sorts the order is kept (and goes stale as particles move)."""
    g = dict(I.grid_params("linear64"), shape_order=1, resort_every=3, nzeta=64)
    beam = hq.Beam(I.random_beam(50_000, 0.5, 0.5, 1.0, 2.0, energy_spread=1e-3))
    grid = hq.Grid(g, precision="fp64")
    for i in range(40):
        grid.advance(i)
        if i > 0 and i % 3 == 0:
            raw = grid.plasma_state(initial_order=False)
            key = cells(g, raw)
            assert bool((key[1:] >= key[:-1]).all()), i
        grid.beam_deposit([beam], i)
        grid.solve(i)
    org = raw["origin"].cpu()
    assert torch.equal(torch.sort(org).values, torch.arange(org.numel()))
    assert not torch.equal(org, torch.arange(org.numel()))
    grid.close()


def test_resort_is_stable_at_slice_zero_order(hq):
    """One re-sort of the unperturbed placement (slice 1, before any particle left its cell)
    must keep every particle where it is: the sort is stable and the placement already sorted."""
    g = dict(nx=32, ny=32, nzeta=2, xmin=-4.0, xmax=4.0, ymin=-4.0, ymax=4.0, zeta_min=-1.0, zeta_max=1.0,
             shape_order=1, ppc_x=2, ppc_y=2, n_pc_iter=1, pc_mix=0.05, psi_guard=0.02, resort_every=1)
    grid = hq.Grid(g, precision="fp64")
    grid.sweep([])
    raw = grid.plasma_state(initial_order=False)
    grid.close()
    # 2 x 2 particles per cell: cell-row-major with sub-cells, sorted by cell they stay in order
    assert torch.equal(raw["origin"].cpu(), torch.arange(32 * 32 * 4))


def test_resort_fp32_blowout_reduced(hq):
    g = dict(I.scaled_grid(I.grid_params("blowout512"), 128, 128, 256), resort_every=8)
    beams = I.workload_beams("blowout512", n_driver=200_000)
    sp = O.GridSpec(**{k: v for k, v in g.items() if k != "resort_every"})
    ref = O.sweep(sp, [O.as_beam(b) for b in beams], record=("ez", "psi"))
    out, st, raw, removed = sweep_gpu(hq, g, beams, "fp32", ("ez", "psi"))
    g0 = dict(g, resort_every=0)
    out0, st0, _, removed0 = sweep_gpu(hq, g0, beams, "fp32", ("ez", "psi"))
    zc = sp.zeta_max - (np.arange(sp.nzeta) + 0.5) * sp.dzeta
    first = torch.as_tensor(zc >= -2 * math.pi)
    bucket = torch.as_tensor(zc >= -7.0)
    c = sp.nx // 2
    e_axis = rel(out["ez"][first, c, c], ref.fields["ez"][first, c, c])
    e_bucket = rel(out["ez"][bucket], ref.fields["ez"][bucket])
    e_psi = rel(out["psi"][bucket], ref.fields["psi"][bucket])
    d_unsorted = rel(out["ez"][bucket], out0["ez"][bucket])
    print(f"fp32 blowout128 re-sorted every 8: on-axis Ez {e_axis:.2e}, bucket Ez {e_bucket:.2e}, psi {e_psi:.2e}, "
          f"vs unsorted {d_unsorted:.2e}, removed {removed} / {removed0} / oracle {ref.removed}")
    assert e_axis <= 1e-4 and e_bucket <= 1e-3, (e_axis, e_bucket)
    # against the unsorted FP32 sweep: the same removals (up to the FP32 atomics' run-to-run
    # noise) and the same plasma positions
    assert abs(removed - removed0) <= 2, (removed, removed0)
    dpos = max(rel(st[k], st0[k]) for k in ("x", "y"))
    assert dpos <= 1e-4, dpos


def test_resort_refuses_the_adjoint(hq):
    g = dict(nx=32, ny=32, nzeta=8, xmin=-4.0, xmax=4.0, ymin=-4.0, ymax=4.0, zeta_min=-1.0, zeta_max=1.0,
             shape_order=1, n_pc_iter=2, pc_mix=0.05, psi_guard=0.02, resort_every=4)
    grid = hq.Grid(g, precision="fp64")
    sums = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(hq.HQError) as e:
        grid.forward_ckpt([hq.Beam(I.random_beam(1000, 0.5, 0.5, 0.5, 0.5))], -1, sums, 4)
    assert e.value.status == 7
    grid.close()
