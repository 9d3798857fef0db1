"""Deterministic FP64 mode (hq_grid_desc.deterministic): the plasma and beam deposits and the
witness sums accumulate in 64-bit fixed point with integer atomics, so the order in which the
GPU performs the additions no longer shows in the result.

Checked: two sweeps on separate grids give bitwise identical fields on every slice, plasma
state, witness sums and pushed beams; the mode meets the oracle at the FP64 bars of the atomic
path (10x the oracle's own rounding floor per field and slice, 30x for the plasma state); an
out-of-range contribution is reported as HQ_ERR_NUMERIC by hq_sync; with the explicit solver
too (its source deposits in fixed point, its dot products in a fixed order) two runs agree bit
for bit; FP32 and the checkpointed forward refuse the mode.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2109_10277_gb300 import inputs as I
from test_gpu_parity import assert_fp64_sweep, plasma_perm, reordered

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hq():
    from paper_2109_10277_gb300 import hq as _hq
    _hq.load()
    torch.cuda.set_device(0)
    return _hq


def setup():
    g = I.scaled_grid(I.grid_params("adjoint256"), 48, 48, 48, deterministic=1)
    beams = I.workload_beams("adjoint256", grid=g)
    return g, beams


def run(hq, g, beams, dt=5.0):
    grid = hq.Grid(g, precision="fp64")
    out = grid.alloc_out(O.FIELD_NAMES)
    hb = [hq.Beam(b) for b in beams]
    sums = torch.zeros(3, dtype=torch.float64, device="cuda")
    grid.sweep(hb, dt=dt, out=out, witness=1, witness_sums=sums)
    removed = grid.sync()
    st = grid.plasma_state()
    grid.close()
    return out, st, removed, [{k: b.t[k].clone() for k in b.t} for b in hb], sums


def test_deterministic_sweeps_are_bitwise_identical(hq):
    g, beams = setup()
    a = run(hq, g, beams)
    b = run(hq, g, beams)
    for k in O.FIELD_NAMES:
        assert torch.equal(a[0][k], b[0][k]), k
    for k in ("x", "y", "psi", "ux", "uy", "w", "alive"):
        assert torch.equal(a[1][k], b[1][k]), k
    assert a[2] == b[2]
    for ba, bb in zip(a[3], b[3]):
        for k in ba:
            assert torch.equal(ba[k], bb[k]), k
    assert torch.equal(a[4], b[4])
    # the atomic FP64 path on the same input, for the record: its two runs differ in the last bits
    g0 = dict(g, deterministic=0)
    c, d = run(hq, g0, beams), run(hq, g0, beams)
    diff = sum(int((c[0][k] != d[0][k]).sum()) for k in O.FIELD_NAMES)
    print(f"atomic FP64 path: {diff} field values differ between two runs; deterministic mode: 0")


def test_deterministic_explicit_solver(hq):
    """The explicit B_perp solver in the deterministic mode (its source deposits in fixed point, its
    dot products summed in a fixed order): two runs bitwise equal, and the oracle's bars."""
    g, beams = setup()
    g = dict(g, bperp_solver="explicit", n_pc_iter=4)
    a = run(hq, g, beams)
    b = run(hq, g, beams)
    for k in O.FIELD_NAMES:
        assert torch.equal(a[0][k], b[0][k]), k
    for ba, bb in zip(a[3], b[3]):
        for k in ba:
            assert torch.equal(ba[k], bb[k]), k
    sp = O.GridSpec(**{k: v for k, v in g.items() if k != "deterministic"})
    ref = O.sweep(sp, [O.as_beam(x) for x in beams], dt=5.0, witness=(1,))
    ref_perm = O.sweep(sp, [O.as_beam(x) for x in reordered(beams)], dt=5.0, witness=(1,),
                       plasma_perm=plasma_perm(g), reverse_ion_order=True, deposit_noise=2.0 ** -52)
    assert_fp64_sweep(a[0], ref, ref_perm, O.FIELD_NAMES, spec=sp)


def test_deterministic_matches_oracle(hq):
    g, beams = setup()
    sp = O.GridSpec(**{k: v for k, v in g.items() if k != "deterministic"})
    ref = O.sweep(sp, [O.as_beam(b) for b in beams], dt=5.0, witness=(1,))
    ref_perm = O.sweep(sp, [O.as_beam(b) for b in reordered(beams)], dt=5.0, witness=(1,),
                       plasma_perm=plasma_perm(g), reverse_ion_order=True, deposit_noise=2.0 ** -52)
    out, st, removed, hb, sums = run(hq, g, beams)
    assert_fp64_sweep(out, ref, ref_perm, O.FIELD_NAMES, spec=sp)
    for k in ("x", "y", "psi", "ux", "uy"):
        d = float((st[k].double().cpu() - ref.plasma[k]).abs().max())
        f = float((ref_perm.plasma[k] - ref.plasma[k]).abs().max())
        assert d <= max(1e-12, 30 * f), (k, d, f)
    assert removed == ref.removed
    s = sums.cpu()
    for j in range(3):
        r, rp = float(ref.witness[1][j]), float(ref_perm.witness[1][j])
        assert abs(float(s[j]) - r) <= max(1e-12 * abs(r), 30 * abs(rp - r)), j
    perm = [np.random.default_rng(0).permutation(len(b["x"])) for b in beams]
    for bi in range(2):
        inv = np.argsort(perm[bi])
        for k in ("x", "y", "zeta", "ux", "uy", "uz"):
            a = hb[bi][k].cpu()
            b = ref.beams[bi][k]
            c = ref_perm.beams[bi][k][inv]
            scale = float((b - b.mean()).abs().max()) + 1e-30
            dd, ff = float((a - b).abs().max()) / scale, float((c - b).abs().max()) / scale
            assert dd <= max(1e-12, 30 * ff), (bi, k, dd, ff)


def test_deterministic_overflow_is_reported(hq):
    """A beam weight that takes a deposit contribution beyond the fixed-point range (2^31): the
    contribution is dropped and hq_sync reports HQ_ERR_NUMERIC (the grid stays usable)."""
    g, beams = setup()
    bad = dict(beams[0])
    bad["w"] = np.full_like(bad["w"], 1e12)
    grid = hq.Grid(g, precision="fp64")
    grid.sweep([hq.Beam(bad)])
    with pytest.raises(hq.HQError) as e:
        grid.sync()
    assert e.value.status == 4
    grid.sweep([hq.Beam(beams[0])])
    assert grid.sync() >= 0
    grid.close()


def test_deterministic_refusals(hq):
    g, beams = setup()
    with pytest.raises(hq.HQError) as e:
        hq.Grid(g, precision="fp32")
    assert e.value.status == 7
    grid = hq.Grid(g, precision="fp64")
    sums = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(hq.HQError) as e:
        grid.forward_ckpt([hq.Beam(beams[0])], -1, sums, 8)
    assert e.value.status == 7
    grid.close()
