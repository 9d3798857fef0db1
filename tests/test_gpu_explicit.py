"""The explicit B_perp solver (Sec. 3.2: a Helmholtz-like equation in chi, solved here by
preconditioned conjugate gradients with a shifted DST-I) through the C ABI, against the
FP64 oracle's explicit solver with the same iteration count.

Bars as for the predictor-corrector sweeps: FP64 within 10x the oracle's own rounding floor
(reordered particles, one-ulp deposit noise) of each field's peak; FP32/bf16x3: on-axis Ez
<= 1e-4 and every recorded field <= 1e-3 rel-L2.  Also: the adjoint refuses this solver.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2109_10277_gb300 import inputs as I
from test_gpu_parity import assert_fp64_sweep, plasma_perm, reordered, rel, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hq():
    from paper_2109_10277_gb300 import hq as _hq
    _hq.load()
    torch.cuda.set_device(0)
    return _hq


def grid(n, nz, order=1, **kw):
    g = dict(nx=n, ny=n, nzeta=nz, xmin=-6.0, xmax=6.0, ymin=-6.0, ymax=6.0, zeta_min=-7.0, zeta_max=5.0,
             shape_order=order, n_pc_iter=4, pc_mix=0.05, psi_guard=0.02, bperp_solver="explicit")
    g.update(kw)
    return g


@pytest.mark.parametrize("order", [1, 2])
def test_explicit_fp64_matches_oracle(hq, order):
    g = grid(32, 24, order)
    beams = [I.random_beam(20_000, 0.5, 0.5, 1.0, 0.5, energy_spread=1e-3)]
    sp = O.GridSpec(**g)
    ref = O.sweep(sp, [O.as_beam(b) for b in beams])
    ref_perm = O.sweep(sp, [O.as_beam(b) for b in reordered(beams)], plasma_perm=plasma_perm(g),
                       reverse_ion_order=True, deposit_noise=2.0 ** -52)
    out, st, removed, _, _ = run_gpu(hq, g, beams, "fp64")
    assert_fp64_sweep(out, ref, ref_perm, O.FIELD_NAMES, spec=sp)
    assert removed == ref.removed


@pytest.mark.parametrize("n,nz", [(64, 64), (256, 96)])
def test_explicit_fp32_matches_oracle(hq, n, nz):
    """64^2 (streamed solve) and 256^2 (resident fold-matrix solve with the shifted table)."""
    g = grid(n, nz)
    beams = [I.random_beam(100_000, 0.4, 0.4, 1.0, 0.5, energy_spread=1e-3)]
    rec = ("ez", "psi", "bx", "by")
    ref = O.sweep(O.GridSpec(**g), [O.as_beam(b) for b in beams], record=rec)
    out, _, _, _, _ = run_gpu(hq, g, beams, "fp32", fields=rec)
    c = n // 2
    axis = rel(out["ez"][:, c, c], ref.fields["ez"][:, c, c])
    errs = {k: rel(out[k], ref.fields[k]) for k in rec}
    print(f"explicit fp32 {n}^2: on-axis Ez {axis:.2e}, rel-L2 {({k: f'{v:.1e}' for k, v in errs.items()})}")
    assert axis <= 1e-4 and max(errs.values()) <= 1e-3, (axis, errs)


def test_explicit_refuses_the_adjoint(hq):
    g = grid(32, 8)
    grid_ = hq.Grid(g, precision="fp64")
    sums = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(hq.HQError) as e:
        grid_.forward_ckpt([hq.Beam(I.random_beam(1000, 0.5, 0.5, 1.0, 0.5))], -1, sums, 4)
    assert e.value.status == 7
    grid_.close()
