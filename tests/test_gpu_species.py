"""Plasma species through the C ABI (hq_grid_desc.species; Sec. 6: plasmas of several species
and profiles, ion motion) against the FP64 oracle with the same species.

Bars as for the single-species sweeps: FP64 every field and slice within 10x the oracle's own
rounding floor, every species' plasma state within 30x; FP32/bf16x3 on-axis Ez <= 1e-4 and the
recorded fields <= 1e-3 rel-L2.  Cases: electrons with mobile ions of mass 100 m_e and different
particles per cell (no immobile background: the species neutralize each other), the electrons
split into two half-density species with different profiles, and a positron plasma.  Also the
refusals (explicit solver, re-sort, checkpointed forward).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2109_10277_gb300 import inputs as I
from test_gpu_parity import assert_fp64_sweep, rel, reordered

pytestmark = pytest.mark.gpu

ION = dict(charge=1.0, mass=100.0, n0_scale=1.0, ppc_x=2, ppc_y=1, neutralize=False)
ELE = dict(charge=-1.0, mass=1.0, n0_scale=1.0, ppc_x=1, ppc_y=1, neutralize=False)
CASES = {
    "electrons+ions": [ELE, ION],
    "split electrons": [dict(ELE, n0_scale=0.5, neutralize=True),
                        dict(ELE, n0_scale=0.5, neutralize=True, ppc_x=2, ppc_y=2,
                             radial_profile=[1.0, 1.0, 0.8, 0.3, 0.0], profile_rmax=6.0)],
    "positrons": [dict(charge=1.0, mass=1.0, n0_scale=1.0, ppc_x=1, ppc_y=1, neutralize=True)],
}


@pytest.fixture(scope="module")
def hq():
    from paper_2109_10277_gb300 import hq as _hq
    _hq.load()
    torch.cuda.set_device(0)
    return _hq


def spec_of(g, species):
    sp = tuple(O.Species(s["charge"], s["mass"], s["n0_scale"], s["ppc_x"], s["ppc_y"], s.get("radial_profile"),
                         s.get("profile_rmax", 0.0), bool(s["neutralize"])) for s in species)
    return O.GridSpec(**{k: v for k, v in g.items() if k != "species"}, species=sp)


def run(hq, g, beams, precision, fields):
    grid = hq.Grid(g, precision=precision)
    out = grid.alloc_out(fields)
    grid.sweep([hq.Beam(b) for b in beams], out=out)
    removed = grid.sync()
    st = grid.plasma_state()
    grid.close()
    return out, st, removed


def species_blocks(g, st):
    out, off = [], 0
    for s in g["species"]:
        n = g["nx"] * g["ny"] * s["ppc_x"] * s["ppc_y"]
        out.append({k: v[off:off + n] for k, v in st.items()})
        off += n
    assert off == st["x"].numel()
    return out


@pytest.mark.parametrize("case", list(CASES))
def test_species_fp64_matches_oracle(hq, case):
    g = dict(nx=40, ny=40, nzeta=32, xmin=-5.0, xmax=5.0, ymin=-5.0, ymax=5.0, zeta_min=-6.0, zeta_max=2.0,
             shape_order=2, n_pc_iter=3, pc_mix=0.05, psi_guard=0.02, species=CASES[case])
    beams = [I.random_beam(20_000, 0.5, 0.5, 0.8, 1.0, energy_spread=1e-3)]
    sp = spec_of(g, CASES[case])
    ref = O.sweep(sp, [O.as_beam(b) for b in beams])
    perm = torch.as_tensor(np.random.default_rng(1).permutation(
        g["nx"] * g["ny"] * CASES[case][0]["ppc_x"] * CASES[case][0]["ppc_y"]))
    ref_perm = O.sweep(sp, [O.as_beam(b) for b in reordered(beams)], plasma_perm=perm,
                       reverse_ion_order=True, deposit_noise=2.0 ** -52)
    out, st, removed = run(hq, g, beams, "fp64", O.FIELD_NAMES)
    assert_fp64_sweep(out, ref, ref_perm, O.FIELD_NAMES, spec=sp)
    blocks = species_blocks(g, st)
    for k_sp, (blk, a, b) in enumerate(zip(blocks, ref.plasma_species, ref_perm.plasma_species)):
        for k in ("x", "y", "psi", "ux", "uy"):
            d = float((blk[k].double().cpu() - a[k]).abs().max())
            f = float((b[k] - a[k]).abs().max())
            assert d <= max(1e-12, 30 * f), (case, k_sp, k, d, f)
    assert removed == ref.removed


@pytest.mark.parametrize("case", ["electrons+ions", "positrons"])
def test_species_fp32_matches_oracle(hq, case):
    g = dict(I.grid_params("linear64"), species=CASES[case])
    beams = I.workload_beams("linear64")
    sp = spec_of(g, CASES[case])
    rec = ("ez", "psi", "bx", "rho")
    ref = O.sweep(sp, [O.as_beam(b) for b in beams], record=rec)
    out, _, _ = run(hq, g, beams, "fp32", rec)
    errs = {k: rel(out[k], ref.fields[k]) for k in rec}
    axis = rel(out["ez"][:, 32, 32], ref.fields["ez"][:, 32, 32])
    print(f"fp32 {case}: on-axis Ez {axis:.2e}, rel-L2 {({k: f'{v:.1e}' for k, v in errs.items()})}")
    assert axis <= 1e-4 and max(errs.values()) <= 1e-3, (errs, axis)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_species_explicit_solver(hq, precision):
    """The explicit B_perp solver on electrons with mobile ions (each species' sources, the shift
    sum q^2 n0 / M) against the oracle: FP64 at the floor-based bars, FP32 at the FP32 bars."""
    g = dict(nx=64, ny=64, nzeta=32, xmin=-6.0, xmax=6.0, ymin=-6.0, ymax=6.0, zeta_min=-4.0, zeta_max=2.0,
             shape_order=1, n_pc_iter=4, pc_mix=0.05, psi_guard=0.02, bperp_solver="explicit",
             species=CASES["electrons+ions"])
    beams = [I.random_beam(20_000, 0.5, 0.5, 0.8, 0.5, energy_spread=1e-3)]
    sp = spec_of(g, CASES["electrons+ions"])
    ref = O.sweep(sp, [O.as_beam(b) for b in beams])
    out, _, _ = run(hq, g, beams, precision, O.FIELD_NAMES)
    if precision == "fp64":
        perm = torch.as_tensor(np.random.default_rng(2).permutation(g["nx"] * g["ny"]))
        ref_perm = O.sweep(sp, [O.as_beam(b) for b in reordered(beams)], plasma_perm=perm,
                           reverse_ion_order=True, deposit_noise=2.0 ** -52)
        assert_fp64_sweep(out, ref, ref_perm, O.FIELD_NAMES, spec=sp)
    else:
        errs = {k: rel(out[k], ref.fields[k]) for k in ("ez", "psi", "bx", "by")}
        axis = rel(out["ez"][:, 32, 32], ref.fields["ez"][:, 32, 32])
        print(f"fp32 explicit electrons+ions: on-axis Ez {axis:.2e}, rel-L2 {errs}")
        assert axis <= 1e-4 and max(errs.values()) <= 1e-3, (errs, axis)


def test_species_initial_placement(hq):
    """Each species block of the slice starts where the oracle places that species."""
    g = dict(nx=16, ny=16, nzeta=1, xmin=-2.0, xmax=2.0, ymin=-2.0, ymax=2.0, zeta_min=-1.0, zeta_max=0.0,
             shape_order=1, n_pc_iter=1, species=CASES["split electrons"])
    grid = hq.Grid(g, precision="fp64")
    st = grid.plasma_state()
    grid.close()
    sp = spec_of(g, CASES["split electrons"])
    for blk, s in zip(species_blocks(g, st), sp.species):
        ref = O.plasma_init(sp, species=s)
        for k in ("x", "y", "w"):
            assert torch.allclose(blk[k].cpu(), ref[k], rtol=1e-15, atol=1e-15), k


def test_species_refusals(hq):
    g = dict(nx=16, ny=16, nzeta=4, xmin=-2.0, xmax=2.0, ymin=-2.0, ymax=2.0, zeta_min=-1.0, zeta_max=0.0,
             shape_order=1, n_pc_iter=2, species=CASES["electrons+ions"])
    with pytest.raises(hq.HQError) as e:
        hq.Grid(dict(g, resort_every=4), precision="fp64")
    assert e.value.status == 7
    with pytest.raises(hq.HQError) as e:
        hq.Grid(dict(g, species=[dict(ELE, mass=0.0)]), precision="fp64")
    assert e.value.status == 1
    grid = hq.Grid(g, precision="fp64")
    sums = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(hq.HQError) as e:
        grid.forward_ckpt([hq.Beam(I.random_beam(1000, 0.5, 0.5, 0.5, 0.5))], -1, sums, 2)
    assert e.value.status == 7
    grid.close()
