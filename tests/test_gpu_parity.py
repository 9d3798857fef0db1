"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars (written here, derived in the design doc):
  * FP64 path: rel-L2 <= 1e-12 per output field per slice (the only differences
    are the order of atomic additions and FFT vs matrix DST rounding);
  * FP32/bf16x3 path: each bf16x3 product carries ~2^-17 relative error, so a
    4-product Dirichlet solve is good to a few 1e-5 (rel-L2); sweeps are checked
    with the per-config bounds in the tests below;
  * integer work (beam binning) is bit-exact: the CSR offsets and the set of
    particles per slice.
"""
import math

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


def rel_per_slice(a, b, floor_frac=1e-6):
    """max over slices of ||a_i - b_i|| / max(||b_i||, floor_frac * max_i ||b_i||)."""
    a = a.double().cpu()
    b = b.double().cpu()
    nb = torch.linalg.norm(b.reshape(b.shape[0], -1), dim=1)
    na = torch.linalg.norm((a - b).reshape(b.shape[0], -1), dim=1)
    fl = floor_frac * float(nb.max()) + 1e-300
    return float((na / torch.clamp(nb, min=fl)).max())


def rel(a, b):
    a = a.double().cpu()
    b = b.double().cpu()
    return float(torch.linalg.norm(a - b) / (torch.linalg.norm(b) + 1e-300))


def run_gpu(hq, g, beams, precision, fields=O.FIELD_NAMES, dt=0.0, witness=-1):
    grid = hq.Grid(g, precision=precision)
    out = grid.alloc_out(fields)
    hb = [hq.Beam(b) for b in beams]
    sums = torch.zeros(3, dtype=torch.float64, device="cuda") if witness >= 0 else None
    grid.sweep(hb, dt=dt, out=out, witness=witness, witness_sums=sums)
    removed = grid.sync()
    st = grid.plasma_state()
    grid.close()
    return out, st, removed, hb, sums


# ---------------------------------------------------------------- Poisson solver

@pytest.mark.parametrize("nx,ny", [(64, 64), (48, 40), (32, 128)])
def test_poisson_fp64(hq, nx, ny):
    g = dict(nx=nx, ny=ny, nzeta=4, xmin=-3.0, xmax=3.5, ymin=-2.0, ymax=2.0, zeta_min=0.0, zeta_max=1.0)
    grid = hq.Grid(g, precision="fp64")
    gen = torch.Generator().manual_seed(nx * 7 + ny)
    src = torch.randn(3, ny, nx, generator=gen, dtype=torch.float64)
    got = grid.poisson_solve(src.cuda()).cpu()
    sp = O.GridSpec(**g)
    for r in range(3):
        assert rel(got[r], O.poisson_solve(sp, src[r])) <= 1e-12
    grid.close()


@pytest.mark.parametrize("nx,ny", [(64, 64), (96, 80), (256, 256), (512, 512)])
def test_poisson_bf16x3(hq, nx, ny):
    g = dict(nx=nx, ny=ny, nzeta=4, xmin=-8.0, xmax=8.0, ymin=-7.0, ymax=7.5, zeta_min=0.0, zeta_max=1.0)
    grid = hq.Grid(g, precision="fp32")
    gen = torch.Generator().manual_seed(nx + 3 * ny)
    # smooth + rough parts, like charge densities near a sheath
    xs = torch.linspace(-1, 1, nx, dtype=torch.float64)
    ys = torch.linspace(-1, 1, ny, dtype=torch.float64)
    smooth = torch.exp(-(xs[None, :] ** 2 + ys[:, None] ** 2) / 0.1)
    src = torch.stack([smooth, torch.randn(ny, nx, generator=gen, dtype=torch.float64),
                       smooth * torch.randn(ny, nx, generator=gen, dtype=torch.float64)])
    got = grid.poisson_solve(src.float().cuda()).cpu()
    sp = O.GridSpec(**g)
    errs = [rel(got[r], O.poisson_solve(sp, src[r].float().double())) for r in range(3)]
    print("bf16x3 poisson rel-L2", nx, ny, errs)
    assert max(errs) <= 3e-5, errs
    grid.close()


# ---------------------------------------------------------------- full sweeps, FP64

def test_sweep_fp64_linear64_full_size(hq):
    """The 64^2 x 64, 1e5-particle workload at full size, every field, every slice."""
    g = I.grid_params("linear64")
    beams = I.workload_beams("linear64")
    ref = O.sweep(O.GridSpec(**g), [O.as_beam(b) for b in beams])
    out, st, removed, _, _ = run_gpu(hq, g, beams, "fp64")
    for k in O.FIELD_NAMES:
        e = rel_per_slice(out[k], ref.fields[k])
        assert e <= 1e-12, (k, e)
    for k in ("x", "y", "psi", "ux", "uy"):
        assert rel(st[k], ref.plasma[k]) <= 1e-12, k
    assert removed == ref.removed == 0


@pytest.mark.parametrize("order,ppc,profile", [(0, (1, 1), False), (1, (2, 1), True), (2, (1, 1), False),
                                               (3, (2, 2), True)])
def test_sweep_fp64_ragged(hq, order, ppc, profile):
    """Non-power-of-two, non-square grid (direct DST path), all shape orders."""
    g = dict(nx=40, ny=48, nzeta=20, xmin=-5.0, xmax=5.0, ymin=-6.0, ymax=6.0, zeta_min=-4.0, zeta_max=4.0,
             shape_order=order, ppc_x=ppc[0], ppc_y=ppc[1], n_pc_iter=3, pc_mix=0.05, psi_guard=0.02)
    if profile:
        g.update(radial_profile=[1.0, 1.0, 0.9, 0.5, 0.2, 0.0, 0.0, 0.0], profile_rmax=7.0, n0_scale=1.3)
    beams = [I.random_beam(6000, 0.5, 0.4, 0.8, 0.5, zeta0=1.0, energy_spread=1e-3)]
    sp = O.GridSpec(**g)
    ref = O.sweep(sp, [O.as_beam(b) for b in beams])
    out, st, removed, _, _ = run_gpu(hq, g, beams, "fp64")
    for k in O.FIELD_NAMES:
        assert rel_per_slice(out[k], ref.fields[k]) <= 1e-12, k
    assert rel(st["x"], ref.plasma["x"]) <= 1e-12
    assert removed == ref.removed


def test_beam_push_and_witness_fp64(hq):
    g = I.scaled_grid(I.grid_params("adjoint256"), 48, 48, 48)
    beams = I.workload_beams("adjoint256", grid=g)
    ref = O.sweep(O.GridSpec(**g), [O.as_beam(b) for b in beams], dt=5.0, witness=(1,), record=("ez",))
    out, st, removed, hb, sums = run_gpu(hq, g, beams, "fp64", fields=("ez",), dt=5.0, witness=1)
    assert rel_per_slice(out["ez"], ref.fields["ez"]) <= 1e-12
    for bi in range(2):
        for k in ("x", "y", "zeta", "ux", "uy", "uz"):
            a = hb[bi].t[k].cpu()
            b = ref.beams[bi][k]
            scale = float(b.abs().max()) + 1e-30
            assert float((a - b).abs().max()) <= 1e-12 * scale, (bi, k)
    s = sums.cpu()
    for j in range(3):
        assert abs(float(s[j]) - float(ref.witness[1][j])) <= 1e-12 * abs(float(ref.witness[1][j])) + 1e-300, j


def test_beam_binning_is_exact(hq):
    """Integer work: per-slice particle counts of the device counting sort equal the oracle's
    (read through the witness charge sum, with a power-of-two weight so every sum is exact)."""
    g = dict(nx=32, ny=32, nzeta=37, xmin=-4.0, xmax=4.0, ymin=-4.0, ymax=4.0, zeta_min=-3.0, zeta_max=3.0,
             shape_order=1, n_pc_iter=0)
    b = I.random_beam(20000, 0.7, 0.7, 2.0, 1.0)
    b["w"] = np.full_like(b["w"], 2.0 ** -30)
    sp = O.GridSpec(**g)
    bins = O.beam_bins(sp, torch.as_tensor(b["zeta"]))
    counts = torch.bincount(bins[bins >= 0], minlength=sp.nzeta)
    grid = hq.Grid(g, precision="fp64")
    hb = [hq.Beam(b)]
    sums = torch.zeros(sp.nzeta, 3, dtype=torch.float64, device="cuda")
    for i in range(sp.nzeta):
        grid.advance(i)
        grid.beam_deposit(hb, i)
        grid.solve(i)
        grid.witness_accumulate(hb[0], i, sums[i])
    grid.sync()
    grid.close()
    got = (-sums[:, 0].cpu() * 2.0 ** 30)
    assert torch.equal(got, counts.double())


def test_fine_grained_api_matches_sweep_and_enforces_order(hq):
    g = I.scaled_grid(I.grid_params("linear64"), 32, 32, 10)
    beams = [hq.Beam(I.random_beam(3000, 0.5, 0.5, 1.0, 0.2))]
    grid = hq.Grid(g, precision="fp64")
    with pytest.raises(hq.HQError) as e:
        grid.solve(0)
    assert e.value.status == 6
    out = grid.alloc_out(("ez", "bx"))
    for i in range(g["nzeta"]):
        grid.advance(i)
        grid.beam_deposit(beams, i)
        grid.solve(i)
        grid.store(out, i)
    with pytest.raises(hq.HQError) as e:
        grid.advance(g["nzeta"] + 5)
    assert e.value.status == 1
    grid.sync()
    out2 = grid.alloc_out(("ez", "bx"))
    grid.sweep(beams, out=out2)
    grid.sync()
    # same arithmetic, different order of atomic additions
    assert rel_per_slice(out2["ez"], out["ez"]) <= 1e-12
    assert rel_per_slice(out2["bx"], out["bx"]) <= 1e-12
    grid.close()


# ---------------------------------------------------------------- FP32 / bf16x3

def test_sweep_fp32_linear(hq):
    g = I.grid_params("linear64")
    beams = I.workload_beams("linear64")
    ref = O.sweep(O.GridSpec(**g), [O.as_beam(b) for b in beams], record=("ez", "psi", "bx", "rho"))
    out, _, removed, _, _ = run_gpu(hq, g, beams, "fp32", fields=("ez", "psi", "bx", "rho"))
    errs = {k: rel(out[k], ref.fields[k]) for k in ("ez", "psi", "bx", "rho")}
    axis = rel(out["ez"][:, 32, 32], ref.fields["ez"][:, 32, 32])
    print("fp32 linear64 rel-L2", errs, "on-axis Ez", axis)
    assert axis <= 1e-4 and max(errs.values()) <= 1e-3, (errs, axis)


def test_sweep_fp32_blowout_reduced(hq):
    """Blowout driver (n_b = 5) on a 128^2 x 256 grid of the 512^2 box: bucket and first period."""
    g = I.scaled_grid(I.grid_params("blowout512"), 128, 128, 256)
    beams = I.workload_beams("blowout512", n_driver=200_000)
    sp = O.GridSpec(**g)
    ref = O.sweep(sp, [O.as_beam(b) for b in beams], record=("ez", "psi"))
    out, _, removed, _, _ = run_gpu(hq, g, beams, "fp32", fields=("ez", "psi"))
    zc = sp.zeta_max - (np.arange(sp.nzeta) + 0.5) * sp.dzeta
    first = torch.as_tensor(zc >= -2 * math.pi)
    bucket = torch.as_tensor(zc >= -7.0)
    c = sp.nx // 2
    e_axis = rel(out["ez"][first, c, c], ref.fields["ez"][first, c, c])
    e_bucket = rel(out["ez"][bucket], ref.fields["ez"][bucket])
    e_psi = rel(out["psi"][bucket], ref.fields["psi"][bucket])
    print("fp32 blowout128: on-axis Ez first period", e_axis, "bucket Ez", e_bucket, "psi", e_psi,
          "removed", removed, ref.removed)
    assert e_axis <= 1e-3 and e_bucket <= 1e-2, (e_axis, e_bucket)


# ---------------------------------------------------------------- full-size workload checks

def test_blowout512_head_full_size(hq):
    """Sampled parity at the full 512^2 / 1e6-particle size: the first 128 slices of the
    sweep (zeta from 7 down to 4.5, the head of the driver up to n_b ~ 1)."""
    g = I.grid_params("blowout512")
    beams = I.workload_beams("blowout512")
    nsamp = 128
    ref = O.sweep(O.GridSpec(**g), [O.as_beam(b) for b in beams], n_slices=nsamp, record=("rho", "jz", "ez", "psi"))
    assert float(ref.fields["rho"].abs().max()) > 0.1  # the beam is in the sample
    for prec, tol in (("fp64", 1e-12), ("fp32", 1e-3)):
        gg = dict(g)
        grid = hq.Grid(gg, precision=prec)
        out = grid.alloc_out(("rho", "jz", "ez", "psi"), nslots=nsamp)
        hb = [hq.Beam(b) for b in beams]
        for i in range(nsamp):
            grid.advance(i)
            grid.beam_deposit(hb, i)
            grid.solve(i)
            grid.store(out, i)
        grid.sync()
        grid.close()
        for k in ("rho", "jz", "psi", "ez"):
            e = rel_per_slice(out[k], ref.fields[k], floor_frac=1e-3)
            print(prec, k, e)
            assert e <= tol, (prec, k, e)


def test_blowout512_full_sweep_properties(hq):
    """The benchmark sweep itself (512^2 x 1024, 1e6 particles, FP32/bf16x3): finite fields,
    total (rho - Jz) neutral on every slice, a blowout (rho reaches the ion density)."""
    g = I.grid_params("blowout512")
    beams = I.workload_beams("blowout512")
    out, st, removed, _, _ = run_gpu(hq, g, beams, "fp32", fields=("rho", "jz", "ez"))
    rho, jz = out["rho"].double(), out["jz"].double()
    assert torch.isfinite(out["ez"]).all()
    sp = O.GridSpec(**g)
    tot = (rho - jz).sum(dim=(1, 2))
    ion_total = float(sp.nx * sp.ny)  # ~1 per interior node
    assert float(tot.abs().max()) <= 1e-3 * ion_total, float(tot.abs().max())
    assert float(rho.max()) > 0.9   # electrons fully expelled somewhere: rho ~ +1 (ions only)
    print("blowout512 fp32: max|Ez|", float(out["ez"].abs().max()), "removed", removed)


def test_zero_beam_full_size_fp32(hq):
    g = I.grid_params("blowout512")
    out, st, removed, _, _ = run_gpu(hq, g, [], "fp32", fields=("ez", "psi", "bx"))
    for k in ("ez", "psi", "bx"):
        assert float(out[k].abs().max()) <= 1e-4, k
    assert removed == 0
