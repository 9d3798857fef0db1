"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars:
  * Poisson solves, FP64: rel-L2 <= 1e-12 (a single linear operation).
  * Whole sweeps, FP64: the quasi-static sweep amplifies last-bit rounding
    differences, and the GPU's deposits are unordered atomic sums (the GPU run
    twice differs from itself by up to ~1e-10 of Bz's peak).  The bar is
    measured on the oracle: a second oracle run with the particles in another
    order, the ion background summed in reverse stencil order and every plasma
    deposit node value perturbed by one ulp (relative 2^-52, the size of the
    error an unordered summation leaves) gives, per field and slice, the
    sweep's own rounding floor f (deviation over the field's peak slice norm).
    One such sample swings by ~10x from slice to slice (even/odd alternation),
    and a perturbation made at slice j is carried to every later slice, so the
    floor envelope at slice i is the running maximum of f over slices <= i.
    The GPU's deviation must be below max(1e-12, 10 x envelope).
  * FP32/bf16x3 path: each bf16x3 product carries ~2^-17 relative error, so a
    4-product Dirichlet solve is good to a few 1e-5 (rel-L2); sweeps are held to
    the on-axis Ez (first plasma period) <= 1e-4 and bucket <= 1e-3 bounds.  At the
    head of the 512^2 driver every field is held to 1e-4 of its peak, although psi
    there (~1e-6) is the difference of unit charge densities: the FP32 path keeps
    the psi source ion-subtracted per particle (an all-FP32 evaluation of the method,
    printed for reference, is off by ~100% there).
  * integer work (beam binning) is bit-exact: per-slice particle counts.
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


def peak_err(a, b):
    """Per-slice ||a_i - b_i|| / max_j ||b_j|| (deviation on the field's own scale)."""
    a = a.double().cpu()
    b = b.double().cpu()
    nb = torch.linalg.norm(b.reshape(b.shape[0], -1), dim=1)
    na = torch.linalg.norm((a - b).reshape(b.shape[0], -1), dim=1)
    return na / (float(nb.max()) + 1e-300)


def reordered(beams, seed=0):
    """The same beams with their particles in another order (changes only summation order)."""
    out = []
    for b in beams:
        perm = np.random.default_rng(seed).permutation(len(b["x"]))
        c = dict(b)
        for k in ("x", "y", "zeta", "ux", "uy", "uz", "w"):
            c[k] = np.asarray(b[k])[perm]
        out.append(c)
    return out


def plasma_perm(g, seed=1):
    n = g["nx"] * g["ny"] * g.get("ppc_x", 1) * g.get("ppc_y", 1)
    return torch.as_tensor(np.random.default_rng(seed).permutation(n))


def assert_fp64_sweep(out, ref, ref_perm, fields, factor=10.0, spec=None):
    for k in fields:
        e = peak_err(out[k], ref.fields[k])
        f = peak_err(ref_perm.fields[k], ref.fields[k])
        env = torch.cummax(f, dim=0).values
        bar = torch.clamp(factor * env, min=1e-12)
        worst = int(torch.argmax(e / bar))
        print(f"fp64 {k}: max dev {float(e.max()):.2e}, reorder floor {float(f.max()):.2e}, "
              f"worst slice {worst}: {float(e[worst]):.2e} vs bar {float(bar[worst]):.2e}")
        assert bool((e <= bar).all()), (k, worst, float(e[worst]), float(bar[worst]))


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
    sp = O.GridSpec(**g)
    ref = O.sweep(sp, [O.as_beam(b) for b in beams])
    ref_perm = O.sweep(sp, [O.as_beam(b) for b in reordered(beams)], plasma_perm=plasma_perm(g),
                     reverse_ion_order=True, deposit_noise=2.0 ** -52)
    out, st, removed, _, _ = run_gpu(hq, g, beams, "fp64")
    assert_fp64_sweep(out, ref, ref_perm, O.FIELD_NAMES, spec=sp)
    for k in ("x", "y", "psi", "ux", "uy"):
        d = float((st[k].double().cpu() - ref.plasma[k]).abs().max())
        f = float((ref_perm.plasma[k] - ref.plasma[k]).abs().max())
        assert d <= max(1e-12, 30 * f), (k, d, f)
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
    ref_perm = O.sweep(sp, [O.as_beam(b) for b in reordered(beams)], plasma_perm=plasma_perm(g),
                     reverse_ion_order=True, deposit_noise=2.0 ** -52)
    out, st, removed, _, _ = run_gpu(hq, g, beams, "fp64")
    assert_fp64_sweep(out, ref, ref_perm, O.FIELD_NAMES, spec=sp)
    assert removed == ref.removed


@pytest.mark.parametrize("solver", ["pc", "explicit"])
def test_beam_push_and_witness_fp64(hq, solver):
    """The beam push with both B_perp solvers (the explicit one takes the beam J_perp of slice i-1
    from before that slice's push)."""
    g = I.scaled_grid(I.grid_params("adjoint256"), 48, 48, 48, bperp_solver=solver)
    beams = I.workload_beams("adjoint256", grid=g)
    sp = O.GridSpec(**g)
    ref = O.sweep(sp, [O.as_beam(b) for b in beams], dt=5.0, witness=(1,), record=("ez",))
    perm = [np.random.default_rng(0).permutation(len(b["x"])) for b in beams]
    ref_perm = O.sweep(sp, [O.as_beam(b) for b in reordered(beams)], dt=5.0, witness=(1,), record=("ez",),
                       plasma_perm=plasma_perm(g),
                     reverse_ion_order=True, deposit_noise=2.0 ** -52)
    out, st, removed, hb, sums = run_gpu(hq, g, beams, "fp64", fields=("ez",), dt=5.0, witness=1)
    assert_fp64_sweep(out, ref, ref_perm, ("ez",))
    for bi in range(2):
        inv = np.argsort(perm[bi])
        for k in ("x", "y", "zeta", "ux", "uy", "uz"):
            a = hb[bi].t[k].cpu()
            b = ref.beams[bi][k]
            c = ref_perm.beams[bi][k][inv]
            scale = float((b - b.mean()).abs().max()) + 1e-30  # spread of the coordinate
            d, f = float((a - b).abs().max()) / scale, float((c - b).abs().max()) / scale
            assert d <= max(1e-12, 30 * f), (bi, k, d, f)
    s = sums.cpu()
    for j in range(3):
        r, rp = float(ref.witness[1][j]), float(ref_perm.witness[1][j])
        assert abs(float(s[j]) - r) <= max(1e-12 * abs(r), 30 * abs(rp - r)), j


def test_beam_push_fp32(hq):
    """The FP32/bf16x3 path's beam push (the cubic1024 time steps): the pushed beam phase space
    and the witness sums against the FP64 oracle, on the adjoint256 box at 64^2 (the folded DST
    path is not needed; the push reads the FP32 gather and B_perp records).  Bars: every
    coordinate within 1e-4 of its spread over the beam and within 1e-3 of its largest change
    in the step (the push's own increment), the witness sums within 1e-4."""
    g = I.scaled_grid(I.grid_params("adjoint256"), 64, 64, 64)
    beams = I.workload_beams("adjoint256", grid=g)
    sp = O.GridSpec(**g)
    ref = O.sweep(sp, [O.as_beam(b) for b in beams], dt=5.0, witness=(1,), record=())
    _, _, _, hb, sums = run_gpu(hq, g, beams, "fp32", fields=(), dt=5.0, witness=1)
    worst = 0.0
    for bi in range(2):
        for k in ("x", "y", "zeta", "ux", "uy", "uz"):
            a = hb[bi].t[k].cpu()
            b = ref.beams[bi][k]
            moved = float((b - torch.as_tensor(beams[bi][k])).abs().max()) + 1e-30
            d = float((a - b).abs().max())
            scale = float((b - b.mean()).abs().max()) + 1e-30
            worst = max(worst, d / scale)
            print(f"fp32 beam push beam {bi} {k}: max dev {d:.2e} of spread {scale:.2e} (moved up to {moved:.2e})")
            assert d <= 1e-4 * scale and d <= 1e-3 * moved, (bi, k, d, scale, moved)
    s_ = sums.cpu()
    for j in range(3):
        r = float(ref.witness[1][j])
        assert abs(float(s_[j]) - r) <= 1e-4 * abs(r), (j, float(s_[j]), r)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_witness_sums_without_push(hq, monkeypatch, precision):
    """Without a beam push the sweep sums slice i-1's witness on a second stream beside slice
    i's final pass (and deposits slice i's beam there).  The witness sums equal the oracle's
    (FP64: within the reordering floor; FP32: 1e-4) and the per-step order's (HQ_NO_FORK=1)."""
    g = I.scaled_grid(I.grid_params("adjoint256"), 128, 128, 48)
    beams = I.workload_beams("adjoint256", grid=g)
    sp = O.GridSpec(**g)
    ref = O.sweep(sp, [O.as_beam(b) for b in beams], witness=(1,), record=("ez",))
    ref_perm = O.sweep(sp, [O.as_beam(b) for b in reordered(beams)], witness=(1,), record=("ez",),
                       plasma_perm=plasma_perm(g), reverse_ion_order=True, deposit_noise=2.0 ** -52)
    res = {}
    for mode in ("fork", "steps"):
        if mode == "steps":
            monkeypatch.setenv("HQ_NO_FORK", "1")
        out, _, _, _, sums = run_gpu(hq, g, beams, precision, fields=("ez",), witness=1)
        res[mode] = (out, sums.cpu())
        monkeypatch.delenv("HQ_NO_FORK", raising=False)
    s0, s2 = float(ref.witness[1][0]), float(ref.witness[1][2])
    scale = [abs(s0), math.sqrt(abs(s0 * s2)), abs(s2)]   # |sum qw Ez| <= sqrt(S0 S2)
    for mode, (out, s) in res.items():
        if precision == "fp64":
            assert_fp64_sweep(out, ref, ref_perm, ("ez",))
        for j in range(3):
            r, rp = float(ref.witness[1][j]), float(ref_perm.witness[1][j])
            bar = max(1e-12 * abs(r), 30 * abs(rp - r)) if precision == "fp64" else 1e-4 * scale[j]
            print(f"{precision} witness sum {j} ({mode}): {float(s[j]):.12e} vs oracle {r:.12e}")
            assert abs(float(s[j]) - r) <= bar, (mode, j, float(s[j]), r)
    assert float(res["fork"][1].abs().sum()) > 0


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
    # same arithmetic, different order of atomic additions: agreement on the fields' scale
    assert float(peak_err(out2["ez"], out["ez"]).max()) <= 1e-9
    assert float(peak_err(out2["bx"], out["bx"]).max()) <= 1e-9
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
    assert e_axis <= 1e-4 and e_bucket <= 1e-3, (e_axis, e_bucket)


# ---------------------------------------------------------------- full-size workload checks

def test_blowout512_head_full_size(hq):
    """Sampled parity at the full 512^2 / 1e6-particle size: the first 128 slices of the
    sweep (zeta from 7 down to 4.5, the head of the driver up to n_b ~ 1)."""
    g = I.grid_params("blowout512")
    beams = I.workload_beams("blowout512")
    nsamp = 128
    sp = O.GridSpec(**g)
    rec = ("rho", "jz", "ez", "psi")
    ref = O.sweep(sp, [O.as_beam(b) for b in beams], n_slices=nsamp, record=rec)
    ref_perm = O.sweep(sp, [O.as_beam(b) for b in reordered(beams)], n_slices=nsamp, record=rec,
                       plasma_perm=plasma_perm(g),
                     reverse_ion_order=True, deposit_noise=2.0 ** -52)
    with O.working_precision(torch.float32):
        ref_f32 = O.sweep(sp, [O.as_beam(b) for b in beams], n_slices=nsamp, record=rec)
    assert float(ref.fields["rho"].abs().max()) > 0.1  # the beam is in the sample
    for prec in ("fp64", "fp32"):
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
        if prec == "fp64":
            assert_fp64_sweep(out, ref, ref_perm, rec, spec=sp)
        else:
            c = g["nx"] // 2
            axis = rel(out["ez"][:, c, c], ref.fields["ez"][:, c, c])
            axis_f = rel(ref_f32.fields["ez"][:, c, c].double(), ref.fields["ez"][:, c, c])
            print("fp32 on-axis Ez rel-L2", axis, "all-FP32 oracle", axis_f)
            assert axis <= 1e-4, (axis, axis_f)
            for k in rec:
                e = peak_err(out[k], ref.fields[k])
                f = peak_err(ref_f32.fields[k].double(), ref.fields[k])
                bar = torch.full_like(e, 1e-4)
                worst = int(torch.argmax(e / bar))
                print(f"fp32 {k}: max dev {float(e.max()):.2e} (bar 1e-4), all-FP32 oracle {float(f.max()):.2e}, "
                      f"worst slice {worst}: {float(e[worst]):.2e}")
                assert bool((e <= bar).all()), (k, worst, float(e[worst]), float(bar[worst]))


def test_blowout512_full_sweep_properties(hq):
    """The benchmark sweep itself (512^2 x 1024, 1e6 particles, FP32/bf16x3): finite fields,
    total (rho - Jz) neutral on every slice, a blowout (rho reaches the ion density), and inside
    the electron-free channel the ion-channel force ExmBy = x/2 (psi's source there is the ion
    density alone; the oracle's blowout pin) on the slices whose axis row is electron-free over
    at least 16 nodes each side: slope within 1 % of 1/2 in the median (measured 0.4997 over 210
    slices) and within 6 % on every slice (the channel's first slices, where the sheath is still
    close to the fitted inner half, measured 0.480; the oracle's 128^2 channel shows the same,
    0.494 at its front)."""
    g = I.grid_params("blowout512")
    beams = I.workload_beams("blowout512")
    out, st, removed, _, _ = run_gpu(hq, g, beams, "fp32", fields=("rho", "jz", "ez", "exmby"))
    rho, jz = out["rho"].double(), out["jz"].double()
    assert torch.isfinite(out["ez"]).all()
    sp = O.GridSpec(**g)
    tot = (rho - jz).sum(dim=(1, 2))
    ion_total = float(sp.nx * sp.ny)  # ~1 per interior node
    assert float(tot.abs().max()) <= 1e-3 * ion_total, float(tot.abs().max())
    assert float(rho.max()) > 0.9   # electrons fully expelled somewhere: rho ~ +1 (ions only)
    print("blowout512 fp32: max|Ez|", float(out["ez"].abs().max()), "removed", removed)
    c = sp.nx // 2
    src = (rho[:, c, :] - jz[:, c, :]).cpu().numpy()
    ex = out["exmby"][:, c, :].double().cpu().numpy()
    slopes = []
    for i in range(sp.nzeta):
        k = 0
        while c + k + 1 < sp.nx - 1 and abs(src[i, c + k + 1] - 1.0) < 1e-5 and abs(src[i, c - k - 1] - 1.0) < 1e-5:
            k += 1
        if k >= 16:
            h = k // 2
            xs = sp.xmin + np.arange(c - h, c + h + 1) * sp.dx
            slopes.append(np.polyfit(xs, ex[i, c - h:c + h + 1], 1)[0])
    slopes = np.asarray(slopes)
    print(f"ion channel: {slopes.size} slices, ExmBy slope {slopes.min():.4f} .. {slopes.max():.4f} "
          f"(median {np.median(slopes):.4f})")
    assert slopes.size >= 20
    assert abs(np.median(slopes) - 0.5) <= 0.005 and np.all(np.abs(slopes - 0.5) <= 0.03), slopes


def test_blowout512_full_sweep_vs_oracle(hq):
    """The benchmark sweep itself against the FP64 oracle: 512^2 x 1024 slices, 1e6-particle
    blowout driver (n_b = 5), FP32/bf16x3, all slices.  The oracle records the bucket window
    |x|, |y| <= 3 and the plasma at 8 slices.  Bars (FP32/split): on-axis Ez over the first
    plasma period (zeta >= -2 pi behind the driver centre) <= 1e-4 rel-L2, Ez across the
    bucket (zeta >= -7) <= 1e-3.  Stated: psi over the bucket, the plasma displacement at 8
    slices and the number of particles removed."""
    g = I.grid_params("blowout512")
    beams = I.workload_beams("blowout512")
    sp = O.GridSpec(**g)
    lo, hi = 160, 353                       # nodes with |x|, |y| <= 3 (dx = 1/32, x_j = -8 + j dx)
    samples = (64, 192, 320, 448, 576, 704, 832, 960)
    torch.set_num_threads(max(1, torch.get_num_threads()))
    ref = O.sweep(sp, [O.as_beam(b) for b in beams], record=("ez", "psi"), crop=(lo, hi, lo, hi),
                  record_plasma_at=samples)
    grid = hq.Grid(g, precision="fp32")
    out = grid.alloc_out(("ez", "psi"))
    hb = [hq.Beam(b) for b in beams]
    plasma = {}
    for i in range(sp.nzeta):
        grid.advance(i)
        if i in samples:
            plasma[i] = {k: v.double().cpu() for k, v in grid.plasma_state().items() if k in ("x", "y", "alive")}
        grid.beam_deposit(hb, i)
        grid.solve(i)
        grid.store(out, i)
    removed = grid.sync()
    grid.close()
    ez = out["ez"][:, lo:hi, lo:hi].double().cpu()
    psi = out["psi"][:, lo:hi, lo:hi].double().cpu()
    zc = sp.zeta_max - (np.arange(sp.nzeta) + 0.5) * sp.dzeta
    first = torch.as_tensor(zc >= -2 * math.pi)
    bucket = torch.as_tensor(zc >= -7.0)
    c = sp.nx // 2 - lo
    e_axis = rel(ez[first, c, c], ref.fields["ez"][first, c, c])
    e_bucket = rel(ez[bucket], ref.fields["ez"][bucket])
    e_psi = rel(psi[bucket], ref.fields["psi"][bucket])
    st0 = O.plasma_init(sp)
    traj = {}
    for i in samples:
        a, b = plasma[i], ref.plasma_at[i]
        both = a["alive"].bool() & b["alive"]
        disp = torch.cat([(b["x"] - st0["x"])[both], (b["y"] - st0["y"])[both]])
        dev = torch.cat([(a["x"] - b["x"])[both], (a["y"] - b["y"])[both]])
        traj[i] = float(torch.linalg.norm(dev) / torch.linalg.norm(disp))
    print(f"blowout512 full sweep fp32: on-axis Ez first period {e_axis:.2e}, bucket Ez {e_bucket:.2e}, "
          f"bucket psi {e_psi:.2e}; plasma displacement rel-L2 per sampled slice "
          f"{ {k: f'{v:.1e}' for k, v in traj.items()} }; removed {removed} (oracle {ref.removed})")
    assert e_axis <= 1e-4 and e_bucket <= 1e-3, (e_axis, e_bucket)
    assert max(traj.values()) <= 1e-2, traj


def test_zero_beam_full_size_fp32(hq):
    g = I.grid_params("blowout512")
    out, st, removed, _, _ = run_gpu(hq, g, [], "fp32", fields=("ez", "psi", "bx"))
    for k in ("ez", "psi", "bx"):
        assert float(out[k].abs().max()) <= 1e-4, k
    assert removed == 0


def test_cubic1024_full_size_sampled(hq):
    """The 1024^2, 4 ppc, cubic-shape workload at full size (4.2M plasma particles per slice,
    1e7 + 2e6 beam particles), FP32/bf16x3, through the first 224 slices (into the driver).
    The oracle cannot run the sweep, so each stage is checked one by one at full size:
      * deposit: the oracle's FP64 deposit of the GPU's own plasma state reproduces the GPU's
        J_perp (the beam carries no transverse momentum) to FP32 rounding;
      * solves: the oracle's Poisson solve of the GPU's own sources reproduces its psi, Ez and
        Bz within the bf16x3 bar (folded DST-I with K = 512: the TMA ring wraps);
      * properties: every field finite, psi > -1 (no sheath collapse this early)."""
    g = I.grid_params("cubic1024")
    beams = I.workload_beams("cubic1024")
    sp = O.GridSpec(**g)
    rec = ("rho", "jx", "jy", "jz", "psi", "ez", "bz")
    grid = hq.Grid(g, precision="fp32")
    out = grid.alloc_out(rec, nslots=1)
    hb = [hq.Beam(b) for b in beams]
    checked = 0
    for i in range(224):
        grid.advance(i)
        if i in (160, 223):
            st = {k: v.double().cpu() if v.dtype != torch.uint8 else v.cpu().bool() for k, v in grid.plasma_state().items()}
        grid.beam_deposit(hb, i)
        grid.solve(i)
        if i in (160, 223):
            grid.store(out, 0)
            grid.sync()
            f = {k: out[k][0].double().cpu() for k in rec}
            for k in rec:
                assert torch.isfinite(f[k]).all(), (i, k)
            assert float(f["psi"].min()) > -1.0
            # deposit stage: plasma J_perp from the GPU's particles through the oracle's deposit
            _, jx_o, jy_o, _, _ = O.plasma_deposit_full(sp, st)
            for k, ref in (("jx", jx_o), ("jy", jy_o)):
                e = rel(f[k], ref.reshape(sp.ny, sp.nx))
                print(f"cubic1024 slice {i}: deposit {k} rel-L2 {e:.2e}")
                assert e <= 1e-5, (i, k, e)
            # solve stage: the GPU's own sources through the oracle's solver.  Bz, the curl of
            # J_perp, is here (a round driver) a small residual of two large terms,
            # L^-1(dy Jx) - L^-1(dx Jy); its error is measured on the scale of one term.
            def wall0(t):
                t = t.clone()
                t[0, :] = 0
                t[:, 0] = 0
                return t
            srcs = {"psi": -(f["rho"] - f["jz"]),
                    "ez": O.ddx(sp, f["jx"]) + O.ddy(sp, f["jy"]),
                    "bz": O.ddy(sp, f["jx"]) - O.ddx(sp, f["jy"])}
            for k, src in srcs.items():
                ref = O.poisson_solve(sp, wall0(src))
                scale = ref if k != "bz" else O.poisson_solve(sp, wall0(O.ddy(sp, f["jx"])))
                e = float(torch.linalg.norm(f[k] - ref) / torch.linalg.norm(scale))
                print(f"cubic1024 slice {i}: solve {k} error {e:.2e} (of the {'field' if k != 'bz' else 'dy Jx term'})")
                assert e <= 3e-5, (i, k, e)
            checked += 1
    grid.sync()
    grid.close()
    assert checked == 2


def test_sweep_graph_replay_matches_stream_launches(hq, monkeypatch):
    """hq_sweep_step replays a captured CUDA graph.  On a linear-regime sweep (128^2, folded
    DST; FP32 atomics order is its only run-to-run difference, measured here between two
    plain-launch sweeps): the replay reproduces plain stream launches (HQ_NO_GRAPH=1), a sweep
    with other output buffers is re-captured and fills them, and the fine-grained calls still
    work after a graph sweep."""
    g = I.scaled_grid(I.grid_params("linear64"), 128, 128, 64)
    beams = I.workload_beams("linear64")
    outs = {}
    for mode in ("graph", "stream"):
        if mode == "stream":
            monkeypatch.setenv("HQ_NO_GRAPH", "1")
        grid = hq.Grid(g, precision="fp32")
        hb = [hq.Beam(b) for b in beams]
        a = grid.alloc_out(("ez", "psi"))
        grid.sweep(hb, out=a)       # captured (or plain) and run
        grid.sweep(hb, out=a)       # replayed
        b = grid.alloc_out(("ez", "psi"))
        grid.sweep(hb, out=b)       # new output buffers: re-captured
        grid.sync()
        c = grid.alloc_out(("ez",), nslots=1)
        for i in range(4):          # fine-grained API after a sweep
            grid.advance(i)
            grid.beam_deposit(hb, i)
            grid.solve(i)
        grid.store(c, 0)
        grid.sync()
        grid.close()
        outs[mode] = (a, b, c)
        monkeypatch.delenv("HQ_NO_GRAPH", raising=False)
    (ga, gb, gc), (sa, sb, sc) = outs["graph"], outs["stream"]
    for k in ("ez", "psi"):
        floor = float(peak_err(sb[k], sa[k]).max())          # plain launches against themselves
        bar = max(10.0 * floor, 1e-6)
        errs = [float(peak_err(gb[k], ga[k]).max()), float(peak_err(ga[k], sa[k]).max()),
                float(peak_err(gb[k], sb[k]).max())]
        print(f"graph replay {k}: run-to-run floor {floor:.1e}, deviations {errs}")
        assert max(errs) <= bar, (k, errs, bar)
        assert float(gb[k].abs().max()) > 0
    assert float(peak_err(gc["ez"], sc["ez"]).max()) <= 1e-5


def test_sources_in_solve_launch_match_separate_kernels(hq, monkeypatch):
    """FP32: the psi/Ez/Bz and B_perp sources formed in the solve launch's first phase give
    the same sweep as separate source kernels (HQ_SEPARATE_SRC=1), within the run-to-run
    floor of the FP32 atomics (two sweeps of the same build)."""
    g = I.scaled_grid(I.grid_params("linear64"), 128, 128, 64)
    beams = [I.random_beam(100_000, 0.3, 0.3, 1.0, 0.5, energy_spread=1e-3)]
    outs = {}
    for mode in ("fused", "fused2", "separate"):
        if mode == "separate":
            monkeypatch.setenv("HQ_SEPARATE_SRC", "1")
        outs[mode] = run_gpu(hq, g, beams, "fp32", fields=("ez", "psi", "bx"))[0]
        monkeypatch.delenv("HQ_SEPARATE_SRC", raising=False)
    for k in ("ez", "psi", "bx"):
        floor = float(peak_err(outs["fused2"][k], outs["fused"][k]).max())
        dev = float(peak_err(outs["separate"][k], outs["fused"][k]).max())
        print(f"fused vs separate sources {k}: {dev:.1e} (run-to-run {floor:.1e})")
        assert dev <= max(10 * floor, 1e-6), (k, dev, floor)


@pytest.mark.parametrize("switch", ["HQ_NO_F4CACHE", "HQ_NO_SRCCACHE"])
def test_slice_caches_match_full_evaluation(hq, monkeypatch, switch):
    """FP32, the two per-slice caches of the predictor-corrector.  HQ_NO_F4CACHE: the trial
    passes after a slice's first, and the final pass, read ExmBy, EypBx, Ez, Bz back from the
    per-particle copy the first trial pass kept and gather Bx, By alone.  HQ_NO_SRCCACHE: the B_perp
    source phases after a slice's first read back the part of the sources that does not depend
    on the trial J_perp.  With either switch set the sweep evaluates everything every time; it
    matches the cached sweep within the run-to-run floor of the FP32 atomics (quadratic shape,
    2 ppc, a driver strong enough to move particles across cells within the predictor-corrector)."""
    g = dict(I.scaled_grid(I.grid_params("linear64"), 128, 128, 64), shape_order=2, ppc_x=2)
    beams = [I.random_beam(100_000, 0.3, 0.3, 1.0, 2.0, energy_spread=1e-3)]
    outs = {}
    for mode in ("cached", "cached2", "full"):
        if mode == "full":
            monkeypatch.setenv(switch, "1")
        outs[mode] = run_gpu(hq, g, beams, "fp32", fields=("ez", "psi", "bx", "by"))[0]
        monkeypatch.delenv(switch, raising=False)
    for k in ("ez", "psi", "bx", "by"):
        floor = float(peak_err(outs["cached2"][k], outs["cached"][k]).max())
        dev = float(peak_err(outs["full"][k], outs["cached"][k]).max())
        print(f"{switch}: cached vs full {k}: {dev:.1e} (run-to-run {floor:.1e})")
        assert dev <= max(10 * floor, 1e-6), (k, dev, floor)


@pytest.mark.parametrize("n", [256, 512])
def test_resident_fold_matrix_solve_matches_streamed(hq, monkeypatch, n):
    """FP32 square grids of 256 and 512 cells run the solve that keeps each CTA's slice of the
    fold matrix in shared memory; it gives the same sweep as the solve that streams it
    (HQ_NO_RS=1), within the run-to-run floor of the FP32 atomics."""
    g = I.scaled_grid(I.grid_params("linear64"), n, n, 64)
    beams = [I.random_beam(100_000, 0.3, 0.3, 1.0, 0.5, energy_spread=1e-3)]
    outs = {}
    for mode in ("rs", "rs2", "streamed"):
        if mode == "streamed":
            monkeypatch.setenv("HQ_NO_RS", "1")
        outs[mode] = run_gpu(hq, g, beams, "fp32", fields=("ez", "psi", "bx"))[0]
        monkeypatch.delenv("HQ_NO_RS", raising=False)
    for k in ("ez", "psi", "bx"):
        floor = float(peak_err(outs["rs2"][k], outs["rs"][k]).max())
        dev = float(peak_err(outs["streamed"][k], outs["rs"][k]).max())
        print(f"n={n} resident vs streamed fold matrix {k}: {dev:.1e} (run-to-run {floor:.1e})")
        assert dev <= max(10 * floor, 1e-6), (k, dev, floor)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_pc_residuals_match_oracle(hq, precision):
    """The per-slice predictor-corrector residual ||B_m - B_m-1|| / ||B_m|| of the last iteration
    (hq_pc_residuals) against the oracle's: FP64 within 1e-8 relative, FP32 within 1e-2 (the residual
    is a difference of iterates, ~1e-3 of B at the smallest here, so the FP32/bf16x3 field error of
    ~1e-5 shows ~100x larger in it; measured 1.9e-3), on every slice where the oracle's residual is
    above 1e-9 (zero where B_perp is zero ahead of the beam)."""
    g = I.grid_params("linear64")
    beams = I.workload_beams("linear64")
    ref = O.sweep(O.GridSpec(**g), [O.as_beam(b) for b in beams], record=())
    grid = hq.Grid(dict(g, pc_residuals=1), precision=precision)
    grid.sweep([hq.Beam(b) for b in beams])
    got = grid.pc_residuals()
    grid.close()
    plain = hq.Grid(g, precision=precision)   # not recorded unless asked for
    with pytest.raises(hq.HQError) as e:
        plain.pc_residuals()
    assert e.value.status == 6
    plain.close()
    tol = 1e-8 if precision == "fp64" else 1e-2
    worst = 0.0
    for i, (a, r) in enumerate(zip(got, ref.pc_residual)):
        if r > 1e-9:
            worst = max(worst, abs(a - r) / r)
            assert abs(a - r) <= tol * r, (i, a, r)
        else:
            assert a <= 1e-6, (i, a, r)
    print(f"{precision} P-C residual: worst relative difference {worst:.2e}; oracle range "
          f"{min(x for x in ref.pc_residual if x > 0):.2e} .. {max(ref.pc_residual):.2e}")

