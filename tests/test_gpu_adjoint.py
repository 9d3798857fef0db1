"""The hand-written reverse-zeta adjoint (hq_sweep_forward_ckpt + hq_sweep_adjoint)
against the oracle's taped FP64 adjoint (autograd through the oracle sweep, itself
pinned to central finite differences in test_oracle_adjoint.py).

Bars: gradients within 1e-5 (FP64 path) and 1e-3 (FP32/bf16x3 path) relative,
checked as the relative L2 error of each gradient vector and of
directional derivatives along random directions.  Both single-segment (no
recompute) and multi-segment (checkpoint restore + recompute) runs are covered.
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


def case(order=1, nz=24, n=24):
    g = dict(nx=n, ny=n, nzeta=nz, xmin=-6.0, xmax=6.0, ymin=-6.0, ymax=6.0, zeta_min=-7.0, zeta_max=5.0,
             shape_order=order, n_pc_iter=2, pc_mix=0.05, psi_guard=0.02,
             radial_profile=[1.0, 1.0, 0.8, 0.5, 0.3], profile_rmax=8.5)
    d = I.fixed_ppc_beam(g, 0.8, 1.0, 2.0)
    w = I.fixed_ppc_beam(g, 0.5, 0.6, 10.0, zeta0=-3.0, gamma=I.GAMMA_WITNESS)
    return g, d, w


def oracle_grads(g, d, w, kind):
    sp = O.GridSpec(**g)
    wd = torch.tensor(d["w"], dtype=torch.float64, requires_grad=True)
    ww = torch.tensor(w["w"], dtype=torch.float64, requires_grad=True)
    n0 = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    prof = torch.tensor(g["radial_profile"], dtype=torch.float64, requires_grad=True)
    bd, bw = O.as_beam(d), O.as_beam(w)
    bd["w"], bw["w"] = wd, ww
    r = O.sweep(sp, [bd, bw], witness=(1,), record=(), n0_scale=n0, radial_profile=prof)
    L = O.witness_loss(r, 1, kind)
    L.backward()
    return float(L), wd.grad, ww.grad, float(n0.grad), prof.grad


def gpu_grads(hq, g, d, w, kind, precision, k):
    grid = hq.Grid(g, precision=precision)
    beams = [hq.Beam(d), hq.Beam(w)]
    sums = torch.zeros(3, dtype=torch.float64, device="cuda")
    grid.forward_ckpt(beams, 1, sums, k)
    s = [float(v) for v in sums.cpu()]
    L, dls = hq.witness_loss_grad(kind, *s)
    res = grid.adjoint(beams, 1, dls)
    grid.sync()
    out = (L, res["beam_w"][0].cpu(), res["beam_w"][1].cpu(), float(res["n0_scale"][0]), res["profile"].cpu())
    grid.close()
    return out


def rel(a, b):
    return float(torch.linalg.norm(a - b) / (torch.linalg.norm(b) + 1e-300))


def directional(a, b, seed=0, k=3):
    """Derivatives along random positive weight perturbations v: |v.(a - b)| relative to
    sum_i |v_i b_i|, the size of the terms summed (the gradient has both signs, so
    |v.b| itself can be much smaller than its terms)."""
    rng = np.random.default_rng(seed)
    worst = 0.0
    for _ in range(k):
        v = torch.tensor(np.abs(rng.standard_normal(a.shape[0])), dtype=torch.float64)
        x, y = float((a * v).sum()), float((b * v).sum())
        worst = max(worst, abs(x - y) / (float((b * v).abs().sum()) + 1e-300))
    return worst


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-5), ("fp32", 1e-3)])
@pytest.mark.parametrize("kind,order,k", [("mean", 1, 24), ("mean", 1, 5), ("mean+rms", 2, 7)])
def test_adjoint_matches_taped_oracle(hq, precision, tol, kind, order, k):
    g, d, w = case(order=order)
    L0, gd0, gw0, gn0, gp0 = oracle_grads(g, d, w, kind)
    L1, gd1, gw1, gn1, gp1 = gpu_grads(hq, g, d, w, kind, precision, k)
    errs = {"loss": abs(L1 - L0) / abs(L0), "driver_w": rel(gd1, gd0), "witness_w": rel(gw1, gw0),
            "driver_dir": directional(gd1, gd0), "n0": abs(gn1 - gn0) / abs(gn0), "profile": rel(gp1, gp0)}
    print(precision, kind, order, k, {a: f"{b:.2e}" for a, b in errs.items()})
    loss_tol = 1e-10 if precision == "fp64" else 1e-3
    assert errs["loss"] <= loss_tol, errs
    for key in ("driver_w", "witness_w", "driver_dir", "n0", "profile"):
        assert errs[key] <= tol, (key, errs)


def test_sweep_loss_autograd_to_beam_parameters(hq):
    """torch.autograd through SweepLoss: gradient of the mean witness Ez w.r.t. the driver's
    peak density, sigma_r, sigma_z, the witness position and n0, against the oracle's taped
    adjoint through the same weight recipe."""
    g, d, w = case(order=1)
    dx = (g["xmax"] - g["xmin"]) / g["nx"]
    dz = (g["zeta_max"] - g["zeta_min"]) / g["nzeta"]

    def weights(beam, nb, sr, sz, z0):
        x, y, z = (torch.as_tensor(beam[k], dtype=torch.float64) for k in ("x", "y", "zeta"))
        return nb * torch.exp(-(x * x + y * y) / (2 * sr * sr)) * torch.exp(-((z - z0) ** 2) / (2 * sz * sz)) * dx * dx * dz

    p0 = [2.0, 0.8, 1.0, -3.0]

    def params():
        return [torch.tensor(v, dtype=torch.float64, requires_grad=True) for v in p0] + \
               [torch.tensor(1.0, dtype=torch.float64, requires_grad=True)]

    g = dict(g)
    g.pop("radial_profile")
    g.pop("profile_rmax")
    # oracle
    nb, sr, sz, z0, n0 = params()
    sp = O.GridSpec(**g)
    bd, bw = O.as_beam(d), O.as_beam(w)
    bd["w"] = weights(d, nb, sr, sz, 0.0)
    bw["w"] = weights(w, 10.0, 0.5, 0.6, z0)
    r = O.sweep(sp, [bd, bw], witness=(1,), record=(), n0_scale=n0)
    Lo = O.witness_loss(r, 1, "mean")
    Lo.backward()
    ref = [float(t.grad) for t in (nb, sr, sz, z0, n0)]
    # GPU, FP64
    grid = hq.Grid(g, precision="fp64")
    beams = [hq.Beam(d), hq.Beam(w)]
    nb, sr, sz, z0, n0 = params()
    wd = weights(d, nb, sr, sz, 0.0).cuda()
    ww = weights(w, 10.0, 0.5, 0.6, z0).cuda()
    L = hq.SweepLoss.apply(grid, beams, 1, "mean", 8, n0, torch.empty(0), wd, ww)
    L.backward()
    got = [float(t.grad) for t in (nb, sr, sz, z0, n0)]
    grid.close()
    assert abs(float(L) - float(Lo)) <= 1e-10 * abs(float(Lo))
    for a, b, name in zip(got, ref, ("n_b", "sigma_r", "sigma_z", "zeta0", "n0")):
        assert abs(a - b) <= 1e-5 * abs(b), (name, a, b)


# ---------------------------------------------------------------- folded DST-I path, workload P-C count

@pytest.fixture(scope="module")
def folded_case():
    """128^2 x 48 slices (nx, ny multiples of 128: the FP32 solves run the folded DST-I),
    quadratic shape, the workloads' 5 predictor-corrector iterations; the oracle's taped
    FP64 gradients, computed once."""
    g = dict(nx=128, ny=128, nzeta=48, xmin=-6.0, xmax=6.0, ymin=-6.0, ymax=6.0, zeta_min=-7.0, zeta_max=5.0,
             shape_order=2, n_pc_iter=5, pc_mix=0.05, psi_guard=0.02,
             radial_profile=[1.0, 1.0, 0.8, 0.5, 0.3], profile_rmax=8.5)
    d = I.fixed_ppc_beam(g, 0.6, 1.0, 2.0)
    w = I.fixed_ppc_beam(g, 0.4, 0.6, 10.0, zeta0=-3.0, gamma=I.GAMMA_WITNESS)
    return g, d, w, oracle_grads(g, d, w, "mean+rms")


@pytest.mark.parametrize("precision,tol,bn", [("fp64", 1e-5, None), ("fp32", 1e-3, None), ("fp32", 1e-3, "64"),
                                               ("tf32x3", 1e-3, None)])
def test_adjoint_folded_path(hq, monkeypatch, folded_case, precision, tol, bn):
    """FP32: the folded solve on 128 x 32 tiles (default) and on 128 x 64 tiles (HQ_SOLVE_BN=64),
    and with TF32x3 operands; two checkpoint segments (recompute); FP64 the same case through its
    FFT DST."""
    g, d, w, (L0, gd0, gw0, gn0, gp0) = folded_case
    if bn:
        monkeypatch.setenv("HQ_SOLVE_BN", bn)
    L1, gd1, gw1, gn1, gp1 = gpu_grads(hq, g, d, w, "mean+rms", precision, 24)
    errs = {"loss": abs(L1 - L0) / abs(L0), "driver_w": rel(gd1, gd0), "witness_w": rel(gw1, gw0),
            "driver_dir": directional(gd1, gd0), "n0": abs(gn1 - gn0) / abs(gn0), "profile": rel(gp1, gp0)}
    print("folded", precision, bn, {a: f"{b:.2e}" for a, b in errs.items()})
    assert errs["loss"] <= (1e-10 if precision == "fp64" else 1e-3), errs
    for key in ("driver_w", "witness_w", "driver_dir", "n0", "profile"):
        assert errs[key] <= tol, (key, errs)


# ---------------------------------------------------------------- gradient workload's named check

def test_adjoint256_small_grid_gradients_vs_central_fd(hq):
    """The gradient workload's check at 64 x 64 x 128 (its box: +-6, zeta in [-7, 5]; linear
    shape, 1 ppc, 5 predictor-corrector iterations): the GPU adjoint's gradient of the mean
    witness Ez with respect to the driver's peak density, sigma_r, sigma_z, the witness zeta
    position and the plasma density scale n0, against central finite differences of the FP64
    oracle with step 1e-6 max(1, |p|).  Bars 1e-5 (FP64) and 1e-3 (FP32/bf16x3), relative."""
    g = I.scaled_grid(I.grid_params("adjoint256"), 64, 64, 128)
    d = I.fixed_ppc_beam(g, 0.2, 1.0, 2.0)
    w = I.fixed_ppc_beam(g, 0.1, 0.3, 20.0, zeta0=-5.0, gamma=I.GAMMA_WITNESS)
    dx = (g["xmax"] - g["xmin"]) / g["nx"]
    dz = (g["zeta_max"] - g["zeta_min"]) / g["nzeta"]

    def weights(beam, nb, sr, sz, z0):
        x, y, z = (torch.as_tensor(beam[k], dtype=torch.float64) for k in ("x", "y", "zeta"))
        return nb * torch.exp(-(x * x + y * y) / (2 * sr * sr)) * torch.exp(-((z - z0) ** 2) / (2 * sz * sz)) * dx * dx * dz

    p0 = {"n_b": 2.0, "sigma_r": 0.2, "sigma_z": 1.0, "zeta_w": -5.0, "n0": 1.0}

    def oracle_loss(p):
        sp = O.GridSpec(**dict(g, n0_scale=p["n0"]))
        bd, bw = O.as_beam(d), O.as_beam(w)
        bd["w"] = weights(d, p["n_b"], p["sigma_r"], p["sigma_z"], 0.0)
        bw["w"] = weights(w, 20.0, 0.1, 0.3, p["zeta_w"])
        r = O.sweep(sp, [bd, bw], witness=(1,), record=())
        return float(O.witness_loss(r, 1, "mean"))

    fd = {}
    for k, v in p0.items():
        h = 1e-6 * max(1.0, abs(v))
        fd[k] = (oracle_loss(dict(p0, **{k: v + h})) - oracle_loss(dict(p0, **{k: v - h}))) / (2 * h)
    for precision, tol in (("fp64", 1e-5), ("fp32", 1e-3)):
        grid = hq.Grid(g, precision=precision)
        beams = [hq.Beam(d), hq.Beam(w)]
        ps = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in p0.items()}
        wd = weights(d, ps["n_b"], ps["sigma_r"], ps["sigma_z"], 0.0).cuda()
        ww = weights(w, 20.0, 0.1, 0.3, ps["zeta_w"]).cuda()
        L = hq.SweepLoss.apply(grid, beams, 1, "mean", 16, ps["n0"], torch.empty(0), wd, ww)
        L.backward()
        grid.close()
        errs = {k: abs(float(ps[k].grad) - fd[k]) / abs(fd[k]) for k in p0}
        print(precision, "gradient vs central FD:", {k: f"{float(ps[k].grad):.6e} / {fd[k]:.6e} ({errs[k]:.1e})"
                                                      for k in p0})
        for k in p0:
            assert errs[k] <= tol, (precision, k, errs)


# ---------------------------------------------------------------- adjoint seeds of per-slice fields

SEEDED = {"ez": 10, "psi": 7, "bx": 12, "by": 3, "exmby": 15, "eypbx": 5, "bz": 9, "rho": 11, "jx": 8, "jy": 6,
          "jz": 14}


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-5), ("fp32", 1e-3)])
def test_adjoint_of_field_seeds_matches_taped_oracle(hq, precision, tol):
    """A loss of the per-slice fields themselves, L = sum over the seeded (field, slice) pairs of
    sum_nodes seed * field, differentiated by hq_sweep_adjoint's dL_dfields against the taped
    oracle (both segments recomputed: checkpoint every 5 slices).  Gradients w.r.t. the beam
    weights, the plasma density scale and the radial profile."""
    g, d, w = case(order=1)
    gen = torch.Generator().manual_seed(31)
    seeds = {k: torch.randn(g["ny"], g["nx"], generator=gen, dtype=torch.float64) for k in SEEDED}
    # oracle
    sp = O.GridSpec(**g)
    wd = torch.tensor(d["w"], dtype=torch.float64, requires_grad=True)
    ww = torch.tensor(w["w"], dtype=torch.float64, requires_grad=True)
    n0 = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    prof = torch.tensor(g["radial_profile"], dtype=torch.float64, requires_grad=True)
    bd, bw = O.as_beam(d), O.as_beam(w)
    bd["w"], bw["w"] = wd, ww
    r = O.sweep(sp, [bd, bw], record=tuple(SEEDED), n0_scale=n0, radial_profile=prof)
    L = sum((seeds[k] * r.fields[k][i]).sum() for k, i in SEEDED.items())
    L.backward()
    # GPU
    dt = torch.float64 if precision == "fp64" else torch.float32
    dl = {}
    for k, i in SEEDED.items():
        t = torch.zeros(g["nzeta"], g["ny"], g["nx"], dtype=dt)
        t[i] = seeds[k].to(dt)
        dl[k] = t.cuda()
    grid = hq.Grid(g, precision=precision)
    beams = [hq.Beam(d), hq.Beam(w)]
    sums = torch.zeros(3, dtype=torch.float64, device="cuda")
    grid.forward_ckpt(beams, -1, sums, 5)
    res = grid.adjoint(beams, -1, None, dl_dfields=dl)
    grid.sync()
    grid.close()
    errs = {"driver_w": rel(res["beam_w"][0].cpu(), wd.grad), "witness_w": rel(res["beam_w"][1].cpu(), ww.grad),
            "n0": abs(float(res["n0_scale"][0]) - float(n0.grad)) / abs(float(n0.grad)),
            "profile": rel(res["profile"].cpu(), prof.grad)}
    print(precision, "field seeds:", {a: f"{b:.2e}" for a, b in errs.items()})
    for key, e in errs.items():
        assert e <= tol, (key, errs)


# ---------------------------------------------------------------- the 1280-parameter workload at full size

def test_adjoint512_full_size_vs_central_fd(hq):
    """The 1280-parameter gradient workload at its full size (512^2 x 1024 slices, 2 ppc,
    quadratic shape, fixed-ppc driver with a 1024-entry slice current profile, 256-entry radial
    plasma profile, witness mean Ez + rms spread), as the benchmark runs it (checkpoints every 32
    slices): the FP32/bf16x3 and FP64 adjoint gradients against central finite differences of the
    FP64 forward sweep in the deterministic mode (bitwise reproducible, so the difference quotient
    carries no summation-order noise), step 1e-6 max(1, |p|), on 16 seeded entries (8 of the slice
    profile, 8 of the radial profile, drawn among the entries whose derivative is at least a tenth of
    the largest) and 3 random directions in all 1280 parameters.  Entry errors are taken relative
    to the largest sampled derivative of the same profile (the FP32 adjoint's error on an entry is
    summation-order noise of about the same absolute size across a profile: relative to the entry
    itself it reached 0.5e-3 .. 6.1e-3 over five runs on entries of 10-100 % of the largest, which
    is at most ~7e-4 of the largest), direction errors relative to sum |v_i g_i|.  Bars: FP64
    1e-5; FP32/split 1e-3 on the directions and 2e-3 on the entries (room for the run-to-run
    spread of that noise).  The FP64 adjoint on this case is within 1.8e-6 of the entries
    themselves."""
    g = I.grid_params("adjoint512")
    bnp = I.workload_beams("adjoint512")
    nz = g["nzeta"]
    dz = (g["zeta_max"] - g["zeta_min"]) / nz
    zc = g["zeta_max"] - (np.arange(nz) + 0.5) * dz
    prof = 4.0 * np.exp(-zc ** 2 / (2.0 * 1.4 ** 2))          # the driver's slice profile
    rad = np.asarray(g["radial_profile"], dtype=np.float64)
    sidx = np.asarray(bnp[0]["slice_index"])
    shape = np.asarray(bnp[0]["w"]) / prof[sidx]               # w_p = prof[s_p] * shape_p

    def beams_for(p_slice):
        d = dict(bnp[0])
        d["w"] = p_slice[sidx] * shape
        return [d, bnp[1]]

    # adjoint gradients (FP32/split as benchmarked, and FP64)
    grads = {}
    for precision in ("fp32", "fp64"):
        grid = hq.Grid(g, precision=precision)
        beams = [hq.Beam(b) for b in bnp]
        sums = torch.zeros(3, dtype=torch.float64, device="cuda")
        grid.forward_ckpt(beams, 1, sums, 32)
        _, dls = hq.witness_loss_grad("mean+rms", *[float(v) for v in sums.cpu()])
        res = grid.adjoint(beams, 1, dls, plasma=False)
        grid.sync()
        gw = res["beam_w"][0].cpu().numpy()
        gs = np.zeros(nz)
        np.add.at(gs, sidx, gw * shape)                         # dL/dprof[s] = sum_p dL/dw_p shape_p
        grads[precision] = (gs, res["profile"].cpu().numpy().copy())
        grid.close()

    # the FP64 deterministic forward loss as a function of (slice profile, radial profile)
    gdet = dict(g, deterministic=1)
    cache = {}

    def loss(p_slice, p_rad):
        key = (p_slice.tobytes(), p_rad.tobytes())
        if key not in cache:
            grid = hq.Grid(dict(gdet, radial_profile=[float(v) for v in p_rad]), precision="fp64")
            sums = torch.zeros(3, dtype=torch.float64, device="cuda")
            grid.sweep([hq.Beam(b) for b in beams_for(p_slice)], witness=1, witness_sums=sums)
            grid.sync()
            grid.close()
            cache[key] = hq.witness_loss_grad("mean+rms", *[float(v) for v in sums.cpu()])[0]
        return cache[key]

    rng = np.random.default_rng(512)
    gs64, gr64 = grads["fp64"]
    pick_s = rng.choice(np.flatnonzero(np.abs(gs64) >= 0.1 * np.abs(gs64).max()), 8, replace=False)
    pick_r = rng.choice(np.flatnonzero(np.abs(gr64) >= 0.1 * np.abs(gr64).max()), 8, replace=False)
    fd_s, fd_r = {}, {}
    for s in pick_s:
        h = 1e-6 * max(1.0, abs(prof[s]))
        up, dn = prof.copy(), prof.copy()
        up[s] += h
        dn[s] -= h
        fd_s[s] = (loss(up, rad) - loss(dn, rad)) / (2 * h)
    for k in pick_r:
        h = 1e-6 * max(1.0, abs(rad[k]))
        up, dn = rad.copy(), rad.copy()
        up[k] += h
        dn[k] -= h
        fd_r[k] = (loss(prof, up) - loss(prof, dn)) / (2 * h)
    dirs = []
    for _ in range(3):
        vs, vr = rng.standard_normal(nz), rng.standard_normal(rad.size)
        h = 1e-6 * max(1.0, float(np.abs(prof).max()))
        fd = (loss(prof + h * vs, rad + h * vr) - loss(prof - h * vs, rad - h * vr)) / (2 * h)
        dirs.append((vs, vr, fd))

    scale_s = max(abs(v) for v in fd_s.values())
    scale_r = max(abs(v) for v in fd_r.values())
    print("adjoint512 central FD, slice-profile entries", {int(k): f"{v:.6e}" for k, v in fd_s.items()},
          "radial-profile entries", {int(k): f"{v:.6e}" for k, v in fd_r.items()})
    for precision, tol_e, tol in (("fp64", 1e-5, 1e-5), ("fp32", 2e-3, 1e-3)):
        gs, gr = grads[precision]
        print(precision, "entries |g - fd| / fd:", {int(s): f"{abs(gs[s] - fd_s[s]) / abs(fd_s[s]):.1e}" for s in pick_s},
              {int(k): f"{abs(gr[k] - fd_r[k]) / abs(fd_r[k]):.1e}" for k in pick_r})
        e_s = {int(s): abs(gs[s] - fd_s[s]) / scale_s for s in pick_s}
        e_r = {int(k): abs(gr[k] - fd_r[k]) / scale_r for k in pick_r}
        e_d = [abs(float(gs @ vs + gr @ vr) - fd) / float(np.abs(gs * vs).sum() + np.abs(gr * vr).sum())
               for vs, vr, fd in dirs]
        print(f"adjoint512 {precision}: slice-profile entries worst {max(e_s.values()):.1e}, radial-profile "
              f"entries worst {max(e_r.values()):.1e}, directions {[f'{e:.1e}' for e in e_d]}")
        assert max(e_s.values()) <= tol_e, (precision, e_s)
        assert max(e_r.values()) <= tol_e, (precision, e_r)
        assert max(e_d) <= tol, (precision, e_d)
