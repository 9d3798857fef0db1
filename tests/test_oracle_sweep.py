"""Whole-loop pins for the oracle's quasi-static sweep (Sec. 2 slice routine, Fig. 1).

  * no beam: every field but chi is exactly zero and the plasma does not move;
  * an on-axis beam on a symmetric grid gives the mirror/swap parities;
  * Ez and -d(psi)/d(zeta), solved independently, agree to O(dzeta^2, dx^2);
  * sum over nodes of the plasma (rho - Jz) is conserved slice to slice;
  * a weak driver reproduces the discrete linear wake, Phi_hat = rho_hat_b/(lambda - 1),
    Ez = int cos(zeta' - zeta) Phi dzeta', with rho_b from the driver's closed form, at the
    workloads' predictor-corrector setting, the error falling as dzeta and dx shrink;
  * the predictor-corrector's lag behind a converged iteration is second order in dzeta;
  * beam binning matches a brute-force per-particle floor.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2109_10277_gb300 import inputs as I


def linear_grid(nx=32, nz=32, order=1, npc=5, **kw):
    g = dict(nx=nx, ny=nx, nzeta=nz, xmin=-6.0, xmax=6.0, ymin=-6.0, ymax=6.0,
             zeta_min=-7.0, zeta_max=5.0, shape_order=order, n_pc_iter=npc, pc_mix=0.05)
    g.update(kw)
    return g


def test_zero_beam_invariant():
    g = linear_grid(nx=24, nz=12, order=2)
    sp = O.GridSpec(**g)
    r = O.sweep(sp, [])
    for k, v in r.fields.items():
        if k != "chi":
            assert torch.all(v == 0), k
    st0 = O.plasma_init(sp)
    for k in ("x", "y", "ux", "uy", "psi"):
        assert torch.equal(r.plasma[k], st0[k]), k


@pytest.mark.parametrize("order", [1, 2])
def test_symmetry_on_axis_beam(order):
    g = linear_grid(nx=32, nz=24, order=order)
    sp = O.GridSpec(**g)
    beam = O.as_beam(I.fixed_ppc_beam(g, 0.8, 1.0, 0.5))
    r = O.sweep(sp, [beam])
    N = sp.nx
    mx = lambda F: torch.cat([F[..., :1], F[..., 1:].flip(-1)], -1)  # noqa: E731  node j -> N-j
    my = lambda F: torch.cat([F[..., :1, :], F[..., 1:, :].flip(-2)], -2)  # noqa: E731
    sw = lambda F: F.transpose(-1, -2)  # noqa: E731
    f = r.fields
    tol = lambda F: 1e-10 * float(F.abs().max()) + 1e-300  # noqa: E731
    for k in ("rho", "jz", "psi", "ez", "chi"):
        assert float((f[k] - mx(f[k])).abs().max()) <= tol(f[k]), k
        assert float((f[k] - my(f[k])).abs().max()) <= tol(f[k]), k
        assert float((f[k] - sw(f[k])).abs().max()) <= tol(f[k]), k
    assert float((f["bx"] + my(f["bx"])).abs().max()) <= tol(f["bx"])
    assert float((f["bx"] - mx(f["bx"])).abs().max()) <= tol(f["bx"])
    assert float((f["by"] + mx(f["by"])).abs().max()) <= tol(f["by"])
    assert float((f["bx"] + sw(f["by"])).abs().max()) <= tol(f["bx"])
    assert float((f["exmby"] + mx(f["exmby"])).abs().max()) <= tol(f["exmby"])
    assert float((f["eypbx"] - sw(f["exmby"])).abs().max()) <= tol(f["exmby"])
    # curl(J_perp) is odd in x, odd in y and antisymmetric under x <-> y (zero only in the continuum)
    assert float((f["bz"] + mx(f["bz"])).abs().max()) <= tol(f["bz"])
    assert float((f["bz"] + my(f["bz"])).abs().max()) <= tol(f["bz"])
    assert float((f["bz"] + sw(f["bz"])).abs().max()) <= tol(f["bz"])
    assert float(f["ez"].abs().max()) > 0


def test_ez_is_minus_dzeta_psi():
    errs = []
    for nz in (32, 64):
        g = linear_grid(nx=32, nz=nz, npc=20)
        sp = O.GridSpec(**g)
        beam = O.as_beam(I.fixed_ppc_beam(g, 1.0, 1.0, 1e-3))
        r = O.sweep(sp, [beam], record=("ez", "psi"))
        ez, psi = r.fields["ez"], r.fields["psi"]
        dpsi = -(psi[:-2] - psi[2:]) / (2 * sp.dzeta)
        e = ez[1:-1]
        errs.append(float(torch.linalg.norm(e - dpsi) / torch.linalg.norm(e)))
    assert errs[0] < 0.05 and errs[1] < errs[0], errs


def test_plasma_rho_minus_jz_conserved():
    # plasma column that ends 1.7 k_p^-1 inside the wall, so no weighted particle deposits on it
    prof = [1.0 if k <= 7 else 0.0 for k in range(17)]
    g = linear_grid(nx=32, nz=32, order=2, radial_profile=prof, profile_rmax=6.0 * math.sqrt(2.0))
    sp = O.GridSpec(**g)
    beam = O.as_beam(I.fixed_ppc_beam(g, 0.6, 1.0, 0.2))
    r = O.sweep(sp, [beam], record=("rho", "jz"))
    st0 = O.plasma_init(sp)
    ion = O.ion_background(sp, st0)
    csr = O.beam_csr(sp, O.beam_bins(sp, beam["zeta"]))
    sums = []
    for i in range(sp.nzeta):
        brho, bjz = O.beam_deposit_slice(sp, beam, csr[1][csr[0][i]:csr[0][i + 1]], ("rho", "jz"))
        plasma = r.fields["rho"][i] - r.fields["jz"][i] - ion - (brho - bjz)
        sums.append(float(plasma.sum()))
    expect = O.PLASMA_Q * float(st0["w"].sum()) / (sp.dx * sp.dy)
    assert max(abs(s - expect) for s in sums) <= 1e-12 * abs(expect)
    assert float(r.fields["jz"].abs().max()) > 1e-3  # the plasma did respond


def analytic_beam_rho(sp, sr, sz, nb0, zeta0=0.0, charge=-1.0):
    """Charge density q n_b of the fixed-ppc Gaussian driver on the nodes of every slice, from
    its closed form n_b = nb0 exp(-r^2 / 2 sr^2) exp(-(zeta - zeta0)^2 / 2 sz^2) at the node
    positions and slice centres (not through the oracle's deposit)."""
    xs = sp.xmin + np.arange(sp.nx) * sp.dx
    ys = sp.ymin + np.arange(sp.ny) * sp.dy
    zc = sp.zeta_max - (np.arange(sp.nzeta) + 0.5) * sp.dzeta
    r2 = xs[None, :] ** 2 + ys[:, None] ** 2
    out = charge * nb0 * np.exp(-r2 / (2 * sr ** 2))[None] * np.exp(-(zc - zeta0) ** 2 / (2 * sz ** 2))[:, None, None]
    out[:, 0, :] = 0.0
    out[:, :, 0] = 0.0
    return out


def screened_solve(sp, s):
    """Phi with (L - 1) Phi = s on the interior nodes (L the 5-point Laplacian, Phi = 0 on the
    wall), through scipy's DST-I (independent of the oracle's matrix DST)."""
    import scipy.fft as F
    kx = np.arange(1, sp.nx)
    ky = np.arange(1, sp.ny)
    lam = (-(4.0 / sp.dx ** 2) * np.sin(np.pi * kx / (2 * sp.nx)) ** 2)[None, :] + \
          (-(4.0 / sp.dy ** 2) * np.sin(np.pi * ky / (2 * sp.ny)) ** 2)[:, None]
    hat = F.dstn(s[1:, 1:], type=1) / (lam - 1.0)
    out = np.zeros_like(s)
    out[1:, 1:] = F.idstn(hat, type=1)
    return out


def linear_wake_error(nx, nz, nb0, npc=5, sr=1.0, sz=1.0):
    """rel-L2 of the oracle's on-axis Ez against the discrete linear wake of a weak fixed-ppc
    driver over the head of the box to one plasma period behind the driver centre.

    Linear cold-fluid response (from the psi, Ez equations of Sec. 2 with a small density
    perturbation): (L - 1) Phi = q n_b on each slice and Ez(zeta) = int_zeta^zeta_max
    cos(zeta' - zeta) Phi(zeta') dzeta' with Phi piecewise constant over the slices.  The
    driver density comes from its closed form, the solve from scipy's DST-I."""
    g = linear_grid(nx=nx, nz=nz, npc=npc)
    sp = O.GridSpec(**g)
    beam = O.as_beam(I.fixed_ppc_beam(g, sr, sz, nb0))
    r = O.sweep(sp, [beam], record=("ez",))
    ez = r.fields["ez"][:, nx // 2, nx // 2].numpy()
    dz = sp.dzeta
    zc = sp.zeta_max - (np.arange(nz) + 0.5) * dz
    rho_b = analytic_beam_rho(sp, sr, sz, nb0)
    phi = np.array([screened_solve(sp, rho_b[i])[nx // 2, nx // 2] for i in range(nz)])
    lin = np.zeros(nz)
    for i in range(nz):
        for k in range(i + 1):  # Phi constant over each slice; integrate cos(z' - zeta_i) from zeta_i up
            hi = zc[k] + dz / 2
            lo = max(zc[k] - dz / 2, zc[i])
            lin[i] += phi[k] * (math.sin(hi - zc[i]) - math.sin(lo - zc[i]))
    win = zc >= -2 * math.pi  # head of the box to one plasma period behind the driver centre
    return float(np.sqrt(((ez - lin)[win] ** 2).sum() / (lin[win] ** 2).sum()))


def test_linear_wake_closed_form():
    """At the workloads' predictor-corrector setting (5 iterations, mixing 0.05)."""
    e64 = linear_wake_error(64, 64, 1e-3)
    assert e64 < 5e-2, e64


@pytest.mark.slow
def test_linear_wake_converges_under_refinement():
    """The same error falls when dzeta is halved (the predictor-corrector's lag behind the
    converged B_perp is O(dzeta^2)) and again when dx is halved too (measured: 4.5 %,
    2.7 %, 0.9 %)."""
    e64 = linear_wake_error(64, 64, 1e-3)
    e64z = linear_wake_error(64, 128, 1e-3)
    e128 = linear_wake_error(128, 128, 1e-3)
    assert e64z < 0.75 * e64 and e128 < 0.4 * e64 and e128 < 1.5e-2, (e64, e64z, e128)


@pytest.mark.slow
def test_predictor_corrector_lag_is_second_order_in_dzeta():
    """Reading of the predictor-corrector: guess 2B(i-1) - B(i-2), 5 iterations mixing 0.05.
    Its fields differ from those of an iteration run to convergence (150 iterations, residual
    ~1e-5) by an amount that falls at least 4x when dzeta is halved (second order: the guess's
    extrapolation error is O(dzeta^2) and the lag it leaves decays over the next slices), so
    the setting converges to the solution of the discrete equations as dzeta -> 0."""
    lag = []
    for nz in (32, 64):
        g = dict(nx=32, ny=32, nzeta=nz, xmin=-6.0, xmax=6.0, ymin=-6.0, ymax=6.0, zeta_min=-7.0, zeta_max=5.0,
                 shape_order=1, n_pc_iter=5, pc_mix=0.05)
        beam = O.as_beam(I.fixed_ppc_beam(g, 0.6, 1.0, 1e-2))
        r5 = O.sweep(O.GridSpec(**g), [beam], record=("bx", "ez", "psi"))
        rc = O.sweep(O.GridSpec(**dict(g, n_pc_iter=150)), [beam], record=("bx", "ez", "psi"))
        assert max(rc.pc_residual) < 1e-3
        lag.append({k: float(torch.linalg.norm(r5.fields[k] - rc.fields[k]) / torch.linalg.norm(rc.fields[k]))
                    for k in ("bx", "ez", "psi")})
    for k in ("bx", "ez", "psi"):
        assert lag[1][k] < 0.25 * lag[0][k], (k, lag)


def test_beam_binning_brute_force():
    g = linear_grid(nx=16, nz=40)
    sp = O.GridSpec(**g)
    b = I.random_beam(3000, 0.5, 0.5, 3.0, 1.0, zeta0=-1.0)
    beam = O.as_beam(b)
    bins = O.beam_bins(sp, beam["zeta"])
    off, order = O.beam_csr(sp, bins)
    ref = []
    for z in b["zeta"]:
        t = math.floor((sp.zeta_max - float(z)) / sp.dzeta)
        ref.append(t if 0 <= t < sp.nzeta else -1)
    ref = np.array(ref)
    assert np.array_equal(bins.numpy(), ref)
    for i in range(sp.nzeta):
        members = sorted(order[off[i]:off[i + 1]].tolist())
        assert members == sorted(np.nonzero(ref == i)[0].tolist())
    assert int(off[-1]) == int((ref >= 0).sum())


def test_plasma_permutation_only_reorders_sums():
    """The plasma_perm option changes the summation order, not the arithmetic."""
    g = linear_grid(nx=24, nz=16, order=2)
    sp = O.GridSpec(**g)
    beam = O.as_beam(I.fixed_ppc_beam(g, 0.8, 1.0, 0.3))
    a = O.sweep(sp, [beam], record=("ez", "bx"))
    perm = torch.as_tensor(np.random.default_rng(3).permutation(sp.nx * sp.ny))
    b = O.sweep(sp, [beam], record=("ez", "bx"), plasma_perm=perm)
    for k in ("ez", "bx"):
        assert float((a.fields[k] - b.fields[k]).abs().max()) <= 1e-9 * float(a.fields[k].abs().max())
    assert torch.allclose(a.plasma["x"], b.plasma["x"], rtol=0, atol=1e-12)


def test_working_precision_knob():
    """working_precision(float32) runs the same steps in single precision (a floor probe):
    fields come out FP32, differ from the FP64 sweep by a small nonzero amount, and the
    default precision is restored afterwards (an FP64 rerun is bit-identical)."""
    g = linear_grid(nx=24, nz=14, order=2)
    sp = O.GridSpec(**g)
    beams = [O.as_beam(I.random_beam(3000, 0.6, 0.6, 1.0, 0.8, zeta0=2.0, seed=5))]
    ref = O.sweep(sp, beams, record=("ez", "psi"))
    with O.working_precision(torch.float32):
        r32 = O.sweep(sp, [O.as_beam(I.random_beam(3000, 0.6, 0.6, 1.0, 0.8, zeta0=2.0, seed=5))],
                      record=("ez", "psi"))
    again = O.sweep(sp, [O.as_beam(I.random_beam(3000, 0.6, 0.6, 1.0, 0.8, zeta0=2.0, seed=5))],
                    record=("ez", "psi"))
    for k in ("ez", "psi"):
        assert r32.fields[k].dtype == torch.float32
        d = float(torch.linalg.norm(r32.fields[k].double() - ref.fields[k]) / torch.linalg.norm(ref.fields[k]))
        assert 0.0 < d < 1e-3, (k, d)
        assert torch.equal(again.fields[k], ref.fields[k])


def test_fp64_sweep_floor_from_dst_rounding():
    """The 64^2 FP64 workload (1e5-particle driver) run twice by the oracle, once with the
    matrix DST-I and once with the FFT DST-I: the same sums in another order.  The sweep
    amplifies that last-bit difference to well above 1e-12 on some field-slices (measured:
    rho 3.4e-11, Bx 1.6e-10, Bz 6.8e-11 per-slice rel-L2), so no implementation whose
    transform rounds differently from the oracle's can reach a flat 1e-12 per field and
    slice; both runs still agree to ~1e-10 of each field's own scale."""
    g = I.grid_params("linear64")
    sp = O.GridSpec(**g)
    beams = [O.as_beam(b) for b in I.workload_beams("linear64")]
    rec = ("rho", "ez", "bx", "bz")
    a = O.sweep(sp, beams, record=rec)
    with O.dst_algorithm("fft"):
        b = O.sweep(sp, beams, record=rec)
    worst = {}
    for k in rec:
        A, B = a.fields[k], b.fields[k]
        nb = torch.linalg.norm(A.reshape(A.shape[0], -1), dim=1)
        nd = torch.linalg.norm((A - B).reshape(A.shape[0], -1), dim=1)
        worst[k] = float((nd / torch.clamp(nb, min=1e-6 * float(nb.max()))).max())
        assert float(nd.max()) <= 1e-9 * float(nb.max()), k
    assert max(worst.values()) > 1e-11, worst
