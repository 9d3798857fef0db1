"""Pin of the oracle in the blowout regime (the regime of the benchmark sweep, where no closed
form of the wake exists): the ion-channel focusing force.

Behind a dense narrow driver (n_b = 5, k_p sigma_r = 0.25) the plasma electrons are expelled from
a region around the axis.  There the source of the psi equation of Sec. 3.2, -(rho - J_z), is
minus the ion density, 1 (the electrons' rho - J_z is the density of their markers, Sec. 3.2
deposition identity, and none are left; the beam's rho_b (1 - beta_b) is ~1e-9), so
psi = -r^2/4 + h with h harmonic, and h is constant near the axis up to O(r^4) for a channel with
the grid's 4-fold symmetry: the transverse force ExmBy = -d psi / dx is x/2 (the 5-point Laplacian
of -r^2/4 is exactly -1 and its central difference exactly x/2, so the discrete solution keeps
this).  By Ez's equation with ExmBy independent of zeta, Ez is flat across the channel.

A dropped or sign-flipped ion background, a wrong psi source sign, a factor in the central
difference or in the Dirichlet solve, or a push that fails to expel the electrons breaks it.
"""
import numpy as np
import pytest

import oracle as O
from paper_2109_10277_gb300 import inputs as I


@pytest.fixture(scope="module")
def bubble():
    g = dict(nx=128, ny=128, nzeta=192, xmin=-4.0, xmax=4.0, ymin=-4.0, ymax=4.0, zeta_min=-6.0, zeta_max=6.0,
             shape_order=2, n_pc_iter=5, pc_mix=0.05, psi_guard=0.02)
    d = I.fixed_ppc_beam(g, 0.25, 0.8, 5.0, zeta0=2.0)
    sp = O.GridSpec(**g)
    r = O.sweep(sp, [O.as_beam(d)], record=("exmby", "rho", "jz", "ez"))
    return sp, r


def channel_rows(sp, r, min_half=8):
    """(slice, half-width) of the slices whose axis row is electron-free over >= min_half nodes
    on each side of the axis node (rho - J_z within 1e-9 of the ion density 1)."""
    src = (r.fields["rho"] - r.fields["jz"]).numpy()
    c = sp.nx // 2
    out = []
    for i in range(sp.nzeta):
        row = src[i, c]
        k = 0
        while c + k + 1 < sp.nx - 1 and abs(row[c + k + 1] - 1.0) < 1e-9 and abs(row[c - k - 1] - 1.0) < 1e-9:
            k += 1
        if k >= min_half:
            out.append((i, k))
    return out


def test_ion_channel_focusing_force_is_x_over_2(bubble):
    sp, r = bubble
    rows = channel_rows(sp, r)
    assert len(rows) >= 20, rows          # the driver does blow the electrons out
    c = sp.nx // 2
    ex = r.fields["exmby"].numpy()
    slopes = []
    for i, k in rows:
        h = k // 2                          # the inner half of the channel
        xs = sp.xmin + np.arange(c - h, c + h + 1) * sp.dx
        slopes.append(np.polyfit(xs, ex[i, c, c - h:c + h + 1], 1)[0])
    slopes = np.asarray(slopes)
    print(f"{len(rows)} channel slices, ExmBy slope {slopes.min():.4f} .. {slopes.max():.4f} "
          f"(median {np.median(slopes):.4f})")
    assert np.all(np.abs(slopes - 0.5) <= 0.01), slopes          # measured 0.494 .. 0.499
    assert abs(np.median(slopes) - 0.5) <= 0.004, slopes


def test_ez_is_flat_across_the_channel(bubble):
    sp, r = bubble
    rows = channel_rows(sp, r)
    assert len(rows) >= 20, rows
    c = sp.nx // 2
    ez = r.fields["ez"].numpy()
    peak = max(abs(ez[i, c, c]) for i, _ in rows)
    spread = max(np.ptp(ez[i, c, c - k // 2:c + k // 2 + 1]) for i, k in rows)
    print(f"Ez spread across the inner channel {spread:.2e} of peak on-axis |Ez| {peak:.3f}")
    assert spread <= 1e-2 * peak, (spread, peak)
