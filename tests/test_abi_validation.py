"""Argument checks of the C ABI that run on the host before any device work: hq_grid_create's
(every refused descriptor returns its status, HQ_ERR_ARG = 1 for a malformed value and
HQ_ERR_UNSUPPORTED = 7 for a valid but unsupported combination, a message naming the field,
and a NULL handle) and hq_poisson_solve_static's."""
import ctypes as C
import math
import os

import pytest

ARG, UNSUPPORTED = 1, 7


@pytest.fixture(scope="module")
def lib():
    from paper_2109_10277_gb300 import build, hq
    if not os.path.exists(hq.LIB_PATH):
        build.build()
    return hq.load()


def base():
    from paper_2109_10277_gb300 import hq
    return hq.GridDesc(64, 64, 8, -1.0, 1.0, -1.0, 1.0, 0.0, 1.0, 1, 1, 1, None, 0, 0.0, 1.0, 5, 0.05, 0.02,
                       hq.HQ_PREC_FP64)


def species(**kw):
    from paper_2109_10277_gb300 import hq
    s = dict(charge=-1.0, mass=1.0, n0_scale=1.0, ppc_x=1, ppc_y=1, radial_profile=None, n_profile=0,
             profile_rmax=0.0, neutralize=1)
    s.update(kw)
    return hq.SpeciesDesc(**s)


def refuse(lib, d, status, word):
    h = C.c_void_p(12345)
    assert lib.hq_grid_create(C.byref(d), None, C.byref(h)) == status
    assert h.value is None
    msg = lib.hq_last_error(None).decode()
    assert word in msg, msg


def edit(**kw):
    d = base()
    for k, v in kw.items():
        setattr(d, k, v)
    return d


CASES = [
    (dict(nx=7), ARG, "nx"),
    (dict(ny=4097), ARG, "nx, ny"),
    (dict(nzeta=0), ARG, "nzeta"),
    (dict(xmax=-1.0), ARG, "box"),
    (dict(ymin=math.nan), ARG, "box"),
    (dict(zeta_max=math.inf), ARG, "box"),
    (dict(shape_order=4), ARG, "shape_order"),
    (dict(ppc_x=0), ARG, "ppc"),
    (dict(ppc_y=17), ARG, "ppc"),
    (dict(n_pc_iter=-1), ARG, "n_pc_iter"),
    (dict(n_pc_iter=1001), ARG, "n_pc_iter"),
    (dict(pc_mix=math.nan), ARG, "pc_mix"),
    (dict(n0_scale=math.inf), ARG, "n0_scale"),
    (dict(precision=3), ARG, "precision"),
    (dict(bperp_solver=2), ARG, "bperp_solver"),
    (dict(bperp_solver=1, n_pc_iter=0), ARG, "explicit"),
    (dict(bperp_solver=1, n_pc_iter=65), ARG, "explicit"),
    (dict(bperp_solver=1, n0_scale=0.0), ARG, "shift"),
    (dict(resort_every=-1), ARG, "resort_every"),
    (dict(pc_residuals=2), ARG, "pc_residuals"),
    (dict(deterministic=2), ARG, "deterministic"),
    (dict(deterministic=1, precision=1), UNSUPPORTED, "FP64"),
    (dict(deterministic=1, precision=2), UNSUPPORTED, "FP64"),
    (dict(n_species=5), ARG, "n_species"),
    (dict(n_species=1), ARG, "n_species"),       # no species array
    (dict(nx=4096, ny=4096, ppc_x=16, ppc_y=16), ARG, "too many"),
]


@pytest.mark.parametrize("fields,status,word", CASES)
def test_descriptor_is_refused(lib, fields, status, word):
    refuse(lib, edit(**fields), status, word)


def test_radial_profile_needs_two_samples_and_a_radius(lib):
    prof = (C.c_double * 1)(1.0)
    d = edit(radial_profile=C.cast(prof, C.POINTER(C.c_double)), n_profile=1, profile_rmax=2.0)
    refuse(lib, d, ARG, "radial profile")
    prof2 = (C.c_double * 2)(1.0, 0.5)
    d = edit(radial_profile=C.cast(prof2, C.POINTER(C.c_double)), n_profile=2, profile_rmax=0.0)
    refuse(lib, d, ARG, "radial profile")


@pytest.mark.parametrize("bad,word", [
    (dict(mass=0.0), "mass"),
    (dict(mass=-1.0), "mass"),
    (dict(charge=0.0), "charge"),
    (dict(charge=math.nan), "charge"),
    (dict(ppc_x=17), "ppc"),
    (dict(neutralize=2), "neutralize"),
    (dict(n_profile=1, profile_rmax=1.0), "radial profile"),
])
def test_species_is_refused(lib, bad, word):
    arr = (C.c_double * 2)(1.0, 1.0)
    kw = dict(bad)
    if "n_profile" in kw:
        kw["radial_profile"] = C.cast(arr, C.POINTER(C.c_double))
    sp = (type(species()) * 2)(species(), species(**kw))
    from paper_2109_10277_gb300 import hq
    d = edit(species=C.cast(sp, C.POINTER(hq.SpeciesDesc)), n_species=2)
    refuse(lib, d, ARG, word)


def test_species_with_the_resort_is_unsupported(lib):
    from paper_2109_10277_gb300 import hq
    sp = (hq.SpeciesDesc * 1)(species())
    d = edit(species=C.cast(sp, C.POINTER(hq.SpeciesDesc)), n_species=1, resort_every=4)
    refuse(lib, d, UNSUPPORTED, "re-sort")


def test_explicit_solver_shift_counts_the_species(lib):
    """The explicit solver's preconditioner shift is sum q^2 n0 / M over the species: species of
    zero density leave none, and the descriptor is refused even with n0_scale set."""
    from paper_2109_10277_gb300 import hq
    sp = (hq.SpeciesDesc * 2)(species(n0_scale=0.0), species(charge=1.0, mass=100.0, n0_scale=0.0))
    d = edit(species=C.cast(sp, C.POINTER(hq.SpeciesDesc)), n_species=2, bperp_solver=1, n0_scale=1.0)
    refuse(lib, d, ARG, "shift")


@pytest.mark.parametrize("args,word", [
    ((None, 16, 64, 64, 0.1, 0.1, 1), "NULL"),
    ((16, None, 64, 64, 0.1, 0.1, 1), "NULL"),
    ((16, 16, 7, 64, 0.1, 0.1, 1), "8..512"),
    ((16, 16, 64, 513, 0.1, 0.1, 1), "8..512"),
    ((16, 16, 64, 64, 0.1, 0.1, 0), "nrhs"),
    ((16, 16, 64, 64, 0.1, 0.1, 4), "nrhs"),
    ((16, 16, 64, 64, 0.0, 0.1, 1), "dx and dy"),
    ((16, 16, 64, 64, 0.1, math.nan, 1), "dx and dy"),
])
def test_allocation_free_solve_checks_its_arguments(lib, args, word):
    """hq_poisson_solve_static refuses out-of-range arguments with HQ_ERR_ARG before it looks at
    the device or the (never dereferenced, here fake) pointers."""
    src, dst, nx, ny, dx, dy, nrhs = args
    st = lib.hq_poisson_solve_static(C.c_void_p(src) if src else None, C.c_void_p(dst) if dst else None,
                                     nx, ny, C.c_double(dx), C.c_double(dy), nrhs, None)
    assert st == ARG
    assert word in lib.hq_last_error(None).decode()
