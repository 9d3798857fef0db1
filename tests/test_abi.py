"""Host-side checks of the C ABI: the library builds, loads, exports every entry
point declared in include/hq.h, and refuses to run without an sm_103a device
(no CPU fallback).  No compute call is made here."""
import ctypes as C
import os
import re

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "hq.h")).read()
    return sorted(set(re.findall(r"^\s*(?:hq_status|const char\*)\s+(hq_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2109_10277_gb300 import build, hq
    if not os.path.exists(hq.LIB_PATH):
        build.build()
    return hq.load()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("hq_grid_create", "hq_beam_deposit", "hq_advance_slice", "hq_solve_fields", "hq_sweep_step"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2109_10277_gb300 import hq
    for n in declared_symbols():
        assert hasattr(lib, n), n
    assert set(declared_symbols()) == set(hq.EXPORTS)


def test_null_arguments_are_rejected(lib):
    assert lib.hq_grid_create(None, None, None) == 1  # HQ_ERR_ARG
    assert b"NULL" in lib.hq_last_error(None)
    assert lib.hq_advance_slice(None, 0) == 1
    # hq_sync(NULL) synchronizes the device and reports the allocation-free solves' status:
    # HQ_ERR_CUDA without a device, HQ_OK on an idle one
    assert lib.hq_sync(None, None) == (0 if torch.cuda.is_available() else 2)


def test_bad_descriptor_is_rejected(lib):
    from paper_2109_10277_gb300 import hq
    d = hq.GridDesc(4, 64, 8, -1, 1, -1, 1, 0, 1, 1, 1, 1, None, 0, 0.0, 1.0, 5, 0.05, 0.02, 0)
    h = C.c_void_p()
    assert lib.hq_grid_create(C.byref(d), None, C.byref(h)) == 1
    assert b"nx" in lib.hq_last_error(None)
    d = hq.GridDesc(64, 64, 8, -1, 1, -1, 1, 0, 1, 7, 1, 1, None, 0, 0.0, 1.0, 5, 0.05, 0.02, 0)
    assert lib.hq_grid_create(C.byref(d), None, C.byref(h)) == 1
    assert b"shape_order" in lib.hq_last_error(None)


def test_precision_values(lib):
    """The precisions the header declares, the binding's names for them, and an unknown value
    refused as an argument error before any device work."""
    from paper_2109_10277_gb300 import hq
    text = open(os.path.join(ROOT, "include", "hq.h")).read()
    for name, val in (("HQ_PREC_FP64", 0), ("HQ_PREC_FP32_BF16X3", 1), ("HQ_PREC_FP32_TF32X3", 2)):
        assert re.search(rf"\b{name} = {val}\b", text), name
        assert getattr(hq, name) == val
    assert hq.PRECISIONS["tf32x3"] == 2 and hq.PRECISIONS["fp32"] == 1
    d = hq.GridDesc(64, 64, 8, -1, 1, -1, 1, 0, 1, 1, 1, 1, None, 0, 0.0, 1.0, 5, 0.05, 0.02, 3)
    h = C.c_void_p()
    assert lib.hq_grid_create(C.byref(d), None, C.byref(h)) == 1
    assert b"precision" in lib.hq_last_error(None)
    with pytest.raises(ValueError):
        hq.Grid(dict(nx=64, ny=64, nzeta=8, xmin=-1, xmax=1, ymin=-1, ymax=1, zeta_min=0, zeta_max=1),
                precision="fp16")


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU refusal")
def test_no_device_fails_loudly(lib):
    from paper_2109_10277_gb300 import hq
    d = hq.GridDesc(64, 64, 8, -1, 1, -1, 1, 0, 1, 1, 1, 1, None, 0, 0.0, 1.0, 5, 0.05, 0.02, 0)
    h = C.c_void_p()
    st = lib.hq_grid_create(C.byref(d), None, C.byref(h))
    assert st in (2, 7)  # HQ_ERR_CUDA / HQ_ERR_UNSUPPORTED, never a silent CPU path
    assert not h.value
    with pytest.raises(RuntimeError):  # HQError or torch refusing the stream
        hq.Grid(dict(nx=64, ny=64, nzeta=8, xmin=-1, xmax=1, ymin=-1, ymax=1, zeta_min=0, zeta_max=1))


def test_every_runtime_switch_is_documented():
    """Each HQ_* environment variable the library reads is listed in include/hq.h."""
    csrc = os.path.join(ROOT, "paper_2109_10277_gb300", "csrc")
    read = set()
    for f in os.listdir(csrc):
        if f.endswith((".cu", ".cuh")):
            read |= set(re.findall(r'getenv\("(HQ_\w+)"\)', open(os.path.join(csrc, f)).read()))
    header = open(os.path.join(ROOT, "include", "hq.h")).read()
    assert read, "no switches found"
    for name in sorted(read):
        assert re.search(rf"^\s*\*\s+{name}=", header, re.M), name


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors of the C structs have the header's sizes and field offsets (compiled
    with the host C compiler against include/hq.h)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    from paper_2109_10277_gb300 import hq
    checks = {"hq_grid_desc": (hq.GridDesc, ("n_pc_iter", "precision", "bperp_solver", "resort_every",
                                             "deterministic", "species", "n_species", "pc_residuals")),
              "hq_species_desc": (hq.SpeciesDesc, ("mass", "ppc_y", "radial_profile", "neutralize")),
              "hq_beam_view": (hq.BeamView, ("w", "charge", "mass")),
              "hq_field_out": (hq.FieldOut, ("bz",)),
              "hq_plasma_view": (hq.PlasmaView, ("alive", "origin"))}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{os.path.join(ROOT, "include", "hq.h")}"',
             "int main(void) {"]
    for name, (_, fields) in checks.items():
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for f in fields:
            lines.append(f'  printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "sizes.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "sizes"
    r = subprocess.run([cc, str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    for name, (cls, fields) in checks.items():
        assert int(got[name]) == C.sizeof(cls), name
        for f in fields:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, (name, f)
