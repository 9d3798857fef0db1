"""The allocation-free Poisson entry point, hq_poisson_solve_static.

Some callers cannot allocate device memory: a host application that reserved the
device memory pool up front and lets no library allocate from it, or a latency-
critical loop where a cudaMalloc or cudaFree would stall the device.
hq_poisson_solve_static serves them with all its scratch in one fixed static device
array.  This test calls it through the C ABI several times in a row:

  * different grid sizes one after the other (a call must not see the previous call's
    leftovers in the shared array), each against the regular grid-based solve
    hq_poisson_solve and against the FP64 oracle's Dirichlet solve, within the bf16x3
    Poisson tolerance used by the other GPU tests (3e-5 relative L2);
  * the first geometry again with new sources (the cached tables are reused);
  * the same nx, ny with another dx (the tables are rebuilt: the solution scales as dx^2);
  * a non-finite source: hq_sync(NULL) reports HQ_ERR_NUMERIC once, then HQ_OK;
  * sizes beyond the static array's limit are refused with a clear message.

The file name sorts last so that a run stopping at the first failure has already run
every other test.
"""
import ctypes as C

import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu

TOL = 3e-5  # bf16x3 Dirichlet solve, as in test_gpu_parity.test_poisson_bf16x3


def rel(a, b):
    a, b = a.double().cpu(), b.double().cpu()
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def static_solve(lib, src, nx, ny, dx, dy, stream):
    out = torch.full_like(src, float("nan"))
    st = lib.hq_poisson_solve_static(C.c_void_p(src.data_ptr()), C.c_void_p(out.data_ptr()), nx, ny, dx, dy,
                                     src.shape[0], C.c_void_p(stream.cuda_stream))
    assert st == 0, lib.hq_last_error(None)
    return out


def test_static_scratch_solve_matches_grid_solve_and_oracle():
    from paper_2109_10277_gb300 import hq
    lib = hq.load()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    gen = torch.Generator(device="cuda").manual_seed(20211)
    cases = [  # (nx, ny, nrhs, box): the second call is smaller and non-square; the third repeats the first
        (512, 512, 3, (-8.0, 8.0, -8.0, 8.0)),
        (96, 80, 2, (-5.0, 5.0, -3.0, 4.0)),
        (512, 512, 3, (-8.0, 8.0, -8.0, 8.0)),
    ]
    for nx, ny, nrhs, (x0, x1, y0, y1) in cases:
        g = dict(nx=nx, ny=ny, nzeta=4, xmin=x0, xmax=x1, ymin=y0, ymax=y1, zeta_min=0.0, zeta_max=1.0)
        src = torch.randn(nrhs, ny, nx, dtype=torch.float32, device="cuda", generator=gen)
        grid = hq.Grid(g, precision="fp32", stream=stream)
        ref = grid.poisson_solve(src)
        out = static_solve(lib, src, nx, ny, (x1 - x0) / nx, (y1 - y0) / ny, stream)
        assert lib.hq_sync(None, None) == 0, lib.hq_last_error(None)
        assert torch.isfinite(out).all()
        e = rel(out, ref)
        assert e <= TOL, (nx, ny, e)
        sp = O.GridSpec(**g)
        for r in range(nrhs):
            eo = rel(out[r], O.poisson_solve(sp, src[r].double().cpu()))
            assert eo <= TOL, (nx, ny, r, eo)
        grid.close()


def test_static_scratch_rebuilds_tables_for_a_new_spacing():
    from paper_2109_10277_gb300 import hq
    lib = hq.load()
    stream = torch.cuda.current_stream()
    src = torch.randn(1, 64, 64, dtype=torch.float32, device="cuda")
    a = static_solve(lib, src, 64, 64, 0.1, 0.1, stream)
    b = static_solve(lib, src, 64, 64, 0.2, 0.2, stream)   # same nx, ny; 5-point operator scales as 1/dx^2
    assert lib.hq_sync(None, None) == 0
    assert rel(b, 4.0 * a) <= TOL
    sp = O.GridSpec(nx=64, ny=64, nzeta=1, xmin=0.0, xmax=12.8, ymin=0.0, ymax=12.8, zeta_min=0.0, zeta_max=1.0)
    assert rel(b[0], O.poisson_solve(sp, src[0].double().cpu())) <= TOL


def test_static_scratch_reports_nonfinite_results():
    from paper_2109_10277_gb300 import hq
    lib = hq.load()
    stream = torch.cuda.current_stream()
    src = torch.randn(1, 64, 64, dtype=torch.float32, device="cuda")
    src[0, 10, 10] = float("inf")
    static_solve(lib, src, 64, 64, 0.1, 0.1, stream)
    assert lib.hq_sync(None, None) == 4  # HQ_ERR_NUMERIC
    assert b"non-finite" in lib.hq_last_error(None)
    assert lib.hq_sync(None, None) == 0  # reported once, then cleared
    src[0, 10, 10] = 0.0
    out = static_solve(lib, src, 64, 64, 0.1, 0.1, stream)
    assert lib.hq_sync(None, None) == 0
    assert torch.isfinite(out).all()


def test_static_scratch_rejects_sizes_beyond_its_limit():
    from paper_2109_10277_gb300 import hq
    lib = hq.load()
    src = torch.zeros(1, 1024, 1024, dtype=torch.float32, device="cuda")
    out = torch.zeros_like(src)
    st = lib.hq_poisson_solve_static(C.c_void_p(src.data_ptr()), C.c_void_p(out.data_ptr()), 1024, 1024, 0.1, 0.1, 1,
                                     None)
    assert st == 1  # HQ_ERR_ARG
    assert b"512" in lib.hq_last_error(None)
    st = lib.hq_poisson_solve_static(C.c_void_p(src.data_ptr()), C.c_void_p(out.data_ptr()), 64, 64, 0.1, 0.1, 4,
                                     None)
    assert st == 1 and b"nrhs" in lib.hq_last_error(None)
