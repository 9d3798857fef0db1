"""The allocation-free Poisson entry point, hq_poisson_solve_static.

Some callers cannot allocate device memory (a host application that reserved the
device pool up front, a latency-critical loop where cudaMalloc would stall the
device).  hq_poisson_solve_static serves them with all its scratch in one fixed
static device array.  This test calls it through the C ABI, twice in a row with
different grid sizes (so the second call must not see the first call's leftovers
in the shared array), and checks each result against the regular grid-based
solve hq_poisson_solve within the bf16x3 Poisson tolerance used by the other
GPU tests (3e-5 relative L2).  It also checks that a size beyond the static
array's limit is refused with a clear message.  The file name sorts last so that
a run stopping at the first failure has already run every other test.
"""
import ctypes as C

import pytest
import torch

pytestmark = pytest.mark.gpu

TOL = 3e-5  # bf16x3 Dirichlet solve, as in test_gpu_parity.test_poisson_bf16x3


def rel(a, b):
    a, b = a.double(), b.double()
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def test_static_scratch_solve_matches_grid_solve():
    from paper_2109_10277_gb300 import hq
    lib = hq.load()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    gen = torch.Generator(device="cuda").manual_seed(20211)
    cases = [  # (nx, ny, nrhs, box): the second call is smaller and non-square
        (512, 512, 3, (-8.0, 8.0, -8.0, 8.0)),
        (96, 80, 2, (-5.0, 5.0, -3.0, 4.0)),
    ]
    for nx, ny, nrhs, (x0, x1, y0, y1) in cases:
        g = dict(nx=nx, ny=ny, nzeta=4, xmin=x0, xmax=x1, ymin=y0, ymax=y1, zeta_min=0.0, zeta_max=1.0)
        src = torch.randn(nrhs, ny, nx, dtype=torch.float32, device="cuda", generator=gen)
        grid = hq.Grid(g, precision="fp32", stream=stream)
        ref = grid.poisson_solve(src)
        out = torch.full_like(src, float("nan"))
        st = lib.hq_poisson_solve_static(C.c_void_p(src.data_ptr()), C.c_void_p(out.data_ptr()), nx, ny,
                                         (x1 - x0) / nx, (y1 - y0) / ny, nrhs, C.c_void_p(stream.cuda_stream))
        assert st == 0, lib.hq_last_error(None)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        e = rel(out, ref)
        assert e <= TOL, (nx, ny, e)
        grid.close()


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
