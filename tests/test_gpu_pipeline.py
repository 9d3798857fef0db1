"""The temporal-decomposition pipeline (Sec. 5.2) on the CUDA library: one rank running every
time step box by box (HqEngine: the per-slice C-ABI calls, the next box's beam joining on each
box's last slice) against the serial loop of whole sweeps on the same GPU (hq_sweep_step), and
against the FP64 oracle's serial loop.  The multi-rank message logic is covered on CPU ranks.

Bars (FP64): pipeline vs serial GPU loop, beam coordinates and witness sums within 1e-11 of the
coordinate's spread (the two differ only in the order of atomic additions); vs the oracle, 30x
the oracle's own rounding floor (a rerun with reordered particles and one-ulp deposit noise).
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2109_10277_gb300 import inputs as I
from paper_2109_10277_gb300 import pipeline as PL
from test_gpu_parity import plasma_perm

pytestmark = pytest.mark.gpu

NSTEP = 3
DT = 2.5


@pytest.fixture(scope="module")
def hq():
    from paper_2109_10277_gb300 import hq as _hq
    _hq.load()
    torch.cuda.set_device(0)
    return _hq


def setup(solver):
    g = dict(nx=48, ny=48, nzeta=32, xmin=-4.0, xmax=4.0, ymin=-4.0, ymax=4.0, zeta_min=-3.0, zeta_max=1.0,
             shape_order=2, n_pc_iter=4, pc_mix=0.05, psi_guard=0.02, bperp_solver=solver)
    drv = I.random_beam(30_000, 0.5, 0.5, 1.2, 0.3, zeta0=-0.8, gamma=math.sqrt(5.0))
    wit = I.random_beam(10_000, 0.3, 0.3, 0.3, 1.0, zeta0=-2.2, gamma=3.0, seed=I.SEED_WITNESS)
    wit["ux"] = 0.05 * np.random.Generator(np.random.PCG64(11)).standard_normal(10_000)
    return g, [drv, wit]


def gpu_serial(hq, g, beams):
    grid = hq.Grid(g, precision="fp64")
    hb = [hq.Beam(b) for b in beams]
    sums = []
    for _ in range(NSTEP):
        s = torch.zeros(3, dtype=torch.float64, device="cuda")
        grid.sweep(hb, dt=DT, witness=1, witness_sums=s)
        sums.append(s)
    grid.sync()
    grid.close()
    return [{k: b.t[k].cpu() for k in PL.KEYS} for b in hb], [s.cpu() for s in sums]


def gpu_pipeline(hq, g, beams, n_boxes):
    grid = hq.Grid(g, precision="fp64")
    eng = PL.HqEngine(grid, [(b["charge"], b["mass"]) for b in beams], DT, witness=1)
    plan = PL.Plan(nzeta=g["nzeta"], n_boxes=n_boxes, n_steps=NSTEP)
    res = PL.run_rank(eng, plan, 0, PL.LocalTransport(), [PL.with_ids(b, "cuda") for b in beams])
    grid.sync()
    grid.close()
    final = PL.assemble([res], 2)
    return ([{k: v.cpu() for k, v in b.items()} for b in final],
            [res.diagnostics[t]["witness_sums"].cpu() for t in range(NSTEP)])


def oracle_serial(g, beams, perturbed=False):
    sp = O.GridSpec(**g)
    bs = [O.as_beam(b) for b in beams]
    sums = []
    for t in range(NSTEP):
        kw = {}
        if perturbed:
            kw = dict(plasma_perm=plasma_perm(g, seed=t + 1), reverse_ion_order=True, deposit_noise=2.0 ** -52,
                      noise_seed=t)
        r = O.sweep(sp, bs, dt=DT, record=(), witness=[1], **kw)
        bs = r.beams
        sums.append(torch.stack(list(r.witness[1])))
    return bs, sums


def spread(v):
    return float((v - v.mean()).abs().max()) + 1e-30


@pytest.mark.parametrize("solver,n_boxes", [("pc", 4), ("pc", 32), ("explicit", 5)])
def test_pipeline_matches_serial_sweeps(hq, solver, n_boxes):
    g, beams = setup(solver)
    pipe, psums = gpu_pipeline(hq, g, beams, n_boxes)
    ser, ssums = gpu_serial(hq, g, beams)
    for s in range(2):
        assert torch.equal(pipe[s]["id"], torch.arange(len(beams[s]["x"])))
        for k in PL.KEYS:
            d = float((pipe[s][k] - ser[s][k]).abs().max()) / spread(ser[s][k])
            assert d <= 1e-11, (s, k, d)
    for t in range(NSTEP):
        assert torch.allclose(psums[t], ssums[t], rtol=1e-11, atol=0.0), (t, psums[t], ssums[t])


def test_pipeline_matches_oracle(hq):
    g, beams = setup("pc")
    pipe, psums = gpu_pipeline(hq, g, beams, 4)
    ref, rsums = oracle_serial(g, beams)
    refp, rpsums = oracle_serial(g, beams, perturbed=True)
    for s in range(2):
        for k in PL.KEYS:
            d = float((pipe[s][k] - ref[s][k]).abs().max()) / spread(ref[s][k])
            f = float((refp[s][k] - ref[s][k]).abs().max()) / spread(ref[s][k])
            assert d <= max(1e-12, 30 * f), (s, k, d, f)
    for t in range(NSTEP):
        for j in range(3):
            r, rp = float(rsums[t][j]), float(rpsums[t][j])
            assert abs(float(psums[t][j]) - r) <= max(1e-12 * abs(r), 30 * abs(rp - r)), (t, j)


def stream_pipeline(hq, g, beams, world, n_boxes, precision="fp64"):
    def make(rank, stream):
        grid = hq.Grid(g, precision=precision, stream=stream)
        return PL.HqEngine(grid, [(b["charge"], b["mass"]) for b in beams], DT, witness=1)
    plan = PL.Plan(nzeta=g["nzeta"], n_boxes=n_boxes, n_steps=NSTEP, world=world)
    res = PL.run_streams(make, plan, [PL.with_ids(b, "cuda") for b in beams])
    torch.cuda.synchronize()
    final = PL.assemble(res, 2)
    diag = {t: d for r in res for t, d in r.diagnostics.items()}
    return ([{k: v.cpu() for k, v in b.items()} for b in final], [diag[t]["witness_sums"].cpu() for t in range(NSTEP)])


@pytest.mark.parametrize("world,n_boxes", [(2, 4), (3, 8)])
def test_stream_ranks_reproduce_serial_sweeps_bitwise(hq, world, n_boxes):
    """Time steps pipelined on one GPU (ranks as threads with their own streams), deterministic
    FP64 mode: the beam after the last step and every step's witness sums are bit for bit those of
    the serial loop of whole sweeps, although the steps overlap on the device."""
    g, beams = setup("pc")
    g = dict(g, deterministic=1)
    pipe, psums = stream_pipeline(hq, g, beams, world, n_boxes)
    ser, ssums = gpu_serial(hq, g, beams)
    for s_ in range(2):
        assert torch.equal(pipe[s_]["id"], torch.arange(len(beams[s_]["x"])))
        for k in PL.KEYS:
            assert torch.equal(pipe[s_][k], ser[s_][k]), (s_, k)
    for t in range(NSTEP):
        assert torch.equal(psums[t], ssums[t]), t


def test_stream_ranks_fp32(hq):
    """The same pipelined on one GPU in FP32: within the FP32 run-to-run noise of the serial loop."""
    g, beams = setup("pc")
    pipe, psums = stream_pipeline(hq, g, beams, 2, 4, precision="fp32")
    grid = hq.Grid(g, precision="fp32")
    hb = [hq.Beam(b) for b in beams]
    for _ in range(NSTEP):
        grid.sweep(hb, dt=DT)
    grid.sync()
    grid.close()
    for s_ in range(2):
        for k in PL.KEYS:
            ref = hb[s_].t[k].cpu()
            d = float((pipe[s_][k] - ref).abs().max()) / spread(ref)
            assert d <= 1e-4, (s_, k, d)


def test_sweep_slices_in_chunks_is_the_sweep(hq):
    """hq_sweep_slices over consecutive ranges equals one hq_sweep_step bit for bit (deterministic
    FP64): fields of every slice, plasma state after the tail, pushed beams; an out-of-order range
    is refused with HQ_ERR_STATE."""
    g, beams = setup("pc")
    g = dict(g, deterministic=1)
    outs = []
    states = []
    pushed = []
    for chunks in ([(0, g["nzeta"])], [(0, 10), (10, 11), (11, 23), (23, g["nzeta"])]):
        grid = hq.Grid(g, precision="fp64")
        out = grid.alloc_out(("rho", "ez", "psi", "bx", "by"))
        hb = [hq.Beam(b) for b in beams]
        if len(chunks) == 1:
            grid.sweep(hb, dt=DT, out=out)
        else:
            for a, b in chunks:
                grid.sweep_slices(hb, a, b, dt=DT, out=out)
        grid.sync()
        outs.append(out)
        states.append(grid.plasma_state())
        pushed.append([{k: v.clone() for k, v in b.t.items()} for b in hb])
        grid.close()
    for k in outs[0]:
        assert torch.equal(outs[0][k], outs[1][k]), k
    for k in ("x", "y", "psi", "ux", "uy", "alive"):
        assert torch.equal(states[0][k], states[1][k]), k
    for a, b in zip(pushed[0], pushed[1]):
        for k in a:
            assert torch.equal(a[k], b[k]), k
    grid = hq.Grid(g, precision="fp64")
    with pytest.raises(hq.HQError) as e:
        grid.sweep_slices([hq.Beam(beams[0])], 5, 8)
    assert e.value.status == 6
    grid.close()
