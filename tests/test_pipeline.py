"""The temporal-decomposition pipeline (Sec. 5.2) on CPU ranks.

The pipeline's host logic (which rank computes which step, box partition, routing of pushed
particles into the next step's boxes, the one-box look-ahead for the predictor-corrector's
J_perp(i+1), the beam messages) runs with an engine built on the FP64 oracle's slice loop.  Since
each box keeps its particles in the serial order, the pipeline must reproduce the serial time
loop (one oracle sweep per step) exactly, on one rank and on two and three gloo ranks; particles
cross slices and boxes every step, some enter from ahead of the box and some leave behind it.
"""
import math
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle as O
from paper_2109_10277_gb300 import inputs as I
from paper_2109_10277_gb300 import pipeline as PL

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NSTEP = 4
DT = 2.5
WITNESS = 1


class OracleEngine:
    """Pipeline engine on the oracle's slice loop (O.SliceLoop), one per time step."""

    def __init__(self, spec, species, dt, witness=-1):
        self.spec, self.species, self.dt, self.witness = spec, species, dt, witness
        self.n_species = len(species)
        self.device = torch.device("cpu")
        self.boxes_seen = []

    def slices(self, s, b):
        t = torch.floor((self.spec.zeta_max - b["zeta"]) / self.spec.dzeta)
        nz = self.spec.nzeta
        out = torch.where(t < 0, torch.full_like(t, -1.0), torch.where(t >= nz, torch.full_like(t, nz), t))
        return torch.where(torch.isfinite(t), out, torch.full_like(t, -2.0)).to(torch.int64)

    def begin_step(self, t):
        self.loop = O.SliceLoop(self.spec)
        self.wsum = [torch.zeros((), dtype=torch.float64)] * 3

    def _beam(self, s, b):
        q, m = self.species[s]
        return dict(b, charge=q, mass=m)

    def run_box(self, t, k, slices, parts, next_parts):
        self.boxes_seen.append((t, k))
        beams = [self._beam(s, b) for s, b in enumerate(parts)]
        bins = [self.slices(s, b) for s, b in enumerate(beams)]
        nz = self.spec.nzeta
        for i in slices:
            cur = [(b, torch.nonzero(bins[s] == i).reshape(-1)) for s, b in enumerate(beams)]
            nxt = []
            if i + 1 < nz:
                if i + 1 < slices.stop:
                    nxt = [(b, torch.nonzero(bins[s] == i + 1).reshape(-1)) for s, b in enumerate(beams)]
                else:
                    nb_ = [self._beam(s, b) for s, b in enumerate(next_parts())]
                    nxt = [(b, torch.nonzero(self.slices(s, b) == i + 1).reshape(-1)) for s, b in enumerate(nb_)]
            wit = [self.witness] if self.witness >= 0 else []
            _, _, beams, ws = self.loop.slice(i, cur, nxt, self.dt, wit)
            for w in ws:
                self.wsum = [a + b for a, b in zip(self.wsum, w)]
        return [{k: b[k] for k in PL.KEYS + ("id",)} for b in beams]

    def end_step(self, t):
        return {"witness_sums": torch.stack(self.wsum)}


def setup():
    """32^2 x 16 slices; a low-energy driver (u_z = 2: it slips ~0.27 per step, about one slice)
    and a witness, with particles placed ahead of the box and near its tail."""
    g = dict(nx=32, ny=32, nzeta=16, xmin=-4.0, xmax=4.0, ymin=-4.0, ymax=4.0, zeta_min=-3.0, zeta_max=1.0,
             shape_order=1, n_pc_iter=3, pc_mix=0.05, psi_guard=0.02)
    drv = I.random_beam(3000, 0.5, 0.5, 1.2, 0.3, zeta0=-0.8, gamma=math.sqrt(5.0))
    wit = I.random_beam(1000, 0.3, 0.3, 0.3, 1.0, zeta0=-2.2, gamma=3.0, seed=I.SEED_WITNESS)
    rng = np.random.Generator(np.random.PCG64(11))
    wit["ux"] = 0.05 * rng.standard_normal(1000)
    return g, [drv, wit]


def serial(g, beams):
    spec = O.GridSpec(**g)
    bs = []
    for b in beams:
        ob = O.as_beam(b)
        ob["id"] = torch.arange(len(b["x"]), dtype=torch.int64)
        bs.append(ob)
    sums = []
    for _ in range(NSTEP):
        r = O.sweep(spec, bs, dt=DT, record=(), witness=[WITNESS])
        bs = r.beams
        sums.append(torch.stack(list(r.witness[WITNESS])))
    return bs, sums


def run_pipeline(g, beams, n_boxes, rank=0, world=1, transport=None):
    spec = O.GridSpec(**g)
    eng = OracleEngine(spec, [(b["charge"], b["mass"]) for b in beams], DT, WITNESS)
    plan = PL.Plan(nzeta=g["nzeta"], n_boxes=n_boxes, n_steps=NSTEP, world=world)
    init = [PL.with_ids(b, "cpu") for b in beams] if rank == 0 else None
    res = PL.run_rank(eng, plan, rank, transport or PL.LocalTransport(), init)
    return res, eng


def check_against_serial(results, ref_beams, ref_sums):
    final = PL.assemble(results, 2)
    for s in range(2):
        assert torch.equal(final[s]["id"], ref_beams[s]["id"])
        for k in PL.KEYS:
            assert torch.equal(final[s][k], ref_beams[s][k]), (s, k)
    diag = {t: d for r in results for t, d in r.diagnostics.items()}
    assert sorted(diag) == list(range(NSTEP))
    for t in range(NSTEP):
        assert torch.equal(diag[t]["witness_sums"], ref_sums[t]), t


@pytest.fixture(scope="module")
def reference():
    g, beams = setup()
    return g, beams, serial(g, beams)


def test_setup_exercises_the_routing(reference):
    """The workload crosses boxes: particles slip more than one box length over the run, some
    leave behind the tail, and some sit ahead of the head (in no slice, so never pushed: they
    ride along in box 0 unchanged)."""
    g, beams, (ref, _) = reference
    spec = O.GridSpec(**g)
    b0 = [O.beam_bins(spec, torch.as_tensor(b["zeta"])) for b in beams]
    b1 = [O.beam_bins(spec, r["zeta"]) for r in ref]
    drv0 = torch.as_tensor(beams[0]["zeta"])
    ahead = drv0 > spec.zeta_max
    assert int(ahead.sum()) > 0 and torch.equal(ref[0]["zeta"][ahead], drv0[ahead])
    assert int(((b0[0] >= 0) & (b1[0] < 0)).sum()) > 0                                            # left
    moved = (b1[0] - b0[0])[(b0[0] >= 0) & (b1[0] >= 0)]
    assert int(moved.min()) >= 0 and int(moved.max()) >= g["nzeta"] // 4   # more than one box of 4


def test_plan():
    p = PL.Plan(nzeta=10, n_boxes=4, n_steps=7, world=3)
    boxes = [list(p.box_slices(k)) for k in range(4)]
    assert sum(boxes, []) == list(range(10)) and all(boxes)
    assert [p.box_of_slice(i) for i in range(10)] == [k for k in range(4) for _ in boxes[k]]
    assert sorted(sum([list(p.steps_of(r)) for r in range(3)], [])) == list(range(7))
    assert [p.rank_of(t) for t in range(7)] == [0, 1, 2, 0, 1, 2, 0]
    assert len({p.tag(t, k) for t in range(7) for k in range(4)}) == 28
    with pytest.raises(ValueError):
        PL.Plan(nzeta=4, n_boxes=5, n_steps=1)


def test_ideal_efficiency():
    """Sec. 5.2: eta_ideal = (1 + (n_ranks - 1) / n_steps)^-1: 1 on one rank, -> 1 for n_steps >> n_ranks,
    and for the reference set-up's 256 ranks over 1000 steps 1000 / 1255."""
    assert PL.ideal_efficiency(1, 10) == 1.0
    assert PL.ideal_efficiency(256, 1000) == pytest.approx(1000.0 / 1255.0, rel=1e-15)
    assert PL.ideal_efficiency(8, 10 ** 9) == pytest.approx(1.0, abs=1e-8)
    # t(n) = (n_steps + n - 1) / n step times for a pipeline of n ranks: eta = t(1) / (n t(n))
    for n, s in ((2, 3), (16, 100), (512, 2048)):
        assert PL.ideal_efficiency(n, s) == pytest.approx(s / (n * (s + n - 1) / n), rel=1e-14)


def test_pack_roundtrip():
    g, beams = setup()
    b = [PL.with_ids(x, "cpu") for x in beams]
    b[1] = PL.take(b[1], torch.tensor([5, 2, 900]))
    counts, payload = PL.pack(b)
    assert counts.tolist() == [3000, 3] and payload.shape == (3003, PL.S_BEAM)
    back = PL.unpack(counts, payload)
    for s in range(2):
        for k in PL.KEYS + ("id",):
            assert torch.equal(back[s][k], b[s][k])


@pytest.mark.parametrize("n_boxes", [1, 4, 16])
def test_one_rank_matches_the_serial_loop(reference, n_boxes):
    g, beams, (ref, sums) = reference
    res, eng = run_pipeline(g, beams, n_boxes)
    assert eng.boxes_seen == [(t, k) for t in range(NSTEP) for k in range(n_boxes)]
    check_against_serial([res], ref, sums)
    assert res.bytes_sent > 0 and res.bytes_sent == res.bytes_received


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n_boxes, out_dir):
    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g, beams = setup()
    res, eng = run_pipeline(g, beams, n_boxes, rank=rank, world=world, transport=PL.DistTransport())
    torch.save({"res": res, "boxes": eng.boxes_seen}, os.path.join(out_dir, f"rank{rank}.pt"))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(600)
@pytest.mark.parametrize("world,n_boxes", [(2, 4), (3, 5)])
def test_gloo_ranks_match_the_serial_loop(reference, tmp_path, world, n_boxes):
    g, beams, (ref, sums) = reference
    mp.start_processes(_rank_main, args=(world, _free_port(), n_boxes, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    got = [torch.load(tmp_path / f"rank{r}.pt", weights_only=False) for r in range(world)]
    results = [x["res"] for x in got]
    for r, x in enumerate(got):
        assert x["res"].steps == list(range(r, NSTEP, world))
        assert x["boxes"] == [(t, k) for t in range(r, NSTEP, world) for k in range(n_boxes)]
    check_against_serial(results, ref, sums)
    # every step but the last hands the beam on: what one rank sends the next one receives
    sent = sum(r.bytes_sent for r in results)
    assert sent == sum(r.bytes_received for r in results) and sent > 0
    last = PL.Plan(nzeta=g["nzeta"], n_boxes=n_boxes, n_steps=NSTEP, world=world).rank_of(NSTEP - 1)
    assert results[last].final is not None and all(r.final is None for i, r in enumerate(results) if i != last)
