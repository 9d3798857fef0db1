#!/usr/bin/env python
"""Throughput of the quasi-static sweep (arXiv:2109.10277, Sec. 2) on GB300.

Metric: plasma particle-slice pushes per second, i.e. plasma particles per slice
x slices x sweeps / time of hq_sweep_step (predictor-corrector trial passes are
not counted; the raw pass count is reported beside it).  The workload is the
512^2 x 1024-slice blowout sweep: +-8 box, 1 particle per cell (262,144 per
slice), quadratic shape, 5 predictor-corrector iterations, a seeded 1e6-particle
Gaussian driver (sigma_r = 0.2, sigma_z = 1.4, n_b = 5).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hq|reference]

One JSON line on rank 0.  N > 1 runs N independent replicas (one per GPU, the
sweep does not shard), value = all replicas' particle-slices / max time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "plasma particle-slice pushes/s, FP32-split vs FP64 on 1 GB300; adjoint/forward time"
UNIT = "particle-slices/s"
WORKLOAD = "blowout512"
WORKLOAD_DESC = ("512x512 grid on +-8 k_p^-1 x 1024 slices over zeta in [-13, 7]; 1 plasma particle per cell "
                 "(262144 per slice), quadratic shape; seeded 1e6-particle Gaussian driver sigma_r=0.2, "
                 "sigma_z=1.4, n_b/n0=5; predictor-corrector 5 iterations, mixing 0.05")
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
# algorithmic bytes per particle of the FP32 particle passes (particle streams read + written)
BYTES_TRIAL = 49    # ux, uy, w (12) + AB5 history sum (20) + cell/frac/1+Psi cache (16) + alive (1)
BYTES_FINAL = 221   # reads: x, y, Psi (24), ux, uy, w (12), AB5 history 4x5x4 (80), cache (16), alive (1);
                    # writes: x, y, Psi (24), ux, uy (8), f_i (20), history sum (20), cache (16)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("hq", "reference"), default="hq")
    ap.add_argument("--precision", choices=("fp32", "fp64"), default="fp32")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison sweep")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--cpu-slices", type=int, default=12, help="oracle sample: slices of the workload")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint/forward timing")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the cubic1024 and adjoint512 legs and the cuFFT DST comparator")
    ap.add_argument("--cubic-steps", type=int, default=9,
                    help="timed beam time steps of the cubic1024 leg after its first (untimed) one: "
                         "the workload defines 10 in all")
    ap.add_argument("--precision-steps", type=int, default=100,
                    help="beam time steps of the FP32-vs-FP64 witness emittance leg")
    ap.add_argument("--case", choices=("sweep", "poisson"), default="sweep",
                    help="poisson: only repeated Dirichlet solves on the workload grid (for ncu captures)")
    ap.add_argument("--nzeta", type=int, default=0,
                    help="override the workload's slice count (a short sweep of the same kernels, for ncu "
                         "captures; the line then names the reduced workload)")
    ap.add_argument("--rhs", type=int, default=3, choices=(1, 2, 3),
                    help="right-hand sides per solve of the poisson case (3: the psi/Ez/Bz solve, 2: B_perp)")
    return ap.parse_args()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class Clocks:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    def __init__(self, dev: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={CLOCK_QUERY}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(dev)], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            cols = [c.strip() for c in line.split(",")]
            if len(cols) < 9:
                continue
            try:
                sm.append(float(cols[1]))
                mx = float(cols[2])
            except ValueError:
                continue
            for n, v in zip(names, cols[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(backend: str):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(world, v: float, device) -> float:
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_sample(n_slices: int) -> dict:
    """The oracle as it stands on the first n_slices of the workload (host cores)."""
    import torch

    import oracle as O
    from paper_2109_10277_gb300 import inputs as I
    g = I.grid_params(WORKLOAD)
    beams = [O.as_beam(b) for b in I.workload_beams(WORKLOAD)]
    sp = O.GridSpec(**g)
    t0 = time.perf_counter()
    with O.dst_algorithm("fft"):   # the O(n^2 log n) DST-I, not the O(n^3) matrix definition
        O.sweep(sp, beams, n_slices=n_slices, record=())
    dt = time.perf_counter() - t0
    p = g["nx"] * g["ny"] * g["ppc_x"] * g["ppc_y"]
    return {"value": p * n_slices / dt, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
            "sample": f"first {n_slices} of 1024 slices of the {WORKLOAD} sweep ({p} particles/slice, "
                      f"full 1e6-particle driver binned), FP64 torch-CPU oracle with the FFT DST-I, {dt:.1f} s"}


def bench_config(world: int, nzeta: int = 0) -> dict:
    """The workload a bench line measures (the same for both arms)."""
    from paper_2109_10277_gb300 import inputs as I
    g = I.grid_params(WORKLOAD)
    nz = nzeta if nzeta > 0 else g["nzeta"]
    return {"workload": f"{WORKLOAD}: {WORKLOAD_DESC}" + (f" (reduced: the first {nz} slices only)" if nzeta > 0 else ""),
            "particles_per_slice": g["nx"] * g["ny"] * g["ppc_x"] * g["ppc_y"], "slices": nz,
            "parallelism": f"replicas x{world}", "l2": "flushed between steps (256 MiB write, outside the timed events)"}


def run_reference(args):
    import torch
    world, rank, _ = dist_setup("gloo")
    if rank != 0:
        return
    n = max(1, min(args.cpu_slices, 4))
    for _ in range(args.warmup):
        oracle_sample(n)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        res = oracle_sample(n)
        times.append(time.perf_counter() - t0)
    from paper_2109_10277_gb300 import inputs as I
    g = I.grid_params(WORKLOAD)
    p = g["nx"] * g["ny"]
    value = p * n * args.steps / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(args.gpus), "sample_slices_per_step": n,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
                             "sample": res["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


# dram__bytes_read.sum + dram__bytes_write.sum per launch from one ncu capture of each kernel
# (profiles/: k_dst_solve_rs R = 3, R = 2 of the first and of the later predictor-corrector
# iterations weighted 1:1:4 as in a slice; the trial pass's first and later iterations 1:4;
# the final pass)
NCU_TRAFFIC = {"dst": (6.902016e6 + 16.344832e6 + 4 * 7.961856e6) / 6, "trial": (21.229824e6 + 4 * 21.23648e6) / 5,
               "final": 46.436608e6 + 4.096e3}


def dst_flops_per_sweep(g: dict) -> float:
    """Executed bf16 flops of the tensor-core DST-I per sweep: per solve of R right-hand
    sides, 4 products of 2 M N K with M = R x padded rows, times 3 (bf16x3).  With nx, ny
    multiples of 128 the solve uses the folded DST-I: every output contracts over K = n/2."""
    nxp = -(-g["nx"] // 128) * 128
    nyp = -(-g["ny"] // 128) * 128
    folded = g["nx"] % 128 == 0 and g["ny"] % 128 == 0
    kx, ky = (nxp // 2, nyp // 2) if folded else (nxp, nyp)
    per_rhs = 2 * (2.0 * nyp * nxp * kx) + 2 * (2.0 * nxp * nyp * ky)
    rhs_per_slice = 3 + 2 * g["n_pc_iter"]
    return 3.0 * per_rhs * rhs_per_slice * g["nzeta"]


def adjoint_leg(hq, I, stream, flush, name="adjoint256", ckpt_every=32):
    """Adjoint/forward time on the 256^2 x 512 gradient workload (FP32/bf16x3, fixed-ppc driver
    and witness, loss = charge-weighted mean Ez of the witness, checkpoint every 32 slices)."""
    import torch
    g = I.grid_params(name)
    beams = [hq.Beam(b) for b in I.workload_beams(name)]
    free0 = torch.cuda.mem_get_info()[0]
    grid = hq.Grid(g, precision="fp32", stream=stream)
    sums = torch.zeros(3, dtype=torch.float64, device="cuda")
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    for _ in range(2):  # warm-up: forward, checkpointed forward + adjoint
        sums.zero_()
        grid.sweep(beams, witness=1, witness_sums=sums)
        sums.zero_()
        grid.forward_ckpt(beams, 1, sums, ckpt_every)
        grid.adjoint(beams, 1, hq.witness_loss_grad("mean", *[float(v) for v in sums.cpu()])[1])
    grid.sync()
    a, b, c, d, e = ev(), ev(), ev(), ev(), ev()
    flush.fill_(3)
    sums.zero_()
    a.record(stream)
    grid.sweep(beams, witness=1, witness_sums=sums)
    b.record(stream)
    flush.fill_(4)
    sums.zero_()
    c.record(stream)
    grid.forward_ckpt(beams, 1, sums, ckpt_every)
    d.record(stream)
    s = [float(v) for v in sums.cpu()]
    loss, dls = hq.witness_loss_grad("mean", *s)
    c2 = ev()
    c2.record(stream)
    grid.adjoint(beams, 1, dls)
    e.record(stream)
    torch.cuda.synchronize()
    used = free0 - torch.cuda.mem_get_info()[0]
    grid.close()
    fwd, ck, adj = a.elapsed_time(b), c.elapsed_time(d), c2.elapsed_time(e)
    return {"workload": f"{name}: 256x256 x 512 slices, 1 ppc, linear shape, fixed-ppc driver (n_b=2) and witness, "
                        f"loss = mean witness Ez, FP32/bf16x3, checkpoint every {ckpt_every}",
            "forward_ms": fwd, "forward_ckpt_ms": ck, "adjoint_ms": adj, "adjoint_over_forward": adj / fwd,
            "ckpt_forward_plus_adjoint_over_forward": (ck + adj) / fwd, "loss": loss,
            "device_bytes_used": int(used)}


def cubic_leg(hq, I, stream, flush, steps=1):
    """1024^2 x 1024 slices, 4 ppc (4.2M plasma particles per slice), cubic shape, driver 1e7 +
    witness 2e6 macroparticles, beam push with dt = 20 after every slice: per-slice throughput."""
    import torch
    g = I.grid_params("cubic1024")
    free0 = torch.cuda.mem_get_info()[0]
    grid = hq.Grid(g, precision="fp32", stream=stream)
    beams = [hq.Beam(b) for b in I.workload_beams("cubic1024")]
    p = g["nx"] * g["ny"] * g["ppc_x"] * g["ppc_y"]
    m0 = grid.beam_moments(beams[1])
    grid.sweep(beams, dt=20.0)   # warm-up: also the first beam time step
    grid.sync()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.fill_(5)
    a.record(stream)
    for _ in range(steps):
        grid.sweep(beams, dt=20.0)
    b.record(stream)
    torch.cuda.synchronize()
    removed = grid.sync()
    m1 = grid.beam_moments(beams[1])
    used = free0 - torch.cuda.mem_get_info()[0]
    ms = a.elapsed_time(b)
    grid.close()
    return {"workload": "cubic1024: 1024x1024 grid on +-10 x 1024 slices over [-18, 6], 4 ppc (4,194,304 per slice), "
                        "cubic shape, driver 1e7 (sigma_r=0.15, sigma_z=1.2, n_b=10) + witness 2e6 (zeta0=-6), "
                        "beam push dt=20 per time step, FP32/bf16x3",
            "time_steps": steps + 1, "timed_steps": steps, "ms_per_step": ms / steps,
            "ms_per_slice": ms / steps / g["nzeta"],
            "value": p * g["nzeta"] * steps / (ms / 1e3), "unit": "particle-slices/s",
            "removed_particles": removed,
            "witness_eps_x_initial": hq.emittance(m0)[0], "witness_eps_x_final": hq.emittance(m1)[0], "device_bytes_used": int(used)}


def explicit_leg(hq, I, stream, flush, iters=6):
    """The headline workload with the explicit B_perp solver (Helmholtz-like equation in chi,
    `iters` preconditioned conjugate-gradient iterations) instead of the predictor-corrector."""
    import torch
    g = dict(I.grid_params(WORKLOAD), bperp_solver="explicit", n_pc_iter=iters)
    grid = hq.Grid(g, precision="fp32", stream=stream)
    hb = [hq.Beam(b) for b in I.workload_beams(WORKLOAD)]
    sums = torch.zeros(3, dtype=torch.float64, device="cuda")
    grid.sweep(hb, witness=0, witness_sums=sums)
    grid.sync()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.fill_(7)
    sums.zero_()
    a.record(stream)
    grid.sweep(hb, witness=0, witness_sums=sums)
    b.record(stream)
    torch.cuda.synchronize()
    removed = grid.sync()
    grid.close()
    ms = a.elapsed_time(b)
    p = g["nx"] * g["ny"] * g["ppc_x"] * g["ppc_y"]
    return {"workload": f"{WORKLOAD} with the explicit B_perp solver, {iters} PCG iterations per slice",
            "ms_per_step": ms, "value": p * g["nzeta"] / (ms / 1e3), "unit": UNIT, "removed_particles": removed,
            "witness_sums": [float(v) for v in sums.cpu()]}


def tf32_leg(hq, I, stream, flush):
    """The headline workload with TF32x3 tensor-core DST operands (HQ_PREC_FP32_TF32X3: ~21
    significant bits per operand against bf16x3's 16, twice the operand bytes and instructions;
    the solve streams the fold matrix)."""
    import torch
    g = I.grid_params(WORKLOAD)
    grid = hq.Grid(g, precision="tf32x3", stream=stream)
    hb = [hq.Beam(b) for b in I.workload_beams(WORKLOAD)]
    sums = torch.zeros(3, dtype=torch.float64, device="cuda")
    grid.sweep(hb, witness=0, witness_sums=sums)
    grid.sync()
    ts = []
    for k in range(2):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(11 + k)
        sums.zero_()
        a.record(stream)
        grid.sweep(hb, witness=0, witness_sums=sums)
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    removed = grid.sync()
    grid.close()
    ms = min(ts)
    p = g["nx"] * g["ny"] * g["ppc_x"] * g["ppc_y"]
    return {"workload": f"{WORKLOAD} with TF32x3 DST operands", "ms_per_step": ms,
            "value": p * g["nzeta"] / (ms / 1e3), "unit": UNIT, "removed_particles": removed,
            "witness_sums": [float(v) for v in sums.cpu()]}


def pipeline_leg(hq, I, steps=8, ranks=2, boxes=8, dt=6.0):
    """The temporal decomposition of Sec. 5.2 on one GPU: `steps` beam time steps of the headline
    workload (beam push Delta t = 6, the Appendix's time step), serially as graph-replayed sweeps,
    then pipelined over `ranks` ranks that are threads with their own CUDA streams (consecutive
    steps overlap on the device, the beam handed over box by box)."""
    import torch
    from paper_2109_10277_gb300 import pipeline as PL
    g = I.grid_params(WORKLOAD)
    beams = I.workload_beams(WORKLOAD)
    grid = hq.Grid(g, precision="fp32")
    hb = [hq.Beam(b) for b in beams]
    grid.sweep(hb)
    grid.sync()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        grid.sweep(hb, dt=dt)
    grid.sync()
    t_ser = time.perf_counter() - t0
    grid.close()
    del grid, hb

    def make(rank, s):
        return PL.HqEngine(hq.Grid(g, precision="fp32", stream=s),
                           [(b.get("charge", -1.0), b.get("mass", 1.0)) for b in beams], dt)
    plan = PL.Plan(nzeta=g["nzeta"], n_boxes=boxes, n_steps=steps, world=ranks)
    init = [PL.with_ids(b, "cuda") for b in beams]
    # warm-up: a first pipelined run pays one-time costs (module loading, per-thread stream and
    # allocator set-up) that the timed one must not include
    PL.run_streams(make, PL.Plan(nzeta=g["nzeta"], n_boxes=boxes, n_steps=ranks, world=ranks),
                   [PL.with_ids(b, "cuda") for b in beams])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = PL.run_streams(make, plan, init)
    torch.cuda.synchronize()
    t_pipe = time.perf_counter() - t0
    p = g["nx"] * g["ny"] * g["ppc_x"] * g["ppc_y"]
    return {"workload": f"{WORKLOAD}, {steps} beam time steps of dt={dt}", "ranks": ranks, "boxes": boxes,
            "serial_ms_per_step": 1e3 * t_ser / steps, "pipeline_ms_per_step": 1e3 * t_pipe / steps,
            "speedup": t_ser / t_pipe, "value": p * g["nzeta"] * steps / t_pipe, "unit": UNIT,
            "ideal_efficiency_sec52": PL.ideal_efficiency(ranks, steps),
            "beam_bytes_handed_over_per_step": sum(r.bytes_sent for r in res) / max(1, steps - 1),
            "timing": "host wall clock around the whole run (both include their host work)"}


def species_leg(hq, I, stream, flush, mass=1836.0):
    """The headline workload with the ions moving: electrons and hydrogen ions (M = 1836 m_e) placed
    alike, no immobile background (twice the plasma particles, the multi-species kernels)."""
    import torch
    sp = [dict(charge=-1.0, mass=1.0, n0_scale=1.0, ppc_x=1, ppc_y=1, neutralize=False),
          dict(charge=1.0, mass=mass, n0_scale=1.0, ppc_x=1, ppc_y=1, neutralize=False)]
    g = dict(I.grid_params(WORKLOAD), species=sp)
    grid = hq.Grid(g, precision="fp32", stream=stream)
    hb = [hq.Beam(b) for b in I.workload_beams(WORKLOAD)]
    grid.sweep(hb)
    grid.sync()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.fill_(9)
    a.record(stream)
    grid.sweep(hb)
    b.record(stream)
    torch.cuda.synchronize()
    removed = grid.sync()
    grid.close()
    ms = a.elapsed_time(b)
    p = 2 * g["nx"] * g["ny"]
    return {"workload": f"{WORKLOAD} with mobile hydrogen ions (electrons + ions, 1 ppc each, no background)",
            "ms_per_step": ms, "value": p * g["nzeta"] / (ms / 1e3), "unit": UNIT, "removed_particles": removed}


def precision_leg(hq, I, stream, steps=100, dt=20.0):
    """Witness emittance over many beam time steps, FP32/bf16x3 against the FP64 GPU path (the
    paper's single- vs double-precision study, Sec. 6): a driver and a witness whose centroid
    starts one sigma off axis, `steps` time steps of dt; the witness's normalised emittance and
    centroid from hq_beam_moments after every step."""
    import numpy as np
    import torch
    g = dict(nx=128, ny=128, nzeta=128, xmin=-6.0, xmax=6.0, ymin=-6.0, ymax=6.0, zeta_min=-7.0, zeta_max=5.0,
             shape_order=1, n_pc_iter=5, pc_mix=0.05, psi_guard=0.02)
    driver = I.random_beam(200_000, 0.4, 0.4, 1.0, 0.5, energy_spread=1e-3)
    wit = I.random_beam(50_000, 0.15, 0.15, 0.3, 2.0, zeta0=-3.5, gamma=I.GAMMA_WITNESS, seed=I.SEED_WITNESS)
    rng = np.random.Generator(np.random.PCG64(7))
    wit["x"] = wit["x"] + 0.15
    wit["ux"] = 0.05 * rng.standard_normal(len(wit["x"]))
    wit["uy"] = 0.05 * rng.standard_normal(len(wit["x"]))
    res = {}
    for prec in ("fp64", "fp32"):
        grid = hq.Grid(g, precision=prec, stream=stream)
        hb = [hq.Beam(driver), hq.Beam(wit)]
        ms = [grid.beam_moments(hb[1])]
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            grid.sweep(hb, dt=dt)
            ms.append(grid.beam_moments(hb[1]))
        b.record(stream)
        torch.cuda.synchronize()
        grid.close()
        m = torch.stack(ms).cpu()
        em = np.array([list(hq.emittance(v)) + [float(v[1] / v[0])] for v in m])
        res[prec] = (em, a.elapsed_time(b) / steps)
    e64, e32 = res["fp64"][0], res["fp32"][0]
    rel = np.abs(e32 - e64) / np.abs(e64)
    return {"workload": f"128x128 x 128 slices on +-6 x [-7, 5], 1 ppc, linear shape; driver 2e5 (sigma 0.4/1.0, n_b=0.5), "
                        f"witness 5e4 (sigma 0.15/0.3, n_b=2, zeta0=-3.5, 1 GeV, centroid offset 0.15, u_perp spread 0.05); "
                        f"{steps} time steps of dt={dt}",
            "eps_x_initial": float(e64[0, 0]), "eps_x_final_fp64": float(e64[-1, 0]), "eps_x_final_fp32": float(e32[-1, 0]),
            "rel_diff_eps_x_final": float(rel[-1, 0]), "rel_diff_eps_y_final": float(rel[-1, 1]),
            "rel_diff_eps_max_over_steps": float(rel[:, :2].max()), "rel_diff_centroid_final": float(rel[-1, 2]),
            "ms_per_step_fp64": res["fp64"][1], "ms_per_step_fp32": res["fp32"][1]}


def adjoint_scale_leg(hq, I, stream, flush, ckpt_every=32):
    """adjoint512: 512^2 x 1024 slices, 2 ppc, quadratic, 256-entry radial profile, fixed-ppc driver
    with a free 1024-entry slice current profile; loss = witness mean Ez + rms spread; one full
    gradient: adjoint/forward time and peak device memory."""
    import torch
    g = I.grid_params("adjoint512")
    free0 = torch.cuda.mem_get_info()[0]
    grid = hq.Grid(g, precision="fp32", stream=stream)
    bnp = I.workload_beams("adjoint512")
    beams = [hq.Beam(b) for b in bnp]
    sums = torch.zeros(3, dtype=torch.float64, device="cuda")
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    sums.zero_()
    grid.sweep(beams, witness=1, witness_sums=sums)   # warm-up
    grid.sync()
    a, b, c, d, e = ev(), ev(), ev(), ev(), ev()
    flush.fill_(6)
    sums.zero_()
    a.record(stream)
    grid.sweep(beams, witness=1, witness_sums=sums)
    b.record(stream)
    sums.zero_()
    c.record(stream)
    grid.forward_ckpt(beams, 1, sums, ckpt_every)
    d.record(stream)
    loss, dls = hq.witness_loss_grad("mean+rms", *[float(v) for v in sums.cpu()])
    grid.sync()
    used_fwd = free0 - torch.cuda.mem_get_info()[0]
    e0 = ev()
    e0.record(stream)
    res = grid.adjoint(beams, 1, dls)
    e.record(stream)
    torch.cuda.synchronize()
    used = free0 - torch.cuda.mem_get_info()[0]
    # gradient w.r.t. the driver's 1024-entry slice current profile: w_p = prof[s_p] * shape_p
    s_idx = torch.as_tensor(bnp[0]["slice_index"], device="cuda")
    w0 = beams[0].t["w"]
    nz = g["nzeta"]
    zc = g["zeta_max"] - (torch.arange(nz, device="cuda", dtype=torch.float64) + 0.5) * (
        (g["zeta_max"] - g["zeta_min"]) / nz)
    prof = 4.0 * torch.exp(-zc ** 2 / (2.0 * 1.4 ** 2))
    dprof = torch.zeros(nz, dtype=torch.float64, device="cuda").index_add_(0, s_idx, res["beam_w"][0] * w0 / prof[s_idx])
    fwd, ck, adj = a.elapsed_time(b), c.elapsed_time(d), e0.elapsed_time(e)
    out = {"workload": "adjoint512: 512x512 x 1024 slices, 2 ppc, quadratic, 256-entry radial profile, fixed-ppc "
                       "driver with a 1024-entry slice current profile (peak n_b=4) + witness, loss = witness mean "
                       f"Ez + rms Ez spread, FP32/bf16x3, checkpoint every {ckpt_every}",
           "forward_ms": fwd, "forward_ckpt_ms": ck, "adjoint_ms": adj, "adjoint_over_forward": adj / fwd,
           "ckpt_forward_plus_adjoint_over_forward": (ck + adj) / fwd, "loss": loss,
           "grad_norms": {"slice_profile": float(torch.linalg.norm(dprof)),
                          "radial_profile": float(torch.linalg.norm(res["profile"])),
                          "n0_scale": float(res["n0_scale"][0])},
           "grads_finite": bool(torch.isfinite(dprof).all() and torch.isfinite(res["profile"]).all()),
           "device_bytes_peak": int(used), "device_bytes_forward_ckpt": int(used_fwd)}
    grid.close()
    return out


def cufft_dst_solve(src, lam_inv):
    """Library comparator: the same Dirichlet solve through cuFFT (torch.fft): DST-I of each row via
    the FFT of its odd extension, along x then y, scale, and the same two transforms again."""
    import torch

    def dst_rows(v):   # DST-I along the last axis, nodes 0..n-1 with node 0 on the wall
        n = v.shape[-1]
        ext = torch.cat([v, torch.zeros_like(v[..., :1]), -v[..., 1:].flip(-1)], dim=-1)
        return -0.5 * torch.fft.rfft(ext, dim=-1)[..., :n].imag

    t = dst_rows(src)
    t = dst_rows(t.transpose(-1, -2)).transpose(-1, -2)
    t = t * lam_inv
    t = dst_rows(t)
    return dst_rows(t.transpose(-1, -2)).transpose(-1, -2)


def dst_comparator(hq, I, stream):
    """Times the tensor-core Dirichlet solve (3 rhs, 512^2) against the cuFFT-based one."""
    import math
    import torch
    g = I.grid_params(WORKLOAD)
    nx, ny = g["nx"], g["ny"]
    dx, dy = (g["xmax"] - g["xmin"]) / nx, (g["ymax"] - g["ymin"]) / ny
    grid = hq.Grid(g, precision="fp32", stream=stream)
    gen = torch.Generator(device="cuda").manual_seed(7)
    src = torch.randn(3, ny, nx, device="cuda", generator=gen)
    src[:, 0, :] = 0
    src[:, :, 0] = 0
    k = torch.arange(nx, device="cuda", dtype=torch.float64)
    l = torch.arange(ny, device="cuda", dtype=torch.float64)
    lam = -(4 / dx ** 2) * torch.sin(math.pi * k / (2 * nx)) ** 2 - (4 / dy ** 2) * torch.sin(math.pi * l[:, None] / (2 * ny)) ** 2
    lam_inv = torch.where(lam != 0, (4.0 / (nx * ny)) / lam, torch.zeros_like(lam)).float()
    lam_inv[0, :] = 0
    lam_inv[:, 0] = 0
    ours = grid.poisson_solve(src)
    lib = cufft_dst_solve(src, lam_inv)
    torch.cuda.synchronize()
    agree = float(torch.linalg.norm(ours - lib) / torch.linalg.norm(lib))

    def timed(fn, n=50):
        for _ in range(5):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(n):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return 1e3 * a.elapsed_time(b) / n

    us_ours = timed(lambda: grid.poisson_solve(src))
    us_lib = timed(lambda: cufft_dst_solve(src, lam_inv))
    grid.close()
    return {"case": "Dirichlet solve, 512x512, 3 right-hand sides, FP32 data",
            "tensor_core_dst_us": us_ours, "cufft_dst_us": us_lib, "rel_l2_between": agree,
            "note": "tensor-core path: one fused cooperative launch (plus the source copy kernel); cuFFT path: "
                    "torch.fft rfft of the odd extension, 4 batched transforms + elementwise ops"}


def run_hq(args):
    import torch
    world, rank, local = dist_setup("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2109_10277_gb300 import hq
    from paper_2109_10277_gb300 import inputs as I
    peaks, peak_src = load_peaks()

    g = I.grid_params(WORKLOAD)
    beams_np = I.workload_beams(WORKLOAD)
    if args.nzeta > 0:
        g["nzeta"] = args.nzeta   # same slice thickness window from zeta_max: the head of the box
        g["zeta_min"] = g["zeta_max"] - args.nzeta * (I.grid_params(WORKLOAD)["zeta_max"] -
                                                      I.grid_params(WORKLOAD)["zeta_min"]) / I.grid_params(WORKLOAD)["nzeta"]
    p = g["nx"] * g["ny"] * g["ppc_x"] * g["ppc_y"]
    nz = g["nzeta"]
    stream = torch.cuda.current_stream()
    grid = hq.Grid(g, precision=args.precision, stream=stream)
    hb = [hq.Beam(b) for b in beams_np]
    sums = torch.zeros(3, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 126 MB L2

    def step():
        sums.zero_()
        grid.sweep(hb, witness=0, witness_sums=sums)

    for _ in range(args.warmup):
        step()
    grid.sync()

    # ---- timed region: K sweeps, inputs resident in HBM, L2 flushed between sweeps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    clk = Clocks(local)
    t_host = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    t_host = time.perf_counter() - t_host
    clocks = clk.stop()
    removed = grid.sync()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    ms = allmax(world, ms, dev)
    value = p * nz * args.steps * world / (ms / 1e3)

    # ---- end to end through the public API with host buffers: H2D beams, sweep, D2H result
    host = [{k: b.t[k].cpu().pin_memory() for k in b.t} for b in hb]
    res_host = torch.zeros(3, dtype=torch.float64).pin_memory()
    e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    h2d = sum(t.numel() * t.element_size() for hbuf in host for t in hbuf.values())
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        e2e_ev[k][0].record(stream)
        for b, hbuf in zip(hb, host):
            for key, t in hbuf.items():
                b.t[key].copy_(t, non_blocking=True)
        step()
        res_host.copy_(sums, non_blocking=True)
        e2e_ev[k][1].record(stream)
    torch.cuda.synchronize()
    e2e_ms = allmax(world, sum(a.elapsed_time(b) for a, b in e2e_ev), dev)
    e2e_value = p * nz * args.steps * world / (e2e_ms / 1e3)

    # ---- one more sweep with per-kernel-class CUDA events (launch stream) for the roofline
    grid.profile(True)
    step()
    prof = grid.profile_read()
    grid.profile(False)
    launches_per_sweep = sum(v[1] for v in prof.values())
    shares = {k: v[0] for k, v in prof.items()}
    tot = sum(shares.values()) or 1.0
    dom = max(shares, key=shares.get)
    roofs = {}
    if prof["dst"][0] > 0:
        fl = dst_flops_per_sweep(g) if args.precision == "fp32" else None
        if fl:
            ach = fl / (prof["dst"][0] / 1e3) / 1e12
            pk = peaks["bf16_tflops_sustained"]
            roofs["dst"] = {"bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                            "traffic": NCU_TRAFFIC.get("dst") if g["nx"] == 512 and g["ny"] == 512 else None,
                            "avg_launch_us": 1e3 * prof["dst"][0] / max(1, prof["dst"][1]),
                            "peak_src": f"bf16 sustained, {peak_src}"}
    for k, nb in (("trial", BYTES_TRIAL), ("final", BYTES_FINAL)):
        if prof[k][0] > 0 and args.precision == "fp32":
            nl = max(1, prof[k][1])
            ach = nb * p * nl / (prof[k][0] / 1e3) / 1e9
            pk = peaks["hbm_gbs"]
            roofs[k] = {"bound": "hbm", "achieved": ach, "peak": pk, "unit": "GB/s", "frac": ach / pk,
                        "traffic": NCU_TRAFFIC.get(k) if g["nx"] == 512 and g["ny"] == 512 else None,
                        "avg_launch_us": 1e3 * prof[k][0] / nl, "peak_src": f"hbm copy, {peak_src}"}
    roof = dict(roofs.get(dom, next(iter(roofs.values()), {})))
    if roof:
        roof["kernel"] = dom

    # ---- FP64 GPU path on the same workload (speedup of FP32/bf16x3 over plain FP64)
    fp64 = None
    if not args.no_fp64 and args.precision == "fp32":
        g64 = hq.Grid(g, precision="fp64", stream=stream)
        sums64 = torch.zeros(3, dtype=torch.float64, device=dev)
        g64.sweep(hb, witness=0, witness_sums=sums64)
        g64.sync()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(1)
        a.record(stream)
        g64.sweep(hb, witness=0, witness_sums=sums64)
        b.record(stream)
        torch.cuda.synchronize()
        ms64 = a.elapsed_time(b)
        g64.close()
        # the same sweep in the deterministic FP64 mode (fixed-point deposits, bitwise reproducible)
        gdet = hq.Grid(dict(g, deterministic=1), precision="fp64", stream=stream)
        gdet.sweep(hb, witness=0, witness_sums=sums64)
        gdet.sync()
        flush.fill_(2)
        a.record(stream)
        gdet.sweep(hb, witness=0, witness_sums=sums64)
        b.record(stream)
        torch.cuda.synchronize()
        msdet = a.elapsed_time(b)
        gdet.close()
        fp64 = {"value": p * nz / (ms64 / 1e3), "ms_per_step": ms64,
                "fp32_speedup": (p * nz * args.steps / (ms / 1e3)) / (p * nz / (ms64 / 1e3)),
                "deterministic_ms_per_step": msdet, "deterministic_over_atomic": msdet / ms64}

    adjoint = None
    if not args.no_adjoint and args.precision == "fp32":
        adjoint = adjoint_leg(hq, I, stream, flush)

    cubic = adjoint512 = dstcmp = precision = explicit = species = pipeline = tf32 = None
    if not args.no_extra and args.precision == "fp32" and rank == 0:
        grid.close()
        grid = None
        torch.cuda.empty_cache()
        cubic = cubic_leg(hq, I, stream, flush, args.cubic_steps)
        torch.cuda.empty_cache()
        if not args.no_adjoint:
            adjoint512 = adjoint_scale_leg(hq, I, stream, flush)
            torch.cuda.empty_cache()
        dstcmp = dst_comparator(hq, I, stream)
        precision = precision_leg(hq, I, stream, steps=args.precision_steps)
        explicit = explicit_leg(hq, I, stream, flush)
        species = species_leg(hq, I, stream, flush)
        tf32 = tf32_leg(hq, I, stream, flush)
        pipeline = pipeline_leg(hq, I)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = oracle_sample(args.cpu_slices)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
            "config": bench_config(world, args.nzeta),
            "precision": "FP32 push/gather/deposit, FP64 x/y/Psi accumulators, bf16x3 tensor-core DST-I"
            if args.precision == "fp32" else "FP64 everywhere, FP64 FFT DST-I",
            "raw_particle_passes_per_s": value * (1 + g["n_pc_iter"]), "host_wall_s": t_host,
            "roofline": roof, "rooflines": roofs,
            "kernel_ms_per_sweep": {k: round(v[0], 3) for k, v in prof.items()},
            "kernel_share": {k: round(v / tot, 4) for k, v in shares.items()},
            "clocks": clocks,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 24},
            "gpu_launches": launches_per_sweep * args.steps,
            "fp64": fp64, "adjoint": adjoint, "cubic1024": cubic, "adjoint512": adjoint512,
            "dst_comparator": dstcmp, "precision_study": precision, "explicit_solver": explicit, "ion_motion": species,
            "temporal_pipeline_1gpu": pipeline, "tf32x3": tf32,
            "cpu_baseline": cpu,
            "removed_particles": removed,
        }
        print(json.dumps(line), flush=True)
    if grid is not None:
        grid.close()


def run_poisson_case(args):
    """A few Dirichlet solves of --rhs right-hand sides on the workload grid: the DST kernels alone."""
    import torch
    from paper_2109_10277_gb300 import hq
    from paper_2109_10277_gb300 import inputs as I
    g = I.grid_params(WORKLOAD)
    grid = hq.Grid(g, precision=args.precision)
    dt = torch.float32 if args.precision == "fp32" else torch.float64
    src = torch.randn(args.rhs, g["ny"], g["nx"], dtype=dt, device="cuda")
    for _ in range(args.warmup + args.steps):
        grid.poisson_solve(src)
    grid.sync()
    grid.close()
    print(json.dumps({"case": "poisson", "rhs": args.rhs, "solves": args.warmup + args.steps}))


def main():
    args = parse()
    if args.case == "poisson":
        run_poisson_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_hq(args)


if __name__ == "__main__":
    main()
