"""Temporal domain decomposition of the time loop (Sec. 5.2), over torch.distributed ranks.

Rank r of R computes every box of the time steps t = r, r + R, r + 2R, ... (t = r mod R).  The
zeta extent is cut into n_boxes boxes of consecutive slices, indexed here in sweep order: box k
holds slices [floor(k nzeta / n_boxes), floor((k + 1) nzeta / n_boxes)), box 0 at the head
(Sec. 5.2 counts the boxes from the tail, b = n_boxes - 1 - k).  For each box the rank

  1. receives the beam particles of box k at time t from rank (t - 1) mod R (the particles that
     step t - 1 left in that box; step 0 takes them from the initial beam),
  2. solves the box's slices with its own plasma slice, carried over from box k - 1 of the same
     step (the plasma starts unperturbed ahead of the beam at every step, Sec. 2), pushing each
     slice's beam particles with that slice's fields,
  3. sends to rank (t + 1) mod R the particles that now lie in box k.

Only beam particles travel.  A message holds, per beam species, an n x 8 float64 block (x, y,
zeta, ux, uy, uz, w and the particle's index in the initial beam), so a rank sends
N_t = n_beam,r x S_beam scalars per step (Sec. 5.2) with S_beam = 8.

Readings (the paper gives the loop, not these details):
  * A beam particle only slips toward the tail (d zeta / dt = v_z - 1 < 0), so a particle of box
    k at time t lies in a box k' >= k at t + 1, and box k's message for t + 1 is complete once its
    sender has finished box k at time t.  A particle ahead of the head (zeta above zeta_max) lies
    in no slice and is never pushed, so it rides along, unchanged, in box 0's message; one behind
    the tail, or with a non-finite zeta, leaves the pipeline for good and is kept, frozen, by the
    rank that pushed it out (the serial loop never touches such a particle again either).
  * The B_perp solvers take the beam's J_perp of slice i + 1 (Sec. 3.2); on the last slice of box
    k that is the first slice of box k + 1, so the rank receives box k + 1 before it solves the
    last slice of box k.  Neighbouring ranks then run one box plus one slice apart.
  * Within a box the particles are ordered by their index in the initial beam, the order of the
    serial sweep, so an engine whose sums follow particle order reproduces the serial time loop
    exactly.

The compute of a box is an engine (``HqEngine`` runs it on the CUDA library); the transport is
torch.distributed point-to-point (gloo for CPU tensors, NCCL for CUDA tensors), an in-process
queue for a single rank, or, on one GPU, ranks as threads with their own CUDA streams
(``run_streams``): consecutive time steps then run concurrently on the device, the beam
handed over through stream events.
"""
from __future__ import annotations

import bisect
import collections
import threading
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Protocol, Sequence

import torch

KEYS = ("x", "y", "zeta", "ux", "uy", "uz", "w")
S_BEAM = len(KEYS) + 1          # scalars per particle in a message; the index rides as a float64

Bunch = Dict[str, torch.Tensor]   # KEYS -> float64 [n], "id" -> int64 [n]


def ideal_efficiency(n_ranks: int, n_steps: int) -> float:
    """Sec. 5.2: the pipeline's fill and drain bound its efficiency by (1 + (n_ranks - 1) / n_steps)^-1."""
    if n_ranks < 1 or n_steps < 1:
        raise ValueError("n_ranks and n_steps must be >= 1")
    return 1.0 / (1.0 + (n_ranks - 1) / n_steps)


@dataclass(frozen=True)
class Plan:
    """Which rank computes which time step, and which slices form which box."""
    nzeta: int
    n_boxes: int
    n_steps: int
    world: int = 1

    def __post_init__(self):
        if not 1 <= self.n_boxes <= self.nzeta:
            raise ValueError("n_boxes must be in 1..nzeta")
        if self.n_steps < 0 or self.world < 1:
            raise ValueError("n_steps must be >= 0 and world >= 1")

    @property
    def starts(self) -> List[int]:
        return [(k * self.nzeta) // self.n_boxes for k in range(self.n_boxes + 1)]

    def box_slices(self, k: int) -> range:
        s = self.starts
        return range(s[k], s[k + 1])

    def box_of_slice(self, i: int) -> int:
        return bisect.bisect_right(self.starts, i) - 1

    def steps_of(self, rank: int) -> range:
        return range(rank, self.n_steps, self.world)

    def rank_of(self, t: int) -> int:
        return t % self.world

    def tag(self, t: int, k: int) -> int:
        return t * self.n_boxes + k


# ---------------------------------------------------------------- particle bunches

def take(b: Bunch, idx: torch.Tensor) -> Bunch:
    return {k: v.index_select(0, idx) for k, v in b.items()}


def concat(parts: Sequence[Bunch], like: Bunch) -> Bunch:
    """Concatenation of `parts`, ordered by the particles' initial index (empty: like's types)."""
    parts = [p for p in parts if p["id"].numel()]
    if not parts:
        return {k: v[:0] for k, v in like.items()}
    cat = {k: torch.cat([p[k] for p in parts]) for k in like}
    return take(cat, torch.argsort(cat["id"]))


def with_ids(arrays: dict, device) -> Bunch:
    """A bunch from plain arrays (x, y, zeta, ux, uy, uz, w); ids are 0..n-1."""
    b = {k: torch.as_tensor(arrays[k], dtype=torch.float64, device=device).contiguous() for k in KEYS}
    b["id"] = torch.arange(b["x"].numel(), dtype=torch.int64, device=device)
    return b


def pack(bunches: Sequence[Bunch]) -> tuple:
    """(counts int64 [n_species], payload float64 [sum n, S_BEAM]) of one box message."""
    dev = bunches[0]["x"].device
    counts = torch.tensor([int(b["id"].numel()) for b in bunches], dtype=torch.int64, device=dev)
    rows = [torch.stack([b[k] for k in KEYS] + [b["id"].to(torch.float64)], dim=1) for b in bunches]
    payload = torch.cat(rows) if rows else torch.zeros((0, S_BEAM), dtype=torch.float64, device=dev)
    return counts, payload.contiguous()


def unpack(counts: torch.Tensor, payload: torch.Tensor) -> List[Bunch]:
    out, o = [], 0
    for n in counts.tolist():
        blk = payload[o:o + n]
        b = {k: blk[:, j].contiguous() for j, k in enumerate(KEYS)}
        b["id"] = blk[:, len(KEYS)].to(torch.int64)
        out.append(b)
        o += n
    return out


# ---------------------------------------------------------------- transports

class Transport(Protocol):
    def send(self, dst: int, tag: int, counts: torch.Tensor, payload: torch.Tensor) -> None: ...
    def recv(self, src: int, tag: int, n_species: int, device) -> tuple: ...
    def flush(self) -> None: ...


class LocalTransport:
    """Single rank: messages to itself, kept in order per tag."""

    def __init__(self):
        self.q = collections.defaultdict(collections.deque)

    def send(self, dst, tag, counts, payload):
        self.q[tag].append((counts, payload))

    def recv(self, src, tag, n_species, device):
        if not self.q[tag]:
            raise RuntimeError(f"pipeline: no message with tag {tag} (a step was computed out of order)")
        return self.q[tag].popleft()

    def flush(self):
        pass


class StreamTransport:
    """Ranks as threads of one process on one GPU, each with its own CUDA stream (the time steps
    of the pipeline overlap on the device).  A message carries an event recorded on the sender's
    stream after its payload was written; the receiver's stream waits on it.  A receive that
    finds nothing within `timeout` seconds raises (a rank that failed or never sends)."""

    def __init__(self, timeout: float = 600.0):
        self.cv = threading.Condition()
        self.q = collections.defaultdict(collections.deque)
        self.timeout = timeout
        self.failed = False

    def send(self, dst, tag, counts, payload):
        ev = torch.cuda.Event()
        ev.record(torch.cuda.current_stream())
        with self.cv:
            self.q[tag].append((counts, payload, ev))
            self.cv.notify_all()

    def recv(self, src, tag, n_species, device):
        with self.cv:
            if not self.cv.wait_for(lambda: self.q[tag] or self.failed, timeout=self.timeout):
                raise RuntimeError(f"pipeline: no message with tag {tag} within {self.timeout} s")
            if self.failed and not self.q[tag]:
                raise RuntimeError("pipeline: another rank failed")
            counts, payload, ev = self.q[tag].popleft()
        cur = torch.cuda.current_stream()
        cur.wait_event(ev)
        # the tensors were allocated on the sender's stream: keep them from being reused there
        # before this stream has read them
        counts.record_stream(cur)
        payload.record_stream(cur)
        return counts, payload

    def fail(self):
        with self.cv:
            self.failed = True
            self.cv.notify_all()

    def flush(self):
        pass


class DistTransport:
    """torch.distributed point-to-point: non-blocking sends (each tensor kept alive until its send
    completes), blocking receives in the order the sender issued the messages.  The header of a
    message (the per-species counts) and its payload go under tags 2 tag and 2 tag + 1."""

    def __init__(self):
        import torch.distributed as dist
        self.dist = dist
        self.pending = []

    def send(self, dst, tag, counts, payload):
        self.pending.append((self.dist.isend(counts, dst, tag=2 * tag), counts))
        if payload.shape[0]:
            self.pending.append((self.dist.isend(payload, dst, tag=2 * tag + 1), payload))

    def recv(self, src, tag, n_species, device):
        counts = torch.empty(n_species, dtype=torch.int64, device=device)
        self.dist.recv(counts, src, tag=2 * tag)
        n = int(counts.sum())
        payload = torch.empty((n, S_BEAM), dtype=torch.float64, device=device)
        if n:
            self.dist.recv(payload, src, tag=2 * tag + 1)
        return counts, payload

    def flush(self):
        for w, _ in self.pending:
            w.wait()
        self.pending.clear()


# ---------------------------------------------------------------- engines

class Engine(Protocol):
    """The compute of one rank: a quasi-static sweep run box by box."""
    n_species: int
    device: object

    def slices(self, s: int, b: Bunch) -> torch.Tensor:
        """Slice of every particle of species s: 0..nzeta-1, -1 ahead, nzeta behind, -2 not finite."""

    def begin_step(self, t: int) -> None: ...

    def run_box(self, t: int, k: int, slices: range, parts: List[Bunch],
                next_parts: Callable[[], Optional[List[Bunch]]]) -> List[Bunch]:
        """Solves `slices` with the box's particles `parts` (one bunch per species) and returns
        them pushed.  next_parts() yields the next box's particles (None after the last box)."""

    def end_step(self, t: int) -> dict: ...


class HqEngine:
    """Engine on the CUDA library: a box is hq_sweep_slices over its slices (advance, beam deposit,
    solve, witness sums, push per slice), the next box's particles joining the beam deposit on
    the box's last slice; everything is queued on the grid's stream."""

    def __init__(self, grid, species: Sequence[tuple], dt: float, witness: int = -1):
        from . import hq
        self.hq = hq
        self.grid = grid
        self.species = [(float(q), float(m)) for q, m in species]
        self.n_species = len(self.species)
        if not 1 <= 2 * self.n_species <= 4:
            raise ValueError("HqEngine takes 1 or 2 beam species (two boxes of views at a time)")
        self.dt = float(dt)
        self.witness = int(witness)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.sums = torch.zeros(3, dtype=torch.float64, device=self.device)

    def _beam(self, s: int, b: Bunch):
        q, m = self.species[s]
        return self.hq.Beam({k: b[k] for k in KEYS}, device=self.device, charge=q, mass=m)

    def slices(self, s, b):
        return self.grid.beam_slices(self._beam(s, b)).to(torch.int64)

    def begin_step(self, t):
        self.sums.zero_()

    def run_box(self, t, k, slices, parts, next_parts):
        beams = [self._beam(s, b) for s, b in enumerate(parts)]
        first, last = slices[0], slices[-1]
        w = self.witness
        sums = self.sums if w >= 0 else None
        # the box's slices but its last in one library call, then the last one with the next box's
        # particles (received as late as possible: they are needed for J_perp(i + 1) only there)
        if last > first:
            self.grid.sweep_slices(beams, first, last, (), self.dt, witness=w, witness_sums=sums)
        nxt = next_parts() if last + 1 < self.grid.nzeta else None
        nb = [self._beam(s, b) for s, b in enumerate(nxt)] if nxt is not None else []
        self.grid.sweep_slices(beams, last, last + 1, nb, self.dt, witness=w, witness_sums=sums)
        return parts

    def end_step(self, t):
        return {"witness_sums": self.sums.clone()} if self.witness >= 0 else {}


# ---------------------------------------------------------------- the pipeline

@dataclass
class RankResult:
    steps: List[int] = field(default_factory=list)
    diagnostics: Dict[int, dict] = field(default_factory=dict)
    lost: List[List[Bunch]] = field(default_factory=list)    # per species: particles that left the box
    final: Optional[List[List[Bunch]]] = None                # per species: the beam after the last step
    bytes_sent: int = 0
    bytes_received: int = 0


def run_rank(engine: Engine, plan: Plan, rank: int, transport: Transport,
             initial: Optional[Sequence[Bunch]] = None) -> RankResult:
    """Runs this rank's time steps (t = rank mod world) and returns what it holds at the end.
    `initial` (one bunch per species, ids included, on engine.device) is needed on the rank of
    step 0 only."""
    ns = engine.n_species
    res = RankResult(lost=[[] for _ in range(ns)])
    dev = engine.device
    nz, nb = plan.nzeta, plan.n_boxes

    def route(bunches: Sequence[Bunch], boxes: Dict[int, List[List[Bunch]]]):
        """Files each particle under the box it now lies in (ahead -> box 0); the rest is lost."""
        for s, b in enumerate(bunches):
            if b["id"].numel() == 0:
                continue
            sl = engine.slices(s, b)
            box = torch.full_like(sl, -1)
            inside = (sl >= 0) & (sl < nz)
            starts = torch.tensor(plan.starts[1:], dtype=sl.dtype, device=sl.device)
            box[inside] = torch.searchsorted(starts, sl[inside], right=True)
            box[sl == -1] = 0
            for kk in torch.unique(box).tolist():
                sel = take(b, torch.nonzero(box == kk).reshape(-1))
                if kk < 0:
                    res.lost[s].append(sel)
                else:
                    boxes.setdefault(kk, [[] for _ in range(ns)])[s].append(sel)

    template = None
    for t in plan.steps_of(rank):
        res.steps.append(t)
        local: Dict[int, List[Bunch]] = {}
        if t == 0:
            if initial is None or len(initial) != ns:
                raise ValueError("the rank of step 0 needs the initial beam (one bunch per species)")
            routed: Dict[int, List[List[Bunch]]] = {}
            route(initial, routed)
            for k in range(nb):
                local[k] = [concat(routed.get(k, [[] for _ in range(ns)])[s], initial[s]) for s in range(ns)]
            template = initial

        def get_box(k: int) -> List[Bunch]:
            if k in local:
                return local.pop(k)
            counts, payload = transport.recv(plan.rank_of(t - 1), plan.tag(t, k), ns, dev)
            res.bytes_received += counts.numel() * 8 + payload.numel() * 8
            return unpack(counts, payload)

        out: Dict[int, List[List[Bunch]]] = {}
        final = [[] for _ in range(ns)]
        engine.begin_step(t)
        cur = get_box(0)
        if template is None:
            template = cur
        for k in range(nb):
            held: Dict[str, List[Bunch]] = {}

            def next_parts(k=k, held=held):
                if k + 1 >= nb:
                    return None
                if "v" not in held:
                    held["v"] = get_box(k + 1)
                return held["v"]

            pushed = engine.run_box(t, k, plan.box_slices(k), cur, next_parts)
            route(pushed, out)
            if any(kk < k for kk in out):
                raise RuntimeError("pipeline: a beam particle moved toward the head (v_z > c)")
            mine = out.pop(k, [[] for _ in range(ns)])
            msg = [concat(mine[s], template[s]) for s in range(ns)]
            if t + 1 < plan.n_steps:
                counts, payload = pack(msg)
                transport.send(plan.rank_of(t + 1), plan.tag(t + 1, k), counts, payload)
                res.bytes_sent += counts.numel() * 8 + payload.numel() * 8
            else:
                for s in range(ns):
                    final[s].append(msg[s])
            cur = next_parts()
        res.diagnostics[t] = engine.end_step(t)
        if t + 1 == plan.n_steps:
            res.final = final
    transport.flush()
    return res


def run_streams(make_engine: Callable[[int, object], Engine], plan: Plan,
                initial: Sequence[Bunch]) -> List[RankResult]:
    """The pipeline on one GPU: plan.world ranks as threads, rank r on its own CUDA stream with
    the engine make_engine(r, stream) (e.g. an HqEngine over a grid created on that stream), so
    consecutive time steps run concurrently, one box (plus a slice) apart.  `initial` (on the
    GPU) seeds step 0.  Returns the ranks' results (rank order); re-raises a rank's error."""
    transport = StreamTransport()
    results: List[Optional[RankResult]] = [None] * plan.world
    errors: List[BaseException] = []
    device = torch.cuda.current_device()
    ready = torch.cuda.Event()
    ready.record(torch.cuda.current_stream())

    def body(rank: int):
        try:
            torch.cuda.set_device(device)
            stream = torch.cuda.Stream()
            stream.wait_event(ready)
            with torch.cuda.stream(stream):
                eng = make_engine(rank, stream)
                results[rank] = run_rank(eng, plan, rank, transport, initial if rank == 0 else None)
                stream.synchronize()
        except BaseException as e:  # noqa: BLE001 - reported to the caller below
            errors.append(e)
            transport.fail()

    threads = [threading.Thread(target=body, args=(r,), name=f"pipeline-rank-{r}") for r in range(plan.world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if errors:
        raise errors[0]
    return results


def assemble(results: Sequence[RankResult], n_species: int) -> List[Bunch]:
    """The whole beam after the last step, one bunch per species ordered by initial index: the
    last step's boxes and every particle that left the pipeline, from all ranks."""
    out = []
    for s in range(n_species):
        parts = []
        for r in results:
            parts += r.lost[s]
            if r.final is not None:
                parts += r.final[s]
        like = next((p for p in parts), None)
        if like is None:
            raise ValueError("no particles of species %d in any result" % s)
        out.append(concat(parts, like))
    return out
