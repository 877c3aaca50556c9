"""Continuous-batching serving loop: solve requests (shock tubes and
homogeneous relaxations) arrive over time, are admitted against an HBM
budget, keep their particle state resident on the device while they run,
and overlap with one another on the GPU; finished requests return their
per-cell moments and free their memory at once, so waiting requests enter
while others are still in flight.

Layout of the loop:

* A fixed pool of slots, each one libtrmc context (its own work counter,
  status word and overflow slabs) and one CUDA stream, created before the
  first request.  A context serves one request at a time, so launches of
  different requests never share a work counter; requests in different
  slots run concurrently on the GPU.
* Admission is first come, first served: the head of the queue enters when a
  slot is free and its resident bytes fit in what the budget has left.  A
  request larger than the whole budget is rejected, never queued.
* A request is a solve to a physical end time t_end (or, if it names none,
  a fixed number of steps): a homogeneous relaxation runs t_end / dt steps
  of its fixed dt; a shock tube runs ceil(t_end / dt_0) steps, dt_0 its
  first CFL step, which the GPU computes from the initial data and the
  host reads back without blocking; the simulated time actually reached
  (the sum of the CFL steps) comes back with the result.
* Each admitted request advances in chunks of steps issued on its stream,
  at most `depth` chunks ahead of the GPU, so the host keeps every active
  request fed without blocking on any of them.  After the last step the
  moments kernel runs and the table is copied to pinned host memory; the
  request is complete when that copy has landed.
* The random draws of a request are keyed by (seed, request id, cell,
  step), never by its slot or by what else runs, so a request's result is
  bit-identical whether it runs alone or in a mix.

The policy (Admission) and the loop (ServingLoop) are host logic and run
with any engine: GpuEngine drives libtrmc, tests also drive them with a
simulated engine on the CPU.
"""
import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import trmc as T

MEAN_RELAX_CELL = (8192 - 64) / np.log(8192 / 64)     # mean of a log-uniform cell size in [64, 8192]
SHOCK_CELLS = 400          # cells of a shock-tube request on [0, 1] (the shock-tube workload's geometry)
RELAX_DT = 0.05            # time step of a relaxation request
T_END = {"shock": 0.2, "relax": 1.0}   # end times of solve requests: Sec. 5.1's tube; relaxation to t = 1


@dataclass
class Request:
    rid: int
    kind: str                  # "shock" (1D Riemann tube, specular walls) or "relax" (homogeneous cells)
    n_particles: int
    eps: float
    steps: int                 # time steps (fixed when t_end is None, else set once known)
    arrival: float = 0.0       # seconds after the loop starts
    admitted: float = None
    done: float = None
    rejected: bool = False
    error: str = None
    slot: int = None
    bytes: int = 0
    counts: np.ndarray = field(default=None, repr=False)   # particles per cell (set by plan())
    particles: int = 0         # particles actually placed (rounding of the cell layout)
    result: np.ndarray = field(default=None, repr=False)   # moments per cell after the last step
    t_end: float = None        # a solve to this physical time (None: run `steps` steps)
    t_reached: float = None    # simulated time after the last step (solves)

    @property
    def latency(self):
        return None if self.done is None else self.done - self.arrival


def requests_from(stream, steps=None, first_id=0, t_end=None):
    """Requests from the dicts of synth.poisson_requests: `steps` steps each,
    or, with steps None, solves to the end time t_end[kind] (default T_END)."""
    if steps is None:
        ends = dict(T_END, **(t_end or {}))
        return [Request(first_id + i, d["kind"], d["n_particles"], d["eps"], 0, d["arrival"], t_end=ends[d["kind"]])
                for i, d in enumerate(stream)]
    return [Request(first_id + i, d["kind"], d["n_particles"], d["eps"], steps, d["arrival"])
            for i, d in enumerate(stream)]


# ------------------------------------------------------------ memory accounting
def _alloc(nbytes):
    """Bytes the caching allocator hands out for one tensor of nbytes: small
    blocks are rounded to 512 B, large ones (above 1 MiB) to 2 MiB."""
    nbytes = max(int(nbytes), 1)
    if nbytes <= 1 << 20:
        return (nbytes + 511) // 512 * 512
    return (nbytes + (2 << 20) - 1) // (2 << 20) * (2 << 20)


def shock_mean(req):
    """Mean particles per cell of a shock-tube request."""
    return req.n_particles / SHOCK_CELLS


def plan(req):
    """Fix the cell layout of a request on the host (deterministic in its
    id): a shock tube of SHOCK_CELLS cells, its particles density-weighted
    across the interface, or homogeneous cells of log-uniform size in
    [64, 8192].  Sets req.counts and req.particles (and, for a relaxation
    solve, req.steps)."""
    from . import synth
    if req.counts is None:
        if req.kind == "shock":
            req.counts = synth.shock_tube_counts(SHOCK_CELLS, shock_mean(req))
        elif req.kind == "relax":
            nc = max(1, int(round(req.n_particles / MEAN_RELAX_CELL)))
            req.counts = synth.loguniform_ints(nc, 64, 8192, g=synth.rng((1 << 40) + req.rid))
        else:
            raise ValueError(f"unknown request kind {req.kind!r}")
        req.particles = int(req.counts.sum())
        if req.kind == "relax" and req.t_end is not None:
            req.steps = int(np.ceil(req.t_end / RELAX_DT - 1e-9))
    return req


def footprint(kind, n_cells, n_particles, precision=T.FP32_MIXED):
    """Device bytes a request holds while it is resident: its particle
    state (with the sort's second buffers for a shock tube), the per-cell
    tables, the initial-data table and the result table, each rounded as the
    caching allocator rounds it."""
    nc, n = n_cells, n_particles
    tubes = 1 if kind == "shock" else 0
    rb = 8 if precision == T.FP64 else 4
    b = 0
    if kind == "shock":
        b += 2 * _alloc(3 * n * rb) + 2 * _alloc(n * rb)            # v, v_alt, x, x_alt
        b += 2 * _alloc(8 * (nc + 1))                                # cell_start, cell_start_alt
        b += _alloc(8 * tubes) + _alloc(88 * tubes)                  # dt, domains
        b += _alloc(8 * 3 * nc) + _alloc(8 * (nc + 1))               # the sort's counters in the context
        b += 3 * _alloc(16)                                          # a solve's first CFL speed, clock and read-back
    else:
        b += _alloc(3 * n * rb)
        b += _alloc(8 * (nc + 1))
    b += _alloc(4 * nc) + _alloc(32 * nc) + _alloc(8 * nc) + _alloc(8 * nc)   # m_max, cell_param, key, vmax2
    if precision == T.FP32_MIXED:
        b += _alloc(32 * nc)                                          # cell_carry
    b += _alloc(8 * T.INIT_COLS * nc)                                 # initial-data table
    b += _alloc(8 * T.MOM_COLS * nc)                                  # result table
    return b


# ------------------------------------------------------------ admission policy
class Admission:
    """First-come-first-served admission under a byte budget and a slot
    count.  The head of the queue blocks the ones behind it (no overtaking),
    so admission order is arrival order."""

    def __init__(self, budget_bytes, n_slots, footprint_fn):
        self.budget = int(budget_bytes)
        self.free_slots = list(range(n_slots))[::-1]
        self.used = 0
        self.peak = 0
        self.queue = collections.deque()
        self.footprint = footprint_fn

    def offer(self, req):
        req.bytes = self.footprint(req)
        if req.bytes > self.budget:
            req.rejected = True
            req.error = f"needs {req.bytes} bytes, budget {self.budget}"
            return False
        self.queue.append(req)
        return True

    def admit(self):
        out = []
        while self.queue and self.free_slots and self.used + self.queue[0].bytes <= self.budget:
            req = self.queue.popleft()
            req.slot = self.free_slots.pop()
            self.used += req.bytes
            self.peak = max(self.peak, self.used)
            out.append(req)
        return out

    def release(self, req):
        self.used -= req.bytes
        self.free_slots.append(req.slot)


# ------------------------------------------------------------ the loop
class ServingLoop:
    """Runs a list of Requests through `engine` in real time (arrival
    times are seconds after run() starts).  engine must provide n_slots,
    start(req) -> job and release(job); a job provides pump() (issue what it
    may, never block) and finished() (True once its result is on the
    host)."""

    def __init__(self, engine, budget_bytes, clock=time.perf_counter, sleep=time.sleep, poll_s=100e-6):
        self.engine = engine
        self.budget = budget_bytes
        self.clock = clock
        self.sleep = sleep
        self.poll_s = poll_s

    def run(self, requests):
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        pending = collections.deque(reqs)
        adm = Admission(self.budget, self.engine.n_slots, self.engine.footprint)
        active = []
        t0 = self.clock()
        while pending or adm.queue or active:
            now = self.clock() - t0
            while pending and pending[0].arrival <= now:
                adm.offer(pending.popleft())
            for req in adm.admit():
                req.admitted = self.clock() - t0
                try:
                    active.append(self.engine.start(req))
                except Exception as e:          # e.g. the allocator ran out: fail this request only
                    req.error = f"start failed: {e}"
                    adm.release(req)
            busy = False
            for job in list(active):
                busy |= job.pump()
                if job.finished():
                    job.req.done = self.clock() - t0
                    adm.release(job.req)
                    self.engine.release(job)
                    active.remove(job)
                    busy = True
            if not busy:
                wait = self.poll_s
                if not active and not adm.queue and pending:
                    wait = max(0.0, pending[0].arrival - (self.clock() - t0))
                self.sleep(wait)
        self.peak_bytes = adm.peak
        return reqs


def summary(reqs):
    """Latency percentiles (ms) and particle-steps/s over the completed
    requests, from the first arrival to the last completion."""
    done = [r for r in reqs if r.done is not None and r.error is None]
    if not done:
        return dict(completed=0, rejected=sum(r.rejected for r in reqs), failed=sum(r.error is not None for r in reqs))
    lat = np.array([r.latency for r in done]) * 1e3
    span = max(r.done for r in done) - min(r.arrival for r in done)
    work = float(sum(r.particles * r.steps for r in done))
    return dict(completed=len(done), rejected=sum(r.rejected for r in reqs),
                failed=sum(r.error is not None and not r.rejected for r in reqs),
                p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                mean_ms=float(lat.mean()), max_ms=float(lat.max()), span_s=span,
                particle_steps_per_s=work / span if span > 0 else None,
                wait_ms_mean=float(np.mean([(r.admitted - r.arrival) * 1e3 for r in done])))


# ------------------------------------------------------------ the GPU engine
class _GpuJob:
    def __init__(self, engine, req, slot):
        import torch
        from .workloads import BatchedRelaxation, ShockTubes
        self.req, self.slot, self.engine = req, slot, engine
        ctx, stream = engine.ctxs[slot], engine.streams[slot]
        self.stream = stream
        self.ctx = ctx
        plan(req)
        nc = len(req.counts)
        self.dt0 = None
        self.t_sim = None
        with torch.cuda.stream(stream):
            if req.kind == "shock":
                self.sim = ShockTubes((req.eps,), n_cells=nc, mean_per_cell=shock_mean(req),
                                      precision=engine.precision, seed=engine.seed, ctx=ctx, problem_base=req.rid)
                if req.t_end is not None:
                    # the first CFL step from the initial data, read back without blocking
                    vm = self.sim.state.cell_vmax2[:nc].max()
                    self.vm_host = torch.empty(1, dtype=torch.float64, pin_memory=True)
                    self.vm_host.copy_(vm.reshape(1), non_blocking=True)
                    self.dt0 = torch.cuda.Event()
                    self.dt0.record(stream)
                    self.t_sim = torch.zeros(1, dtype=torch.float64, device="cuda")
            else:
                self.sim = BatchedRelaxation(counts=req.counts, eps_lo=req.eps, eps_hi=req.eps,
                                             precision=engine.precision, seed=req.rid, ctx=ctx,
                                             problem_base=req.rid, problem_per_cell=False, dt=RELAX_DT)
        assert self.sim.n_particles == req.particles
        self.issued = 0
        self.inflight = collections.deque()
        self.final = None
        self.t_check = None

    def _steps_known(self):
        if self.dt0 is None:
            return True
        if not self.dt0.query():
            return False
        dt = self.sim.cfl * (1.0 / len(self.req.counts)) / float(np.sqrt(self.vm_host.item()))
        self.req.steps = max(1, int(np.ceil(self.req.t_end / dt - 1e-9)))
        self.dt0 = None
        return True

    def pump(self):
        import torch
        issued = False
        while self.inflight and self.inflight[0].query():
            self.inflight.popleft()
        if not self._steps_known():
            return False
        with torch.cuda.stream(self.stream):
            while len(self.inflight) < self.engine.depth and self.issued < self.req.steps:
                k = min(self.engine.chunk, self.req.steps - self.issued)
                for _ in range(k):
                    self.sim.step()
                    if self.t_sim is not None:
                        self.t_sim += self.sim.dt[0]
                self.issued += k
                ev = torch.cuda.Event()
                ev.record(self.stream)
                self.inflight.append(ev)
                issued = True
            if self.issued == self.req.steps and self.final is None and self.t_sim is not None:
                # a solve ends at the first step that reaches t_end: read the
                # simulated time (and the last CFL step) back without blocking
                # and, if the CFL steps shrank on the way, add the steps still
                # missing
                if self.t_check is None:
                    self.t_host = torch.empty(2, dtype=torch.float64, pin_memory=True)
                    self.t_host.copy_(torch.cat([self.t_sim, self.sim.dt[:1]]), non_blocking=True)
                    self.t_check = torch.cuda.Event()
                    self.t_check.record(self.stream)
                    return True
                if not self.t_check.query():
                    return issued
                t, dt = (float(x) for x in self.t_host.tolist())
                if t < self.req.t_end:
                    self.req.steps += max(1, int(np.ceil((self.req.t_end - t) / dt - 1e-9)))
                    self.t_check = None
                    return True
            if self.issued == self.req.steps and self.final is None and (self.t_sim is None or self.t_check is not None):
                st = self.sim.state
                self.out = torch.empty((st.n_cells, T.MOM_COLS), dtype=torch.float64, device="cuda")
                T.trmc_moments(self.ctx, st, self.out, stream=self.stream)
                self.host = torch.empty(self.out.shape, dtype=torch.float64, pin_memory=True)
                self.host.copy_(self.out, non_blocking=True)
                self.final = torch.cuda.Event()
                self.final.record(self.stream)
                issued = True
        return issued

    def finished(self):
        if self.final is None or not self.final.query():
            return False
        try:
            T.trmc_check(self.ctx, self.stream)
        except T.TrmcError as e:
            self.req.error = str(e)
        self.req.result = self.host.numpy().copy()
        if self.req.t_end is not None:
            self.req.t_reached = float(self.t_host[0]) if self.t_sim is not None else self.req.steps * RELAX_DT
        return True


class GpuEngine:
    """Slots of libtrmc contexts and CUDA streams for ServingLoop."""

    def __init__(self, n_slots=8, precision=T.FP32_MIXED, seed=0, workspace_bytes=512 << 20, chunk=4, depth=2):
        import torch
        self.n_slots = n_slots
        self.precision = precision
        self.seed = seed
        self.chunk = chunk
        self.depth = depth
        self.workspace_bytes = workspace_bytes
        self.ctxs = [T.trmc_create(precision, seed, workspace_bytes) for _ in range(n_slots)]
        self.streams = [torch.cuda.Stream() for _ in range(n_slots)]

    @property
    def fixed_bytes(self):
        """Device bytes the engine holds whatever runs (the contexts' workspaces)."""
        return self.n_slots * (self.workspace_bytes + 4096)

    def footprint(self, req):
        plan(req)
        return footprint(req.kind, len(req.counts), req.particles, self.precision)

    def start(self, req):
        return _GpuJob(self, req, req.slot)

    def release(self, job):
        job.sim = None
        job.out = None

    def close(self):
        import torch
        torch.cuda.synchronize()
        for c in self.ctxs:
            T.trmc_destroy(c)
        self.ctxs = []


def serve(requests, budget_bytes=150 << 30, n_slots=8, precision=T.FP32_MIXED, seed=0, workspace_bytes=512 << 20,
          chunk=4, depth=2, engine=None):
    """Run requests through a fresh (or given) GPU engine; the budget covers
    the engine's workspaces and every resident request."""
    own = engine is None
    if own:
        engine = GpuEngine(n_slots, precision, seed, workspace_bytes, chunk, depth)
    try:
        loop = ServingLoop(engine, budget_bytes - engine.fixed_bytes)
        out = loop.run(requests)
        out_peak = loop.peak_bytes + engine.fixed_bytes
    finally:
        if own:
            engine.close()
    return out, out_peak
