"""Runtime helpers around the C ABI: CUDA-graph stepping, the launch-shape
autotuner and largest-first cell ordering.  Everything here only decides
how the library's kernels are launched: the results are bit-identical for
every launch shape and cell order (the library sums every cell's moments in
one canonical order whatever the CTA size), and the autotuner puts the
simulation back where it found it.

* GraphStepper captures a fixed number of whole time steps (transport +
  sort + collide, or collide alone) into one CUDA graph and replays it.  The
  collision draws are keyed by a device step counter that every collide
  launch advances (trmc_state.step_dev), so replays step the simulation
  exactly as eager calls would.  A graph holds an even number of steps when
  the workload transports: the sort's ping-pong buffers are then back in
  their original roles at the end of every replay.
* autotune_collide times candidate (CTA size, CTAs per SM) shapes on the
  live workload in interleaved rounds (every candidate once per round, so a
  drift over the sweep falls on all of them alike), keeps the one with the
  smallest median and then restores the state it stepped (velocities,
  positions, cell starts, RAD depths, carries, step counters).
  autotune_schedule then sweeps the work schedule inside a cell at that
  shape: the particles per warp (the largest tree level one warp takes alone)
  and the levels whose collisions are precomputed as records (collisions per
  thread).  autotune_transport does the same for the sort schedule (threads
  per CTA of the counting sort's count and scatter kernels, one CTA per
  cell), and autotune runs all three.
* largest_first orders cells by particle count, biggest first, so the
  longest cells start early and the launch does not end on one of them.
"""
import numpy as np

from . import trmc as T

DEFAULT_SHAPES = ((256, 3), (256, 2), (128, 4), (128, 3), (160, 3), (192, 2), (64, 8), (512, 1))
SORT_SCHEDULES = (0, 64, 128, 256)     # transport threads per cell CTA (0: by mean cell size)
# (particles per warp, records per thread); (0, 0) is the library's default
WORK_SCHEDULES = ((0, 0), (32, 4), (128, 4), (512, 4), (0, 2), (0, 8))


def largest_first(cell_start):
    counts = np.diff(np.asarray(cell_start, dtype=np.int64))
    return np.argsort(-counts, kind="stable").astype(np.int32)


class GraphStepper:
    """Replays `steps_per_graph` steps of `sim` (an object with .state,
    .ctx and .step()) from one captured CUDA graph; `step_kwargs` (e.g. a
    statistics buffer, which then accumulates over replays) are passed to
    the captured steps."""

    def __init__(self, sim, steps_per_graph=2, warmup=2, step_kwargs=None):
        import torch
        kw = dict(step_kwargs or {})
        self.sim = sim
        transports = getattr(sim, "transports", False)
        if transports and steps_per_graph % 2:
            raise ValueError("a transporting workload needs an even number of steps per graph")
        if sim.state.step_dev is None:
            sim.state.use_device_step(getattr(sim, "step_index", 0))
        self.steps_per_graph = steps_per_graph
        self.stream = torch.cuda.Stream()
        self.stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(self.stream):
            for _ in range(warmup):            # first calls allocate and configure, outside the capture
                sim.step()
        self.stream.synchronize()
        T.trmc_check(sim.ctx)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            for _ in range(steps_per_graph):
                sim.step(**kw)
        torch.cuda.current_stream().wait_stream(self.stream)

    def replay(self, times=1):
        for _ in range(times):
            self.graph.replay()


def _snapshot(sim):
    """Copies of every tensor of the simulation's state and its step index."""
    import torch
    st = sim.state
    keep = {k: v.clone() for k, v in vars(st).items() if isinstance(v, torch.Tensor)}
    extra = {k: v.clone() for k, v in vars(sim).items() if isinstance(v, torch.Tensor)}
    return keep, extra, getattr(sim, "step_index", None)


def _restore(sim, snap):
    """Copy the snapshot back.  Transport swaps the roles of a state's
    primary and *_alt tensors; the data go back under the names they had, and
    the C struct is refilled to match."""
    keep, extra, step_index = snap
    st = sim.state
    for k, v in keep.items():
        cur = getattr(st, k)
        if cur.data_ptr() != v.data_ptr():
            cur.copy_(v)
    for k, v in extra.items():
        getattr(sim, k).copy_(v)
    if step_index is not None:
        sim.step_index = step_index
    st._fill()


def _sweep(sim, choices, apply, which, rounds, steps, flush_bytes):
    """Time every choice in `rounds` interleaved rounds (each round sets every
    choice in turn, takes one untimed step and `steps` timed ones, an L2
    flush before each), so that a drift of the state or of the GPU over the
    sweep falls on all choices alike; keep the choice with the smallest
    median, restore the simulation and return ({choice: median ms}, best).
    `which` picks the timed part of a step: 0 transport, 1 collide."""
    import torch
    flush = torch.empty(flush_bytes, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    snap = _snapshot(sim)
    samples = {c: [] for c in choices}
    for _ in range(rounds):
        for c in choices:
            apply(c)
            sim.step()                                # configure this choice outside the timing
            for _ in range(steps):
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                flush.zero_()
                sim.step(events=ev)
                torch.cuda.synchronize()
                samples[c].append(ev[which].elapsed_time(ev[which + 1]))
    times = {c: float(np.median(v)) for c, v in samples.items()}
    best = min(times, key=times.get)
    apply(best)
    T.trmc_check(sim.ctx)
    _restore(sim, snap)
    torch.cuda.synchronize()
    return times, best


def autotune_collide(sim, shapes=DEFAULT_SHAPES, steps=2, rounds=4, flush_bytes=256 << 20):
    """The fastest (threads, CTAs per SM) collide launch shape for the live
    workload (median collide time over interleaved rounds); the simulation is
    put back in the state it had.  Returns ({shape: median ms}, best), the
    best shape left set."""
    return _sweep(sim, shapes, lambda c: T.trmc_set_collide_launch(sim.ctx, *c), 1, rounds, steps, flush_bytes)


def autotune_schedule(sim, choices=WORK_SCHEDULES, steps=2, rounds=4, flush_bytes=256 << 20):
    """The fastest work schedule inside a cell (particles per warp, records
    per thread) at the current launch shape, timed like autotune_collide.
    Returns ({schedule: median ms}, best), the best left set."""
    return _sweep(sim, choices, lambda c: T.trmc_set_collide_schedule(sim.ctx, *c), 1, rounds, steps, flush_bytes)


def autotune_transport(sim, choices=SORT_SCHEDULES, steps=2, rounds=4, flush_bytes=256 << 20):
    """The fastest sort schedule (threads per CTA of the counting sort's count
    and scatter kernels; 0 lets the library pick from the mean cell size),
    timed on the transport like autotune_collide.  A workload without
    transport returns ({}, None)."""
    if not getattr(sim, "transports", False):
        return {}, None
    return _sweep(sim, choices, lambda c: T.trmc_set_transport_launch(sim.ctx, c), 0, rounds, steps, flush_bytes)


def autotune(sim, shapes=DEFAULT_SHAPES, schedules=SORT_SCHEDULES, steps=2, work=WORK_SCHEDULES, rounds=4):
    """The collide launch shape, then the work schedule inside a cell at that
    shape, and the sort schedule for the live workload (all left set; the
    simulation is restored)."""
    collide_times, shape = autotune_collide(sim, shapes, steps, rounds)
    work_times, wsched = autotune_schedule(sim, work, steps, rounds)
    sort_times, sched = autotune_transport(sim, schedules, steps, rounds)
    return {"collide": collide_times, "collide_best": shape, "work": work_times, "work_best": wsched,
            "sort": sort_times, "sort_best": sched}
