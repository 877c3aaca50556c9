"""Runtime helpers around the C ABI: CUDA-graph stepping, the launch-shape
autotuner and largest-first cell ordering.  Everything here only decides
how the library's kernels are launched; results do not change.

* GraphStepper captures a fixed number of whole time steps (transport +
  sort + collide, or collide alone) into one CUDA graph and replays it.  The
  collision draws are keyed by a device step counter that every collide
  launch advances (trmc_state.step_dev), so replays step the simulation
  exactly as eager calls would.  A graph holds an even number of steps when
  the workload transports: the sort's ping-pong buffers are then back in
  their original roles at the end of every replay.
* autotune_collide times candidate (CTA size, CTAs per SM) shapes on the
  live workload and keeps the fastest.
* largest_first orders cells by particle count, biggest first, so the
  longest cells start early and the launch does not end on one of them.
"""
import numpy as np

from . import trmc as T

DEFAULT_SHAPES = ((128, 4), (96, 4), (96, 5), (128, 3), (160, 3), (192, 2), (256, 2), (64, 8))


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


def autotune_collide(sim, shapes=DEFAULT_SHAPES, steps=6, flush_bytes=256 << 20):
    """Time `steps` collide launches of the live workload for every (threads,
    CTAs per SM) shape, with an L2 flush before each, and keep the fastest.
    Returns {shape: mean collide ms} and leaves the best shape set."""
    import torch
    flush = torch.empty(flush_bytes, dtype=torch.uint8, device="cuda")
    times = {}
    for shape in shapes:
        T.trmc_set_collide_launch(sim.ctx, *shape)
        sim.step()                                    # configure this shape outside the timing
        ms = []
        for _ in range(steps):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            flush.zero_()
            sim.step(events=ev)
            torch.cuda.synchronize()
            ms.append(ev[1].elapsed_time(ev[2]))
        times[shape] = float(np.median(ms))
    best = min(times, key=times.get)
    T.trmc_set_collide_launch(sim.ctx, *best)
    T.trmc_check(sim.ctx)
    return times, best
