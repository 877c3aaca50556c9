"""The serving loop on the GPU: a request's result is bit-identical alone
and in an overlapping mix (and to the same workload stepped directly), the
HBM budget bounds what the requests hold on the device, and every result
keeps the conserved particle counts."""
import numpy as np
import pytest

from tests.gpu_common import T, ensure_built, need_gpu, torch

pytestmark = pytest.mark.gpu

SPECS = [("shock", 30_000, 1e-2), ("relax", 40_000, 1e-3), ("shock", 61_000, 1e-4), ("relax", 20_000, 0.5),
         ("shock", 12_000, 1.0), ("relax", 70_000, 1e-4)]


def test_alone_equals_in_mix():
    need_gpu()
    ensure_built()
    from paper_1009_2768_gb300.serving import Request, serve
    mix = [Request(i, k, n, e, steps=6, arrival=0.0005 * i) for i, (k, n, e) in enumerate(SPECS)]
    out, _ = serve(mix, n_slots=3, workspace_bytes=64 << 20, chunk=2)
    assert all(r.error is None and r.done is not None for r in out)
    for i, (k, n, e) in enumerate(SPECS):
        alone = Request(i, k, n, e, steps=6)
        serve([alone], n_slots=1, workspace_bytes=64 << 20, chunk=3)
        assert alone.error is None
        assert np.array_equal(alone.result, mix[i].result), f"request {i} ({k}) differs alone and in the mix"
        res = mix[i].result
        assert np.all(np.isfinite(res))
        assert int(res[:, 0].sum()) == mix[i].particles               # walls and homogeneous cells keep every particle
        if k == "relax":
            assert np.array_equal(res[:, 0].astype(np.int64), mix[i].counts)


def test_served_result_equals_direct_stepping():
    need_gpu()
    ensure_built()
    from paper_1009_2768_gb300.serving import Request, plan, serve, shock_mean
    from paper_1009_2768_gb300.workloads import BatchedRelaxation, ShockTubes
    for rid, (k, n, e) in enumerate(SPECS[:2]):
        req = plan(Request(rid, k, n, e, steps=5))
        serve([req], n_slots=1, workspace_bytes=64 << 20, chunk=2)
        ctx = T.trmc_create(T.FP32_MIXED, 0, 64 << 20)
        if k == "shock":
            sim = ShockTubes((e,), n_cells=len(req.counts), mean_per_cell=shock_mean(req), precision=T.FP32_MIXED,
                             ctx=ctx, problem_base=rid)
        else:
            sim = BatchedRelaxation(counts=req.counts, eps_lo=e, eps_hi=e, precision=T.FP32_MIXED, seed=rid, ctx=ctx,
                                    problem_base=rid, problem_per_cell=False)
        for _ in range(5):
            sim.step()
        out = torch.empty((sim.state.n_cells, T.MOM_COLS), dtype=torch.float64, device="cuda")
        T.trmc_moments(ctx, sim.state, out)
        T.trmc_check(ctx)
        assert np.array_equal(out.cpu().numpy(), req.result)
        del sim
        T.trmc_destroy(ctx)


def test_budget_bounds_resident_requests():
    need_gpu()
    ensure_built()
    from paper_1009_2768_gb300.serving import GpuEngine, Request, serve
    reqs = [Request(i, "shock", 200_000, 1e-2, 4, arrival=0.0) for i in range(8)]
    eng = GpuEngine(n_slots=4, workspace_bytes=64 << 20, chunk=2)
    big = max(eng.footprint(r) for r in reqs)
    assert all(eng.footprint(r) == big for r in reqs)
    budget = eng.fixed_bytes + 2 * big + big // 2     # room for two requests at a time, though four slots are free
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    torch.cuda.reset_peak_memory_stats()
    out, peak = serve(reqs, budget_bytes=budget, engine=eng)
    torch.cuda.synchronize()
    grew = torch.cuda.max_memory_allocated() - base
    eng.close()
    assert all(r.done is not None and r.error is None for r in out)
    assert peak <= budget
    assert grew <= peak - eng.fixed_bytes, (grew, peak - eng.fixed_bytes)   # the accounting covers the tensors
    ev = sorted([(r.admitted, 1) for r in out] + [(r.done, -1) for r in out], key=lambda t: (t[0], t[1]))
    live = np.cumsum([d for _, d in ev])
    assert live.max() == 2
    # mixed sizes: the bytes resident at any time stay within the budget
    mixed = [Request(10 + i, "shock" if i % 2 else "relax", 100_000 + 40_000 * i, 1e-2, 3, arrival=0.0)
             for i in range(8)]
    eng = GpuEngine(n_slots=4, workspace_bytes=64 << 20, chunk=2)
    budget = eng.fixed_bytes + 2 * max(eng.footprint(r) for r in mixed)
    out, peak = serve(mixed, budget_bytes=budget, engine=eng)
    eng.close()
    assert all(r.done is not None and r.error is None for r in out)
    ev = sorted([(r.admitted, r.bytes) for r in out] + [(r.done, -r.bytes) for r in out], key=lambda t: (t[0], t[1]))
    assert np.cumsum([b for _, b in ev]).max() <= budget - eng.fixed_bytes
    # a request that can never fit is rejected, the others still run
    eng2 = GpuEngine(n_slots=2, workspace_bytes=64 << 20)
    small = Request(100, "shock", 50_000, 1e-2, 2)
    huge = Request(101, "relax", 5_000_000, 1e-2, 2)
    out2, _ = serve([huge, small], budget_bytes=eng2.fixed_bytes + eng2.footprint(small), engine=eng2)
    eng2.close()
    assert huge.rejected and huge.done is None
    assert small.done is not None and small.error is None
