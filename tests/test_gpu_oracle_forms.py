"""The batched, graph-replayed and served forms of the step against the FP64
CPU oracle, and the FP32-mixed form's error against it.

* A batched relaxation stepped from a captured CUDA graph (FP64) equals the
  oracle stepping the same initial state with the same keys: velocities
  within 1e-12 of each cell's speed scale, RAD depths exact.
* A served solve (FP64 engine, one slot, the request run to its physical end
  time) equals the oracle stepping the same request's initial state the same
  number of steps: per-cell moments within 1e-12, the simulated time reached
  equal to the oracle's sum of CFL steps.
* FP32-mixed: a batched relaxation (bi-Maxwellian cells, VHS 0.6, TRMC-RAD)
  tracks the FP64 oracle on the same keys far more closely than the oracle
  tracks itself with other keys (the Monte Carlo noise), and the mean
  anisotropy of its cells after the run equals the oracle's within the
  Monte Carlo error of the difference.
"""
import numpy as np
import pytest

from oracle.stepper import OracleSim
from tests.gpu_common import T, assert_velocity_parity, ensure_built, need_gpu, torch

pytestmark = pytest.mark.gpu


def gpu_moments(sim):
    mom = torch.zeros((sim.state.n_cells, T.MOM_COLS), dtype=torch.float64, device="cuda")
    T.trmc_moments(sim.ctx, sim.state, mom)
    return mom.cpu().numpy()


def test_graph_replayed_batched_step_matches_the_oracle():
    need_gpu()
    ensure_built()
    from paper_1009_2768_gb300.runtime import GraphStepper
    from paper_1009_2768_gb300.workloads import BatchedRelaxation
    sim = BatchedRelaxation(n_cells=300, lo=2, hi=3000, precision=T.FP64, seed=5, order="adaptive")
    orc = OracleSim(sim, seed=5)
    g = GraphStepper(sim, steps_per_graph=2, warmup=1)      # 1 eager step
    g.replay(2)                                             # + 4 replayed steps
    torch.cuda.synchronize()
    T.trmc_check(sim.ctx)
    for _ in range(5):
        orc.step(threads=4)
    n = orc.n
    assert_velocity_parity(sim.state.v[:, :n].cpu().numpy(), orc.v, orc.cs)
    assert np.array_equal(sim.state.m_max.cpu().numpy(), orc.ms)
    sim.close()


@pytest.mark.parametrize("kind,n,eps", [("shock", 24_000, 1e-2), ("relax", 30_000, 1e-3)])
def test_served_solve_matches_the_oracle(kind, n, eps):
    need_gpu()
    ensure_built()
    from paper_1009_2768_gb300.serving import T_END, Request, plan, serve, shock_mean
    from paper_1009_2768_gb300.workloads import BatchedRelaxation, ShockTubes
    t_end = {"shock": 0.01, "relax": T_END["relax"]}[kind]
    req = plan(Request(7, kind, n, eps, 0, t_end=t_end))
    out, _ = serve([req], n_slots=1, precision=T.FP64, workspace_bytes=64 << 20, chunk=3)
    assert req.error is None and req.steps > 0
    # the same request's initial state, built and stepped by the oracle
    ctx = T.trmc_create(T.FP64, 0, 64 << 20)
    if kind == "shock":
        sim = ShockTubes((eps,), n_cells=len(req.counts), mean_per_cell=shock_mean(req), precision=T.FP64, ctx=ctx,
                         problem_base=req.rid)
    else:
        sim = BatchedRelaxation(counts=req.counts, eps_lo=eps, eps_hi=eps, precision=T.FP64, seed=req.rid, ctx=ctx,
                                problem_base=req.rid, problem_per_cell=False)
    orc = OracleSim(sim, seed=0)
    T.trmc_destroy(ctx)
    t = 0.0
    for _ in range(req.steps):
        orc.step(threads=4)
        if kind == "shock":
            t += float(orc.cp[0, 1])
    ref = orc.moments()
    got = req.result
    assert np.array_equal(got[:, 0], ref[:, 0])                           # particles per cell
    scale = np.maximum(np.abs(ref), 1.0)
    assert np.all(np.abs(got[:, 1:9] - ref[:, 1:9]) <= 1e-12 * scale[:, 1:9])
    if kind == "shock":
        assert req.t_reached >= t_end and abs(req.t_reached - t) <= 1e-12 * t
    else:
        assert req.steps == 20 and abs(req.t_reached - 1.0) < 1e-12


def test_fp32_mixed_batched_tracks_the_oracle_within_noise():
    need_gpu()
    ensure_built()
    from paper_1009_2768_gb300.workloads import BatchedRelaxation
    steps = 10
    sim = BatchedRelaxation(n_cells=600, lo=64, hi=2048, precision=T.FP32_MIXED, seed=8, eps_lo=1e-2, eps_hi=1.0)
    orc, other = OracleSim(sim, seed=8), OracleSim(sim, seed=9)
    m0 = gpu_moments(sim)
    for _ in range(steps):
        sim.step()
    T.trmc_check(sim.ctx)
    got = gpu_moments(sim)
    for _ in range(steps):
        orc.step(threads=8)
        other.step(threads=8)
    ref, alt = orc.moments(), other.moments()
    an = lambda m: (m[:, 6] - m[:, 5]) / m[:, 5]
    a0 = np.abs(an(m0)).sum()
    err = np.abs(an(got) - an(ref)).sum() / a0
    noise = np.abs(an(alt) - an(ref)).sum() / a0
    assert err < 0.5 * noise, (err, noise)
    d = an(got) - an(ref)
    assert abs(d.mean()) <= 4.0 * d.std(ddof=1) / np.sqrt(len(d)) + 1e-12
    # conservation of every cell (stored floats plus the FP64 carry)
    n = sim.n_particles
    cs = sim.state.cell_start.cpu().numpy()
    v = sim.state.v[:, :n].double().cpu().numpy()
    carry = sim.state.cell_carry.cpu().numpy()
    for c in range(0, len(cs) - 1, 37):
        a, b = cs[c], cs[c + 1]
        p = v[:, a:b].sum(1) + carry[c, :3]
        e = (v[:, a:b] ** 2).sum() + carry[c, 3]
        assert np.all(np.abs(p - m0[c, 2:5] * (b - a)) <= 1e-9 * np.abs(v[:, a:b]).sum())
        assert abs(e - 2 * m0[c, 8] * (b - a)) <= 1e-9 * e
    sim.close()
