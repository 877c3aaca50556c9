"""The benchmark workloads at their full sizes, built and launched exactly as
bench.py times them (its make_sim and LAUNCH): the collide results are
checked where the oracle can follow them one cell at a time, and by
properties that hold at any size where it cannot.

- FP64 shock tubes (4 x 400 cells, 8e5 particles): after a few steps, the
  cells of one collide launch -- the four longest of the previous launch and
  an even sample of every tube -- are recomputed by the oracle from the
  launch's own inputs (velocities after transport, per-cell dt and RAD state,
  cell keys) and must match within 1e-12 relative, RAD states exactly.
- FP32-mixed stationary shock (1e7 particles) and batched relaxation (4096
  cells): every cell's momentum and energy, stored floats plus the FP64
  carry, are unchanged by a collide launch, within FP64 rounding."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1009_2768_gb300 import synth
from tests.gpu_common import T, assert_velocity_parity, need_gpu, oracle_params, torch

pytestmark = pytest.mark.gpu


def bench_sim(workload):
    import bench
    sim, _, _ = bench.make_sim(workload, 0)
    T.trmc_set_collide_launch(sim.ctx, *bench.LAUNCH[workload])
    return sim


def one_step(sim, before_collide=None):
    """The workload's own step, split so the state between transport and
    collide can be read."""
    if getattr(sim, "transports", False):
        T.trmc_transport(sim.ctx, sim.state, sim.domains, getattr(sim, "n_tubes", 1), sim.cfl, sim.dt,
                         sim.step_index)
    snap = before_collide() if before_collide else None
    T.trmc_collide(sim.ctx, sim.state, sim.params, sim.step_index)
    sim.step_index += 1
    return snap


def test_shock_tubes_full_size_sampled_cells_match_oracle():
    need_gpu()
    sim = bench_sim("shock")
    for _ in range(4):
        one_step(sim)
    T.trmc_check(sim.ctx)
    st = sim.state

    def snapshot():
        torch.cuda.synchronize()
        return {"cs": st.cell_start.cpu().numpy().copy(), "v": st.v.cpu().numpy().copy(),
                "m": st.m_max.cpu().numpy().copy(), "cp": st.cell_param.cpu().numpy().copy(),
                "key": st.cell_key.cpu().numpy().view(np.uint64).copy(),
                "cost": st.cell_cost.cpu().numpy().astype(np.int64)}

    step = sim.step_index
    s = one_step(sim, snapshot)
    T.trmc_check(sim.ctx)
    torch.cuda.synchronize()
    v_after, m_after = st.v.cpu().numpy(), st.m_max.cpu().numpy()
    nc, per_tube = st.n_cells, sim.n_cells_tube
    longest = np.argsort(-s["cost"], kind="stable")[:4]
    sample = {int(c) for c in longest}
    for t in range(sim.n_tubes):
        sample |= {t * per_tube + int(c) for c in np.linspace(0, per_tube - 1, 7).round()}
    cells = sorted(sample)
    assert len(cells) >= 28 and max(cells) < nc
    cs = s["cs"]
    counts = np.array([cs[c + 1] - cs[c] for c in cells])
    sub = synth.starts(counts)
    v_in = np.concatenate([s["v"][:, cs[c]:cs[c + 1]] for c in cells], axis=1)
    v_gpu = np.concatenate([v_after[:, cs[c]:cs[c + 1]] for c in cells], axis=1)
    po = oracle_params(O, sim.params)
    vo, _, mo = O.collide(v_in, sub, po, step, m_state=s["m"][cells], cell_param=s["cp"][cells].ravel(),
                          cell_key=s["key"][cells])
    assert_velocity_parity(v_gpu, vo, sub)
    assert np.array_equal(m_after[cells], mo)
    sim.close()


def cell_sums(v, cs):
    """Per-cell sums of v (3) and of |v|^2 in FP64 (squares of floats are
    exact in FP64; numpy's pairwise sums keep the rounding near 1e-16)."""
    n = int(cs[-1])
    v = v[:, :n].astype(np.float64)
    e = (v * v).sum(axis=0)
    out = np.zeros((len(cs) - 1, 4))
    for c in range(len(cs) - 1):
        a, b = cs[c], cs[c + 1]
        out[c, :3] = v[:, a:b].sum(axis=1)
        out[c, 3] = e[a:b].sum()
    return out


@pytest.mark.parametrize("workload", ["stationary", "batched"])
def test_fp32_workloads_full_size_conserve_every_cell(workload):
    need_gpu()
    sim = bench_sim(workload)
    for _ in range(3):
        one_step(sim)
    T.trmc_check(sim.ctx)
    st = sim.state

    def snapshot():
        torch.cuda.synchronize()
        cs = st.cell_start.cpu().numpy().copy()
        return cs, cell_sums(st.v.cpu().numpy(), cs) + st.cell_carry.cpu().numpy()[:st.n_cells]

    cs, q0 = one_step(sim, snapshot)
    T.trmc_check(sim.ctx)
    torch.cuda.synchronize()
    assert np.array_equal(st.cell_start.cpu().numpy(), cs)       # the collide moves no particle between cells
    q1 = cell_sums(st.v.cpu().numpy(), cs) + st.cell_carry.cpu().numpy()[:st.n_cells]
    scale = np.abs(q0).max(axis=1, keepdims=True) + 1e-300
    err = np.abs(q1 - q0) / scale
    assert err.max() <= 1e-12, (int(err.max(axis=1).argmax()), float(err.max()))
    sim.close()
