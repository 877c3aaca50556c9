"""CUDA-graph stepping, cell ordering and the launch-shape autotuner change
how kernels are launched, never what they compute: states must be
bit-identical to plain eager stepping."""
import numpy as np
import pytest

from tests.gpu_common import T, need_gpu, torch

pytestmark = pytest.mark.gpu


def snapshot(sim):
    st = sim.state
    out = [st.v.cpu().numpy().copy(), st.cell_start.cpu().numpy().copy()]
    if st.x is not None:
        out.append(st.x.cpu().numpy().copy())
    if st.m_max is not None:
        out.append(st.m_max.cpu().numpy().copy())
    return out


def same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("precision", [T.FP64, T.FP32_MIXED])
def test_graph_replay_matches_eager_shock(precision):
    need_gpu()
    from paper_1009_2768_gb300.runtime import GraphStepper
    from paper_1009_2768_gb300.workloads import ShockTubes
    a = ShockTubes((1e-2, 1e-3), n_cells=64, mean_per_cell=200, precision=precision, seed=3)
    a.state.use_device_step(0)
    for _ in range(8):
        a.step()
    b = ShockTubes((1e-2, 1e-3), n_cells=64, mean_per_cell=200, precision=precision, seed=3)
    g = GraphStepper(b, steps_per_graph=2, warmup=2)     # 2 eager warm-up steps
    g.replay(3)                                          # + 6 replayed steps
    torch.cuda.synchronize()
    T.trmc_check(a.ctx)
    T.trmc_check(b.ctx)
    assert int(b.state.step_dev.item()) == 8 == int(a.state.step_dev.item())
    assert same(snapshot(a), snapshot(b))
    a.close()
    b.close()


def test_graph_replay_matches_eager_batched():
    need_gpu()
    from paper_1009_2768_gb300.runtime import GraphStepper
    from paper_1009_2768_gb300.workloads import BatchedRelaxation
    a = BatchedRelaxation(n_cells=300, lo=32, hi=3000, seed=5)
    a.state.use_device_step(0)
    for _ in range(5):
        a.step()
    b = BatchedRelaxation(n_cells=300, lo=32, hi=3000, seed=5)
    g = GraphStepper(b, steps_per_graph=1, warmup=1)
    g.replay(4)
    torch.cuda.synchronize()
    assert same(snapshot(a), snapshot(b))
    a.close()
    b.close()


def test_cell_order_and_launch_shape_do_not_change_results():
    need_gpu()
    from paper_1009_2768_gb300.runtime import largest_first
    from paper_1009_2768_gb300.workloads import BatchedRelaxation
    ref = BatchedRelaxation(n_cells=300, lo=32, hi=3000, seed=6)
    for s in range(3):
        ref.step()
    alt = BatchedRelaxation(n_cells=300, lo=32, hi=3000, seed=6)
    alt.state.set_cell_order(largest_first(alt.state.cell_start.cpu().numpy()))
    for s, shape in enumerate([(64, 8), (256, 2), (96, 4)]):
        T.trmc_set_collide_launch(alt.ctx, *shape)
        alt.step()
    torch.cuda.synchronize()
    assert same(snapshot(ref), snapshot(alt))
    ref.close()
    alt.close()


def test_autotuner_picks_a_measured_shape():
    need_gpu()
    from paper_1009_2768_gb300.runtime import autotune_collide
    from paper_1009_2768_gb300.workloads import BatchedRelaxation
    sim = BatchedRelaxation(n_cells=256, lo=32, hi=2000, seed=7)
    times, best = autotune_collide(sim, shapes=((128, 4), (64, 8)), steps=2)
    assert set(times) == {(128, 4), (64, 8)} and best in times
    assert times[best] == min(times.values())
    sim.close()


@pytest.mark.parametrize("precision", [T.FP64, T.FP32_MIXED])
def test_adaptive_order_does_not_change_results(precision):
    """Cells handed out longest first by the measured times of the previous
    launch (a permutation rewritten before every collide) step exactly like
    the identity order."""
    need_gpu()
    from paper_1009_2768_gb300.workloads import ShockTubes
    a = ShockTubes((1e-1, 1e-3), n_cells=64, mean_per_cell=300, precision=precision, seed=4)
    b = ShockTubes((1e-1, 1e-3), n_cells=64, mean_per_cell=300, precision=precision, seed=4)
    b.state.use_adaptive_order()
    for _ in range(6):
        a.step()
        b.step()
    torch.cuda.synchronize()
    T.trmc_check(b.ctx)
    assert same(snapshot(a), snapshot(b))
    order = b.state.cell_order.cpu().numpy()
    cost = b.state.cell_cost.cpu().numpy().view(np.uint32)
    assert np.array_equal(np.sort(order), np.arange(b.state.n_cells))
    assert cost.max() > 0
    a.close()
    b.close()


def test_autotuner_puts_the_simulation_back():
    """The autotuners step the live workload for every candidate collide
    shape, work schedule or sort schedule and then restore it: the next step
    equals that of an untuned twin."""
    need_gpu()
    from paper_1009_2768_gb300.runtime import autotune_collide, autotune_schedule, autotune_transport
    from paper_1009_2768_gb300.workloads import ShockTubes
    ref = ShockTubes((1e-2, 1e-3), n_cells=48, mean_per_cell=150, seed=9)
    tun = ShockTubes((1e-2, 1e-3), n_cells=48, mean_per_cell=150, seed=9)
    for _ in range(3):
        ref.step()
        tun.step()
    before = snapshot(tun)
    times, best = autotune_collide(tun, shapes=((64, 8), (128, 4), (96, 3)), steps=1)
    assert best in times and same(before, snapshot(tun))
    assert tun.step_index == ref.step_index
    work_times, work = autotune_schedule(tun, choices=((0, 0), (16, 1), (512, 8)), steps=1, rounds=2)
    assert set(work_times) == {(0, 0), (16, 1), (512, 8)} and work_times[work] == min(work_times.values())
    assert same(before, snapshot(tun)) and tun.step_index == ref.step_index
    sort_times, sched = autotune_transport(tun, choices=(0, 64, 256), steps=1)
    assert set(sort_times) == {0, 64, 256} and sort_times[sched] == min(sort_times.values())
    assert same(before, snapshot(tun)) and tun.step_index == ref.step_index
    ref.step()
    tun.step()
    torch.cuda.synchronize()
    assert same(snapshot(ref), snapshot(tun))
    ref.close()
    tun.close()
