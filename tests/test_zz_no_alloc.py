"""trmc_collide_static, the collision step for callers that cannot allocate
device memory where they run it (code where cudaMalloc is forbidden or would
synchronise the device, or a plug-in handed particle arrays but no
allocator).  It must give what trmc_collide gives on the same inputs, call
after call, using only the library's fixed scratch array.  This file is
collected last so that a failure here comes after every other test ran."""
import numpy as np
import pytest

from paper_1009_2768_gb300 import synth
from tests.gpu_common import T, assert_velocity_parity, ctx, need_gpu, torch

pytestmark = pytest.mark.gpu

COUNTS = [2, 64, 300, 889, 2500, 6000]      # the last cell overflows shared memory into the scratch slab


def _states(precision, counts, seed):
    g = synth.rng(seed)
    v = np.concatenate([synth.bimaxwellian(n, 2.0, 0.5, u=(0.2, 0.0, -0.1), g=g) for n in counts], axis=1)
    cs = synth.starts(counts)
    out = []
    for _ in range(2):
        st = T.ParticleState(cs, precision=precision, rad=True)
        st.set_velocities(v)
        st.m_max.fill_(2)
        out.append(st)
    return cs, out


@pytest.mark.parametrize("precision", [T.FP64, T.FP32_MIXED])
def test_static_matches_trmc_collide_two_calls_in_a_row(precision):
    need_gpu()
    cs, (ref, st) = _states(precision, COUNTS, seed=31)
    p = T.collide_params(dt=0.05, eps=0.05, alpha=1.0, rho_scale=1.0 / 500, trunc=T.TRUNC_RAD, m=2)
    c = ctx(precision, seed=0)
    status = torch.zeros(2, dtype=torch.int32, device="cuda")
    for step in (4, 5):
        T.trmc_collide(c, ref, p, step)
        T.trmc_check(c)
        T.trmc_collide_static(st, p, precision, 0, step, max(COUNTS), status)
        torch.cuda.synchronize()
        assert status.tolist() == [0, 0]
        n = int(cs[-1])
        assert_velocity_parity(st.v[:, :n].double().cpu().numpy(), ref.v[:, :n].double().cpu().numpy(), cs)
        assert torch.equal(st.m_max, ref.m_max)
        assert torch.equal(st.cell_vmax2, ref.cell_vmax2)


def test_static_rejects_cells_larger_than_its_scratch():
    need_gpu()
    cs, (_, st) = _states(T.FP64, [100], seed=32)
    p = T.collide_params(dt=0.05, eps=1.0, rho_scale=0.01, trunc=T.TRUNC_FIXED, m=2)
    with pytest.raises(T.TrmcError) as e:
        T.trmc_collide_static(st, p, T.FP64, 0, 0, 1 << 30)
    assert e.value.code == T.ERR_CAPACITY


def test_static_between_calls_of_a_wide_launch_shape():
    """A context whose collide launch uses two CTAs per SM (about twice the
    shared memory per CTA of the default) keeps working after an
    allocation-free call in between, and its results do not depend on it."""
    need_gpu()
    cs, (ref, st) = _states(T.FP64, COUNTS, seed=33)
    p = T.collide_params(dt=0.05, eps=0.05, alpha=1.0, rho_scale=1.0 / 500, trunc=T.TRUNC_RAD, m=2)
    c_ref, c = ctx(T.FP64, seed=0), T.trmc_create(T.FP64, 0, 256 << 20)
    T.trmc_set_collide_launch(c, 256, 2)
    tmp = T.ParticleState(cs, precision=T.FP64, rad=True)
    tmp.set_velocities(st.v[:, :int(cs[-1])].cpu().numpy())
    tmp.m_max.fill_(2)
    for step in (1, 2):
        T.trmc_collide(c_ref, ref, p, step)
        T.trmc_collide(c, st, p, step)
        T.trmc_collide_static(tmp, p, T.FP64, 0, step, max(COUNTS))
        T.trmc_check(c)
        T.trmc_check(c_ref)
    T.trmc_destroy(c)
    n = int(cs[-1])
    # per-cell sums run in the same canonical order for every CTA size
    assert torch.equal(st.v[:, :n], ref.v[:, :n])
    assert torch.equal(tmp.v[:, :n], ref.v[:, :n])


def test_static_reports_a_cell_larger_than_its_bound():
    """With max_cell_particles below the real largest cell, that cell can
    overflow its slab: it is left unchanged and reported in status_dev as
    (TRMC_ERR_CAPACITY, cell) while every other cell is collided."""
    need_gpu()
    counts = [50] * 700 + [6000]
    cs, (_, st) = _states(T.FP64, counts, seed=34)
    before = st.v.clone()
    p = T.collide_params(dt=0.05, eps=0.05, alpha=1.0, rho_scale=1.0 / 500, trunc=T.TRUNC_RAD, m=2)
    status = torch.zeros(2, dtype=torch.int32, device="cuda")
    T.trmc_collide_static(st, p, T.FP64, 0, 1, 50, status)
    torch.cuda.synchronize()
    assert status.tolist() == [T.ERR_CAPACITY, len(counts) - 1]
    assert torch.equal(st.v[:, cs[-2]:cs[-1]], before[:, cs[-2]:cs[-1]])
    assert not torch.equal(st.v[:, :cs[-2]], before[:, :cs[-2]])
