"""Results do not depend on the collide launch shape: every per-cell sum
(moments, the collisions' change, the thermalised set, the Maxwellian
samples, the carry) runs over the same 256 virtual lanes and 8 virtual warps
in a fixed tree whatever the CTA size, so the bound, q, the split and every
velocity have the same bits for every (threads per CTA, CTAs per SM).  Nor on
the work schedule inside a cell (particles per warp, records per thread)."""
import numpy as np
import pytest

from paper_1009_2768_gb300 import synth
from tests.gpu_common import T, need_gpu, torch, ensure_built

pytestmark = pytest.mark.gpu

COUNTS = [2, 3, 17, 64, 255, 257, 889, 2500, 6000, 9001]
SHAPES = [(64, 8), (128, 4), (256, 2), (96, 3), (32, 8), (512, 1)]


def run_shape(precision, shape, params, counts, steps=2, carry=False, schedule=None):
    ensure_built()
    g = synth.rng(77)
    v = np.concatenate([synth.bimaxwellian(n, 2.0, 0.5, u=(0.3, -0.2, 0.1), g=g) for n in counts], axis=1)
    cs = synth.starts(counts)
    nc = len(counts)
    cp = np.stack([np.geomspace(1e-3, 1.0, nc), np.full(nc, 0.05), 1.0 / np.asarray(counts, float) * 2.0,
                   np.full(nc, params.alpha)], axis=1)
    st = T.ParticleState(cs, precision=precision, rad=params.trunc == T.TRUNC_RAD, cell_param=cp, carry=carry)
    st.set_velocities(v)
    if st.m_max is not None:
        st.m_max.fill_(2)
    c = T.trmc_create(precision, 11, 1 << 30)
    T.trmc_set_collide_launch(c, *shape)
    if schedule is not None:
        T.trmc_set_collide_schedule(c, *schedule)
    rep = torch.zeros((nc, T.REPORT_LEN), dtype=torch.int64, device="cuda")
    for s in range(steps):
        T.trmc_collide(c, st, params, 3 + s, report=rep)
    T.trmc_check(c)
    T.trmc_destroy(c)
    out = [st.v.cpu().numpy(), rep.cpu().numpy(), st.cell_vmax2.cpu().numpy()]
    if st.m_max is not None:
        out.append(st.m_max.cpu().numpy())
    if carry:
        out.append(st.cell_carry.cpu().numpy())
    return out


PARAMS = {
    "rad hard spheres": T.collide_params(alpha=1.0, trunc=T.TRUNC_RAD, m=2, indicator=T.IND_PXX),
    "rad M4, vhs 0.6": T.collide_params(alpha=0.6, trunc=T.TRUNC_RAD, m=2, indicator=T.IND_M4),
    "fixed m=4, Maxwell": T.collide_params(alpha=0.0, trunc=T.TRUNC_FIXED, m=4),
    "wb, 1 + min": T.collide_params(alpha=1.0, trunc=T.TRUNC_WB, m=3, m_cap=12, wb_length=T.LEN_MIN),
}


@pytest.mark.parametrize("precision", [T.FP64, T.FP32_MIXED])
@pytest.mark.parametrize("name", sorted(PARAMS))
def test_results_are_bit_identical_across_launch_shapes(precision, name):
    need_gpu()
    carry = precision == T.FP32_MIXED
    ref = run_shape(precision, SHAPES[0], PARAMS[name], COUNTS, carry=carry)
    for shape in SHAPES[1:]:
        got = run_shape(precision, shape, PARAMS[name], COUNTS, carry=carry)
        for a, b in zip(ref, got):
            assert np.array_equal(a, b), f"launch shape {shape} differs from {SHAPES[0]} ({name})"


# (particles per warp, records per thread; 0: the default): levels from one
# collision up in CTA-wide waves, or every level in one warp; records for few
# levels or for the largest ones
SCHEDULES = [(0, 0), (2, 1), (16, 1), (256, 16), (4096, 4), (8192, 16)]


@pytest.mark.parametrize("precision", [T.FP64, T.FP32_MIXED])
@pytest.mark.parametrize("name", sorted(PARAMS))
def test_results_are_bit_identical_across_work_schedules(precision, name):
    # which warps run a level, and which levels' collisions are precomputed,
    # moves work between threads only: same draws, same sums, same bits
    need_gpu()
    carry = precision == T.FP32_MIXED
    ref = run_shape(precision, (128, 4), PARAMS[name], COUNTS, carry=carry, schedule=SCHEDULES[0])
    for sch in SCHEDULES[1:]:
        got = run_shape(precision, (128, 4), PARAMS[name], COUNTS, carry=carry, schedule=sch)
        for a, b in zip(ref, got):
            assert np.array_equal(a, b), f"work schedule {sch} differs from the default ({name})"


def test_work_schedule_arguments_are_checked():
    need_gpu()
    ensure_built()
    c = T.trmc_create(T.FP64, 0, 1 << 20)
    for bad in ((3, 0), (1, 0), (8194, 0), (-2, 0), (0, 17), (0, -1)):
        with pytest.raises(T.TrmcError):
            T.trmc_set_collide_schedule(c, *bad)
    T.trmc_set_collide_schedule(c, 64, 4)
    T.trmc_destroy(c)


@pytest.mark.parametrize("precision,shape", [(T.FP32_MIXED, (256, 3)), (T.FP64, (256, 2))])
def test_whole_mode_with_cells_in_the_slab(precision, shape):
    """Cells a little too large for shared memory (here up to 4100 particles,
    against room for about 3950 FP32 or 3640 FP64 ones) keep the launch in
    the whole-staging kernel, those cells staged in global memory, from the
    second launch of a context on: the same bits as the dual kernel, which
    the smallest CTAs run."""
    need_gpu()
    counts = [3000, 3950, 4100, 2500, 3700, 17]
    params = PARAMS["rad hard spheres"]
    carry = precision == T.FP32_MIXED
    ref = run_shape(precision, (64, 8), params, counts, steps=3, carry=carry)
    got = run_shape(precision, shape, params, counts, steps=3, carry=carry)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", [T.FP64, T.FP32_MIXED])
@pytest.mark.parametrize("alpha,ind", [(0.0, T.IND_M4), (1.0, T.IND_PXX)])
def test_large_cells_moment_prepass_gives_the_same_bits(precision, alpha, ind):
    """Cells of at least 32768 particles get their moment sums from a pre-pass
    that spreads the eight virtual warps over eight CTAs; the allocation-free
    entry point sums them in the cell's own CTA.  Two steps, same bits."""
    need_gpu()
    ensure_built()
    counts = [40000, 5, 70001, 1200, 33000]
    g = synth.rng(21)
    v = np.concatenate([synth.bkw(n, 0.6, g=g) for n in counts], axis=1)
    cs = synth.starts(counts)
    p = T.collide_params(dt=0.05, eps=0.5, alpha=alpha, rho_scale=1.0 / 40000, trunc=T.TRUNC_RAD, m=2, indicator=ind)
    sts = []
    for _ in range(2):
        st = T.ParticleState(cs, precision=precision, rad=True)
        st.set_velocities(v)
        st.m_max.fill_(2)
        sts.append(st)
    c = T.trmc_create(precision, 0, 1 << 30)
    status = torch.zeros(2, dtype=torch.int32, device="cuda")
    for step in (0, 1):
        T.trmc_collide(c, sts[0], p, step)
        T.trmc_check(c)
        T.trmc_collide_static(sts[1], p, precision, 0, step, max(counts), status)
        torch.cuda.synchronize()
        assert status.tolist() == [0, 0]
        for a, b in ((sts[0].v, sts[1].v), (sts[0].m_max, sts[1].m_max), (sts[0].cell_vmax2, sts[1].cell_vmax2)):
            assert torch.equal(a, b)
    T.trmc_destroy(c)


def test_sort_schedule_does_not_change_transport():
    """The counting sort is stable whatever its CTA size: shock tubes stepped
    with 64, 128 or 256 threads per cell CTA (and the library's own pick) end
    in bit-identical states."""
    need_gpu()
    ensure_built()
    from paper_1009_2768_gb300.workloads import ShockTubes
    out = []
    for tt in (0, 64, 128, 256):
        sim = ShockTubes((1e-2, 1e-3), n_cells=64, mean_per_cell=300, precision=T.FP64, seed=4)
        T.trmc_set_transport_launch(sim.ctx, tt)
        for _ in range(4):
            sim.step()
        torch.cuda.synchronize()
        T.trmc_check(sim.ctx)
        st = sim.state
        out.append([st.v.cpu().numpy(), st.x.cpu().numpy(), st.cell_start.cpu().numpy(), st.m_max.cpu().numpy()])
        sim.close()
    for other in out[1:]:
        for a, b in zip(out[0], other):
            assert np.array_equal(a, b)
