"""Parity of the CUDA library (FP64 contexts) with the CPU oracle, through
the C ABI: the per-cell plan records (split quotas, collisions and demand
per level, roles, passes, counters) must be bit-identical and every
velocity must agree within 1e-12 relative; transport and the cell sort
must be bit-identical; init and moments within 1e-12."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1009_2768_gb300 import synth
from tests.gpu_common import (T, TOL_V, assert_velocity_parity, ctx, gpu_collide, need_gpu, oracle_params,
                              torch)

pytestmark = pytest.mark.gpu

COUNTS = [2, 3, 5, 17, 64, 255, 256, 257, 889, 1000, 2500, 4100]


def cells(counts, seed, kind="bimax"):
    g = synth.rng(seed)
    if kind == "bkw":
        v = np.concatenate([synth.bkw(n, 0.6, g=g) for n in counts], axis=1)
    else:
        v = np.concatenate([synth.bimaxwellian(n, 2.0, 0.5, u=(0.3, -0.1, 0.2), g=g) for n in counts], axis=1)
    return v, synth.starts(counts)


def compare(v, cs, p, step, m_state=None, cell_param=None, cell_key=None, workspace=256 << 20, launch=None):
    need_gpu()
    g = gpu_collide(v, cs, p, step, m_state=m_state, cell_param=cell_param, cell_key=cell_key, workspace=workspace,
                    launch=launch)
    vo, rep, ms = O.collide(v, cs, oracle_params(O, p), step, m_state=m_state,
                            cell_param=None if cell_param is None else np.asarray(cell_param, np.float64).ravel(),
                            cell_key=cell_key)
    assert np.array_equal(g["report"], rep), first_report_diff(g["report"], rep)
    assert_velocity_parity(g["v"], vo, cs)
    if m_state is not None:
        assert np.array_equal(g["m_state"], ms)
    return g, vo, rep


def first_report_diff(a, b):
    idx = np.argwhere(a != b)
    if len(idx) == 0:
        return ""
    c, f = idx[0]
    name = T.REPORT_FIELDS[f] if f < 16 else ("Nk", "Ck", "Dk")[(f - 16) // (T.MCAP + 2)] + f"[{(f - 16) % (T.MCAP + 2)}]"
    return f"cell {c} field {name}: gpu {a[c, f]} oracle {b[c, f]}"


@pytest.mark.parametrize("alpha", [0.0, 0.6, 1.0])
@pytest.mark.parametrize("eps", [1e-4, 0.05, 1.0, 50.0])
@pytest.mark.parametrize("trunc,m", [(T.TRUNC_FIXED, 1), (T.TRUNC_FIXED, 4), (T.TRUNC_RAD, 2), (T.TRUNC_UNLIMITED, 2)])
def test_collide_parity(alpha, eps, trunc, m):
    v, cs = cells(COUNTS, seed=int(100 * alpha) + int(1000 * eps) + m)
    p = T.collide_params(dt=0.05, eps=eps, alpha=alpha, rho_scale=1.0 / 500, trunc=trunc, m=m)
    ms = np.full(len(COUNTS), m, np.int32) if trunc == T.TRUNC_RAD else None
    compare(v, cs, p, step=7, m_state=ms)


@pytest.mark.parametrize("length", [T.LEN_K, T.LEN_MIN, T.LEN_MEAN])
@pytest.mark.parametrize("m_max", [0, 1, 2, 5])
@pytest.mark.parametrize("alpha,eps", [(0.0, 1e-3), (1.0, 0.05), (0.6, 1.0), (1.0, 1e-4)])
def test_collide_parity_wb(length, m_max, alpha, eps):
    """TRMC-WB (Sec. 4.4): same tree lengths, same rejected outputs, same
    extended thermalised set as the oracle."""
    v, cs = cells(COUNTS, seed=40 + 7 * length + m_max)
    p = T.collide_params(dt=0.05, eps=eps, alpha=alpha, rho_scale=1.0 / 500, trunc=T.TRUNC_WB, m=m_max,
                         wb_length=length)
    g, vo, rep = compare(v, cs, p, step=5)
    if m_max == 0:      # every output is rejected but a lone one with no thermalised set
        lone = (rep[:, 5] - rep[:, 15] == 0) & (rep[:, 7] == 1)
        assert np.array_equal(rep[:, 15], np.where(lone, 0, rep[:, 7]))


# Cells too large for shared memory, at the default launch (128 x 4) and at
# 256 x 2, the shape of the large-cell workloads.
BIG_LAUNCH = [None, (256, 2)]


@pytest.mark.parametrize("launch", BIG_LAUNCH)
def test_collide_parity_wb_large_cells(launch):
    """Deep trees (q near 1/2 over many levels) in cells that run from the
    overflow slab; enough rejections under every definition."""
    counts = [20000, 9000, 30000]
    v, cs = cells(counts, seed=44)
    for length, m_max in ((T.LEN_MIN, 2), (T.LEN_MEAN, 2), (T.LEN_K, 3)):
        p = T.collide_params(dt=0.7, eps=1.0, alpha=0.0, rho_scale=1.0 / np.array(counts).mean(), trunc=T.TRUNC_WB,
                             m=m_max, wb_length=length)
        g, vo, rep = compare(v, cs, p, step=2, workspace=512 << 20, launch=launch)
        assert rep[:, 15].sum() > 50


def test_collide_parity_rad_continuations():
    # far from equilibrium and a long step: several TRMC-RAD passes per cell
    v, cs = cells([300, 1200, 3000], seed=3)
    p = T.collide_params(dt=2.0, eps=1.0, alpha=0.0, rho_scale=1.0 / 1000, trunc=T.TRUNC_RAD, m=1,
                         indicator=T.IND_PXX)
    g, vo, rep = compare(v, cs, p, step=1, m_state=np.ones(3, np.int32))
    assert rep[:, 1].max() >= 2, "expected at least one continuation pass"


@pytest.mark.parametrize("launch", BIG_LAUNCH)
def test_collide_parity_bkw_m4_indicator(launch):
    v, cs = cells([5000, 20000], seed=4, kind="bkw")
    p = T.collide_params(dt=0.05, eps=1.0, alpha=0.0, rho_scale=1.0 / 20000, trunc=T.TRUNC_RAD, m=2,
                         indicator=T.IND_M4)
    ms = np.array([2, 4], np.int32)
    for step in range(3):
        g, v, rep = compare(v, cs, p, step=step, m_state=ms, launch=launch)
        ms = g["m_state"]


@pytest.mark.parametrize("launch", BIG_LAUNCH)
def test_collide_parity_single_cell_1e5(launch):
    """The homogeneous single-cell workload size (N = 1e5, BKW data): the
    cell does not fit in shared memory; its changed particles are staged
    compact and the rest stays in global memory."""
    v, cs = cells([100000], seed=5, kind="bkw")
    p = T.collide_params(dt=0.05, eps=1.0, alpha=0.0, rho_scale=1e-5, trunc=T.TRUNC_RAD, m=2, indicator=T.IND_M4)
    compare(v, cs, p, step=0, m_state=np.array([2], np.int32), launch=launch)


@pytest.mark.parametrize("launch", BIG_LAUNCH)
@pytest.mark.parametrize("alpha,ind", [(1.0, T.IND_PXX), (0.6, T.IND_M4)])
def test_collide_parity_large_cells_vhs(launch, alpha, ind):
    """Cells too large for shared memory with the VHS bound and the P_xx
    indicator (a second pass over the cell), next to small cells staged
    whole, at every alignment of a cell's first and last particle against
    16 bytes."""
    counts = [13001, 7, 24577, 30002, 8195, 3, 41003]
    v, cs = cells(counts, seed=12)
    p = T.collide_params(dt=0.05, eps=0.02, alpha=alpha, rho_scale=1.0 / 20000, trunc=T.TRUNC_RAD, m=2,
                         indicator=ind)
    compare(v, cs, p, step=4, m_state=np.full(len(counts), 2, np.int32), workspace=512 << 20, launch=launch)


def test_collide_per_cell_params_and_keys():
    counts = [64, 500, 3000, 8192]
    v, cs = cells(counts, seed=6)
    g = synth.rng(7)
    eps = synth.loguniform(len(counts), 1e-4, 10, g=g)
    cp = np.stack([eps, np.full(4, 0.05), 1.0 / np.array(counts, float), np.full(4, 0.6)], axis=1)
    keys = np.array([(11 << 32) | 0, (12 << 32) | 0, (13 << 32) | 0, (14 << 32) | 0], np.uint64)
    p = T.collide_params(trunc=T.TRUNC_RAD, m=2)
    compare(v, cs, p, step=3, m_state=np.full(4, 2, np.int32), cell_param=cp, cell_key=keys)


def test_collide_deterministic_and_batch_independent():
    need_gpu()
    counts = [700, 40, 2000]
    v, cs = cells(counts, seed=8)
    keys = np.array([(5 << 32) | 3, (6 << 32) | 1, (7 << 32) | 9], np.uint64)
    p = T.collide_params(dt=0.3, eps=0.5, alpha=1.0, rho_scale=1e-3, trunc=T.TRUNC_FIXED, m=3)
    a = gpu_collide(v, cs, p, 2, cell_key=keys)
    b = gpu_collide(v, cs, p, 2, cell_key=keys)
    assert np.array_equal(a["v"], b["v"]) and np.array_equal(a["report"], b["report"])
    alone = gpu_collide(v[:, cs[1]:cs[2]], [0, counts[1]], p, 2, cell_key=keys[1:2])
    assert np.array_equal(alone["v"], a["v"][:, cs[1]:cs[2]])


def test_conservation_fp64():
    need_gpu()
    v, cs = cells(COUNTS, seed=9)
    p = T.collide_params(dt=0.05, eps=0.01, alpha=1.0, rho_scale=1.0 / 500, trunc=T.TRUNC_RAD, m=2)
    g = gpu_collide(v, cs, p, 0, m_state=np.full(len(COUNTS), 2, np.int32))
    for c in range(len(COUNTS)):
        a, b = cs[c], cs[c + 1]
        scale = np.abs(v[:, a:b]).sum()
        assert np.all(np.abs(g["v"][:, a:b].sum(1) - v[:, a:b].sum(1)) <= 1e-12 * scale)
        e0 = (v[:, a:b] ** 2).sum()
        assert abs((g["v"][:, a:b] ** 2).sum() - e0) <= 1e-12 * e0


def test_capacity_error_is_reported_and_cell_left_unchanged():
    need_gpu()
    v, cs = cells([20000], seed=10)
    p = T.collide_params(dt=0.05, eps=1.0, rho_scale=1e-4, trunc=T.TRUNC_FIXED, m=2)
    c = ctx(T.FP64, 0, 64 << 10)                     # 64 KiB workspace cannot hold 20000 FP64 particles
    st = T.ParticleState(cs, precision=T.FP64)
    st.set_velocities(v)
    T.trmc_collide(c, st, p, 0)
    with pytest.raises(T.TrmcError) as e:
        T.trmc_check(c)
    assert e.value.code == T.ERR_CAPACITY
    assert np.array_equal(st.v.cpu().numpy(), v)
    T.trmc_check(c)                                  # cleared


def test_argument_errors():
    need_gpu()
    c = ctx()
    st = T.ParticleState([0, 10], precision=T.FP64)
    for bad in (T.collide_params(m=0), T.collide_params(trunc=7), T.collide_params(eps=0.0),
                T.collide_params(m_cap=65), T.collide_params(trunc=T.TRUNC_RAD)):
        with pytest.raises(T.TrmcError) as e:
            T.trmc_collide(c, st, bad, 0)
        assert e.value.code == T.ERR_ARG


# ---------------------------------------------------------------- transport / sort
def tube_state(n_cells, mean, seed, ntubes=1):
    g = synth.rng(seed)
    counts = np.concatenate([synth.shock_tube_counts(n_cells, mean)] * ntubes)
    cs = synth.starts(counts)
    x = np.concatenate([(c % n_cells + g.random(k)) / n_cells for c, k in enumerate(counts)])
    v = synth.maxwellian(int(cs[-1]), g=g)
    doms = [(t * n_cells, n_cells, 0.0, 1.0) for t in range(ntubes)]
    return x, v, cs, doms


def gpu_transport(x, v, cs, doms, dt=None, cfl=0.0, vmax2=None):
    st = T.ParticleState(cs, precision=T.FP64, with_x=True)
    st.set_velocities(v)
    st.set_positions(x)
    if vmax2 is not None:
        st.cell_vmax2.copy_(torch.as_tensor(vmax2))
    dd = T.domains_tensor(doms)
    dtt = torch.as_tensor(np.asarray(dt if dt is not None else np.zeros(len(doms)), np.float64)).cuda()
    c = ctx()
    T.trmc_transport(c, st, dd, len(doms), cfl, dtt)
    T.trmc_check(c)
    n = int(cs[-1])
    return st.x[:n].cpu().numpy(), st.v[:, :n].cpu().numpy(), st.cell_start.cpu().numpy(), dtt.cpu().numpy()


def test_transport_parity_bit_exact():
    need_gpu()
    x, v, cs, doms = tube_state(400, 500, seed=11, ntubes=2)
    dt = O.cfl_dt(v, cs, doms, 0.5)
    xg, vg, csg, _ = gpu_transport(x, v, cs, doms, dt=dt)
    xo, vo, cso = O.transport(x, v, cs, doms, dt)
    assert np.array_equal(csg, cso)
    assert np.array_equal(xg, xo)
    assert np.array_equal(vg, vo)


@pytest.mark.parametrize("n_cells,lo,hi", [(400, 0.0, 1.0), (7, 0.1, 0.83), (1000, -2.5, 3.0)])
def test_transport_parity_at_cell_faces(n_cells, lo, hi):
    """Positions on the cell faces and one ulp either side, where the cell
    index floor((x - lo) / dx) is decided by the last bit of the quotient."""
    need_gpu()
    dx = (hi - lo) / n_cells
    xs, cell = [], []
    for k in range(1, n_cells):
        for f in (lo + k * dx, lo + k * (hi - lo) / n_cells, lo + (k * dx + dx * 1e-17)):
            for y in (f, np.nextafter(f, -np.inf), np.nextafter(f, np.inf)):
                xs.append(y)
                cell.append(k - 1 if y < lo + k * dx else k)
    xs, cell = np.array(xs), np.array(cell)
    order = np.argsort(cell, kind="stable")
    xs, cell = xs[order], cell[order]
    counts = np.bincount(cell, minlength=n_cells)
    cs = synth.starts(counts)
    g = synth.rng(14)
    v = g.standard_normal((3, len(xs))) * 1e-3
    doms = [(0, n_cells, lo, hi)]
    for dt in (0.0, 1e-9):
        xg, vg, csg, _ = gpu_transport(xs, v, cs, doms, dt=[dt])
        xo, vo, cso = O.transport(xs, v, cs, doms, [dt])
        assert np.array_equal(csg, cso) and np.array_equal(xg, xo) and np.array_equal(vg, vo)


def test_transport_cfl_mode_matches_oracle_dt():
    need_gpu()
    x, v, cs, doms = tube_state(64, 300, seed=12, ntubes=3)
    mom = O.moments(v, cs)
    dto = O.cfl_dt(v, cs, doms, 0.5)
    xg, vg, csg, dtg = gpu_transport(x, v, cs, doms, cfl=0.5, vmax2=mom[:, 9])
    assert np.array_equal(dtg, dto)
    xo, vo, cso = O.transport(x, v, cs, doms, dto)
    assert np.array_equal(csg, cso) and np.array_equal(xg, xo) and np.array_equal(vg, vo)


def test_transport_rejects_moves_beyond_one_cell():
    need_gpu()
    x, v, cs, doms = tube_state(32, 50, seed=13)
    with pytest.raises(T.TrmcError) as e:
        gpu_transport(x, v, cs, doms, dt=[10.0])
    assert e.value.code == T.ERR_STATE


# ---------------------------------------------------------------- init / moments
def test_init_parity():
    need_gpu()
    counts = [1000, 3, 0, 2000, 500]
    cs = synth.starts(counts)
    ci = np.zeros((5, T.INIT_COLS))
    ci[0] = [T.INIT_MAXWELL, 0.5, -1, 0, 2.0, 0, 0, 0.0, 0.25]
    ci[1] = [T.INIT_BIMAXWELL, 0, 0, 0, 2.5, 0.25, 0, 0.25, 0.5]
    ci[2] = [T.INIT_MAXWELL, 0, 0, 0, 1.0, 0, 0, 0.5, 0.75]
    ci[3] = [T.INIT_BKW, 0, 0, 0, 1.0, 0, 0.6, 0.75, 1.0]
    ci[4] = [T.INIT_BKW, 0.1, 0, 0, 1.0, 0, 0.8, 0.0, 1.0]
    st = T.ParticleState(cs, precision=T.FP64, with_x=True)
    c = T.trmc_create(T.FP64, 42, 1 << 20)
    T.trmc_init_cells(c, st, torch.as_tensor(ci).cuda())
    T.trmc_check(c)
    T.trmc_destroy(c)
    xo, vo = O.init_cells(ci, cs, 42)
    n = int(cs[-1])
    assert_velocity_parity(st.v[:, :n].cpu().numpy(), vo, cs)
    assert np.allclose(st.x[:n].cpu().numpy(), xo, rtol=0, atol=1e-14)
    mom = O.moments(vo, cs)
    assert np.allclose(st.cell_vmax2.cpu().numpy(), mom[:, 9], rtol=1e-12, atol=0)


def test_moments_parity():
    need_gpu()
    v, cs = cells(COUNTS + [0, 1], seed=14)
    st = T.ParticleState(cs, precision=T.FP64)
    st.set_velocities(v)
    out = torch.zeros((st.n_cells, T.MOM_COLS), dtype=torch.float64, device="cuda")
    T.trmc_moments(ctx(), st, out)
    mo = O.moments(v, cs)
    assert np.allclose(out.cpu().numpy(), mo, rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------- whole steps
def test_shock_tube_chain_parity():
    """Transport (CFL 0.5, specular walls) + sort + VHS hard-sphere collide
    for several steps on a 100-cell shock tube, GPU and oracle each running
    their own chain from the same initial state."""
    need_gpu()
    n_cells = 100
    counts = synth.shock_tube_counts(n_cells, 200)
    cs = synth.starts(counts)
    ci = np.zeros((n_cells, T.INIT_COLS))
    for c in range(n_cells):
        T_ = 1.0 if c < n_cells // 2 else 0.8
        ci[c] = [T.INIT_MAXWELL, 0, 0, 0, T_, 0, 0, c / n_cells, (c + 1) / n_cells]
    w = 0.5625 / cs[-1] * n_cells             # particle mass / cell width: rho_L = 1
    cp = np.tile([1e-2, 0.0, w, 1.0], (n_cells, 1))
    st = T.ParticleState(cs, precision=T.FP64, with_x=True, rad=True, cell_param=cp)
    c = T.trmc_create(T.FP64, 3, 64 << 20)
    T.trmc_init_cells(c, st, torch.as_tensor(ci).cuda())
    xo, vo = O.init_cells(ci, cs, 3)
    cso = cs.copy()
    mo = np.full(n_cells, 2, np.int32)
    doms = [(0, n_cells, 0.0, 1.0)]
    dd = T.domains_tensor(doms)
    dtt = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = T.collide_params(trunc=T.TRUNC_RAD, m=2)
    po = oracle_params(O, p)
    po.seed = 3
    for step in range(5):
        T.trmc_transport(c, st, dd, 1, 0.5, dtt)
        T.trmc_collide(c, st, p, step)
        T.trmc_check(c)
        dto = O.cfl_dt(vo, cso, doms, 0.5)
        xo, vo, cso = O.transport(xo, vo, cso, doms, dto)
        cpo = cp.copy(); cpo[:, 1] = dto[0]
        vo, _, mo = O.collide(vo, cso, po, step, m_state=mo, cell_param=cpo.ravel())
        n = int(cs[-1])
        assert abs(dtt.item() - dto[0]) <= 1e-14 * dto[0]
        assert np.array_equal(st.cell_start.cpu().numpy(), cso)
        assert np.allclose(st.x[:n].cpu().numpy(), xo, rtol=0, atol=1e-12)
        assert_velocity_parity(st.v[:, :n].cpu().numpy(), vo, cso, tol=1e-11)
        assert np.array_equal(st.m_max.cpu().numpy(), mo)
    T.trmc_destroy(c)


def test_collide_parity_deep_continuation_with_tiny_pool():
    """Deep trees (tau ~ 0.83) from m = 32: the TRMC-RAD continuation to
    levels 33..64 works on a thermalised pool of a few particles, which
    cannot supply the leaves; the depth is lowered until the plan fits."""
    counts = [885, 916, 111, 3000]
    v, cs = cells(counts, seed=15)
    p = T.collide_params(dt=1.8, eps=1.0, alpha=0.0, rho_scale=0.0, trunc=T.TRUNC_RAD, m=32, indicator=T.IND_PXX)
    cp = np.stack([np.ones(4), np.full(4, 1.8), 1.0 / np.array(counts, float), np.zeros(4)], axis=1)
    g, vo, rep = compare(v, cs, p, step=2, m_state=np.full(4, 32, np.int32), cell_param=cp)
    assert rep[:, 1].max() >= 2 and rep[:, 11].sum() > 0, "expected continuations with depth reductions"


# ---------------------------------------------------------------- reservoirs
def shock_state(n_int, mean, seed):
    from paper_1009_2768_gb300.workloads import rankine_hugoniot
    left, right = rankine_hugoniot(3.0)
    dx = 1.0 / n_int
    mass = (0.5 * left[0] + 0.5 * right[0]) / (n_int * mean)
    nc = n_int + 2
    counts = np.array([int(round((left if (c - 0.5) * dx < 0.5 else right)[0] * dx / mass)) for c in range(nc)])
    cs = synth.starts(counts)
    ci = np.zeros((nc, T.INIT_COLS))
    for c in range(nc):
        rho, u, Tm = left if (c - 0.5) * dx < 0.5 else right
        ci[c] = [T.INIT_MAXWELL, u, 0, 0, Tm, 0, 0, (c - 1) * dx, c * dx]
    dom = (0, nc, 0.0, 1.0, T.BC_RESERVOIR, left, right, mass)
    return cs, ci, dom, mass


def test_reservoir_transport_parity():
    need_gpu()
    cs, ci, dom, mass = shock_state(40, 300, seed=16)
    xo0, vo0 = O.init_cells(ci, cs, 21)
    cap = int(cs[-1] * 1.5)
    st = T.ParticleState(cs, capacity=cap, precision=T.FP64, with_x=True)
    st.set_velocities(vo0)
    st.set_positions(xo0)
    c = T.trmc_create(T.FP64, 21, 1 << 20)
    dd = T.domains_tensor([dom])
    dt = O.cfl_dt(vo0, cs, [O.domain(*dom)], 0.5)
    dtt = torch.as_tensor(dt).cuda()
    T.trmc_transport(c, st, dd, 1, 0.0, dtt, 9)
    T.trmc_check(c)
    xo, vo, cso = O.transport(xo0, vo0, cs, [O.domain(*dom)], dt, step=9, seed=21, capacity=cap)
    n = int(cso[-1])
    assert np.array_equal(st.cell_start.cpu().numpy(), cso)
    assert np.array_equal(st.x[:n].cpu().numpy(), xo)
    g0, g1 = cso[1], cso[-2]                       # refilled ghosts: [0, g0) and [g1, n)
    vg = st.v[:, :n].cpu().numpy()
    assert np.array_equal(vg[:, g0:g1], vo[:, g0:g1])                       # moved particles: exact
    assert np.allclose(vg[:, :g0], vo[:, :g0], rtol=1e-12, atol=1e-12)      # Maxwellian draws: ulps
    assert np.allclose(vg[:, g1:], vo[:, g1:], rtol=1e-12, atol=1e-12)
    T.trmc_destroy(c)


def test_stationary_shock_keeps_rankine_hugoniot_end_states():
    """Mach 3 stationary shock (Sec. 5.2): after 300 steps the upstream and
    downstream thirds still carry the Rankine-Hugoniot states (density ratio
    3, temperature ratio 11/3, velocity ratio 1/3)."""
    need_gpu()
    from paper_1009_2768_gb300.workloads import StationaryShock
    sim = StationaryShock(n_cells=200, mean_per_cell=400, eps=1e-3, precision=T.FP32_MIXED, seed=2)
    for _ in range(300):
        sim.step()
    T.trmc_check(sim.ctx)
    mom = torch.zeros((sim.state.n_cells, T.MOM_COLS), dtype=torch.float64, device="cuda")
    T.trmc_moments(sim.ctx, sim.state, mom)
    m = mom.cpu().numpy()[1:-1]
    up, down = m[10:60], m[140:190]
    (rl, ul, tl), (rr, ur, tr) = sim.left, sim.right
    assert abs(rr / rl - 3.0) < 1e-12 and abs(tr / tl - 11.0 / 3.0) < 1e-12 and abs(ur / ul - 1.0 / 3.0) < 1e-12
    assert abs(up[:, 1].mean() / rl - 1) < 0.03 and abs(down[:, 1].mean() / rr - 1) < 0.03
    assert abs(up[:, 5].mean() / tl - 1) < 0.03 and abs(down[:, 5].mean() / tr - 1) < 0.03
    assert abs(up[:, 2].mean() / ul - 1) < 0.03 and abs(down[:, 2].mean() / ur - 1) < 0.05
    sim.close()
