"""Pins of the oracle's free transport, cell sort, initial data and moments.

* transport: hand-worked positions, velocities and cells, including wall
  reflections; speeds, per-domain counts and energy are unchanged;
* the cell sort agrees with numpy's stable argsort (an independent sort);
* CFL: dt * max|v| = cfl * dx;
* initial data: Maxwellian (KS), bi-Maxwellian variances, BKW
  (|v|^2 / K ~ chi^2_5 at K = 0.6, M_4 = 15 K (2 - K)), uniform positions;
* moments: a hand-worked two- and four-particle cell.
"""
import numpy as np
from scipy import stats

from oracle import oracle as O
from paper_1009_2768_gb300 import synth


def test_transport_hand_example():
    # domain [0,1], 4 cells of width 0.25; dt = 1
    x = np.array([0.10, 0.30, 0.90, 0.60, 0.99])
    v = np.array([[-0.30, 0.05, 0.20, -0.40, 0.0],
                  [1.0, 2.0, 3.0, 4.0, 5.0],
                  [0.5, 0.5, 0.5, 0.5, 0.5]])
    # sorted by cell: cell 0: x=0.10; cell 1: 0.30; cell 2: 0.60; cell 3: 0.90, 0.99
    order = [0, 1, 3, 2, 4]
    x, v = x[order], v[:, order]
    cs = np.array([0, 1, 2, 3, 5])
    xo, vo, cso = O.transport(x, v, cs, [(0, 4, 0.0, 1.0)], [1.0])
    # hand results: 0.10-0.30 -> -0.20 -> 0.20 (vx +0.30, cell 0); 0.30+0.05=0.35 (cell 1);
    # 0.60-0.40=0.20 (cell 0); 0.90+0.20=1.10 -> 0.90 (vx -0.20, cell 3); 0.99 (cell 3)
    assert np.array_equal(cso, [0, 2, 3, 3, 5])
    assert np.allclose(xo, [0.20, 0.20, 0.35, 0.90, 0.99], atol=1e-15)
    assert np.allclose(vo[0], [0.30, -0.40, 0.05, -0.20, 0.0], atol=1e-15)
    assert np.array_equal(vo[1], [1.0, 4.0, 2.0, 3.0, 5.0])     # stable: old order within a cell


def test_transport_sort_matches_numpy_stable_sort():
    g = synth.rng(20)
    counts = synth.shock_tube_counts(64, 50)
    cs = synth.starts(counts)
    n = int(cs[-1])
    x = np.concatenate([(c + g.random(k)) / 64 for c, k in enumerate(counts)])
    v = synth.maxwellian(n, T=1.0, g=g)
    doms = [(0, 32, 0.0, 0.5), (32, 32, 0.5, 1.0)]       # two independent tubes
    dt = O.cfl_dt(v, cs, doms, 0.5)
    xo, vo, cso = O.transport(x, v, cs, doms, dt)
    # independent recomputation of the keys, then numpy's stable sort
    key = np.empty(n, np.int64)
    xn = x.copy(); vx = v[0].copy()
    for d, (cb, nc, lo, hi) in enumerate(doms):
        sl = slice(cs[cb], cs[cb + nc])
        xn[sl] = x[sl] + v[0][sl] * dt[d]
        left, right = xn[sl] < lo, xn[sl] > hi
        xs = xn[sl]; xs[left] = 2 * lo - xs[left]; xs[right] = 2 * hi - xs[right]; xn[sl] = xs
        vs = vx[sl]; vs[left | right] *= -1; vx[sl] = vs
        key[sl] = cb + np.clip(np.floor((xn[sl] - lo) / ((hi - lo) / nc)).astype(np.int64), 0, nc - 1)
    perm = np.argsort(key, kind="stable")
    assert np.array_equal(xo, xn[perm])
    assert np.array_equal(vo[0], vx[perm]) and np.array_equal(vo[1:], v[1:, perm])
    assert np.array_equal(cso, np.searchsorted(key[perm], np.arange(65), side="left"))
    # particles never leave their tube, speeds unchanged, energy unchanged
    assert cso[32] == cs[32]
    assert np.array_equal(np.sort((vo ** 2).sum(0)), np.sort((v ** 2).sum(0)))
    assert np.all((xo >= 0) & (xo <= 1))


def test_cfl_dt():
    g = synth.rng(21)
    v = synth.maxwellian(1000, g=g)
    dt = O.cfl_dt(v, [0, 500, 1000], [(0, 2, 0.0, 2.0)], 0.5)
    dx = 1.0
    assert abs(dt[0] * np.sqrt((v ** 2).sum(0).max()) - 0.5 * dx) < 1e-15


def _init(kind, n, cols, seed=1, cells=1):
    ci = np.zeros((cells, O.INIT_COLS))
    ci[:, 0] = kind
    for k, val in cols.items():
        ci[:, k] = val
    cs = synth.starts([n] * cells)
    return O.init_cells(ci, cs, seed)


def test_init_maxwellian():
    x, v = _init(O.INIT_MAXWELL, 40000, {1: 0.5, 2: -1.0, 3: 0.0, 4: 2.0, 7: 0.25, 8: 0.5})
    z = (v - np.array([[0.5], [-1.0], [0.0]])) / np.sqrt(2.0)
    for c in range(3):
        assert stats.kstest(z[c], "norm").pvalue > 1e-4
    assert np.all((x >= 0.25) & (x < 0.5))
    assert stats.kstest((x - 0.25) / 0.25, "uniform").pvalue > 1e-4


def test_init_bimaxwellian():
    x, v = _init(O.INIT_BIMAXWELL, 40000, {4: 2.5, 5: 0.25})
    for c, T in ((0, 2.5), (1, 0.25), (2, 0.25)):
        assert stats.kstest(v[c] / np.sqrt(T), "norm").pvalue > 1e-4


def test_init_bkw():
    K = 0.6
    x, v = _init(O.INIT_BKW, 60000, {6: K})
    s2 = (v ** 2).sum(0)
    assert stats.kstest(s2 / K, "chi2", args=(5,)).pvalue > 1e-4      # weight of chi_3 is 0 at K = 0.6
    M4 = (s2 ** 2).mean()
    se = (s2 ** 2).std() / np.sqrt(len(s2))
    assert abs(M4 - 15 * K * (2 - K)) < 4 * se
    x, v = _init(O.INIT_BKW, 60000, {6: 0.8}, seed=3)
    s2 = (v ** 2).sum(0)
    assert abs(s2.mean() - 3.0) < 4 * s2.std() / np.sqrt(len(s2))     # unit temperature
    M4 = (s2 ** 2).mean()
    assert abs(M4 - 15 * 0.8 * 1.2) < 4 * (s2 ** 2).std() / np.sqrt(len(s2))


def test_moments_hand_example():
    v = np.array([[1.0, -1.0, 2.0, 0.0, 0.0, 0.0],
                  [0.0, 0.0, 0.0, 0.0, 1.0, 1.0],
                  [0.0, 0.0, 0.0, 0.0, 0.0, 2.0]])
    m = O.moments(v, [0, 2, 6], rho_scale=[0.5, 0.25])
    # cell 0: v = (+-1,0,0): U = 0, |v-U|^2 = 1 each -> T = 1/3, Pxx = 1, M4 = 1, E = 1/2
    assert np.allclose(m[0], [2, 1.0, 0, 0, 0, 1 / 3, 1.0, 1.0, 0.5, 1.0])
    # cell 1: (2,0,0), (0,0,0), (0,1,0), (0,1,2): U = (1/2, 1/2, 1/2);
    # |v-U|^2 = 2.75, 0.75, 0.75, 2.75 -> T = 7/12; (v_x-U_x)^2 = 2.25, .25, .25, .25 -> Pxx = 3/4;
    # |v|^2 = 4, 0, 1, 5 -> M4 = 42/4, E = 10/8, max |v|^2 = 5
    assert np.allclose(m[1], [4, 1.0, 0.5, 0.5, 0.5, 7 / 12, 0.75, 10.5, 1.25, 5.0], rtol=1e-15, atol=0)


# ---------------------------------------------------------------- reservoirs
def res_domain(n_int, lo=0.0, hi=1.0, rlo=(1.0, 0.5, 1.0), rhi=(2.0, -0.3, 0.5), mass=1e-3):
    return O.domain(0, n_int + 2, lo, hi, O.BC_RESERVOIR, rlo, rhi, mass)


def test_reservoir_hand_example():
    # 2 interior cells on [0,1] (dx 0.5) + ghosts [-0.5,0) and [1,1.5); dt = 1
    d = res_domain(2, rlo=(0.0, 0.0, 1.0), rhi=(0.0, 0.0, 1.0), mass=1.0)    # empty reservoirs: no refill
    x = np.array([-0.2, -0.4, 0.1, 0.6, 0.9, 1.2])
    v = np.array([[0.3, 0.1, -0.2, 0.1, 0.2, -0.4], [1, 2, 3, 4, 5, 6], [0, 0, 0, 0, 0, 0.0]])
    cs = np.array([0, 2, 3, 5, 6])
    xo, vo, cso = O.transport(x, v, cs, [d], [1.0])
    # -0.2+0.3=0.1 enters cell 1; -0.4+0.1=-0.3 stays in the ghost: removed; 0.1-0.2=-0.1 leaves: removed;
    # 0.6+0.1=0.7 and 0.9+0.2=1.1 (leaves: removed); 1.2-0.4=0.8 enters cell 2
    assert np.array_equal(cso, [0, 0, 1, 3, 3])
    assert np.allclose(xo, [0.1, 0.7, 0.8], atol=1e-15)
    assert np.array_equal(vo[1], [1, 4, 6])


def test_reservoir_refill_counts_and_law():
    d = res_domain(4, rlo=(1.0, 0.5, 2.0), rhi=(3.0, -1.0, 0.5), mass=1e-4)   # dx 0.25: 2500 and 7500 expected
    cs = np.zeros(7, np.int64)
    xs, vs = [], []
    for step in range(40):
        xo, vo, cso = O.transport(np.zeros(0), np.zeros((3, 0)), cs, [d], [0.0], step=step, seed=3)
        g_lo, g_hi = cso[1] - cso[0], cso[6] - cso[5]
        assert abs(g_lo - 2500) <= 1 and abs(g_hi - 7500) <= 1      # Iround(rho dx / mass)
        assert np.all((xo[:g_lo] >= -0.25) & (xo[:g_lo] < 0.0)) and np.all((xo[g_lo:] >= 1.0) & (xo[g_lo:] < 1.25))
        xs.append(xo[:g_lo]); vs.append(vo[:, :g_lo])
    v = np.concatenate(vs, axis=1)
    assert stats.kstest((v[0] - 0.5) / np.sqrt(2.0), "norm").pvalue > 1e-4
    assert stats.kstest(v[1] / np.sqrt(2.0), "norm").pvalue > 1e-4
    assert stats.kstest((np.concatenate(xs) + 0.25) / 0.25, "uniform").pvalue > 1e-4


def test_reservoir_inflow_is_the_half_range_flux():
    """Particles entering from a reservoir (rho, u, T) per step: (rho/mass)
    dt E[max(v_x, 0)] with E[v_x^+] = u Phi(u/sqrt T) + sqrt T phi(u/sqrt T)
    (uniform positions in the ghost cell, v dt < dx)."""
    rho, u, T, mass, dt = 1.0, 0.4, 1.0, 2e-5, 0.01
    d = res_domain(4, rlo=(rho, u, T), rhi=(0.0, 0.0, 1.0), mass=mass)
    cs = np.zeros(7, np.int64)
    x, v, cs = O.transport(np.zeros(0), np.zeros((3, 0)), cs, [d], [0.0], step=0, seed=5)    # fill the ghost
    entered = []
    for step in range(1, 121):
        x2, v2, cs2 = O.transport(x, v, cs, [d], [dt], step=step, seed=5)
        entered.append(cs2[5] - cs2[1])          # interior particles now (the interior started empty)
        x, v, cs = x2[:cs2[1]], v2[:, :cs2[1]], np.array([0, cs2[1], cs2[1], cs2[1], cs2[1], cs2[1], cs2[1]])
    s = u / np.sqrt(T)
    flux = u * stats.norm.cdf(s) + np.sqrt(T) * stats.norm.pdf(s)
    expect = rho / mass * dt * flux
    e = np.array(entered, float)
    assert abs(e.mean() - expect) <= 4 * e.std(ddof=1) / np.sqrt(len(e)), (e.mean(), expect)
