"""Pins of the oracle's collision step against what the paper and the
mathematics fix, independent of the oracle's own code:

* exact conservation of mass, momentum and energy (Sec. 3.2 (i), Sec. 4.2);
* level occupation E[N_k] = N q tau^k, E[N_{m+1}] = N tau^{m+1} (Eq. WST,
  Alg. 4.2) and the exact distribution of the split for tiny N (brute force);
* the one-step relaxation factor of M_4 - 15 and of P_xx - T for Maxwell
  molecules: q * sum_{k<=m} (a)_k / k! * tau^k with a = 2/3 resp. 1/2, which
  follows from Eq. CF-r and the collision map (Eq. Maxwell_coll); it tends
  to exp(-dt/(3 eps)) resp. exp(-dt/(2 eps)) as m grows;
* the BKW closed-form M_4(t) for Maxwell molecules;
* the Maxwellian limit eps -> 0 (Eq. as_pres) and the Bird-like limit at
  large eps (expected collisions N mu dt / (2 eps));
* adaptive truncation (Sec. 4.3) rules and determinism.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O
from paper_1009_2768_gb300 import synth


def run(v, prm, step=0, m_state=None, cell_start=None):
    cs = cell_start if cell_start is not None else [0, v.shape[1]]
    return O.collide(v, cs, prm, step, m_state=m_state)


def central_m4(v):
    u = v.mean(1, keepdims=True)
    d = v - u
    T = (d ** 2).sum(0).mean() / 3.0
    return ((d ** 2).sum(0) ** 2).mean() / T ** 2


def aniso(v):
    u = v.mean(1, keepdims=True)
    d = v - u
    T = (d ** 2).sum(0).mean() / 3.0
    return ((d[0] ** 2).mean() - T) / T


def rising(a, k):
    r = 1.0
    for j in range(k):
        r *= (a + j) / (j + 1)
    return r


def factor(a, q, m):
    tau = 1.0 - q
    return q * sum(rising(a, k) * tau ** k for k in range(m + 1))


# ---------------------------------------------------------------- conservation
@pytest.mark.parametrize("alpha", [0.0, 0.6, 1.0])
@pytest.mark.parametrize("eps", [1e-4, 0.05, 1.0, 50.0])
@pytest.mark.parametrize("trunc,m", [(O.TRUNC_FIXED, 1), (O.TRUNC_FIXED, 3), (O.TRUNC_RAD, 2), (O.TRUNC_UNLIMITED, 0)])
def test_conservation(alpha, eps, trunc, m):
    g = synth.rng(int(1000 * eps) + int(10 * alpha) + m)
    counts = [2, 3, 5, 17, 64, 400, 2500]
    v = np.concatenate([synth.bimaxwellian(n, 2.0, 0.5, u=(0.3, -0.1, 0.2), g=g) for n in counts], axis=1)
    cs = synth.starts(counts)
    prm = O.collide_params(dt=0.05, eps=eps, alpha=alpha, rho_scale=1.0 / 500, trunc=trunc, m=max(m, 1),
                           indicator=O.IND_PXX)
    ms = np.full(len(counts), 2, np.int32)
    vn, rep, _ = O.collide(v, cs, prm, 3, m_state=ms)
    for c in range(len(counts)):
        a, b = cs[c], cs[c + 1]
        p0, p1 = v[:, a:b].sum(1), vn[:, a:b].sum(1)
        e0, e1 = (v[:, a:b] ** 2).sum(), (vn[:, a:b] ** 2).sum()
        scale = np.abs(v[:, a:b]).sum()
        assert np.all(np.abs(p1 - p0) <= 1e-12 * scale), (c, p0, p1)
        assert abs(e1 - e0) <= 1e-12 * e0, (c, e0, e1)
        r = O.report_dict(rep[c])
        # every particle has exactly one role: uncollided, leaf, thermalised
        assert r["N0"] + r["leaves"] + r["R_final"] == counts[c]
    assert np.all(np.isfinite(vn))


def test_tiny_cells_and_zero_dt_unchanged():
    v = synth.maxwellian(1, g=synth.rng(1))
    prm = O.collide_params(dt=0.05, eps=0.01, alpha=1.0, rho_scale=1.0)
    vn, rep, _ = run(v, prm)
    assert np.array_equal(vn, v)
    v = synth.maxwellian(300, g=synth.rng(2))
    prm = O.collide_params(dt=0.0, eps=1.0, alpha=0.0, rho_scale=1.0)
    vn, rep, _ = run(v, prm)
    assert np.array_equal(vn, v)          # q = 1: nobody collides
    assert O.report_dict(rep[0])["N0"] == 300


# ---------------------------------------------------------------- level occupation
def test_level_occupation_expectation():
    N, eps, m = 3000, 1.0, 3
    q = np.exp(-1.0 * 0.5 / eps)          # mu = rho = 1 (rho_scale = 1/N), dt = 0.5
    tau = 1 - q
    prm = O.collide_params(dt=0.5, eps=eps, alpha=0.0, rho_scale=1.0 / N, trunc=O.TRUNC_FIXED, m=m)
    v = synth.maxwellian(N, g=synth.rng(3))
    nk = []
    for s in range(400):
        _, rep, _ = run(v, prm, step=s)
        nk.append(O.report_dict(rep[0])["Nk"][:m + 2])
    nk = np.array(nk, dtype=float)
    expect = np.array([N * q * tau ** k for k in range(m + 1)] + [N * tau ** (m + 1)])
    se = nk.std(0, ddof=1) / np.sqrt(len(nk))
    assert np.all(np.abs(nk.mean(0) - expect) <= 4 * se + 1e-9), (nk.mean(0), expect, se)


def split_distribution(N, q, m):
    """Exact law of (N_0..N_m, N_{m+1}) under Alg. 4.2 with Iround."""
    q = Fraction(q)
    dist = {}

    def rec(n, rem, acc, p):
        if n > m:
            key = tuple(acc) + (rem,)
            dist[key] = dist.get(key, 0) + p
            return
        x = q * rem
        fl = x.numerator // x.denominator
        frac = x - fl
        for cnt, pc in ((fl, 1 - frac), (fl + 1, frac)):
            if pc == 0:
                continue
            nrem = rem - cnt
            if nrem == 0:
                key = tuple(acc + [cnt]) + (0,) * (m - n) + (0,)
                dist[key] = dist.get(key, 0) + p * pc
            else:
                rec(n + 1, nrem, acc + [cnt], p * pc)

    rec(0, N, [], Fraction(1))
    return dist


@pytest.mark.parametrize("N,m", [(3, 2), (5, 3), (6, 2)])
def test_split_brute_force(N, m):
    dt = 0.7
    q = float(np.exp(-dt))             # eps = 1, mu = 1
    exact = split_distribution(N, q, m)
    prm = O.collide_params(dt=dt, eps=1.0, alpha=0.0, rho_scale=1.0 / N, trunc=O.TRUNC_FIXED, m=m)
    v = synth.maxwellian(N, g=synth.rng(4))
    hist = {}
    S = 6000
    for s in range(S):
        _, rep, _ = run(v, prm, step=s)
        key = tuple(int(x) for x in O.report_dict(rep[0])["Nk"][:m + 2])
        hist[key] = hist.get(key, 0) + 1
    assert set(hist) <= set(exact), set(hist) - set(exact)
    keys = sorted(exact)
    obs = np.array([hist.get(k, 0) for k in keys], float)
    exp = np.array([float(exact[k]) * S for k in keys])
    keep = exp >= 5
    obs_k = np.append(obs[keep], obs[~keep].sum())
    exp_k = np.append(exp[keep], exp[~keep].sum())
    if exp_k[-1] == 0:
        obs_k, exp_k = obs_k[:-1], exp_k[:-1]
    assert stats.chisquare(obs_k, exp_k).pvalue > 1e-4


# ---------------------------------------------------------------- relaxation factors
@pytest.mark.parametrize("m", [1, 2, 4])
def test_m4_step_factor_maxwell(m):
    N, runs = 100000, 40
    q = np.exp(-1.0)                       # dt / eps = 1, mu = 1
    v0 = synth.bkw(N, K=0.6, g=synth.rng(5))
    a0 = central_m4(v0) - 15.0
    prm = O.collide_params(dt=1.0, eps=1.0, alpha=0.0, rho_scale=1.0 / N, trunc=O.TRUNC_FIXED, m=m)
    r = []
    for s in range(runs):
        vn, _, _ = run(v0, prm, step=s)
        r.append((central_m4(vn) - 15.0) / a0)
    r = np.array(r)
    F = factor(2.0 / 3.0, q, m)
    se = r.std(ddof=1) / np.sqrt(runs)
    assert abs(r.mean() - F) <= 4 * se + 0.004, (m, r.mean(), F, se)
    # and it is clearly not the next truncation order
    assert abs(factor(2.0 / 3.0, q, m + 1) - F) > 3 * se


@pytest.mark.parametrize("m", [1, 3])
def test_anisotropy_step_factor_maxwell(m):
    N, runs = 100000, 30
    q = np.exp(-1.0)
    v0 = synth.bimaxwellian(N, 2.0, 0.5, g=synth.rng(6))
    a0 = aniso(v0)
    prm = O.collide_params(dt=1.0, eps=1.0, alpha=0.0, rho_scale=1.0 / N, trunc=O.TRUNC_FIXED, m=m)
    r = np.array([aniso(run(v0, prm, step=s)[0]) / a0 for s in range(runs)])
    G = factor(0.5, q, m)
    se = r.std(ddof=1) / np.sqrt(runs)
    assert abs(r.mean() - G) <= 4 * se + 0.003, (m, r.mean(), G, se)


def test_factor_limit_is_exact_exponential():
    # the truncated Wild sum has no time-discretisation error as m grows
    for dt in (0.05, 1.0):
        q = np.exp(-dt)
        assert abs(factor(2.0 / 3.0, q, 400) - np.exp(-dt / 3)) < 1e-12
        assert abs(factor(0.5, q, 400) - np.exp(-dt / 2)) < 1e-12


@pytest.mark.slow
def test_bkw_m4_trajectory():
    """Maxwell molecules from BKW data (K0 = 0.6): M_4(t) - 15 =
    (M_4(0) - 15) exp(-t/3) with eps = 1 (unit collision rate)."""
    N, seeds, dt, eps = 50000, 4, 0.05, 1.0
    checkpoints = {20: 1.0, 40: 2.0, 100: 5.0, 200: 10.0}
    err = {t: [] for t in checkpoints.values()}
    for sd in range(seeds):
        v = synth.bkw(N, K=0.6, g=synth.rng(100 + sd))
        a0 = central_m4(v) - 15.0
        ms = np.array([2], np.int32)
        prm = O.collide_params(dt=dt, eps=eps, alpha=0.0, rho_scale=1.0 / N, trunc=O.TRUNC_RAD, m=2,
                               indicator=O.IND_M4, seed=sd)
        for s in range(1, 201):
            v, _, ms = run(v, prm, step=s, m_state=ms)
            if s in checkpoints:
                t = checkpoints[s]
                err[t].append((central_m4(v) - 15.0) - a0 * np.exp(-t / 3.0))
    sigma = np.sqrt(720.0 / N) / np.sqrt(seeds)       # Var |v|^4 = 945 - 225 for a Maxwellian
    for t, e in err.items():
        assert abs(np.mean(e)) <= 3 * sigma + 0.03, (t, np.mean(e), sigma)


# ---------------------------------------------------------------- limits
def test_maxwellian_limit():
    N = 20000
    v = synth.bimaxwellian(N, 3.0, 0.3, u=(1.0, 0.5, -0.5), g=synth.rng(7))
    prm = O.collide_params(dt=0.05, eps=1e-9, alpha=1.0, rho_scale=1.0 / N, trunc=O.TRUNC_FIXED, m=4)
    vn, rep, _ = run(v, prm)
    r = O.report_dict(rep[0])
    assert r["N0"] == 0 and r["leaves"] == 0 and r["R_final"] == N
    u = v.mean(1, keepdims=True)
    T = ((v - u) ** 2).sum(0).mean() / 3
    z = (vn - u) / np.sqrt(T)
    for comp in range(3):
        assert stats.kstest(z[comp], "norm").pvalue > 1e-4
    assert np.allclose(vn.mean(1), v.mean(1), atol=1e-13)


def test_bird_like_limit():
    N, eps, dt = 100000, 10.0, 0.05
    prm = O.collide_params(dt=dt, eps=eps, alpha=0.0, rho_scale=1.0 / N, trunc=O.TRUNC_FIXED, m=4)
    v = synth.maxwellian(N, g=synth.rng(8))
    coll = np.array([O.report_dict(run(v, prm, step=s)[1][0])["coll"] for s in range(200)], float)
    bird = N * 1.0 * dt / (2 * eps)          # expected DSMC collisions, mu = 1
    tau = 1 - np.exp(-dt / eps)
    se = coll.std(ddof=1) / np.sqrt(len(coll))
    assert abs(coll.mean() - bird) <= 4 * se + N * tau ** 2, (coll.mean(), bird)


# ---------------------------------------------------------------- adaptivity
def test_rad_rules():
    N = 20000
    # equilibrium: tiny relative change -> accept and halve m (Sec. 4.3)
    v = synth.maxwellian(N, g=synth.rng(9))
    prm = O.collide_params(dt=0.05, eps=1.0, alpha=0.0, rho_scale=1.0 / N, trunc=O.TRUNC_RAD,
                           indicator=O.IND_PXX)
    _, rep, ms = run(v, prm, m_state=np.array([8], np.int32))
    r = O.report_dict(rep[0])
    assert r["passes"] == 1 and r["m_next"] == 4 and ms[0] == 4
    _, rep, ms = run(v, prm, m_state=np.array([1], np.int32))
    assert ms[0] == 1                      # never below m_min
    # far from equilibrium with a large step: rejected, redone with 2m
    v = synth.bimaxwellian(N, 2.7, 0.15, g=synth.rng(10))
    prm = O.collide_params(dt=2.0, eps=1.0, alpha=0.0, rho_scale=1.0 / N, trunc=O.TRUNC_RAD,
                           indicator=O.IND_PXX)
    vn, rep, ms = run(v, prm, m_state=np.array([1], np.int32))
    r = O.report_dict(rep[0])
    assert r["passes"] >= 2 and r["m_last"] == 2 ** (r["passes"] - 1)
    assert abs((vn ** 2).sum() - (v ** 2).sum()) <= 1e-12 * (v ** 2).sum()
    # continuation keeps every level <= m of the first pass: same pass-0 quotas
    prm_fixed = O.collide_params(dt=2.0, eps=1.0, alpha=0.0, rho_scale=1.0 / N, trunc=O.TRUNC_FIXED, m=1)
    _, rep_f, _ = run(v, prm_fixed)
    assert np.array_equal(O.report_dict(rep_f[0])["Nk"], r["Nk"])


def test_determinism_and_batch_independence():
    g = synth.rng(11)
    counts = [100, 37, 900]
    v = np.concatenate([synth.bimaxwellian(n, 2.0, 0.5, g=g) for n in counts], axis=1)
    cs = synth.starts(counts)
    prm = O.collide_params(dt=0.3, eps=0.5, alpha=0.6, rho_scale=1.0 / 300, trunc=O.TRUNC_FIXED, m=3)
    keys = np.array([(7 << 32) | 0, (9 << 32) | 4, (3 << 32) | 2], np.uint64)
    a, ra, _ = O.collide(v, cs, prm, 5, cell_key=keys)
    b, rb, _ = O.collide(v, cs, prm, 5, cell_key=keys, threads=3)
    assert np.array_equal(a, b) and np.array_equal(ra, rb)
    # the middle cell alone gives the same result as inside the batch
    c, rc, _ = O.collide(v[:, cs[1]:cs[2]], [0, counts[1]], prm, 5, cell_key=keys[1:2])
    assert np.array_equal(c, a[:, cs[1]:cs[2]])


def test_tree_label_law():
    """Each level-n collision takes k uniform in {0..n-1} (Alg. 4.1/4.3) and
    needs one sample of f_k and one of f_{n-1-k}; the labels are drawn after
    C_n is fixed, so E[D_k] = E[sum_{n>k} 2 C_n / n] for every level k."""
    N, m, runs = 5000, 16, 300
    prm = O.collide_params(dt=3.0, eps=1.0, alpha=0.0, rho_scale=1.0 / N, trunc=O.TRUNC_FIXED, m=m)
    v = synth.maxwellian(N, g=synth.rng(12))
    diffs = []
    for s in range(runs):
        r = O.report_dict(run(v, prm, step=s)[1][0])
        assert r["feas"] == 0
        Ck, Dk = r["Ck"].astype(float), r["Dk"].astype(float)
        exp = np.array([sum(2.0 * Ck[n] / n for n in range(k + 1, m + 1)) for k in range(m)])
        diffs.append(Dk[:m] - exp)
    diffs = np.array(diffs)
    se = diffs.std(0, ddof=1) / np.sqrt(runs) + 1e-12
    assert np.all(np.abs(diffs.mean(0)) <= 4.5 * se), (diffs.mean(0), se)
