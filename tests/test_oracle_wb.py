"""Pins of the oracle's shape-dependent truncation TRMC-WB (Sec. 4.4):

* Table 1: the lengths of the paper's two example trees under the three
  definitions (Eqs. def:1-3), through the list encoding of Algorithm 4.5;
* with L = k (Eq. def:1) the rejected outputs are exactly those of the
  levels above m_max, and the one-step relaxation factor is the one of the
  fixed truncation at m = m_max (the two are the same truncation);
* with L = 1 + min / 1 + mean the number of rejected outputs per level
  follows the length law of Algorithm 4.1's recursive trees (root label
  uniform, subtrees independent), computed exactly by recursion;
* m_max = 0 thermalises every output; conservation holds in every mode.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_1009_2768_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_tree_lengths.txt")


def golden():
    lengths, trees = {}, {}
    for line in open(GOLDEN):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "lengths":
            lengths[f[1]] = [Fraction(x) for x in f[2:5]]
        elif f[0] == "tree":
            trees[f[1]] = [int(x) for x in f[2:]]
    return lengths, trees


def test_table1_tree_lengths():
    lengths, trees = golden()
    assert set(lengths) == set(trees) == {"left", "right"}
    for name in ("left", "right"):
        got = [O.tree_length(trees[name], d) for d in (O.LEN_K, O.LEN_MIN, O.LEN_MEAN)]
        assert got == [float(x) for x in lengths[name]], (name, got, lengths[name])


def test_tree_length_small_cases_and_malformed_lists():
    assert O.tree_length([0], O.LEN_MIN) == 0.0                  # a sample of f_0
    assert O.tree_length([1, 0, 0], O.LEN_MEAN) == 1.0
    assert O.tree_length([2, 1, 0, 0, 0], O.LEN_MEAN) == 1.5     # 1 + (1 + 0) / 2
    assert O.tree_length([2, 0, 1, 0, 0], O.LEN_MIN) == 1.0
    for bad in ([2, 1, 1, 0, 0], [1, 0], [3, 1, 1, 0, 0, 0, 0, 5], [-1]):
        with pytest.raises(ValueError):
            O.tree_length(bad, O.LEN_K)


# ---------------------------------------------------------------- the law of the lengths
def tail_min(n_max, m_max):
    """P(L_n > m_max) for L = 1 + min over Algorithm 4.1's random trees of
    n collisions: L_n > m iff both subtrees have L > m - 1."""
    P = {}

    def p(n, m):
        if (n, m) in P:
            return P[(n, m)]
        if n == 0:
            r = Fraction(1) if m < 0 else Fraction(0)
        else:
            r = sum(p(j, m - 1) * p(n - 1 - j, m - 1) for j in range(n)) / n
        P[(n, m)] = r
        return r
    return [float(p(n, m_max)) for n in range(n_max + 1)]


def tail_mean(n_max, m_max):
    dist = [{Fraction(0): Fraction(1)}]
    for n in range(1, n_max + 1):
        d = {}
        for j in range(n):
            for a, pa in dist[j].items():
                for b, pb in dist[n - 1 - j].items():
                    v = 1 + (a + b) / 2
                    d[v] = d.get(v, 0) + pa * pb / n
        dist.append(d)
    return [float(sum(p for v, p in d.items() if v > m_max)) for d in dist]


def outputs_per_level(rep):
    r = O.report_dict(rep)
    return np.array([2 * r["Ck"][n] - r["Dk"][n] for n in range(O.MCAP + 2)], np.int64)


def wb_run(length, m_max, q=0.6, n_cells=12, N=20000, seed=3, alpha=0.0):
    g = synth.rng(seed)
    v = np.concatenate([synth.bimaxwellian(N, 2.0, 0.5, g=g) for _ in range(n_cells)], axis=1)
    cs = synth.starts([N] * n_cells)
    dt = -np.log(q)                       # Maxwell molecules, rho = 1: q = exp(-dt / eps) with eps = 1
    prm = O.collide_params(dt=dt, eps=1.0, alpha=alpha, rho_scale=1.0 / N, trunc=O.TRUNC_WB, m=m_max,
                           wb_length=length)
    vn, rep, _ = O.collide(v, cs, prm, 1, threads=4)
    return v, vn, cs, rep


def test_wb_k_rejects_exactly_the_levels_above_m_max():
    for m_max in (1, 2, 4):
        _, _, _, rep = wb_run(O.LEN_K, m_max, n_cells=6, N=5000, seed=m_max)
        for row in rep:
            r = O.report_dict(row)
            out = outputs_per_level(row)
            assert r["passes"] == 1 and r["m_eff0"] > m_max
            assert r["wbrej"] == out[m_max + 1:].sum(), (m_max, r["wbrej"], out)


@pytest.mark.parametrize("length,m_max", [(O.LEN_MIN, 1), (O.LEN_MIN, 2), (O.LEN_MEAN, 2), (O.LEN_MEAN, 3)])
def test_wb_rejections_follow_the_tree_length_law(length, m_max):
    _, _, _, rep = wb_run(length, m_max, q=0.45 if length == O.LEN_MIN else 0.5, seed=10 + m_max)
    out = sum(outputs_per_level(row) for row in rep)
    top = int(np.nonzero(out)[0].max())
    assert top <= (40 if length == O.LEN_MIN else 21)
    tail = (tail_min if length == O.LEN_MIN else tail_mean)(top, m_max)
    expect = sum(out[n] * tail[n] for n in range(1, top + 1))
    var = sum(2 * out[n] * tail[n] * (1 - tail[n]) for n in range(1, top + 1))   # x2: paired products
    got = sum(O.report_dict(row)["wbrej"] for row in rep)
    assert expect > 100
    assert abs(got - expect) <= 5 * np.sqrt(var), (got, expect, np.sqrt(var))
    if length == O.LEN_MIN and m_max == 1:
        # closed form: L > 1 iff both subtrees are non-empty, probability (n - 2) / n
        assert np.allclose(tail[3:], [(n - 2) / n for n in range(3, top + 1)])


def test_wb_m_max_zero_thermalises_every_output():
    v, vn, cs, rep = wb_run(O.LEN_MIN, 0, n_cells=4, N=3000, seed=7)
    for c, row in enumerate(rep):
        r = O.report_dict(row)
        assert r["wbrej"] == r["leaves"] and r["R_final"] == r["N"] - r["N0"]


@pytest.mark.parametrize("length", [O.LEN_K, O.LEN_MIN, O.LEN_MEAN])
@pytest.mark.parametrize("alpha", [0.0, 1.0])
def test_wb_conservation(length, alpha):
    g = synth.rng(20 + length)
    counts = [2, 3, 5, 17, 64, 400, 2500]
    v = np.concatenate([synth.bimaxwellian(n, 2.0, 0.5, u=(0.3, -0.1, 0.2), g=g) for n in counts], axis=1)
    cs = synth.starts(counts)
    for eps in (1e-3, 0.05, 1.0):
        prm = O.collide_params(dt=0.05, eps=eps, alpha=alpha, rho_scale=1.0 / 500, trunc=O.TRUNC_WB, m=2,
                               wb_length=length)
        vn, rep, _ = O.collide(v, cs, prm, 2)
        for c in range(len(counts)):
            a, b = cs[c], cs[c + 1]
            scale = np.abs(v[:, a:b]).sum()
            assert np.all(np.abs(vn[:, a:b].sum(1) - v[:, a:b].sum(1)) <= 1e-12 * scale)
            e0 = (v[:, a:b] ** 2).sum()
            assert abs((vn[:, a:b] ** 2).sum() - e0) <= 1e-12 * e0
            r = O.report_dict(rep[c])
            assert r["N0"] + r["leaves"] + r["R_final"] - r["wbrej"] == counts[c]


def test_wb_k_has_the_fixed_truncation_factor():
    """TRMC-WB with L = k and m_max = m relaxes P_xx - T by the factor of the
    fixed truncation at m (the levels above m are thermalised in both)."""
    N, runs, m = 100000, 24, 2
    q = np.exp(-1.0)
    v0 = synth.bimaxwellian(N, 2.0, 0.5, g=synth.rng(6))

    def aniso(v):
        d = v - v.mean(1, keepdims=True)
        T = (d ** 2).sum(0).mean() / 3.0
        return ((d[0] ** 2).mean() - T) / T
    a0 = aniso(v0)
    prm = O.collide_params(dt=1.0, eps=1.0, alpha=0.0, rho_scale=1.0 / N, trunc=O.TRUNC_WB, m=m, wb_length=O.LEN_K)
    r = np.array([aniso(O.collide(v0, [0, N], prm, s)[0]) / a0 for s in range(runs)])
    tau = 1 - q
    G = q * sum(np.prod([(0.5 + j) / (j + 1) for j in range(k)]) * tau ** k for k in range(m + 1))
    se = r.std(ddof=1) / np.sqrt(runs)
    assert abs(r.mean() - G) <= 4 * se + 0.003, (r.mean(), G, se)
