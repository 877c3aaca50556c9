"""Pins of the oracle's tree plan (the level-synchronous reading of Alg. 4.3:
odd counts, labels, leaf feasibility) against an independent brute-force
enumeration and against the unbiasedness the Wild sum asks of it.

Alg. 4.3 leaves two choices open, and the oracle takes one reading of each:

* an odd number of wanted level-n samples (quota N_n plus demand D_n from
  the levels above) leaves one product of the last pair over: a fair coin
  either sends one quota particle of the level to the thermalised set or
  keeps the surplus product as an extra level-n output; with no quota
  particle at the level the surplus is kept;
* more leaves wanted than the non-uncollided particles can give (a tree is
  never longer than the cell, end of Sec. 4.1): the missing leaves are taken
  from level 0, and only if level 0 is too small is the top level dropped
  into the thermalised set and the plan redone.

Two kinds of pin:

1. For N <= 6 and m <= 3 every random decision of the split (Alg. 4.2,
   Iround), the parity coins and the labels k (Alg. 4.1, uniform in
   {0..n-1}) has finitely many outcomes.  `plan_law` below enumerates them
   all, exactly, in plain Python written from the reading (not from the C
   source): a coin or a label is drawn once per level and collision and
   keeps its value when the plan is redone at a smaller depth, because the
   draws are keyed by (level, collision).  The oracle's plan records over
   tens of thousands of independently keyed cells must follow that law (chi
   square), in cases where the coin, borrowing from level 0 and lowering the
   depth all carry real probability.
2. For cells of 2..17 particles at tau >= 0.5 the coin must leave every
   level's output count unbiased: E[out_n] = E[N_n] + P(N_n = 0 and D_n odd)
   for every level n the plan keeps, out_n = 2 C_n - D_n, because only the
   forced surplus of a level without quota moves the expectation.  With
   E[N_n] = N q tau^n (the split's law, Eq. WST) the outputs of level n then
   follow the Wild sum's coefficient up to that forced surplus.  An
   always-round-up or always-round-down rule fails this by about half the
   probability of an odd count.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O
from paper_1009_2768_gb300 import synth


class _Undecided(Exception):
    def __init__(self, key, outcomes):
        super().__init__(key)
        self.key, self.outcomes = key, outcomes


def _enumerate(trial):
    """Exact law of trial(draw): draw(key, outcomes) returns the value of the
    random variable `key` with law `outcomes` [(value, probability)]; each
    variable is decided once and keeps its value within a trial."""
    law = {}
    pending = [({}, Fraction(1))]
    while pending:
        fixed, p = pending.pop()

        def draw(key, outcomes, fixed=fixed):
            if key not in fixed:
                raise _Undecided(key, outcomes)
            return fixed[key]

        try:
            out = trial(draw)
        except _Undecided as u:
            for val, pv in u.outcomes:
                if pv > 0:
                    f = dict(fixed)
                    f[u.key] = val
                    pending.append((f, p * pv))
            continue
        law[out] = law.get(out, Fraction(0)) + p
    return law


def plan_trial(N, q, m):
    """One step's split and tree plan of a cell of N particles (pass 0,
    fixed order m) as a function of its random decisions; returns the plan
    record (quotas N_0..N_{m+1}, depth kept, uncollided count, collisions
    C_1..C_m, demand D_0..D_m)."""
    q = Fraction(q)

    def trial(draw):
        Nq = [0] * (m + 2)
        rem, m_eff = N, m
        for n in range(m + 1):                        # Alg. 4.2 with Iround
            x = q * rem
            fl = x.numerator // x.denominator
            fr = x - fl
            cnt = fl + (draw(("split", n), [(1, fr), (0, 1 - fr)]) if fr else 0)
            Nq[n] = cnt
            rem -= cnt
            if rem == 0:
                m_eff = n
                break
        else:
            Nq[m + 1] = rem
        top = m_eff
        while True:
            D = [0] * (m + 2)
            C = [0] * (m + 2)
            for n in range(top, 0, -1):                # top level first
                quota = Nq[n]
                T = quota + D[n]
                if T % 2:
                    if quota >= 1 and draw(("coin", n), [(True, Fraction(1, 2)), (False, Fraction(1, 2))]):
                        T -= 1                         # one quota particle joins the thermalised set
                    else:
                        T += 1                         # the surplus product is an extra output
                C[n] = T // 2
                for c in range(C[n]):                  # label k of collision c, uniform in {0..n-1}
                    k = 0 if n == 1 else draw(("label", n, c), [(j, Fraction(1, n)) for j in range(n)])
                    D[k] += 1
                    D[n - 1 - k] += 1
            n0, A = Nq[0], N - Nq[0]
            if D[0] <= A:
                break
            if D[0] - A <= n0:                         # borrow the missing leaves from level 0
                n0 -= D[0] - A
                break
            top -= 1                                   # level 0 too small: drop the top level
        return tuple(Nq), top, n0, tuple(C[1:m + 1]), tuple(D[:m + 1])

    return trial


def plan_law(N, q, m):
    return _enumerate(plan_trial(N, q, m))


def oracle_q(N, rho_scale, dt, eps):
    """q = exp(-mu dt / eps) for Maxwell molecules (Sigma = 1, mu = rho),
    evaluated as the step evaluates it in FP64."""
    rho = float(N) * rho_scale
    return math.exp(-(rho * 1.0 * dt) / eps)


def oracle_records(N, m, q_dt, cells, step=0):
    """Plan records of `cells` independently keyed cells of N particles at
    fixed order m, Maxwell molecules, q = exp(-q_dt) (eps = 1, rho = 1)."""
    counts = [N] * cells
    cs = synth.starts(counts)
    v = synth.maxwellian(N * cells, g=synth.rng(1234 + N + 10 * m))
    prm = O.collide_params(dt=q_dt, eps=1.0, alpha=0.0, rho_scale=1.0 / N, trunc=O.TRUNC_FIXED, m=m)
    _, rep, _ = O.collide(v, cs, prm, step)
    return rep, oracle_q(N, 1.0 / N, q_dt, 1.0)


def record_key(row, m):
    r = O.report_dict(row)
    return (tuple(int(x) for x in r["Nk"][:m + 2]), int(r["m_eff0"]), int(r["N0"]),
            tuple(int(x) for x in r["Ck"][1:m + 1]), tuple(int(x) for x in r["Dk"][:m + 1]))


def chi2_pvalue(law, keys_seen, S):
    keys = sorted(law)
    obs = np.array([keys_seen.get(k, 0) for k in keys], float)
    exp = np.array([float(law[k]) * S for k in keys])
    keep = exp >= 5
    obs_k = np.append(obs[keep], obs[~keep].sum())
    exp_k = np.append(exp[keep], exp[~keep].sum())
    if exp_k[-1] == 0:
        obs_k, exp_k = obs_k[:-1], exp_k[:-1]
    return stats.chisquare(obs_k, exp_k).pvalue


def prob(law, pred):
    return float(sum(p for k, p in law.items() if pred(k)))


# (N, m, dt): q = exp(-dt).  The last cases have deep trees on few particles,
# where the leaf rule is decisive.
CASES = [(6, 3, 0.7), (5, 3, 1.2), (4, 3, 1.6), (6, 2, 1.0), (3, 3, 2.5)]


def test_enumeration_is_a_law():
    # probabilities sum to one; every plan uses each particle once; the
    # enumeration agrees with the closed-form split expectation N q tau^n
    for N, m, dt in CASES:
        q = Fraction(oracle_q(N, 1.0 / N, dt, 1.0))
        law = plan_law(N, q, m)
        assert sum(law.values()) == 1
        for (Nq, top, n0, C, D), p in law.items():
            out = [2 * C[n - 1] - D[n] for n in range(1, m + 1)]
            assert all(o >= 0 for o in out) and sum(out) == D[0]
            assert 0 <= n0 <= Nq[0] and D[0] <= N - n0
        tau = 1 - q
        for n in range(m + 1):
            assert sum(p * k[0][n] for k, p in law.items()) == N * q * tau ** n
        assert sum(p * k[0][m + 1] for k, p in law.items()) == N * tau ** (m + 1)


def test_the_cases_exercise_both_readings():
    laws = {c: plan_law(c[0], Fraction(oracle_q(c[0], 1.0 / c[0], c[2], 1.0)), c[1]) for c in CASES}
    coin = lambda k: any((k[0][n] + k[4][n]) % 2 == 1 and k[0][n] >= 1 for n in range(1, k[1] + 1))
    borrow = lambda k: k[2] < k[0][0]
    split_top = lambda Nq: len(Nq) - 2 if Nq[-1] > 0 else max(n for n in range(len(Nq)) if Nq[n] > 0)
    lowered = lambda k: k[1] < split_top(k[0])
    assert max(prob(l, coin) for l in laws.values()) > 0.3
    assert max(prob(l, borrow) for l in laws.values()) > 0.05
    assert max(prob(l, lowered) for l in laws.values()) > 0.05


@pytest.mark.parametrize("N,m,dt", CASES)
def test_oracle_plan_follows_the_enumerated_law(N, m, dt):
    S = 30000
    rep, q = oracle_records(N, m, dt, S)
    law = plan_law(N, Fraction(q), m)
    seen = {}
    for row in rep:
        k = record_key(row, m)
        seen[k] = seen.get(k, 0) + 1
    assert set(seen) <= set(law), sorted(set(seen) - set(law))[:5]
    assert chi2_pvalue(law, seen, S) > 1e-4


def sample_plans(N, q, m, S, seed):
    """S plans of the reading drawn at random (numpy's generator, not the
    oracle's Philox): the same trial function as the enumeration, with each
    random decision sampled once per trial."""
    g = np.random.default_rng(seed)
    trial = plan_trial(N, Fraction(q), m)
    out = []
    for _ in range(S):
        fixed = {}

        def draw(key, outcomes):
            if key not in fixed:
                p = np.array([float(pv) for _, pv in outcomes])
                fixed[key] = outcomes[int(g.choice(len(outcomes), p=p / p.sum()))][0]
            return fixed[key]

        out.append(trial(draw))
    return out


def plan_summary(keys, N, m):
    """Per plan: outputs of levels 1..m, uncollided, thermalised, depth kept."""
    rows = []
    for Nq, top, n0, C, D in keys:
        out = [2 * C[n - 1] - D[n] for n in range(1, m + 1)]
        rows.append(out + [n0, N - n0 - D[0], top])
    return np.array(rows, float)


@pytest.mark.parametrize("N", [8, 11, 17])
@pytest.mark.parametrize("dt", [0.7, 1.4])
def test_oracle_plan_follows_the_sampled_reading(N, dt):
    """Beyond enumeration: the oracle's plans of cells of 8..17 particles at
    tau >= 0.5, where the coin and the leaf rule act in most cells, against
    plans of the reading drawn with an unrelated generator: the mean outputs
    of every level, the uncollided and thermalised counts and the kept depth
    agree within their statistical errors."""
    m, S = 6, 20000
    rep, q = oracle_records(N, m, dt, S, step=3)
    assert 1.0 - q >= 0.5
    a = plan_summary([record_key(r, m) for r in rep], N, m)
    b = plan_summary(sample_plans(N, q, m, S, seed=N + int(10 * dt)), N, m)
    se = np.sqrt(a.var(0, ddof=1) / S + b.var(0, ddof=1) / S) + 1e-12
    assert np.all(np.abs(a.mean(0) - b.mean(0)) <= 4.5 * se), (a.mean(0), b.mean(0), se)
    # the leaf rule really acted
    assert np.mean(rep[:, O.R_FIELDS.index("feas")] > 0) + np.mean(rep[:, O.R_FIELDS.index("N0")] < rep[:, O.R_NK]) > 0.02


@pytest.mark.parametrize("dt", [0.7, 1.5])
def test_outputs_are_unbiased_per_level(dt):
    """In cells large enough that the leaf rule never acts, the coin leaves
    each level's output count with the expectation of its Wild-sum quota:
    E[out_n - N_n - [N_n = 0 and D_n odd]] = 0 at every level n <= m, with
    out_n = 2 C_n - D_n and E[N_n] = N q tau^n (Eq. WST); only a level
    without quota particles keeps a surplus by force."""
    N, m, cells = 1000, 4, 2000
    rep, q = oracle_records(N, m, dt, cells, step=5)
    assert np.all(rep[:, O.R_FIELDS.index("feas")] == 0)
    assert np.all(rep[:, O.R_FIELDS.index("N0")] == rep[:, O.R_NK])
    Nk = rep[:, O.R_NK:O.R_NK + m + 2].astype(float)
    Ck = rep[:, O.R_CK:O.R_CK + m + 2]
    Dk = rep[:, O.R_DK:O.R_DK + m + 2]
    tossed = 0
    for n in range(1, m + 1):
        out = 2 * Ck[:, n] - Dk[:, n]
        forced = (Nk[:, n] == 0) & (Dk[:, n] % 2 == 1)
        z = out - Nk[:, n] - forced
        tossed += int(np.count_nonzero(((Nk[:, n] + Dk[:, n]) % 2 == 1) & (Nk[:, n] >= 1)))
        zse = max(z.std(ddof=1), 0.1) / np.sqrt(cells)
        assert abs(z.mean()) <= 4.5 * zse, (n, z.mean(), zse)
    assert tossed > 0.3 * cells * m          # the coin was really tossed
