"""FP32-mixed contexts: float velocities and collisions, FP64 moments, bounds,
level probabilities and renormalisation.  Assignments may differ from the
FP64 oracle (q and Sigma come from float data), so these tests check what
must hold regardless: conservation (with the FP64 carry of the storage
rounding), the closed-form relaxation factors of the truncated Wild sum
(Eq. CF-r / Eq. WST) and the BKW fourth moment within 3 sigma."""
import numpy as np
import pytest

from paper_1009_2768_gb300 import synth
from tests.gpu_common import T, ctx, need_gpu, torch

pytestmark = pytest.mark.gpu


def exact_sums(v, cs):
    """Per-cell sum of v (3) and of |v|^2, exactly (float data, FP64 sums of
    at most a few thousand values of similar magnitude, pairwise)."""
    v = v.astype(np.float64)
    out = np.zeros((len(cs) - 1, 4))
    for c in range(len(cs) - 1):
        a, b = cs[c], cs[c + 1]
        out[c, :3] = np.sum(v[:, a:b], axis=1)
        out[c, 3] = np.sum(v[:, a:b] ** 2)
    return out


def test_fp32_conservation_with_carry():
    need_gpu()
    g = synth.rng(40)
    counts = synth.loguniform_ints(64, 16, 6000, g=g)
    cs = synth.starts(counts)
    eps = synth.loguniform(64, 1e-4, 10, g=g)
    cp = np.stack([eps, np.full(64, 0.05), 1.0 / counts, np.full(64, 0.6)], axis=1)
    v = np.concatenate([synth.bimaxwellian(int(n), 2.0, 0.5, u=(0.4, 0.0, -0.2), g=g) for n in counts], axis=1)
    st = T.ParticleState(cs, precision=T.FP32_MIXED, rad=True, cell_param=cp, carry=True)
    st.set_velocities(v)
    c = ctx(T.FP32_MIXED, seed=1)
    n = int(cs[-1])
    q0 = exact_sums(st.v[:, :n].cpu().numpy(), cs)
    scale = np.abs(q0).max(axis=1, keepdims=True) + np.array([[0, 0, 0, 0]])
    drift = []
    for step in range(20):
        T.trmc_collide(c, st, T.collide_params(trunc=T.TRUNC_RAD, m=2), step)
        T.trmc_check(c)
        raw = exact_sums(st.v[:, :n].cpu().numpy(), cs)
        carry = st.cell_carry.cpu().numpy()[:64]
        # sum of stored floats plus the carried rounding defect: conserved
        assert np.all(np.abs(raw + carry - q0) <= 1e-12 * scale), (step, np.abs(raw + carry - q0).max())
        drift.append(np.abs(raw - q0).max(axis=0) / np.abs(q0).max(axis=0))
    # the stored floats alone drift by one step's rounding at most: no accumulation
    drift = np.array(drift)
    assert drift.max() < 1e-5
    assert drift[-5:].max() < 10 * drift[:5].max() + 1e-7


def rising(a, k):
    r = 1.0
    for j in range(k):
        r *= (a + j) / (j + 1)
    return r


def factor(a, q, m):
    tau = 1.0 - q
    return q * sum(rising(a, k) * tau ** k for k in range(m + 1))


def central_m4(v):
    v = v.astype(np.float64)
    d = v - v.mean(1, keepdims=True)
    Tm = (d ** 2).sum(0).mean() / 3.0
    return ((d ** 2).sum(0) ** 2).mean() / Tm ** 2


@pytest.mark.parametrize("m", [1, 2, 4])
def test_fp32_m4_step_factor(m):
    """One step from BKW data at dt/eps = 1: E[M4' - 15] / (M4 - 15) equals
    q sum_{k<=m} ((2/3)_k / k!) tau^k (derived from Eq. CF-r and the map)."""
    need_gpu()
    N, runs = 100000, 40
    v0 = synth.bkw(N, K=0.6, g=synth.rng(41)).astype(np.float32)
    a0 = central_m4(v0) - 15.0
    st = T.ParticleState([0, N], precision=T.FP32_MIXED)
    c = ctx(T.FP32_MIXED, seed=2)
    p = T.collide_params(dt=1.0, eps=1.0, alpha=0.0, rho_scale=1.0 / N, trunc=T.TRUNC_FIXED, m=m)
    r = []
    for s in range(runs):
        st.set_velocities(v0)
        T.trmc_collide(c, st, p, s)
        r.append((central_m4(st.v.cpu().numpy()) - 15.0) / a0)
    T.trmc_check(c)
    r = np.array(r)
    F = factor(2.0 / 3.0, np.exp(-1.0), m)
    se = r.std(ddof=1) / np.sqrt(runs)
    assert abs(r.mean() - F) <= 4 * se + 0.004, (m, r.mean(), F, se)


def test_fp32_bkw_fourth_moment_within_3_sigma():
    """Homogeneous BKW run (Maxwell molecules, K0 = 0.6, N = 1e5, eps = 1,
    dt = 0.05, TRMC-RAD with the M4 indicator) for 200 steps to t = 10:
    M4(t) - 15 = (M4(0) - 15) exp(-t/3) within 3 sigma of the Monte Carlo
    error (8 seeds)."""
    need_gpu()
    from paper_1009_2768_gb300.workloads import HomogeneousBKW
    seeds, checkpoints = 8, {20: 1.0, 40: 2.0, 100: 5.0, 200: 10.0}
    err = {t: [] for t in checkpoints.values()}
    for sd in range(seeds):
        sim = HomogeneousBKW(100000, precision=T.FP32_MIXED, seed=100 + sd)
        a0 = central_m4(sim.state.v.cpu().numpy()) - 15.0
        for s in range(1, 201):
            sim.step()
            if s in checkpoints:
                t = checkpoints[s]
                err[t].append((central_m4(sim.state.v.cpu().numpy()) - 15.0) - a0 * np.exp(-t / 3.0))
        T.trmc_check(sim.ctx)
        sim.close()
    sigma = np.sqrt(720.0 / 1e5) / np.sqrt(seeds)
    for t, e in err.items():
        assert abs(np.mean(e)) <= 3 * sigma, (t, np.mean(e), sigma)
