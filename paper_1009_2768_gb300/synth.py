"""Seeded synthetic inputs (numpy only).

These generators produce the particle sets of the workloads: Maxwellian,
bi-Maxwellian and BKW velocity samples, log-uniform cell sizes and Knudsen
numbers, and the two-state shock-tube layout.  They hold none of the TRMC-R
method's arithmetic and serve the tests and the benchmark on both sides of
a comparison (the CUDA library and the CPU oracle get identical arrays).
"""
import numpy as np


def rng(seed):
    return np.random.default_rng(seed)


def maxwellian(n, T=1.0, u=(0.0, 0.0, 0.0), g=None):
    g = g or rng(0)
    return np.asarray(u, dtype=np.float64)[:, None] + np.sqrt(T) * g.standard_normal((3, n))


def bimaxwellian(n, T_par, T_perp, u=(0.0, 0.0, 0.0), g=None):
    g = g or rng(0)
    v = g.standard_normal((3, n))
    v[0] *= np.sqrt(T_par)
    v[1:] *= np.sqrt(T_perp)
    return v + np.asarray(u, dtype=np.float64)[:, None]


def bkw(n, K=0.6, g=None):
    """BKW similarity solution for Maxwell molecules at shape K (unit
    density and temperature, zero mean): sqrt(K) chi_3 with weight
    (5K-3)/(2K), sqrt(K) chi_5 otherwise, isotropic direction."""
    g = g or rng(0)
    z = g.standard_normal((3, n))
    w_gauss = (5.0 * K - 3.0) / (2.0 * K)
    five = g.random(n) >= w_gauss
    extra = g.standard_normal((2, n))
    r3 = np.sqrt((z ** 2).sum(0))
    r5 = np.sqrt((z ** 2).sum(0) + (extra ** 2).sum(0))
    f = np.where(five, r5 / r3, 1.0)
    return np.sqrt(K) * z * f


def loguniform_ints(n, lo, hi, g=None):
    g = g or rng(0)
    return np.floor(np.exp(g.uniform(np.log(lo), np.log(hi + 1), n))).astype(np.int64).clip(lo, hi)


def loguniform(n, lo, hi, g=None):
    g = g or rng(0)
    return np.exp(g.uniform(np.log(lo), np.log(hi), n))


def starts(counts):
    cs = np.zeros(len(counts) + 1, np.int64)
    cs[1:] = np.cumsum(counts)
    return cs


def shock_tube_counts(n_cells, mean_per_cell, rho_l=1.0, rho_r=0.125):
    """Particles per cell for a Riemann problem with the interface at the
    middle of [0,1], proportional to density with the given mean."""
    half = n_cells // 2
    total = mean_per_cell * n_cells
    w = total / (half * rho_l + (n_cells - half) * rho_r)
    counts = np.empty(n_cells, np.int64)
    counts[:half] = int(round(w * rho_l))
    counts[half:] = int(round(w * rho_r))
    return counts


def poisson_requests(n, rate, n_lo=100_000, n_hi=20_000_000, eps_lo=1e-4, eps_hi=1.0, kinds=("shock", "relax"),
                     g=None):
    """A stream of n solve requests: Poisson arrivals at `rate` per second
    (exponential gaps, first arrival at 0), kind drawn uniformly from
    `kinds`, particle count log-uniform in [n_lo, n_hi], Knudsen number
    log-uniform in [eps_lo, eps_hi].  Returns a list of dicts."""
    g = g or rng(0)
    gaps = g.exponential(1.0 / rate, n)
    gaps[0] = 0.0
    t = np.cumsum(gaps)
    kind = g.integers(0, len(kinds), n)
    npart = loguniform_ints(n, n_lo, n_hi, g=g)
    eps = loguniform(n, eps_lo, eps_hi, g=g)
    return [dict(arrival=float(t[i]), kind=kinds[kind[i]], n_particles=int(npart[i]), eps=float(eps[i]))
            for i in range(n)]
