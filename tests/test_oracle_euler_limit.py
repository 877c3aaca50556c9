"""Pin of the oracle's whole splitting step (transport, sort, collision) in
the fluid limit: a shock tube at eps = 1e-4 (Sec. 5.1), where every cell
relaxes to its local Maxwellian each step, must follow the exact Riemann
solution of the Euler equations of a monatomic gas (gamma = 5/3, p = rho T)
for the tube's initial data (rho, u, p) = (1, 0, 1) | (0.125, 0, 0.1) at
x = 0.5: shock and contact where the exact solution puts them, the density
plateau between them, and a small L1 density error overall.

The exact solution is written here from the textbook shock and rarefaction
relations (pressure functions, star state, wave fan) and is itself checked
against the Rankine-Hugoniot jump conditions and the rarefaction's
isentropic relation before the oracle is compared with it."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1009_2768_gb300 import synth

GAMMA = 5.0 / 3.0
LEFT, RIGHT = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)      # (rho, u, p)


def star_state(L, R, g=GAMMA):
    """Pressure and velocity between the two waves (bisection on the sum of
    the two sides' pressure functions)."""
    def f(p, side):
        rho, _, pk = side
        c = np.sqrt(g * pk / rho)
        if p > pk:                                     # shock
            a, b = 2.0 / ((g + 1.0) * rho), (g - 1.0) / (g + 1.0) * pk
            return (p - pk) * np.sqrt(a / (p + b))
        return 2.0 * c / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)    # rarefaction

    lo, hi = 1e-12, 100.0 * max(L[2], R[2])
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid, L) + f(mid, R) + R[1] - L[1] > 0.0:
            hi = mid
        else:
            lo = mid
    ps = 0.5 * (lo + hi)
    return ps, 0.5 * (L[1] + R[1]) + 0.5 * (f(ps, R) - f(ps, L))


def waves(g=GAMMA):
    """For the tube's data (left rarefaction, right shock): star pressure and
    velocity, the two star densities, the shock speed and the fan's edges."""
    ps, us = star_state(LEFT, RIGHT, g)
    rl, ul, pl = LEFT
    rr, ur, pr = RIGHT
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    k = (g - 1.0) / (g + 1.0)
    rho_sr = rr * (ps / pr + k) / (k * ps / pr + 1.0)
    shock = ur + cr * np.sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g))
    rho_sl = rl * (ps / pl) ** (1.0 / g)
    head, tail = ul - cl, us - cl * (ps / pl) ** ((g - 1.0) / (2.0 * g))
    return dict(ps=ps, us=us, rho_sl=rho_sl, rho_sr=rho_sr, shock=shock, head=head, tail=tail, cl=cl)


def exact_density(xi, g=GAMMA):
    w = waves(g)
    rl, ul, _ = LEFT
    out = np.empty_like(xi)
    for i, s in enumerate(xi):
        if s < w["head"]:
            out[i] = rl
        elif s < w["tail"]:
            out[i] = rl * (2.0 / (g + 1.0) + (g - 1.0) / ((g + 1.0) * w["cl"]) * (ul - s)) ** (2.0 / (g - 1.0))
        elif s < w["us"]:
            out[i] = w["rho_sl"]
        elif s < w["shock"]:
            out[i] = w["rho_sr"]
        else:
            out[i] = RIGHT[0]
    return out


def test_exact_solution_meets_the_jump_conditions():
    w = waves()
    rr, ur, pr = RIGHT
    S, us, ps, rs = w["shock"], w["us"], w["ps"], w["rho_sr"]
    m = rr * (S - ur)                                              # mass flux through the shock
    assert abs(m - rs * (S - us)) < 1e-12 * m
    assert abs(m * (us - ur) - (ps - pr)) < 1e-12 * ps             # momentum
    e_r = pr / ((GAMMA - 1.0) * rr) + 0.5 * ur * ur                # specific total energies
    e_s = ps / ((GAMMA - 1.0) * rs) + 0.5 * us * us
    assert abs(m * (e_s - e_r) - (ps * us - pr * ur)) < 1e-12 * ps * us
    rl, ul, pl = LEFT                                              # rarefaction: isentropic, Riemann invariant
    assert abs(ps / w["rho_sl"] ** GAMMA - pl / rl ** GAMMA) < 1e-12
    c_s = np.sqrt(GAMMA * ps / w["rho_sl"])
    assert abs((ul + 2.0 * w["cl"] / (GAMMA - 1.0)) - (us + 2.0 * c_s / (GAMMA - 1.0))) < 1e-12
    # the fan joins both constant states continuously
    d = exact_density(np.array([w["head"] + 1e-12, w["tail"] - 1e-12]))
    assert abs(d[0] - rl) < 1e-9 and abs(d[1] - w["rho_sl"]) < 1e-9


def run_tube(n_cells=100, mean=500, seed=0, t_end=0.2, eps=1e-4):
    counts = synth.shock_tube_counts(n_cells, mean)
    cs = synth.starts(counts)
    ci = np.zeros((n_cells, 9))
    for c in range(n_cells):                       # Maxwellian, T = p / rho: 1 | 0.8
        ci[c] = [0, 0, 0, 0, 1.0 if c < n_cells // 2 else 0.8, 0, 0, c / n_cells, (c + 1) / n_cells]
    w = 0.5625 / int(cs[-1])                       # particle mass: the tube holds 0.5 * 1 + 0.5 * 0.125
    x, v = O.init_cells(ci, cs, seed)
    doms = [(0, n_cells, 0.0, 1.0)]
    prm = O.collide_params(trunc=O.TRUNC_RAD, m=2, alpha=1.0)
    prm.seed = seed
    ms = np.full(n_cells, 2, np.int32)
    t, step = 0.0, 0
    while t < t_end - 1e-12:
        dt = min(O.cfl_dt(v, cs, doms, 0.5)[0], t_end - t)
        x, v, cs = O.transport(x, v, cs, doms, np.array([dt]))
        cp = np.tile([eps, dt, w * n_cells, 1.0], (n_cells, 1))
        v, _, ms = O.collide(v, cs, prm, step, m_state=ms, cell_param=cp.ravel(), threads=8)
        t += dt
        step += 1
    return np.diff(cs) * w * n_cells              # density per cell


def test_oracle_shock_tube_follows_the_euler_riemann_solution():
    n, t = 100, 0.2
    rho = run_tube(n_cells=n, t_end=t)
    xc = (np.arange(n) + 0.5) / n
    exact = exact_density((xc - 0.5) / t)
    w = waves()
    # shock: the last cell above the midpoint of the post- and pre-shock densities
    x_shock = xc[np.nonzero(rho > 0.5 * (w["rho_sr"] + RIGHT[0]))[0].max()] + 0.5 / n
    assert abs(x_shock - (0.5 + w["shock"] * t)) <= 2.0 / n
    # contact: the last cell above the midpoint of the two star densities
    x_contact = xc[np.nonzero(rho > 0.5 * (w["rho_sl"] + w["rho_sr"]))[0].max()] + 0.5 / n
    assert abs(x_contact - (0.5 + w["us"] * t)) <= 3.0 / n
    # the plateau between contact and shock, away from both
    lo, hi = int((0.5 + w["us"] * t) * n) + 4, int((0.5 + w["shock"] * t) * n) - 3
    assert abs(rho[lo:hi].mean() / w["rho_sr"] - 1.0) < 0.06
    # the undisturbed states near the walls
    assert abs(rho[:15].mean() - LEFT[0]) < 0.03 and abs(rho[-8:].mean() / RIGHT[0] - 1.0) < 0.05
    assert np.abs(rho - exact).mean() < 0.045


@pytest.mark.parametrize("g", [1.4, 2.0])
def test_euler_pin_rejects_another_gamma(g):
    """The comparison above is sharp enough to tell the monatomic gas the
    particles make from other adiabatic exponents."""
    w, w_other = waves(), waves(g)
    assert abs(w_other["shock"] - w["shock"]) * 0.2 > 2.0 / 100 or abs(w_other["rho_sr"] / w["rho_sr"] - 1.0) > 0.06
