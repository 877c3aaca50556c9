"""Set-up of the synthetic workloads through the C ABI (trmc_init_cells),
and one time step of each.  Everything runs in libtrmc; this module only
lays out the cell tables the library reads.

Workloads (synthetic closed-form initial data, no dataset):
  * ShockTubes  -- 1D Riemann shock tubes on [0,1] (left rho=1, T=1; right
    rho=0.125, T=0.8; u=0), specular walls, hard-sphere VHS, CFL 0.5, one
    tube per Knudsen number, all advanced together;
  * HomogeneousBKW -- one space-homogeneous cell of Maxwell molecules with
    BKW initial data (K0 = 0.6, unit density and temperature);
  * BatchedRelaxation -- independent homogeneous cells with log-uniform
    particle counts and Knudsen numbers, bi-Maxwellian initial data.
"""
import numpy as np

from . import synth
from . import trmc as T

def _dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


class ShockTubes:
    transports = True
    def __init__(self, eps_list=(1e-1, 1e-2, 1e-3, 1e-4), n_cells=400, mean_per_cell=500,
                 precision=T.FP64, seed=0, alpha=1.0, trunc=T.TRUNC_RAD, m_init=2, cfl=0.5,
                 workspace=512 << 20, ctx=None, problem_base=0, order="given"):
        import torch
        self.n_tubes = len(eps_list)
        self.n_cells_tube = n_cells
        counts1 = synth.shock_tube_counts(n_cells, mean_per_cell)
        counts = np.tile(counts1, self.n_tubes)
        cs = synth.starts(counts)
        self.n_particles = int(cs[-1])
        nt = int(counts1.sum())
        rho_scale = 0.5625 * n_cells / nt         # tube mass 0.5*1 + 0.5*0.125 over nt particles, per cell width
        nc = n_cells * self.n_tubes
        cp = np.zeros((nc, 4))
        cp[:, 0] = np.repeat(np.asarray(eps_list, float), n_cells)
        cp[:, 2] = rho_scale
        cp[:, 3] = alpha
        tube = np.repeat(np.arange(self.n_tubes, dtype=np.uint64), n_cells)
        keys = ((np.uint64(problem_base) + tube) << np.uint64(32)) | np.tile(np.arange(n_cells, dtype=np.uint64),
                                                                             self.n_tubes)
        ci = np.zeros((nc, T.INIT_COLS))
        c = np.tile(np.arange(n_cells), self.n_tubes)
        ci[:, 0] = T.INIT_MAXWELL
        ci[:, 4] = np.where(c < n_cells // 2, 1.0, 0.8)
        ci[:, 7] = c / n_cells
        ci[:, 8] = (c + 1) / n_cells
        self.state = T.ParticleState(cs, capacity=self.n_particles, precision=precision, with_x=True,
                                     rad=trunc == T.TRUNC_RAD, cell_param=cp, cell_key=keys,
                                     carry=precision == T.FP32_MIXED)
        if trunc == T.TRUNC_RAD:
            self.state.m_max.fill_(m_init)
        if order == "adaptive":
            self.state.use_adaptive_order()
        self.launches_per_step = 6 + (order == "adaptive")   # cfl, count, scan, scatter, refill, [order], collide
        self.own_ctx = ctx is None
        self.ctx = T.trmc_create(precision, seed, workspace) if ctx is None else ctx
        T.trmc_init_cells(self.ctx, self.state, _dev(ci))
        self.domains = T.domains_tensor([(t * n_cells, n_cells, 0.0, 1.0) for t in range(self.n_tubes)])
        self.dt = torch.zeros(self.n_tubes, dtype=torch.float64, device="cuda")
        self.cfl = cfl
        self.params = T.collide_params(trunc=trunc, m=m_init, indicator=T.IND_PXX)
        self.step_index = 0

    def step(self, stats=None, events=None):
        """One splitting step: transport + sort, then collide.  events, if
        given, is a list of three CUDA events recorded before transport,
        between transport and collide, and after collide."""
        if events:
            events[0].record()
        T.trmc_transport(self.ctx, self.state, self.domains, self.n_tubes, self.cfl, self.dt, self.step_index)
        if events:
            events[1].record()
        T.trmc_collide(self.ctx, self.state, self.params, self.step_index, stats=stats)
        if events:
            events[2].record()
        self.step_index += 1

    def close(self):
        if self.own_ctx:
            T.trmc_destroy(self.ctx)


class HomogeneousBKW:
    transports = False
    def __init__(self, n=100000, K0=0.6, eps=1.0, dt=0.05, precision=T.FP64, seed=0, trunc=T.TRUNC_RAD, m_init=2,
                 workspace=256 << 20):
        cs = np.array([0, n], np.int64)
        self.n_particles = n
        self.state = T.ParticleState(cs, precision=precision, rad=trunc == T.TRUNC_RAD, vmax=False)
        if trunc == T.TRUNC_RAD:
            self.state.m_max.fill_(m_init)
        self.ctx = T.trmc_create(precision, seed, workspace)
        ci = np.array([[T.INIT_BKW, 0, 0, 0, 1.0, 0, K0, 0, 1]], float)
        T.trmc_init_cells(self.ctx, self.state, _dev(ci))
        self.params = T.collide_params(dt=dt, eps=eps, alpha=0.0, rho_scale=1.0 / n, trunc=trunc, m=m_init,
                                       indicator=T.IND_M4)
        self.step_index = 0
        # a cell of 32768 particles or more: the moment pre-pass, then collide
        self.launches_per_step = 2 if n >= 32768 else 1

    def step(self, stats=None, events=None):
        if events:
            events[0].record()
            events[1].record()
        T.trmc_collide(self.ctx, self.state, self.params, self.step_index, stats=stats)
        if events:
            events[2].record()
        self.step_index += 1

    def close(self):
        T.trmc_destroy(self.ctx)


class BatchedRelaxation:
    transports = False
    def __init__(self, n_cells=4096, lo=64, hi=8192, eps_lo=1e-4, eps_hi=10.0, alpha=0.6, dt=0.05,
                 precision=T.FP32_MIXED, seed=0, trunc=T.TRUNC_RAD, m_init=2, workspace=1 << 30,
                 order="given", ctx=None, problem_base=0, problem_per_cell=True, counts=None):
        g = synth.rng(seed)
        if counts is None:
            counts = synth.loguniform_ints(n_cells, lo, hi, g=g)
        counts = np.asarray(counts, np.int64)
        n_cells = len(counts)
        eps = synth.loguniform(n_cells, eps_lo, eps_hi, g=g)
        ratio = g.uniform(0.3, 3.0, n_cells)          # T_par / T_perp with T = (T_par + 2 T_perp)/3 = 1
        t_perp = 3.0 / (ratio + 2.0)
        t_par = ratio * t_perp
        cs = synth.starts(counts)
        self.n_particles = int(cs[-1])
        cp = np.stack([eps, np.full(n_cells, dt), 1.0 / counts, np.full(n_cells, alpha)], axis=1)
        c = np.arange(n_cells, dtype=np.uint64)
        if problem_per_cell:                  # every cell its own problem
            keys = (np.uint64(problem_base) + c) << np.uint64(32)
        else:                                 # one problem, cells numbered within it
            keys = (np.uint64(problem_base) << np.uint64(32)) | c
        self.state = T.ParticleState(cs, capacity=self.n_particles, precision=precision, rad=trunc == T.TRUNC_RAD,
                                     cell_param=cp, cell_key=keys, carry=precision == T.FP32_MIXED, vmax=False)
        if trunc == T.TRUNC_RAD:
            self.state.m_max.fill_(m_init)
        self.own_ctx = ctx is None
        self.ctx = T.trmc_create(precision, seed, workspace) if ctx is None else ctx
        ci = np.zeros((n_cells, T.INIT_COLS))
        ci[:, 0] = T.INIT_BIMAXWELL
        ci[:, 4] = t_par
        ci[:, 5] = t_perp
        T.trmc_init_cells(self.ctx, self.state, _dev(ci))
        if order == "largest_first":          # cell sizes never change here: order once
            self.state.set_cell_order(np.argsort(-counts, kind="stable").astype(np.int32))
        elif order == "adaptive":
            self.state.use_adaptive_order()
        self.launches_per_step = 1 + (order == "adaptive")
        self.params = T.collide_params(trunc=trunc, m=m_init, indicator=T.IND_PXX)
        self.step_index = 0

    def step(self, stats=None, events=None):
        if events:
            events[0].record()
            events[1].record()
        T.trmc_collide(self.ctx, self.state, self.params, self.step_index, stats=stats)
        if events:
            events[2].record()
        self.step_index += 1

    def close(self):
        if self.own_ctx:
            T.trmc_destroy(self.ctx)


def rankine_hugoniot(mach, rho_l=1.0, t_l=1.0, gamma=5.0 / 3.0):
    """Downstream state of a normal shock from the Rankine-Hugoniot relations
    (Sec. 5.2) for an upstream state moving at Mach `mach` (p = rho T)."""
    u_l = mach * np.sqrt(gamma * t_l)
    m2 = mach * mach
    rho_r = rho_l * (gamma + 1.0) * m2 / ((gamma - 1.0) * m2 + 2.0)
    u_r = rho_l * u_l / rho_r
    p_r = rho_l * t_l * (2.0 * gamma * m2 - (gamma - 1.0)) / (gamma + 1.0)
    return (rho_l, u_l, t_l), (rho_r, u_r, p_r / rho_r)


class StationaryShock:
    transports = True
    """1D stationary normal shock on [0,1] (Sec. 5.2): upstream Rankine-
    Hugoniot state on the left flowing in through a reservoir, downstream
    state on the right flowing out through the other, initial step at 0.5;
    hard-sphere VHS, CFL time step, ghost cells at both ends (not collided)."""

    def __init__(self, n_cells=4000, mean_per_cell=2500, mach=3.0, eps=1e-3, precision=T.FP32_MIXED, seed=0,
                 alpha=1.0, trunc=T.TRUNC_RAD, m_init=2, cfl=0.5, workspace=1 << 30, headroom=1.25, order="given"):
        import torch
        left, right = rankine_hugoniot(mach)
        self.left, self.right = left, right
        dx = 1.0 / n_cells
        n_total = n_cells * mean_per_cell
        mass = (0.5 * left[0] + 0.5 * right[0]) / n_total           # particle mass
        self.particle_mass = mass
        nc = n_cells + 2
        counts = np.empty(nc, np.int64)
        ci = np.zeros((nc, T.INIT_COLS))
        for c in range(nc):
            xc = (c - 1 + 0.5) * dx
            rho, u, Tm = left if xc < 0.5 else right
            counts[c] = int(round(rho * dx / mass))
            ci[c] = [T.INIT_MAXWELL, u, 0, 0, Tm, 0, 0, (c - 1) * dx, c * dx]
        cs = synth.starts(counts)
        self.n_particles = int(cs[-1])
        cp = np.zeros((nc, 4))
        cp[:, 0] = eps
        cp[[0, -1], 0] = 1e300                 # ghost cells: reservoir particles, never collided
        cp[:, 2] = mass / dx
        cp[:, 3] = alpha
        cap = int(headroom * self.n_particles) + 4 * mean_per_cell
        self.state = T.ParticleState(cs, capacity=cap, precision=precision, with_x=True, rad=trunc == T.TRUNC_RAD,
                                     cell_param=cp, carry=precision == T.FP32_MIXED)
        if trunc == T.TRUNC_RAD:
            self.state.m_max.fill_(m_init)
        if order == "adaptive":
            self.state.use_adaptive_order()
        self.launches_per_step = 6 + (order == "adaptive")   # cfl, count, scan, scatter, refill, [order], collide
        self.ctx = T.trmc_create(precision, seed, workspace)
        T.trmc_init_cells(self.ctx, self.state, _dev(ci))
        self.domains = T.domains_tensor([(0, nc, 0.0, 1.0, T.BC_RESERVOIR, left, right, mass)])
        self.dt = torch.zeros(1, dtype=torch.float64, device="cuda")
        self.cfl = cfl
        self.params = T.collide_params(trunc=trunc, m=m_init, indicator=T.IND_PXX)
        self.step_index = 0

    def step(self, stats=None, events=None):
        if events:
            events[0].record()
        T.trmc_transport(self.ctx, self.state, self.domains, 1, self.cfl, self.dt, self.step_index)
        if events:
            events[1].record()
        T.trmc_collide(self.ctx, self.state, self.params, self.step_index, stats=stats)
        if events:
            events[2].record()
        self.step_index += 1

    def close(self):
        T.trmc_destroy(self.ctx)
