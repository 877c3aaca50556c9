"""The FP64 CPU oracle stepping the same problem as a GPU simulation.

TEST INFRASTRUCTURE ONLY: used by tests/ and by bench.py's oracle
comparison (moment error, CPU baseline).  It reads a GPU simulation's state
once (its tensors copied to the host: velocities, positions, cell tables,
RAD depths, keys, domains, collide parameters, step index) and then runs
only the oracle's own transport and collision step (oracle/*.c) on it.
"""
import ctypes

import numpy as np

from . import oracle as O


class OracleSim:
    """The FP64 CPU oracle stepping the same workload as a GPU simulation,
    from that simulation's current state (velocities, positions, cell
    tables, RAD depths, step index) with the same keys, or with another seed."""

    def __init__(self, sim, seed):
        st = sim.state
        self.O = O
        self.cs = st.cell_start.cpu().numpy().copy()
        n = int(self.cs[-1])
        self.n = n
        self.v = st.v[:, :n].double().cpu().numpy()
        self.transports = bool(getattr(sim, "transports", False))
        self.x = st.x[:n].double().cpu().numpy() if self.transports else None
        self.cp = st.cell_param.cpu().numpy().copy() if st.cell_param is not None else None
        self.keys = st.cell_key.cpu().numpy().view(np.uint64).copy() if st.cell_key is not None else None
        self.ms = st.m_max.cpu().numpy().copy() if st.m_max is not None else None
        if self.transports:
            raw = sim.domains.cpu().numpy().tobytes()
            size = ctypes.sizeof(O.Domain)
            self.doms = [O.Domain.from_buffer_copy(raw, i * size) for i in range(len(raw) // size)]
            self.cfl = sim.cfl
        p = sim.params
        self.prm = O.collide_params(dt=p.dt, eps=p.eps, alpha=p.alpha, rho_scale=p.rho_scale, trunc=p.trunc,
                                    m=p.m_fixed, m_min=p.m_min, m_cap=p.m_cap, delta1=p.delta1, delta2=p.delta2,
                                    indicator=p.indicator, seed=seed, wb_length=p.wb_length)
        self.seed = seed
        self.cap = int(st.capacity)
        self.step_index = int(sim.step_index)
        self.problem_id = int(st.c.problem_id)

    def step(self, threads):
        O = self.O
        if self.transports:
            dt = O.cfl_dt(self.v, self.cs, self.doms, self.cfl)
            self.x, self.v, self.cs = O.transport(self.x, self.v, self.cs, self.doms, dt, step=self.step_index,
                                                  seed=self.seed, problem_id=self.problem_id, cell_key=self.keys,
                                                  capacity=self.cap)
            if self.cp is not None:
                for d, h in zip(self.doms, dt):
                    self.cp[d.cell_begin:d.cell_begin + d.n_cells, 1] = h
        self.v, _, self.ms = O.collide(self.v, self.cs, self.prm, self.step_index, m_state=self.ms,
                                       cell_param=None if self.cp is None else self.cp.ravel(), cell_key=self.keys,
                                       problem_id=self.problem_id, threads=threads)
        self.step_index += 1

    def moments(self):
        return self.O.moments(self.v, self.cs, None if self.cp is None else self.cp[:, 2])
