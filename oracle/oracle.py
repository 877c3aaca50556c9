"""numpy front end of the FP64 CPU oracle (oracle/*.c).

TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the CPU
baseline of bench.py.  The product (the CUDA library and its binding) never
imports this module.  Every routine here just marshals numpy arrays into the
C oracle, which cites the paper passage each step follows.
"""
import ctypes as C
import os

import numpy as np

from .build import build_oracle

TAG_INIT, TAG_SPLIT, TAG_PARITY, TAG_KSEL, TAG_PERM0, TAG_PERMK, TAG_COLL, TAG_MAXW = range(1, 9)
TRUNC_FIXED, TRUNC_RAD, TRUNC_UNLIMITED, TRUNC_WB = 0, 1, 2, 3
LEN_K, LEN_MIN, LEN_MEAN = 1, 2, 3          # tree-length definitions, Eqs. def:1-3
IND_PXX, IND_M4 = 0, 1
INIT_MAXWELL, INIT_BIMAXWELL, INIT_BKW = 0, 1, 2
MCAP = 64
INIT_COLS = 9
MOM_COLS = 10

# report layout (int64 per cell)
R_FIELDS = ["N", "passes", "m_first", "m_last", "m_next", "R_final", "N0", "leaves",
            "coll", "dummy", "exceed", "feas", "pdrop", "psurp", "m_eff0", "wbrej"]
R_NK = 16
R_CK = 16 + MCAP + 2
R_DK = 16 + 2 * (MCAP + 2)
R_LEN = 16 + 3 * (MCAP + 2)


class CollideParams(C.Structure):
    _fields_ = [("dt", C.c_double), ("eps", C.c_double), ("alpha", C.c_double),
                ("rho_scale", C.c_double), ("delta1", C.c_double), ("delta2", C.c_double),
                ("trunc", C.c_int32), ("m_fixed", C.c_int32), ("m_min", C.c_int32),
                ("m_cap", C.c_int32), ("indicator", C.c_int32), ("wb_length", C.c_int32),
                ("seed", C.c_uint64)]


BC_SPECULAR, BC_RESERVOIR = 0, 1
TAG_RESERVOIR = 9


class Domain(C.Structure):
    _fields_ = [("cell_begin", C.c_int32), ("n_cells", C.c_int32),
                ("x_lo", C.c_double), ("x_hi", C.c_double), ("bc", C.c_int32), ("reserved", C.c_int32),
                ("res_lo", C.c_double * 3), ("res_hi", C.c_double * 3), ("particle_mass", C.c_double)]


def domain(cell_begin, n_cells, x_lo, x_hi, bc=BC_SPECULAR, res_lo=(0, 0, 0), res_hi=(0, 0, 0), particle_mass=0.0):
    return Domain(cell_begin, n_cells, x_lo, x_hi, bc, 0, (C.c_double * 3)(*res_lo), (C.c_double * 3)(*res_hi),
                  particle_mass)


def _domains(domains):
    ds = [d if isinstance(d, Domain) else domain(*d) for d in domains]
    return (Domain * len(ds))(*ds)


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build_oracle())
        P = C.c_void_p
        _lib.orc_philox4x64.argtypes = [P, P, P]
        _lib.orc_draw.argtypes = [C.c_uint64] * 6 + [C.c_uint32, C.c_uint32, P]
        _lib.orc_u01.argtypes = [C.c_uint64]; _lib.orc_u01.restype = C.c_double
        _lib.orc_u01_open.argtypes = [C.c_uint64]; _lib.orc_u01_open.restype = C.c_double
        _lib.orc_below.argtypes = [C.c_uint64, C.c_uint32]; _lib.orc_below.restype = C.c_uint32
        _lib.orc_prp_init.argtypes = [P, C.c_uint64, P]
        _lib.orc_prp_fwd.argtypes = [P, C.c_uint64]; _lib.orc_prp_fwd.restype = C.c_uint64
        _lib.orc_prp_inv.argtypes = [P, C.c_uint64]; _lib.orc_prp_inv.restype = C.c_uint64
        _lib.orc_prp_tables.argtypes = [C.c_uint64, P, C.c_int64, P]
        _lib.orc_collide.argtypes = [P, P, P, P, C.c_int32, P, C.c_uint64, C.c_uint64, P, P, P, P, C.c_int]
        _lib.orc_collide_cell.argtypes = [P, P, P, C.c_int64, C.c_uint64, C.c_uint64, C.c_uint64, P, P, P, P]
        _lib.orc_transport.argtypes = [P, P, P, P, P, C.c_int32, P, C.c_int32, P, P, C.c_uint64, C.c_uint64,
                                       C.c_uint64, P, P, P, P, C.c_int64, P]
        _lib.orc_transport.restype = C.c_int64
        _lib.orc_cfl_dt.argtypes = [P, P, P, P, P, C.c_int32, C.c_double, P]
        _lib.orc_init_cells.argtypes = [P, P, C.c_int32, P, C.c_uint64, C.c_uint64, P, P, P, P]
        _lib.orc_moments.argtypes = [P, P, P, P, C.c_int32, P, P]
        _lib.orc_tree_length.argtypes = [P, C.c_int64, C.c_int]
        _lib.orc_tree_length.restype = C.c_double
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def philox(ctr, key):
    ctr = _c(ctr, np.uint64); key = _c(key, np.uint64)
    out = np.zeros(4, np.uint64)
    lib().orc_philox4x64(_p(ctr), _p(key), _p(out))
    return out


def draw(seed, problem, index, aux, cell, step, pass_, tag):
    out = np.zeros(4, np.uint64)
    lib().orc_draw(seed, problem, index, aux, cell, step, pass_, tag, _p(out))
    return out


def u01(w):
    return lib().orc_u01(int(w))


def u01_open(w):
    return lib().orc_u01_open(int(w))


def below(w, n):
    return lib().orc_below(int(w), int(n))


class _Prp(C.Structure):
    _fields_ = [("n", C.c_uint64), ("b", C.c_int), ("key", C.c_uint64 * 4)]


def prp_table(n, key, inverse=False):
    """Return [pi(0), ..., pi(n-1)] (or the inverse permutation)."""
    p = _Prp()
    k = _c(key, np.uint64)
    lib().orc_prp_init(C.byref(p), n, _p(k))
    f = lib().orc_prp_inv if inverse else lib().orc_prp_fwd
    return np.array([f(C.byref(p), i) for i in range(n)], dtype=np.int64)


def prp_tables(n, keys):
    """Forward tables of many permutations of [0, n): keys [K][4] uint64 ->
    [K][n] int32, row j = [pi_j(0), ..., pi_j(n-1)]."""
    k = np.ascontiguousarray(keys, dtype=np.uint64)
    out = np.zeros((k.shape[0], n), dtype=np.int32)
    lib().orc_prp_tables(n, _p(k), k.shape[0], _p(out))
    return out


def collide_params(dt=0.0, eps=1.0, alpha=0.0, rho_scale=1.0, trunc=TRUNC_FIXED, m=2, m_min=1,
                   m_cap=MCAP, delta1=0.005, delta2=0.01, indicator=IND_PXX, seed=0, wb_length=0):
    """For trunc=TRUNC_WB, m is the shape threshold m_max and wb_length one of LEN_*."""
    return CollideParams(dt, eps, alpha, rho_scale, delta1, delta2, trunc, m, m_min, m_cap,
                         indicator, wb_length, seed)


def tree_length(path, definition):
    """Length of the collision tree stored as Algorithm 4.5's list (k, then
    (j, h) of every node in pre-order) under definition LEN_K/LEN_MIN/LEN_MEAN."""
    a = _c(path, np.int32)
    L = lib().orc_tree_length(_p(a), len(a), definition)
    if L < 0:
        raise ValueError("malformed tree list")
    return L


def collide(v, cell_start, prm, step, m_state=None, cell_param=None, cell_key=None,
            problem_id=0, threads=1):
    """Collision step over all cells.  v: (3, Np) float64 (copied).
    Returns (v_new, reports (n_cells, R_LEN) int64, m_state_new)."""
    v = np.array(v, dtype=np.float64, copy=True)
    cs = _c(cell_start, np.int64)
    nc = len(cs) - 1
    ms = None if m_state is None else np.array(m_state, dtype=np.int32, copy=True)
    cp = None if cell_param is None else _c(cell_param, np.float64)
    ck = None if cell_key is None else _c(cell_key, np.uint64)
    rep = np.zeros((nc, R_LEN), np.int64)
    vx, vy, vz = (np.ascontiguousarray(v[i]) for i in range(3))
    rc = lib().orc_collide(_p(vx), _p(vy), _p(vz), _p(cs), nc, _p(ck), problem_id, step,
                           _p(ms), C.byref(prm), _p(cp), _p(rep), threads)
    if rc == 2:
        raise ValueError("oracle collide: a cell's velocities or energy sum are not finite")
    if rc != 0:
        raise ValueError("oracle collide rejected its arguments")
    return np.stack([vx, vy, vz]), rep, ms


def cfl_dt(v, cell_start, domains, cfl):
    doms = _domains(domains)
    out = np.zeros(len(domains), np.float64)
    vx, vy, vz = (_c(v[i], np.float64) for i in range(3))
    lib().orc_cfl_dt(_p(vx), _p(vy), _p(vz), _p(_c(cell_start, np.int64)), doms, len(domains),
                     cfl, _p(out))
    return out


def transport(x, v, cell_start, domains, dt_dom, step=0, seed=0, problem_id=0, cell_key=None, capacity=None):
    """Free transport + boundaries + stable cell sort.  domains: Domain
    structs or tuples (cell_begin, n_cells, x_lo, x_hi[, bc, res_lo, res_hi,
    particle_mass]).  Returns (x, v, cell_start) of the new particle set."""
    x = np.array(x, dtype=np.float64, copy=True)
    v = np.array(v, dtype=np.float64, copy=True)
    cs = np.array(cell_start, dtype=np.int64, copy=True)
    nc = len(cs) - 1
    cap = int(capacity if capacity is not None else 2 * int(cs[-1]) + 100000)
    doms = _domains(domains)
    dt = _c(dt_dom, np.float64)
    ck = None if cell_key is None else _c(cell_key, np.uint64)
    vx, vy, vz = (np.ascontiguousarray(v[i]) for i in range(3))
    xo = np.zeros(cap); vxo = np.zeros(cap); vyo = np.zeros(cap); vzo = np.zeros(cap)
    cso = np.zeros(nc + 1, np.int64)
    n = lib().orc_transport(_p(x), _p(vx), _p(vy), _p(vz), _p(cs), nc, doms, len(doms), _p(dt), _p(ck), problem_id,
                            seed, step, _p(xo), _p(vxo), _p(vyo), _p(vzo), cap, _p(cso))
    if n == -2:
        raise ValueError("oracle transport: non-finite position, velocity or time step")
    if n < 0:
        raise ValueError("oracle transport: particle count exceeds capacity")
    return xo[:n], np.stack([vxo[:n], vyo[:n], vzo[:n]]), cso


def init_cells(cell_init, cell_start, seed, problem_id=0, cell_key=None, with_x=True):
    ci = _c(cell_init, np.float64).reshape(-1, INIT_COLS)
    cs = _c(cell_start, np.int64)
    nc = len(cs) - 1
    np_ = int(cs[-1])
    vx = np.zeros(np_); vy = np.zeros(np_); vz = np.zeros(np_)
    x = np.zeros(np_) if with_x else None
    ck = None if cell_key is None else _c(cell_key, np.uint64)
    lib().orc_init_cells(_p(ci), _p(cs), nc, _p(ck), problem_id, seed, _p(vx), _p(vy), _p(vz), _p(x))
    return x, np.stack([vx, vy, vz])


def moments(v, cell_start, rho_scale=None):
    cs = _c(cell_start, np.int64)
    nc = len(cs) - 1
    out = np.zeros((nc, MOM_COLS))
    vx, vy, vz = (_c(v[i], np.float64) for i in range(3))
    rs = None if rho_scale is None else _c(rho_scale, np.float64)
    lib().orc_moments(_p(vx), _p(vy), _p(vz), _p(cs), nc, _p(rs), _p(out))
    return out


def report_dict(row):
    d = {f: int(row[i]) for i, f in enumerate(R_FIELDS)}
    d["Nk"] = row[R_NK:R_NK + MCAP + 2].copy()
    d["Ck"] = row[R_CK:R_CK + MCAP + 2].copy()
    d["Dk"] = row[R_DK:R_DK + MCAP + 2].copy()
    return d
