"""Python binding of libtrmc (include/trmc.h): argument marshalling only.

Every function has the name of the C entry point it calls and passes
device pointers of torch tensors plus the current torch CUDA stream.  All
computation happens in the CUDA library; if the library is missing or no
GPU is present, the calls raise instead of falling back to anything else.
"""
import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtrmc.so")

OK, ERR_ARG, ERR_CUDA, ERR_NOMEM, ERR_CAPACITY, ERR_TIMEOUT, ERR_STATE = range(7)
FP64, FP32_MIXED = 0, 1
TRUNC_FIXED, TRUNC_RAD, TRUNC_UNLIMITED, TRUNC_WB = 0, 1, 2, 3
LEN_K, LEN_MIN, LEN_MEAN = 1, 2, 3
IND_PXX, IND_M4 = 0, 1
INIT_MAXWELL, INIT_BIMAXWELL, INIT_BKW = 0, 1, 2
MCAP = 64
INIT_COLS = 9
MOM_COLS = 10
REPORT_LEN = 16 + 3 * (MCAP + 2)
REPORT_FIELDS = ["N", "passes", "m_first", "m_last", "m_next", "R_final", "N0", "leaves",
                 "coll", "dummy", "exceed", "feas", "pdrop", "psurp", "m_eff0", "wbrej"]
EXPORTS = ["trmc_create", "trmc_destroy", "trmc_last_error", "trmc_check", "trmc_init_cells",
           "trmc_collide", "trmc_transport", "trmc_moments", "trmc_collide_static", "trmc_set_collide_launch",
           "trmc_set_transport_launch", "trmc_set_collide_schedule",
           "trmc_fp64_selftest", "trmc_split_selftest"]
STATIC_SCRATCH_BYTES = 32 << 20


class TrmcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"trmc status {code}: {msg}")
        self.code = code


class CellParam(C.Structure):
    _fields_ = [("eps", C.c_double), ("dt", C.c_double), ("rho_scale", C.c_double), ("alpha", C.c_double)]


class State(C.Structure):
    _fields_ = [("vx", C.c_void_p), ("vy", C.c_void_p), ("vz", C.c_void_p), ("x", C.c_void_p),
                ("vx_alt", C.c_void_p), ("vy_alt", C.c_void_p), ("vz_alt", C.c_void_p), ("x_alt", C.c_void_p),
                ("cell_start", C.c_void_p), ("cell_start_alt", C.c_void_p), ("m_max", C.c_void_p),
                ("cell_param", C.c_void_p), ("cell_key", C.c_void_p), ("cell_vmax2", C.c_void_p),
                ("step_dev", C.c_void_p), ("cell_order", C.c_void_p), ("cell_carry", C.c_void_p), ("cell_cost", C.c_void_p),
                ("capacity", C.c_int64), ("n_cells", C.c_int32), ("problem_id", C.c_uint32)]


class CollideParams(C.Structure):
    _fields_ = [("dt", C.c_double), ("eps", C.c_double), ("alpha", C.c_double), ("rho_scale", C.c_double),
                ("delta1", C.c_double), ("delta2", C.c_double), ("trunc", C.c_int32), ("m_fixed", C.c_int32),
                ("m_min", C.c_int32), ("m_cap", C.c_int32), ("indicator", C.c_int32), ("wb_length", C.c_int32)]


BC_SPECULAR, BC_RESERVOIR = 0, 1


class Domain(C.Structure):
    _fields_ = [("cell_begin", C.c_int32), ("n_cells", C.c_int32), ("x_lo", C.c_double), ("x_hi", C.c_double),
                ("bc", C.c_int32), ("reserved", C.c_int32), ("res_lo", C.c_double * 3), ("res_hi", C.c_double * 3),
                ("particle_mass", C.c_double)]


def domains_tensor(domains, device="cuda"):
    """Device array of trmc_domain from Domain structs or tuples
    (cell_begin, n_cells, x_lo, x_hi[, bc, res_lo, res_hi, particle_mass])."""
    import torch
    arr = (Domain * len(domains))()
    for i, d in enumerate(domains):
        if isinstance(d, Domain):
            arr[i] = d
            continue
        bc = d[4] if len(d) > 4 else BC_SPECULAR
        rlo = d[5] if len(d) > 5 else (0.0, 0.0, 0.0)
        rhi = d[6] if len(d) > 6 else (0.0, 0.0, 0.0)
        mass = d[7] if len(d) > 7 else 0.0
        arr[i] = Domain(d[0], d[1], d[2], d[3], bc, 0, (C.c_double * 3)(*rlo), (C.c_double * 3)(*rhi), mass)
    raw = np.frombuffer(bytes(arr), dtype=np.uint8).copy()
    return torch.as_tensor(raw).to(device)


class Stats(C.Structure):
    _fields_ = [(f, C.c_ulonglong) for f in
                ("collisions", "dummy", "maxwell", "exceed", "passes", "feas", "cells", "capacity_skips",
                 "changed", "particles", "wb_rejected")]


STATS_FIELDS = [f for f, _ in Stats._fields_]
_lib = None


def load():
    """Load libtrmc.so (built by build.py); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_1009_2768_gb300.build.build() first")
        lib = C.CDLL(LIB_PATH)
        P = C.c_void_p
        lib.trmc_create.argtypes = [C.POINTER(P), C.c_int32, C.c_uint64, C.c_size_t]
        lib.trmc_destroy.argtypes = [P]
        lib.trmc_last_error.argtypes = [P]
        lib.trmc_last_error.restype = C.c_char_p
        lib.trmc_check.argtypes = [P, P]
        lib.trmc_init_cells.argtypes = [P, C.POINTER(State), P, P]
        lib.trmc_collide.argtypes = [P, C.POINTER(State), C.POINTER(CollideParams), C.c_uint64, P, P, P]
        lib.trmc_transport.argtypes = [P, C.POINTER(State), P, C.c_int32, C.c_double, P, C.c_uint64, P]
        lib.trmc_moments.argtypes = [P, C.POINTER(State), P, P]
        lib.trmc_set_collide_launch.argtypes = [P, C.c_int32, C.c_int32]
        lib.trmc_set_transport_launch.argtypes = [P, C.c_int32]
        lib.trmc_set_collide_schedule.argtypes = [P, C.c_int32, C.c_int32]
        lib.trmc_collide_static.argtypes = [C.POINTER(State), C.POINTER(CollideParams), C.c_int32, C.c_uint64,
                                            C.c_uint64, C.c_int32, P, P]
        lib.trmc_fp64_selftest.argtypes = [P, C.c_int32, P, P]
        lib.trmc_split_selftest.argtypes = [P, P, P, C.c_int32, P, P]
        for f in EXPORTS:
            if f != "trmc_last_error":
                getattr(lib, f).restype = C.c_int
        _lib = lib
    return _lib


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _raise(ctx, code):
    if code != OK:
        msg = load().trmc_last_error(ctx).decode() if ctx else "no context"
        raise TrmcError(code, msg)


def trmc_create(precision=FP64, seed=0, workspace_bytes=0):
    ctx = C.c_void_p()
    code = load().trmc_create(C.byref(ctx), precision, seed, workspace_bytes)
    if code != OK:
        raise TrmcError(code, "trmc_create failed")
    return ctx


def trmc_destroy(ctx):
    _raise(None, load().trmc_destroy(ctx))


def trmc_check(ctx, stream=None):
    _raise(ctx, load().trmc_check(ctx, _stream(stream)))


def trmc_set_collide_launch(ctx, threads, ctas_per_sm):
    _raise(ctx, load().trmc_set_collide_launch(ctx, threads, ctas_per_sm))


def trmc_set_collide_schedule(ctx, warp_particles, records_per_thread):
    _raise(ctx, load().trmc_set_collide_schedule(ctx, warp_particles, records_per_thread))


def trmc_set_transport_launch(ctx, threads):
    _raise(ctx, load().trmc_set_transport_launch(ctx, threads))


def trmc_init_cells(ctx, state, cell_init, stream=None):
    _raise(ctx, load().trmc_init_cells(ctx, C.byref(state.c), _ptr(cell_init), _stream(stream)))


def trmc_collide(ctx, state, params, step, report=None, stats=None, stream=None):
    _raise(ctx, load().trmc_collide(ctx, C.byref(state.c), C.byref(params), step, _ptr(report), _ptr(stats),
                                    _stream(stream)))


def trmc_transport(ctx, state, domains, n_domains, cfl, dt, step=0, stream=None):
    code = load().trmc_transport(ctx, C.byref(state.c), _ptr(domains), n_domains, cfl, _ptr(dt), step,
                                 _stream(stream))
    state.after_transport()
    _raise(ctx, code)


def trmc_moments(ctx, state, out, stream=None):
    _raise(ctx, load().trmc_moments(ctx, C.byref(state.c), _ptr(out), _stream(stream)))


def trmc_collide_static(state, params, precision, seed, step, max_cell_particles, status=None, stream=None):
    """Collision step that allocates nothing (no context; scratch is a fixed
    device array inside the library).  status: optional int32 device tensor
    of 2 that receives device-detected errors (code, first cell)."""
    code = load().trmc_collide_static(C.byref(state.c), C.byref(params), precision, seed, step,
                                      max_cell_particles, _ptr(status), _stream(stream))
    if code != OK:
        why = {ERR_ARG: "invalid argument", ERR_CAPACITY: "a cell of max_cell_particles does not fit the static "
               f"scratch of {STATIC_SCRATCH_BYTES >> 20} MiB", ERR_CUDA: "CUDA call failed"}.get(code, "error")
        raise TrmcError(code, f"trmc_collide_static: {why}")


def trmc_fp64_selftest(words, out, stream=None):
    """words: uint64 (as int64) device tensor [n]; out: float64 device tensor [n, 8]."""
    code = load().trmc_fp64_selftest(_ptr(words), words.numel(), _ptr(out), _stream(stream))
    if code != OK:
        raise TrmcError(code, "trmc_fp64_selftest failed")


def trmc_split_selftest(q, R, K, out, stream=None):
    """q: float64, R: int32, K: uint64 (as int64), out: int32 device tensors [n]."""
    code = load().trmc_split_selftest(_ptr(q), _ptr(R), _ptr(K), q.numel(), _ptr(out), _stream(stream))
    if code != OK:
        raise TrmcError(code, "trmc_split_selftest failed")


# ---------------------------------------------------------------- helpers
def collide_params(dt=0.0, eps=1.0, alpha=0.0, rho_scale=1.0, trunc=TRUNC_FIXED, m=2, m_min=1, m_cap=MCAP,
                   delta1=0.005, delta2=0.01, indicator=IND_PXX, wb_length=0):
    """trunc=TRUNC_WB: m is the shape threshold m_max and wb_length one of LEN_*."""
    return CollideParams(dt, eps, alpha, rho_scale, delta1, delta2, trunc, m, m_min, m_cap, indicator, wb_length)


class ParticleState:
    """Device arrays of one particle state (torch tensors) and the C struct
    that names them.  After trmc_transport the roles of the primary and
    *_alt arrays swap; after_transport() keeps the tensors in step."""

    def __init__(self, cell_start, capacity=None, precision=FP64, with_x=False, rad=False,
                 cell_param=None, cell_key=None, problem_id=0, carry=False, vmax=True, device="cuda"):
        import torch
        cs = torch.as_tensor(np.asarray(cell_start, dtype=np.int64)).to(device)
        n_cells = cs.numel() - 1
        n = int(cs[-1].item()) if capacity is None else int(capacity)
        # a whole number of 16-byte vectors per array (every row of v then starts
        # 16-byte aligned, and the transport reads the particles as vectors)
        n = -(-n // 4) * 4
        dt = torch.float64 if precision == FP64 else torch.float32
        self.precision = precision
        self.v = torch.zeros((3, max(n, 1)), dtype=dt, device=device)
        self.x = torch.zeros(max(n, 1), dtype=dt, device=device) if with_x else None
        self.v_alt = torch.zeros_like(self.v) if with_x else None
        self.x_alt = torch.zeros_like(self.x) if with_x else None
        self.cell_start = cs
        self.cell_start_alt = torch.zeros_like(cs) if with_x else None
        self.m_max = torch.full((max(n_cells, 1),), 2, dtype=torch.int32, device=device) if rad else None
        self.cell_param = None
        if cell_param is not None:
            cp = np.asarray(cell_param, dtype=np.float64).reshape(n_cells, 4)
            self.cell_param = torch.as_tensor(cp).to(device)
        self.cell_key = None if cell_key is None else torch.as_tensor(
            np.asarray(cell_key, dtype=np.uint64).view(np.int64)).to(device)
        # per-cell max |v|^2 after each collide: the CFL time step of a transport
        # needs it; homogeneous problems can leave it out (vmax=False) and save
        # the collide step its pass over the final velocities
        self.cell_vmax2 = torch.zeros(max(n_cells, 1), dtype=torch.float64, device=device) if vmax else None
        self.device = device
        self.cell_carry = torch.zeros((max(n_cells, 1), 4), dtype=torch.float64, device=device) if carry else None
        self.step_dev = None           # device step counter (use_device_step)
        self.cell_order = None         # cell processing order (set_cell_order)
        self.cell_cost = None          # measured per-cell time (use_adaptive_order)
        self.n_cells = n_cells
        self.capacity = n
        self.c = State()
        self.c.capacity = n
        self.c.n_cells = n_cells
        self.c.problem_id = problem_id
        self._fill()

    def _fill(self):
        c = self.c
        c.vx, c.vy, c.vz = (self.v[i].data_ptr() for i in range(3))
        c.x = self.x.data_ptr() if self.x is not None else None
        if self.v_alt is not None:
            c.vx_alt, c.vy_alt, c.vz_alt = (self.v_alt[i].data_ptr() for i in range(3))
            c.x_alt = self.x_alt.data_ptr()
            c.cell_start_alt = self.cell_start_alt.data_ptr()
        c.cell_start = self.cell_start.data_ptr()
        c.m_max = self.m_max.data_ptr() if self.m_max is not None else None
        c.cell_param = self.cell_param.data_ptr() if self.cell_param is not None else None
        c.cell_key = self.cell_key.data_ptr() if self.cell_key is not None else None
        c.cell_vmax2 = self.cell_vmax2.data_ptr() if self.cell_vmax2 is not None else None
        c.cell_carry = self.cell_carry.data_ptr() if self.cell_carry is not None else None
        c.step_dev = self.step_dev.data_ptr() if self.step_dev is not None else None
        c.cell_order = self.cell_order.data_ptr() if self.cell_order is not None else None
        c.cell_cost = self.cell_cost.data_ptr() if self.cell_cost is not None else None

    def use_device_step(self, start=0):
        """Key the collision draws with a device counter that each trmc_collide
        advances, so that captured CUDA graphs step on replay."""
        import torch
        self.step_dev = torch.full((1,), start, dtype=torch.int64, device=self.device)
        self._fill()

    def use_adaptive_order(self):
        """Let every collide launch hand out the cells longest first, by the
        times the previous launch measured (identity order at the start)."""
        import torch
        dev = self.device
        self.cell_cost = torch.zeros(max(self.n_cells, 1), dtype=torch.int32, device=dev)
        self.cell_order = torch.arange(max(self.n_cells, 1), dtype=torch.int32, device=dev)
        self._fill()

    def set_cell_order(self, order):
        import torch
        self.cell_order = torch.as_tensor(np.asarray(order, dtype=np.int32)).to(self.device)
        self._fill()

    def after_transport(self):
        if self.c.vx == self.v_alt[0].data_ptr():
            self.v, self.v_alt = self.v_alt, self.v
            self.x, self.x_alt = self.x_alt, self.x
            self.cell_start, self.cell_start_alt = self.cell_start_alt, self.cell_start
        self._fill()

    def set_velocities(self, v):
        import torch
        self.v[:, :v.shape[1]].copy_(torch.as_tensor(np.asarray(v)).to(self.v.dtype))

    def set_positions(self, x):
        import torch
        self.x[:len(x)].copy_(torch.as_tensor(np.asarray(x)).to(self.x.dtype))


def report_dict(row):
    row = np.asarray(row)
    d = {f: int(row[i]) for i, f in enumerate(REPORT_FIELDS)}
    d["Nk"] = row[16:16 + MCAP + 2].copy()
    d["Ck"] = row[16 + MCAP + 2:16 + 2 * (MCAP + 2)].copy()
    d["Dk"] = row[16 + 2 * (MCAP + 2):16 + 3 * (MCAP + 2)].copy()
    return d
