"""The C ABI library builds for sm_103a, loads without a GPU and exports
every entry point declared in include/trmc.h; the binding refuses to run
without the library (no fallback)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "trmc.h")).read()
    return sorted(set(re.findall(r"^\s*(?:trmc_status|const char \*)\s*(trmc_\w+)\s*\(", src, re.M)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("trmc_init_cells", "trmc_collide", "trmc_transport", "trmc_moments",
              "trmc_create", "trmc_destroy", "trmc_last_error", "trmc_check"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1009_2768_gb300 import build
    lib = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(trmc_\w+)$", out, re.M))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing
    import ctypes
    so = ctypes.CDLL(lib)            # loads without a GPU: no CUDA call at load time
    for n in declared():
        assert hasattr(so, n)
    from paper_1009_2768_gb300 import trmc
    assert sorted(trmc.EXPORTS) == declared()


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1009_2768_gb300 import trmc
    monkeypatch.setattr(trmc, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(trmc, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        trmc.trmc_create(trmc.FP64, 0, 0)


def test_struct_layouts_match_header():
    import ctypes
    from paper_1009_2768_gb300 import trmc
    assert ctypes.sizeof(trmc.State) == 18 * 8 + 8 + 4 + 4
    assert ctypes.sizeof(trmc.CollideParams) == 6 * 8 + 6 * 4
    assert ctypes.sizeof(trmc.Domain) == 88
    assert ctypes.sizeof(trmc.CellParam) == 32
    assert ctypes.sizeof(trmc.Stats) == 88


def test_static_entry_point_checks_parameters_on_the_host():
    """trmc_collide_static makes trmc_collide's host checks before any CUDA
    call: invalid parameters come back as TRMC_ERR_ARG, on a machine without
    a GPU too (valid ones get as far as the first CUDA call)."""
    import ctypes
    import math
    from paper_1009_2768_gb300 import build, trmc as T
    build.build()
    lib = T.load()
    st = T.State()
    st.vx = st.vy = st.vz = st.cell_start = st.m_max = 256      # never dereferenced on the host
    st.n_cells, st.capacity = 1, 10

    def code(**kw):
        p = T.collide_params(dt=0.05, eps=1.0, alpha=1.0, rho_scale=0.01, trunc=T.TRUNC_RAD, m=2)
        for k, v in kw.items():
            setattr(p, k, v)
        return lib.trmc_collide_static(ctypes.byref(st), ctypes.byref(p), T.FP64, 0, 0, 100, None, None)

    for bad in ({"rho_scale": -1.0}, {"rho_scale": math.nan}, {"indicator": 7}, {"eps": 0.0}, {"dt": -1.0},
                {"alpha": 1.5}, {"m_cap": 0}, {"m_min": 0}, {"delta2": 0.001}, {"trunc": 9}, {"wb_length": 2}):
        assert code(**bad) == T.ERR_ARG, bad
    assert code() != T.ERR_ARG
