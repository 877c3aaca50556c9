"""Shared helpers of the GPU tests: run the CUDA library through the C ABI
(binding in paper_1009_2768_gb300.trmc) and the CPU oracle on the same
seeded inputs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1009_2768_gb300 import trmc as T  # noqa: E402

TOL_V = 1e-12          # relative velocity tolerance of the FP64 parity contract


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def ensure_built():
    from paper_1009_2768_gb300 import build
    build.build()


_ctx = {}


def ctx(precision=T.FP64, seed=0, workspace=256 << 20):
    key = (precision, seed, workspace)
    if key not in _ctx:
        ensure_built()
        _ctx[key] = T.trmc_create(precision, seed, workspace)
    return _ctx[key]


def gpu_collide(v, cell_start, params, step, precision=T.FP64, seed=0, m_state=None, cell_param=None,
                cell_key=None, problem_id=0, workspace=256 << 20, want_report=True, stats=False, launch=None):
    """One trmc_collide on a cached context; launch = (threads, CTAs per SM)
    for this call only (the context's default, 128 x 4, otherwise)."""
    st = T.ParticleState(cell_start, precision=precision, rad=m_state is not None, cell_param=cell_param,
                         cell_key=cell_key, problem_id=problem_id)
    st.set_velocities(v)
    if m_state is not None:
        st.m_max.copy_(torch.as_tensor(np.asarray(m_state, np.int32)))
    c = ctx(precision, seed, workspace)
    rep = torch.zeros((max(st.n_cells, 1), T.REPORT_LEN), dtype=torch.int64, device="cuda") if want_report else None
    stt = torch.zeros(len(T.STATS_FIELDS), dtype=torch.int64, device="cuda") if stats else None
    if launch is not None:
        T.trmc_set_collide_launch(c, *launch)
    try:
        T.trmc_collide(c, st, params, step, report=rep, stats=stt)
        T.trmc_check(c)
    finally:
        if launch is not None:
            T.trmc_set_collide_launch(c, 128, 4)
    out = {"v": st.v[:, :int(cell_start[-1])].double().cpu().numpy(),
           "report": rep.cpu().numpy()[:st.n_cells] if want_report else None,
           "m_state": st.m_max.cpu().numpy() if m_state is not None else None,
           "vmax2": st.cell_vmax2.cpu().numpy()[:st.n_cells],
           "stats": dict(zip(T.STATS_FIELDS, stt.cpu().numpy().tolist())) if stats else None}
    return out


def oracle_params(O, p):
    return O.collide_params(dt=p.dt, eps=p.eps, alpha=p.alpha, rho_scale=p.rho_scale, trunc=p.trunc, m=p.m_fixed,
                            m_min=p.m_min, m_cap=p.m_cap, delta1=p.delta1, delta2=p.delta2, indicator=p.indicator,
                            seed=0, wb_length=p.wb_length)


def assert_velocity_parity(v_gpu, v_orc, cell_start, tol=TOL_V):
    for c in range(len(cell_start) - 1):
        a, b = cell_start[c], cell_start[c + 1]
        if b == a:
            continue
        scale = max(1.0, np.abs(v_orc[:, a:b]).max())
        err = np.abs(v_gpu[:, a:b] - v_orc[:, a:b]).max()
        assert err <= tol * scale, f"cell {c}: max |dv| = {err:.3e} (scale {scale:.3g})"
