#!/usr/bin/env python
"""Benchmark of the TRMC-R hot path on GB300: one step = free transport with
inflow/outflow reservoirs + stable cell sort + collision step (split,
recursive trees, VHS hard-sphere acceptance, Maxwellian renormalisation,
TRMC-RAD) over the Mach 3 stationary normal shock: 4000 cells of 2500
particles on average (1e7 particles), eps 1e-3, CFL 0.5, FP32 velocities
with FP64 moments.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload stationary|shock|batched|bkw|serving]

--workload selects the step timed (default stationary, the benchmark line):
  stationary  the Mach 3 stationary shock above (FP32-mixed);
  shock   four 1D Riemann shock tubes on [0,1] (one per Knudsen number 1e-1,
          1e-2, 1e-3, 1e-4), 400 cells x 500 particles per cell, specular
          walls, CFL 0.5, FP64;
  batched 4096 independent homogeneous cells, 64..8192 particles log-uniform,
          bi-Maxwellian, VHS alpha 0.6, eps log-uniform 1e-4..10, FP32-mixed;
  bkw     one homogeneous cell of 1e5 Maxwell molecules from BKW data, FP64;
  serving a stream of solve requests (shock tubes and homogeneous relaxations,
          1e5..2e7 particles log-uniform, eps 1e-4..1 log-uniform, FP32-mixed)
          arriving as a Poisson process, swept over --rates requests/s,
          admitted against a 150 GB HBM budget; reports p50/p99 latency and
          particle-steps/s per rate (value: the highest rate's throughput).

Every line states the moment error of the timed form against the FP64 CPU
oracle: the GPU form and the oracle step the same initial state with the same
keys for a few steps, and the oracle with other keys gives the Monte Carlo
noise floor of the same measure; the plain FP64 form of the same workload is
measured beside it (forms).

N > 1 runs N independent replicas (one per rank, launched by torchrun), each
on its own problem ids; value is the total over ranks.  --impl reference
times the CPU oracle (FP64, all host cores) on a bounded sample of the same
workload.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

EPS = (1e-1, 1e-2, 1e-3, 1e-4)
N_CELLS, MEAN = 400, 500
WORKLOAD = ("1D Riemann shock tube on [0,1] (rho 1/0.125, T 1/0.8, u 0), hard-sphere VHS, specular walls, "
            "CFL 0.5, TRMC-RAD (P_xx indicator, delta 0.005/0.01, m0 2); 4 tubes x 400 cells x 500 "
            "particles/cell mean, eps 1e-1/1e-2/1e-3/1e-4, FP64")
METRIC = "particle-steps/s"
DEFAULT_WORKLOAD = "stationary"
COMPARE_STEPS = 20          # steps of the oracle comparison (moment error, CPU baseline)

# Per collide launch, from `ncu` on the same command (one whole-staging launch of the
# stationary shock and the shock tubes, one dual launch of the batched relaxation): DRAM
# traffic (dram__bytes_read.sum + dram__bytes_write.sum), issue and warp activity and the
# leading stall reasons, keyed by the hash of csrc/collide.cu they were taken on; reported
# as null once the kernel source differs.  See profiles/.
NCU_TRAFFIC = {
    "stationary": {"collide_sha": "674f83b37ff2bfd5", "launch": (256, 3), "bytes": 121820928 + 65572352,
              "issue_active_pct": 34.1, "warps_active_pct": 36.7,
              "stalls_per_issue": {"barrier": 7.15, "no_instruction": 3.44, "wait": 2.30, "long_scoreboard": 1.15}},
    "shock": {"collide_sha": "674f83b37ff2bfd5", "launch": (128, 4), "bytes": 19977728 + 96768,
              "issue_active_pct": 17.7, "warps_active_pct": 22.8,
              "stalls_per_issue": {"barrier": 7.06, "wait": 3.99, "short_scoreboard": 3.66, "no_instruction": 3.06}},
    "batched": {"collide_sha": "674f83b37ff2bfd5", "launch": (256, 2), "bytes": 83151104 + 24946944,
              "issue_active_pct": 30.9, "warps_active_pct": 24.8,
              "stalls_per_issue": {"barrier": 5.12, "wait": 2.35, "no_instruction": 1.22, "long_scoreboard": 1.05}},
}

# Collide launch shape (threads per CTA, CTAs per SM) per workload: the fastest of
# runtime.autotune_collide's candidates on GB300 (--tune measures them again).
LAUNCH = {"shock": (128, 4), "stationary": (256, 3), "batched": (256, 2), "bkw": (512, 1)}


def collide_sha():
    """Hash of the collide kernel's code: its sources with comments and
    whitespace removed, so that an edit of comments alone keeps the ncu
    records valid while any change of code voids them."""
    h = hashlib.sha256()
    for f in ("collide.cu", "trmc_device.cuh", "fp64_tables.inc"):
        src = open(os.path.join(ROOT, "paper_1009_2768_gb300", "csrc", f)).read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.out = None

    def start(self):
        try:
            self.out = open(os.devnull if False else f"/tmp/trmc_clocks_{os.getpid()}.csv", "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.gpu)], stdout=self.out,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        self.proc.wait()
        self.out.close()
        rows = []
        for line in open(self.out.name):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.out.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(ms, dist=None):
    """The slowest rank's time (all ranks get it); the input itself without a
    process group.  A device tensor under NCCL, a host tensor otherwise."""
    if dist is None:
        return ms
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(n_per_rank, world, steps, total_ms):
    """Whole-job particle-steps/s of `world` independent replicas of n
    particles each, over `steps` steps timed by the slowest rank."""
    return n_per_rank * world * steps / (total_ms / 1e3)


# ------------------------------------------------------------------ CPU oracle
def oracle_tube_rate(n_cells, mean, steps, threads, seed=0, budget_s=None):
    """Particle-steps/s of the FP64 CPU oracle on one shock tube (eps 1e-2)."""
    from oracle import oracle as O
    from paper_1009_2768_gb300 import synth
    counts = synth.shock_tube_counts(n_cells, mean)
    cs = synth.starts(counts)
    n = int(cs[-1])
    ci = np.zeros((n_cells, O.INIT_COLS))
    for c in range(n_cells):
        ci[c] = [O.INIT_MAXWELL, 0, 0, 0, 1.0 if c < n_cells // 2 else 0.8, 0, 0, c / n_cells, (c + 1) / n_cells]
    x, v = O.init_cells(ci, cs, seed)
    rho_scale = 0.5625 * n_cells / n
    cp = np.tile([1e-2, 0.0, rho_scale, 1.0], (n_cells, 1))
    prm = O.collide_params(trunc=O.TRUNC_RAD, m=2, seed=seed)
    ms = np.full(n_cells, 2, np.int32)
    doms = [(0, n_cells, 0.0, 1.0)]
    done, t0 = 0, time.perf_counter()
    for s in range(steps):
        dt = O.cfl_dt(v, cs, doms, 0.5)
        x, v, cs = O.transport(x, v, cs, doms, dt)
        cp[:, 1] = dt[0]
        v, _, ms = O.collide(v, cs, prm, s, m_state=ms, cell_param=cp.ravel(), threads=threads)
        done += 1
        if budget_s is not None and time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    return n * done / el, n, done, el


def oracle_workload(workload, threads, seed=0):
    """The FP64 CPU oracle set up on a bounded sample of a workload other
    than the shock tubes, with the oracle's own initial-data sampler: returns
    (step function, particles, sample description, threads used).  Same
    generators and parameters as workloads.py."""
    from oracle import oracle as O
    from paper_1009_2768_gb300 import synth
    from paper_1009_2768_gb300.workloads import rankine_hugoniot
    if workload == "batched":
        # the first 512 of the 4096 cells (same log-uniform counts, eps and anisotropy)
        g = synth.rng(seed)
        counts = synth.loguniform_ints(4096, 64, 8192, g=g)
        eps = synth.loguniform(4096, 1e-4, 10.0, g=g)
        ratio = g.uniform(0.3, 3.0, 4096)
        k = 512
        counts, eps, ratio = counts[:k], eps[:k], ratio[:k]
        t_perp = 3.0 / (ratio + 2.0)
        cs = synth.starts(counts)
        ci = np.zeros((k, O.INIT_COLS))
        ci[:, 0] = O.INIT_BIMAXWELL
        ci[:, 4] = ratio * t_perp
        ci[:, 5] = t_perp
        keys = np.arange(k, dtype=np.uint64) << np.uint64(32)
        _, v = O.init_cells(ci, cs, seed, cell_key=keys, with_x=False)
        cp = np.stack([eps, np.full(k, 0.05), 1.0 / counts, np.full(k, 0.6)], axis=1)
        prm = O.collide_params(trunc=O.TRUNC_RAD, m=2, seed=seed)
        ms = np.full(k, 2, np.int32)
        n = int(cs[-1])
        desc = f"cells 0..511 of the 4096 ({n} particles), collide steps"
        def step(s):
            nonlocal v, ms
            v, _, ms = O.collide(v, cs, prm, s, m_state=ms, cell_param=cp.ravel(), cell_key=keys, threads=threads)
    elif workload == "stationary":
        # the whole stationary shock (4000 cells + 2 reservoir ghosts, 1e7 particles), first steps
        left, right = rankine_hugoniot(3.0)
        nc0, mean = 4000, 2500
        dx, mass = 1.0 / nc0, (0.5 * left[0] + 0.5 * right[0]) / (nc0 * mean)
        nc = nc0 + 2
        counts = np.empty(nc, np.int64)
        ci = np.zeros((nc, O.INIT_COLS))
        for c in range(nc):
            rho, u, Tm = left if (c - 0.5) * dx < 0.5 else right
            counts[c] = int(round(rho * dx / mass))
            ci[c] = [O.INIT_MAXWELL, u, 0, 0, Tm, 0, 0, (c - 1) * dx, c * dx]
        cs = synth.starts(counts)
        x, v = O.init_cells(ci, cs, seed)
        cp = np.zeros((nc, 4))
        cp[:, 0] = 1e-3
        cp[[0, -1], 0] = 1e300
        cp[:, 2] = mass / dx
        cp[:, 3] = 1.0
        doms = [O.domain(0, nc, 0.0, 1.0, O.BC_RESERVOIR, left, right, mass)]
        prm = O.collide_params(trunc=O.TRUNC_RAD, m=2, seed=seed)
        ms = np.full(nc, 2, np.int32)
        n = int(cs[-1])
        desc = f"the whole stationary shock ({n} particles), transport + collide, first steps"
        def step(s):
            nonlocal x, v, cs, ms
            dt = O.cfl_dt(v, cs, doms, 0.5)
            x, v, cs = O.transport(x, v, cs, doms, dt, step=s, seed=seed, capacity=int(1.25 * n) + 4 * mean)
            cp[:, 1] = dt[0]
            v, _, ms = O.collide(v, cs, prm, s, m_state=ms, cell_param=cp.ravel(), threads=threads)
    else:                                   # bkw: one cell of 1e5, single-threaded like the workload's one CTA
        n = 100000
        cs = np.array([0, n], np.int64)
        ci = np.array([[O.INIT_BKW, 0, 0, 0, 1.0, 0, 0.6, 0, 1]], np.float64)
        _, v = O.init_cells(ci, cs, seed, with_x=False)
        prm = O.collide_params(dt=0.05, eps=1.0, alpha=0.0, rho_scale=1.0 / n, trunc=O.TRUNC_RAD, m=2,
                               indicator=O.IND_M4, seed=seed)
        ms = np.full(1, 2, np.int32)
        threads = 1
        desc = "the BKW cell (1e5 particles), collide steps, one thread"
        def step(s):
            nonlocal v, ms
            v, _, ms = O.collide(v, cs, prm, s, m_state=ms, threads=1)
    return step, n, desc, threads


def reference_arm(args):
    """The CPU oracle, as it stands, on the machine's host cores, on a bounded
    sample of the workload the GPU arm times: W untimed steps, then K timed."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle.build import build_oracle
    build_oracle()
    threads = os.cpu_count() or 1
    wl = args.workload
    if wl == "serving":
        print(json.dumps({"impl": "reference", "unavailable": "the serving stream has no CPU-oracle form: "
                          "requests are timed end to end on the GPU only"}))
        return
    if wl == "shock":
        # one tube, cells scaled so that W + K steps take about two minutes
        rate, n, _, el = oracle_tube_rate(40, MEAN, 2, threads)
        per_step = n / rate
        cells = int(np.clip(40 * 120.0 / max(per_step * (args.steps + args.warmup) * 10, 1e-9), 8, N_CELLS))
        cells -= cells % 2
        oracle_tube_rate(cells, MEAN, args.warmup, threads)
        rate, n, done, el = oracle_tube_rate(cells, MEAN, args.steps, threads)
        sample = f"one tube (eps 1e-2) of {cells} cells x {MEAN}/cell mean ({n} particles), {done} steps"
        used = threads
    else:
        step, n, desc, used = oracle_workload(wl, threads)
        for s in range(args.warmup):
            step(s)
        t0 = time.perf_counter()
        for s in range(args.steps):
            step(args.warmup + s)
        el = time.perf_counter() - t0
        done = args.steps
        rate = n * done / el
        sample = f"{desc}: {args.warmup} untimed + {done} timed steps in {el:.1f} s"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": rate, "unit": METRIC, "n_gpus": args.gpus,
        "steps": done, "warmup": args.warmup, "ms_per_step": 1e3 * el / done, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[wl], "sample": sample},
        "cpu_baseline": {"value": rate, "unit": METRIC, "cores": used, "cpu_model": cpu_model(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": rate, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


# ------------------------------------------------------------------ GPU arm
WORKLOADS = {
    "shock": WORKLOAD,
    "batched": ("batched homogeneous relaxation: 4096 independent cells, 64..8192 particles log-uniform, "
                "bi-Maxwellian T_par/T_perp in [0.3,3], VHS alpha 0.6, eps log-uniform 1e-4..10, dt 0.05, "
                "TRMC-RAD, FP32-mixed"),
    "bkw": "homogeneous Maxwell molecules, one cell of 1e5 particles, BKW K0 0.6, eps 1, dt 0.05, TRMC-RAD (M4), FP64",
    "stationary": ("1D stationary normal shock, Mach 3, 4000 cells x 2500 particles/cell mean (1e7), hard-sphere "
                   "VHS, eps 1e-3, Rankine-Hugoniot inflow/outflow reservoirs, CFL 0.5, TRMC-RAD, FP32-mixed"),
    "serving": ("serving stream: Poisson arrivals of shock-tube (500 particles/cell, specular walls) and homogeneous-"
                "relaxation (cells 64..8192 log-uniform, bi-Maxwellian) solves, 1e5..2e7 particles log-uniform, eps "
                "1e-4..1 log-uniform, state resident on the device, 150 GB HBM budget, TRMC-RAD, FP32-mixed"),
}


def make_sim(workload, seed, precision=None):
    """The workload's simulation on the GPU (its own precision unless one is
    given), with its data type label."""
    from paper_1009_2768_gb300 import trmc as T
    from paper_1009_2768_gb300.workloads import BatchedRelaxation, HomogeneousBKW, ShockTubes, StationaryShock
    own = {"stationary": T.FP32_MIXED, "shock": T.FP64, "batched": T.FP32_MIXED, "bkw": T.FP64}[workload]
    prec = own if precision is None else precision
    label = "f64" if prec == T.FP64 else "f32 velocities, f64 moments"
    rb = 8 if prec == T.FP64 else 4
    if workload == "stationary":
        return StationaryShock(4000, 2500, precision=prec, seed=seed, order="adaptive"), rb, label
    if workload == "shock":
        return ShockTubes(EPS, N_CELLS, MEAN, precision=prec, seed=seed, order="adaptive"), rb, label
    if workload == "batched":
        return BatchedRelaxation(precision=prec, seed=seed, order="adaptive"), rb, label
    return HomogeneousBKW(100000, precision=prec, seed=seed), rb, label


def time_steps(sim, K, flush, stats=None):
    """K steps, each bracketed by CUDA events on the current stream, with an
    L2 flush before each; returns per-step (transport, collide) ms arrays."""
    import torch
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    for k in range(K):
        flush.zero_()
        sim.step(stats=stats, events=ev[k])
    torch.cuda.synchronize()
    tr = np.array([ev[k][0].elapsed_time(ev[k][1]) for k in range(K)])
    co = np.array([ev[k][1].elapsed_time(ev[k][2]) for k in range(K)])
    return tr, co


def time_graph_steps(sim, K, flush, stats):
    """K steps of a workload without transport, each one replay of a
    captured single-step CUDA graph (cell order + collide), bracketed by
    CUDA events, with an L2 flush before each; (transport, collide) ms."""
    import torch
    from paper_1009_2768_gb300.runtime import GraphStepper
    g = GraphStepper(sim, steps_per_graph=1, warmup=2, step_kwargs={"stats": stats})
    stats.zero_()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K)]
    for k in range(K):
        flush.zero_()
        ev[k][0].record()
        g.replay()
        ev[k][1].record()
    torch.cuda.synchronize()
    co = np.array([ev[k][0].elapsed_time(ev[k][1]) for k in range(K)])
    return np.zeros(K), co


def gpu_moments(sim):
    import torch
    from paper_1009_2768_gb300 import trmc as T
    mom = torch.zeros((sim.state.n_cells, T.MOM_COLS), dtype=torch.float64, device="cuda")
    T.trmc_moments(sim.ctx, sim.state, mom)
    return mom.cpu().numpy()


def l1_rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    ok = np.isfinite(a) & np.isfinite(b)
    den = np.abs(b[ok]).sum()
    return float(np.abs(a[ok] - b[ok]).sum() / den) if den > 0 else 0.0


def moment_measure(workload, got, ref, init):
    """The moment error of one workload (per-cell moment tables
    [N, rho, u, T, P_xx, M_4, E, max|v|^2]): density and temperature
    profiles of the 1D problems (interior cells), the anisotropy
    (P_xx - T)/T per cell of the batched relaxation relative to its initial
    size, the fourth moment of the BKW cell."""
    if workload in ("stationary", "shock"):
        sl = slice(1, -1) if workload == "stationary" else slice(None)
        return {"rho_L1": l1_rel(got[sl, 1], ref[sl, 1]), "T_L1": l1_rel(got[sl, 5], ref[sl, 5])}
    if workload == "batched":
        an = lambda m: (m[:, 6] - m[:, 5]) / m[:, 5]
        return {"aniso_L1": float(np.abs(an(got) - an(ref)).sum() / np.abs(an(init)).sum())}
    return {"M4_abs": float(abs(got[0, 7] - ref[0, 7])), "M4": float(got[0, 7])}


MEASURE_TEXT = {
    "stationary": "L1 relative difference of the interior cells' density and temperature profiles",
    "shock": "L1 relative difference of the four tubes' density and temperature profiles",
    "batched": "sum over cells of |a_gpu - a_oracle| / sum of |a_initial|, a = (P_xx - T)/T per cell",
    "bkw": "|M_4 difference| of the cell (M_4 = <|v|^4>)",
}


def oracle_compare(workload, precision, steps, threads, flush=None, seed=0):
    """The GPU form of `workload` at `precision` and the FP64 oracle step the
    same initial state (the GPU's own initial data, copied) for `steps`
    steps with the same keys; the oracle with the next seed gives the Monte
    Carlo noise floor of the same measure.  Also times the GPU form (median
    step, CUDA events, L2 flushed before each step) and the oracle."""
    import torch
    from paper_1009_2768_gb300 import trmc as T
    sim, rb, label = make_sim(workload, seed, precision)
    if workload in LAUNCH:
        T.trmc_set_collide_launch(sim.ctx, *LAUNCH[workload])
    from oracle.stepper import OracleSim
    orc, orc_b = OracleSim(sim, seed), OracleSim(sim, seed + 1)
    init = gpu_moments(sim)
    ms = []
    for _ in range(steps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        if flush is not None:
            flush.zero_()
        sim.step(events=ev)
        torch.cuda.synchronize()
        ms.append(ev[0].elapsed_time(ev[2]))
    T.trmc_check(sim.ctx)
    got = gpu_moments(sim)
    n = sim.n_particles
    sim.close()
    t0 = time.perf_counter()
    for _ in range(steps):
        orc.step(threads)
    t_orc = time.perf_counter() - t0
    ref = orc.moments()
    for _ in range(steps):
        orc_b.step(threads)
    other = orc_b.moments()
    step_ms = float(np.median(ms))
    return {"precision": label, "steps": steps,
            "error": moment_measure(workload, got, ref, init),
            "noise_floor": moment_measure(workload, other, ref, init),
            "gpu": {"value": n / (step_ms / 1e3), "unit": METRIC, "ms_per_step": step_ms, "particles": n},
            "oracle": {"value": orc.n * steps / t_orc, "unit": METRIC, "seconds": t_orc, "steps": steps,
                       "particles": orc.n, "threads": threads}}


def ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1009_2768_gb300 import build
    build.build()
    from paper_1009_2768_gb300 import trmc as T

    sim, rb, dtype = make_sim(args.workload, rank)
    n = sim.n_particles
    stats = torch.zeros(len(T.STATS_FIELDS), dtype=torch.int64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")      # > L2 (129 MB)
    for _ in range(args.warmup):
        sim.step()
    T.trmc_check(sim.ctx)
    if args.tune:
        # the collide launch shape for this workload's cell sizes, measured on
        # the live state before timing
        from paper_1009_2768_gb300 import runtime as RT
        tuned = RT.autotune(sim, steps=2, rounds=4)
        best = tuned["collide_best"]
        launch = {"threads": best[0], "ctas_per_sm": best[1],
                  "tuned_ms": {f"{k[0]}x{k[1]}": round(v, 4) for k, v in tuned["collide"].items()},
                  "work_schedule": {"warp_particles": tuned["work_best"][0],
                                    "records_per_thread": tuned["work_best"][1]},
                  "work_tuned_ms": {f"{k[0]}/{k[1]}": round(v, 4) for k, v in tuned["work"].items()},
                  "sort_threads": tuned["sort_best"],
                  "sort_tuned_ms": {str(k): round(v, 4) for k, v in tuned["sort"].items()}}
        for _ in range(2):
            sim.step()
        T.trmc_check(sim.ctx)
    else:
        th, per = ((int(v) for v in args.launch.lower().split("x")) if args.launch
                   else LAUNCH.get(args.workload, (128, 4)))
        T.trmc_set_collide_launch(sim.ctx, th, per)
        launch = {"threads": th, "ctas_per_sm": per, "tuned_ms": None}
    K = args.steps
    clocks = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.2)
    t_wall = time.perf_counter()
    if args.workload == "batched":
        # one persistent collide launch per step, replayed from a captured CUDA graph
        tr_ms, co_ms = time_graph_steps(sim, K, flush, stats)
    else:
        tr_ms, co_ms = time_steps(sim, K, flush, stats)
    t_wall = time.perf_counter() - t_wall
    if dist:
        dist.barrier()
    clk = clocks.stop()
    T.trmc_check(sim.ctx)
    step_ms = tr_ms + co_ms
    total_ms = max_over_ranks(float(step_ms.sum()), dist)
    value = replica_throughput(n, world, K, total_ms)
    st = dict(zip(T.STATS_FIELDS, stats.cpu().numpy().tolist()))

    # roofline of the dominant kernel, from the same events
    peak, peak_kind = peaks()
    collide_bytes = 3 * rb * (n + st["changed"] / K)               # read every particle, write the changed ones
    transport_bytes = (2 * rb + 8 * rb) * n                        # count: x, v_x; scatter: read x, v + write x, v
    co_avg, tr_avg = co_ms.mean() / 1e3, tr_ms.mean() / 1e3
    if co_avg >= tr_avg:
        kern, abytes, dur = "collide_kernel", collide_bytes, co_avg
    else:
        kern, abytes, dur = "transport (count+scan+scatter)", transport_bytes, tr_avg
    achieved = abytes / dur / 1e9
    tr_rec = NCU_TRAFFIC.get(args.workload)
    fresh = bool(tr_rec and kern == "collide_kernel" and tr_rec["collide_sha"] == collide_sha()
                 and tuple(tr_rec["launch"]) == (launch["threads"], launch["ctas_per_sm"]))
    traffic = tr_rec["bytes"] if fresh else None
    roof = {"bound": "hbm", "kernel": kern, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": peak_kind, "traffic": traffic,
            "collide_ms": float(co_ms.mean()), "transport_ms": float(tr_ms.mean()),
            "algorithmic_bytes_per_launch": abytes}
    if fresh:
        # what bounds the kernel instead, from the same ncu capture: a kernel
        # whose DRAM throughput and issue rate are both low waits on latency
        top = max(tr_rec["stalls_per_issue"], key=tr_rec["stalls_per_issue"].get)
        roof["limiter"] = {"kind": "latency", "issue_active_pct": tr_rec["issue_active_pct"],
                           "warps_active_pct": tr_rec["warps_active_pct"],
                           "stalls_per_issue": tr_rec["stalls_per_issue"], "top_stall": top}

    # end to end: host-resident state, H2D + step + D2H every step
    e2e = None
    if not args.no_e2e:
        hv = torch.empty_like(sim.state.v, device="cpu").pin_memory()
        hv.copy_(sim.state.v)
        hx = None
        if sim.state.x is not None:
            hx = torch.empty_like(sim.state.x, device="cpu").pin_memory()
            hx.copy_(sim.state.x)
        hcs = sim.state.cell_start.cpu().pin_memory()
        Ke = max(1, min(K, 200))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for k in range(Ke):
            if hx is not None:
                sim.state.x.copy_(hx, non_blocking=True)
            sim.state.v.copy_(hv, non_blocking=True)
            sim.state.cell_start.copy_(hcs, non_blocking=True)
            sim.step()
            if hx is not None:
                hx.copy_(sim.state.x, non_blocking=True)
            hv.copy_(sim.state.v, non_blocking=True)
            hcs.copy_(sim.state.cell_start, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        e_ms = e0.elapsed_time(e1)
        h2d = hv.numel() * hv.element_size() + hcs.numel() * 8 + (hx.numel() * hx.element_size() if hx is not None else 0)
        e2e = {"value": n * world * Ke / (e_ms / 1e3), "unit": METRIC, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": h2d, "steps": Ke}

    # the moment error against the FP64 oracle (same initial state and keys,
    # COMPARE_STEPS steps), the oracle's own rate on that sample (the CPU
    # baseline), and the other precision's form of the same workload
    cpu, moment_error, forms = None, None, None
    if rank == 0 and world == 1 and not args.no_cpu:
        from oracle.build import build_oracle
        build_oracle()
        threads = 1 if args.workload == "bkw" else (os.cpu_count() or 1)
        own = oracle_compare(args.workload, None, COMPARE_STEPS, threads, flush)
        o = own["oracle"]
        cpu = {"value": o["value"], "unit": METRIC, "cores": threads, "cpu_model": cpu_model(), "kind": "oracle",
               "sample": f"the whole workload ({o['particles']} particles) from the GPU's initial state, "
                         f"{o['steps']} steps in {o['seconds']:.1f} s"}
        moment_error = {"what": f"{MEASURE_TEXT[args.workload]}, GPU {own['precision']} vs the FP64 CPU oracle "
                                f"from the same initial state with the same keys, after {COMPARE_STEPS} steps; "
                                f"noise_floor: the same measure between the oracle and the oracle with other keys",
                        "error": own["error"], "noise_floor": own["noise_floor"], "steps": COMPARE_STEPS}
        forms = {"timed_form": {"precision": own["precision"], "value": own["gpu"]["value"],
                                "ms_per_step": own["gpu"]["ms_per_step"], "error": own["error"]}}
        if not args.no_forms:
            other = T.FP64 if args.workload in ("stationary", "batched") else T.FP32_MIXED
            alt = oracle_compare(args.workload, other, COMPARE_STEPS, threads, flush)
            forms["fp64_form" if other == T.FP64 else "fp32_mixed_form"] = {
                "precision": alt["precision"], "value": alt["gpu"]["value"], "ms_per_step": alt["gpu"]["ms_per_step"],
                "error": alt["error"], "noise_floor": alt["noise_floor"],
                "note": f"same workload, {COMPARE_STEPS} eager steps from its initial state, median step time"}

    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "particles_per_gpu": n,
                       "cells_per_gpu": sim.state.n_cells,
                       "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{world}",
                       "cuda_graph": args.workload == "batched",
                       "collide_launch": launch},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "moment_error": moment_error,
            "gpu_launches": sim.launches_per_step * K, "clocks": clk, "forms": forms,
            "step_stats": {k: st[k] / K for k in ("collisions", "dummy", "maxwell", "changed", "passes")},
            "wall_s": t_wall}))
    sim.close()
    if dist:
        dist.destroy_process_group()


def served_vs_oracle(reqs, precision, seed, threads, per_kind=1):
    """The smallest completed requests of each kind against the FP64 oracle:
    the request's initial state is built again (it is deterministic in the
    request id and seed), the oracle steps it as many steps as the request
    ran, with the same keys and with the next seed (the noise floor), and
    the served moment table is compared with both."""
    from oracle.stepper import OracleSim
    from paper_1009_2768_gb300 import trmc as T
    from paper_1009_2768_gb300.serving import shock_mean
    from paper_1009_2768_gb300.workloads import BatchedRelaxation, ShockTubes
    rows = []
    for kind in ("shock", "relax"):
        done = sorted([r for r in reqs if r.kind == kind and r.result is not None and r.error is None],
                      key=lambda r: r.particles)[:per_kind]
        for r in done:
            ctx = T.trmc_create(precision, seed, 64 << 20)
            if kind == "shock":
                sim = ShockTubes((r.eps,), n_cells=len(r.counts), mean_per_cell=shock_mean(r), precision=precision,
                                 seed=seed, ctx=ctx, problem_base=r.rid)
            else:
                sim = BatchedRelaxation(counts=r.counts, eps_lo=r.eps, eps_hi=r.eps, precision=precision, seed=r.rid,
                                        ctx=ctx, problem_base=r.rid, problem_per_cell=False)
            orc, alt = OracleSim(sim, seed), OracleSim(sim, seed + 1)
            T.trmc_destroy(ctx)
            init = orc.moments()
            for _ in range(r.steps):
                orc.step(threads)
                alt.step(threads)
            ref, oth = orc.moments(), alt.moments()
            wl = "shock" if kind == "shock" else "batched"
            rows.append({"rid": r.rid, "kind": kind, "particles": r.particles, "steps": r.steps,
                         "t_reached": r.t_reached, "error": moment_measure(wl, r.result, ref, init),
                         "noise_floor": moment_measure(wl, oth, ref, init)})
    return rows


def serving_bench(args):
    """Rate sweep of the continuous-batching serving loop.  Every request is
    a solve to its physical end time (shock tubes to t = 0.2, relaxations to
    t = 1; --req-steps K runs K steps instead), and its latency runs from its
    arrival to its moments table landing in host memory: set-up of its cell
    tables (host -> device), its steps, the moments kernel and the copy
    back."""
    import torch
    from paper_1009_2768_gb300 import build, synth
    from paper_1009_2768_gb300 import trmc as T
    from paper_1009_2768_gb300.serving import T_END, GpuEngine, ServingLoop, requests_from, summary
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    build.build()
    steps = args.req_steps or None
    budget = int(args.budget_gb * (1 << 30))
    eng = GpuEngine(n_slots=args.slots, precision=T.FP32_MIXED, seed=rank, workspace_bytes=1 << 30,
                    chunk=args.chunk, depth=2)
    rates = [float(r) for r in args.rates.split(",")]
    # warm-up: a few small requests through the same engine (allocator, module load, pinned pool)
    warm = requests_from(synth.poisson_requests(max(args.warmup, 3), 1e4, n_hi=1_000_000, g=synth.rng(99)),
                         steps=steps, first_id=1 << 20, t_end={"shock": 0.01})
    ServingLoop(eng, budget - eng.fixed_bytes).run(warm)
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.2)
    sweep, rid = [], 0
    t_wall = time.perf_counter()
    for i, rate in enumerate(rates):
        n_req = args.requests or int(min(48, max(8, 8 * rate)))
        reqs = requests_from(synth.poisson_requests(n_req, rate, g=synth.rng(1000 * rank + i)), steps=steps,
                             first_id=rid)
        rid += n_req
        torch.cuda.synchronize()
        torch.cuda.reset_peak_memory_stats()
        loop = ServingLoop(eng, budget - eng.fixed_bytes)
        out = loop.run(reqs)
        s = summary(out)
        s.update(rate=rate, requests=n_req, resident_peak_gb=(loop.peak_bytes + eng.fixed_bytes) / 2 ** 30,
                 torch_peak_gb=torch.cuda.max_memory_allocated() / 2 ** 30,
                 mean_particles=float(np.mean([r.particles for r in out])),
                 mean_steps=float(np.mean([r.steps for r in out if r.done is not None])),
                 errors=[r.error for r in out if r.error][:3])
        sweep.append(s)
        last = (i, n_req, rid - n_req, out)
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    eng.close()
    # The plain single-problem FP64 form on the first requests of the highest
    # rate's stream: one slot, FP64 contexts, the same requests (same problem
    # ids and seed), so its latencies and throughput stand beside the served
    # FP32-mixed ones; both forms' moment tables are compared with the FP64
    # oracle on the smallest requests of each kind.
    i, n_req, first, out32 = last
    n64 = min(n_req, args.fp64_requests)
    reqs64 = requests_from(synth.poisson_requests(n_req, rates[i], g=synth.rng(1000 * rank + i))[:n64],
                           steps=steps, first_id=first)
    eng64 = GpuEngine(n_slots=1, precision=T.FP64, seed=rank, workspace_bytes=2 << 30, chunk=args.chunk, depth=2)
    out64 = ServingLoop(eng64, budget - eng64.fixed_bytes).run(reqs64)
    eng64.close()
    s64 = summary(out64)
    svc = np.array([(r.done - r.admitted) * 1e3 for r in out64 if r.done is not None and r.error is None])
    moment_error = None
    if rank == 0 and not args.no_cpu:
        from oracle.build import build_oracle
        build_oracle()
        threads = os.cpu_count() or 1
        moment_error = {"what": "per compared request: density and temperature profiles (shock tubes) or the cells' "
                                "anisotropy (relaxations) after the request's last step, served form vs the FP64 "
                                "CPU oracle stepping the same initial state with the same keys; noise_floor: the "
                                "oracle against itself with other keys",
                        "fp32_mixed_served": served_vs_oracle(out32, T.FP32_MIXED, rank, threads),
                        "fp64_single": served_vs_oracle(out64, T.FP64, rank, threads)}
    fp64_single = {"rate": rates[i], "slots": 1, "requests": n64, "p50_ms": s64.get("p50_ms"),
                   "p99_ms": s64.get("p99_ms"),
                   "service_p50_ms": float(np.percentile(svc, 50)) if svc.size else None,
                   "service_p99_ms": float(np.percentile(svc, 99)) if svc.size else None,
                   "particle_steps_per_s": s64.get("particle_steps_per_s"), "completed": s64.get("completed")}
    top = sweep[-1]
    value = top.get("particle_steps_per_s") or 0.0
    peak, peak_kind = peaks()
    achieved = value * (12 + 12) / 1e9          # FP32: read v, write (at most) every particle, per particle-step
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.req_steps,
            "warmup": len(warm), "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 velocities, f64 moments", "data": "synthetic",
            "config": {"workload": WORKLOADS["serving"], "rates_per_s": rates,
                       "requests": ("solves: shock tubes (400 cells, specular walls, CFL 0.5) to t = %g, "
                                    "relaxations (dt 0.05) to t = %g" % (T_END["shock"], T_END["relax"]))
                       if steps is None else f"{steps} steps each",
                       "slots": args.slots, "chunk": args.chunk, "budget_gb": args.budget_gb,
                       "l2": "requests far larger than L2 on average (mean 3.8e6 particles)",
                       "parallelism": f"replicas x{world}"},
            "serving": sweep,
            "fp64_single": fp64_single,
            "moment_error": moment_error,
            "roofline": {"bound": "hbm", "kernel": "all kernels of the served mix", "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind,
                         "traffic": None},
            "cpu_baseline": None,
            "e2e": {"value": value, "unit": METRIC, "note": "serving is timed end to end (tables in, moments out)",
                    "h2d_bytes_per_step": None, "d2h_bytes_per_step": None},
            "clocks": clk, "wall_s": t_wall}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--tune", action="store_true", help="choose the collide launch shape, the work schedule inside a cell (particles per warp, records per thread) and the sort schedule with the autotuner")
    ap.add_argument("--launch", default="", help="collide launch shape THREADSxCTAS_PER_SM (default: per workload)")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=["stationary", "shock", "batched", "bkw", "serving"])
    ap.add_argument("--rates", default="1,10,50,200", help="serving: arrival rates (requests/s) to sweep")
    ap.add_argument("--requests", type=int, default=0, help="serving: requests per rate (default 8*rate in [8, 48])")
    ap.add_argument("--req-steps", type=int, default=0,
                    help="serving: time steps per request (0: each request is a solve to its physical end time)")
    ap.add_argument("--fp64-requests", type=int, default=16,
                    help="serving: requests of the highest rate run again as FP64 single-problem solves")
    ap.add_argument("--slots", type=int, default=8, help="serving: concurrent requests (contexts + streams)")
    ap.add_argument("--chunk", type=int, default=4, help="serving: steps issued per chunk")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="serving: HBM budget (GiB)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        reference_arm(args)
    elif args.workload == "serving":
        serving_bench(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
