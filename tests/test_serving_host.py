"""Host logic of the serving loop, driven by a simulated engine on a
virtual clock (no GPU): first-come-first-served admission under the byte
budget and the slot count, rejection of requests that can never fit,
completion of every admitted request, the latency bookkeeping, and the
Poisson request stream."""
import numpy as np
import pytest

from paper_1009_2768_gb300 import synth
from paper_1009_2768_gb300.serving import (RELAX_DT, SHOCK_CELLS, T_END, Admission, Request, ServingLoop, footprint,
                                           plan, requests_from, summary)


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-6)


class SimJob:
    def __init__(self, eng, req):
        self.req, self.eng = req, eng
        self.end = eng.clock.t + eng.seconds(req)

    def pump(self):
        return False

    def finished(self):
        if self.eng.clock.t >= self.end:
            self.req.result = np.array([self.req.rid])
            return True
        return False


class SimEngine:
    """Each request runs for particles*steps/rate seconds of virtual time
    once started; tracks resident bytes and busy slots."""

    def __init__(self, clock, n_slots, rate=1e9, fail_rids=()):
        self.clock, self.n_slots, self.rate = clock, n_slots, rate
        self.resident = 0
        self.peak = 0
        self.busy = set()
        self.starts = []
        self.fail_rids = set(fail_rids)

    def seconds(self, req):
        return req.particles * req.steps / self.rate

    def footprint(self, req):
        plan(req)
        return footprint(req.kind, len(req.counts), req.particles)

    def start(self, req):
        if req.rid in self.fail_rids:
            raise MemoryError("simulated allocation failure")
        assert req.slot not in self.busy
        self.busy.add(req.slot)
        self.resident += req.bytes
        self.peak = max(self.peak, self.resident)
        self.starts.append(req.rid)
        return SimJob(self, req)

    def release(self, job):
        self.busy.remove(job.req.slot)
        self.resident -= job.req.bytes


def stream(n, rate, seed, n_lo=100_000, n_hi=2_000_000):
    from paper_1009_2768_gb300.serving import requests_from
    return requests_from(synth.poisson_requests(n, rate, n_lo=n_lo, n_hi=n_hi, g=synth.rng(seed)), steps=20)


def test_admission_is_fcfs_and_respects_budget_and_slots():
    sizes = {0: 40, 1: 50, 2: 30, 3: 100, 4: 10}
    adm = Admission(100, 2, lambda r: sizes[r.rid])
    reqs = [Request(i, "shock", 1, 1.0, 1) for i in range(5)]
    for r in reqs:
        assert adm.offer(r)
    first = adm.admit()
    assert [r.rid for r in first] == [0, 1]             # 2 slots
    assert adm.used == 90 and adm.admit() == []          # no slot; and 2 (30 B) must wait anyway
    adm.release(first[0])
    assert [r.rid for r in adm.admit()] == [2]           # 50 + 30 <= 100
    adm.release(first[1])
    assert adm.admit() == []                             # head is 3 (100 B): blocks 4 behind it
    adm.release(reqs[2])
    assert [r.rid for r in adm.admit()] == [3]
    assert adm.used == 100 and adm.peak == 100


def test_admission_rejects_what_can_never_fit():
    adm = Admission(100, 4, lambda r: 101 if r.rid == 1 else 10)
    ok = [adm.offer(Request(i, "shock", 1, 1.0, 1)) for i in range(3)]
    assert ok == [True, False, True]
    assert [r.rid for r in adm.admit()] == [0, 2]


@pytest.mark.parametrize("n_slots,budget_frac", [(1, 1.0), (4, 0.3), (8, 1.0)])
def test_loop_completes_every_request_in_order(n_slots, budget_frac):
    clock = Clock()
    eng = SimEngine(clock, n_slots)
    reqs = stream(40, rate=50.0, seed=3)
    big = max(eng.footprint(r) for r in reqs)
    budget = max(big, int(budget_frac * sum(eng.footprint(r) for r in reqs)))
    loop = ServingLoop(eng, budget, clock=clock, sleep=clock.sleep)
    out = loop.run(reqs)
    assert all(r.done is not None and r.result[0] == r.rid for r in out)
    assert eng.starts == [r.rid for r in sorted(out, key=lambda r: (r.arrival, r.rid))]   # FCFS
    assert eng.peak <= budget and loop.peak_bytes == eng.peak
    assert eng.resident == 0 and not eng.busy
    for r in out:
        assert r.arrival <= r.admitted <= r.done
        assert r.latency >= eng.seconds(r) - 1e-9
    s = summary(out)
    assert s["completed"] == 40 and s["p50_ms"] <= s["p99_ms"] <= s["max_ms"]


def test_loop_overlaps_requests_and_serves_one_slot_sequentially():
    reqs = [Request(i, "shock", 200_000, 1e-2, 10, arrival=0.0) for i in range(6)]
    clock = Clock()
    eng = SimEngine(clock, 1)
    ServingLoop(eng, 1 << 40, clock=clock, sleep=clock.sleep).run(reqs)
    serial = max(r.done for r in reqs)
    reqs2 = [Request(i, "shock", 200_000, 1e-2, 10, arrival=0.0) for i in range(6)]
    clock2 = Clock()
    eng2 = SimEngine(clock2, 6)
    ServingLoop(eng2, 1 << 40, clock=clock2, sleep=clock2.sleep).run(reqs2)
    # the simulated engine does not slow down with concurrency, so six slots finish ~6x sooner
    assert max(r.done for r in reqs2) < serial / 4


def test_rejected_and_failed_requests_do_not_block_others():
    clock = Clock()
    eng = SimEngine(clock, 2, fail_rids={2})
    reqs = [Request(i, "shock", 100_000 if i != 1 else 50_000_000, 1e-2, 5, arrival=0.01 * i) for i in range(5)]
    budget = eng.footprint(Request(99, "shock", 200_000, 1.0, 1))
    out = ServingLoop(eng, budget, clock=clock, sleep=clock.sleep).run(reqs)
    by = {r.rid: r for r in out}
    assert by[1].rejected and by[1].done is None
    assert by[2].error.startswith("start failed") and by[2].done is None
    assert all(by[i].done is not None for i in (0, 3, 4))
    s = summary(out)
    assert s["completed"] == 3 and s["rejected"] == 1 and s["failed"] == 1


def test_plan_and_footprint():
    a = plan(Request(7, "relax", 1_000_000, 1e-2, 1))
    b = plan(Request(7, "relax", 1_000_000, 1e-2, 1))
    assert np.array_equal(a.counts, b.counts) and a.particles == int(a.counts.sum())
    assert a.counts.min() >= 64 and a.counts.max() <= 8192
    s = plan(Request(8, "shock", 1_000_000, 1e-2, 1))
    assert len(s.counts) == SHOCK_CELLS and abs(s.particles - 1_000_000) < SHOCK_CELLS
    # a solve request: relaxation to t_end = 1 runs 20 steps of dt 0.05; a shock
    # tube's step count waits for its first CFL step (set on the GPU)
    r = plan(Request(9, "relax", 300_000, 1e-2, 0, t_end=T_END["relax"]))
    assert r.steps == round(T_END["relax"] / RELAX_DT) == 20
    sol = requests_from(synth.poisson_requests(6, 10.0, g=synth.rng(3)))
    assert all(q.t_end == T_END[q.kind] for q in sol)
    # resident bytes grow with the particle count and cover the FP32 particle arrays
    f1 = footprint("shock", 2000, 1_000_000)
    assert f1 >= 2 * (12 + 4) * 1_000_000
    assert footprint("shock", 4000, 2_000_000) > f1
    assert footprint("relax", 600, 1_000_000) >= 12 * 1_000_000


def test_poisson_request_stream():
    reqs = synth.poisson_requests(4000, rate=20.0, g=synth.rng(1))
    t = np.array([r["arrival"] for r in reqs])
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0)
    gaps = np.diff(t)
    assert abs(gaps.mean() * 20.0 - 1.0) < 0.06               # mean gap 1/rate (4000 samples: ~1.6% s.e.)
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.08         # exponential: coefficient of variation 1
    n = np.array([r["n_particles"] for r in reqs])
    assert n.min() >= 100_000 and n.max() <= 20_000_000
    ln = np.log(n)                                              # log-uniform: uniform in log
    assert abs(ln.mean() - 0.5 * (np.log(1e5) + np.log(2e7))) < 0.1
    eps = np.array([r["eps"] for r in reqs])
    assert eps.min() >= 1e-4 and eps.max() <= 1.0
    kinds = [r["kind"] for r in reqs]
    assert 0.45 < kinds.count("shock") / len(kinds) < 0.55
