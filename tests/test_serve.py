"""Host logic of the serving loop, with a stand-in engine (CPU only).

Faults are injected on the host: invalid requests, an allocation that fails
at admission, and a specimen whose tick reports an error."""
import itertools
import json

import pytest

from paper_2603_07321_gb300.serve import Request, Scheduler


class FakeEngine:
    """Advances each specimen's strain by rate * h per tick (the first tick
    of a specimen is its initial one); footprint = 1000 bytes per cell^3."""

    def __init__(self, fail_create=(), fail_tick=(), oom_once=(), overflow_once=()):
        self.fail_create = set(fail_create)
        self.fail_tick = set(fail_tick)
        self.oom_once = set(oom_once)
        self.overflow_once = set(overflow_once)
        self.state = {}
        self.created = []
        self.destroyed = []
        self.tick_calls = []

    def validate(self, req):
        return "" if req.n_cells >= 3 else "too small"

    def footprint(self, req):
        return 1000 * req.n_cells ** 3

    def create(self, req):
        if req.rid in self.oom_once:
            self.oom_once.discard(req.rid)
            raise MemoryError("simulated out of memory")
        if req.rid in self.fail_create:
            raise ValueError("simulated invalid specimen")
        self.created.append(req.rid)
        self.state[req.rid] = {"req": req, "strain": 0.0, "init": False, "ticks": 0}
        return req.rid

    def destroy(self, h):
        self.destroyed.append(h)
        self.state.pop(h, None)

    def tick(self, handles):
        self.tick_calls.append(list(handles))
        out = []
        for h in handles:
            s = self.state[h]
            if h in self.fail_tick and s["ticks"] >= 1:
                out.append({"error": "simulated burst failure"})
                continue
            if h in self.overflow_once and s["ticks"] >= 1:
                # the real engine restores the specimen from its state before
                # this tick into a new one with more list memory: same state,
                # new handle, the tick not counted
                self.overflow_once.discard(h)
                new = ("regrown", h)
                self.state[new] = dict(s)
                self.state.pop(h)
                self.destroyed.append(h)
                out.append({"recovered": True, "handle": new, "atom_steps": 0,
                            "bytes": 2 * self.footprint(s["req"]), "neigh_cap": 64,
                            "reason": "neighbour-list overflow"})
                continue
            s["ticks"] += 1
            r = s["req"]
            if not s["init"]:
                s["init"] = True
                s["strain"] += r.strain_rate * 0.2
                out.append({"strain": s["strain"], "v": [1, 2, 3], "source": [-1] * 3,
                            "initial": True, "atom_steps": 3 * r.burst_steps * 4 * r.n_cells ** 3})
            else:
                s["strain"] += r.strain_rate * 1.0
                out.append({"strain": s["strain"], "v": [s["strain"]] * 3, "source": [0] * 3,
                            "initial": False,
                            "atom_steps": 3 * r.burst_steps * 4 * r.n_cells ** 3})
        return out


def _clock():
    c = itertools.count()
    return lambda: next(c) * 0.01


def req(rid, n=10, rate=0.01, target=0.05, t=0.0):
    return Request(rid=rid, n_cells=n, T0=300.0, seed=rid, strain_rate=rate, target_strain=target,
                   arrival_s=t, burst_steps=10)


def test_fifo_admission_by_memory_footprint():
    eng = FakeEngine()
    s = Scheduler(eng, mem_budget_bytes=2 * 1000 * 10 ** 3, max_slots=8, clock=_clock())
    res = s.run([req(0), req(1), req(2)], realtime=False)
    assert all(r.status == "done" for r in res.values())
    # only two fit at a time: the third is admitted after the first leaves
    assert eng.tick_calls[0] == [0, 1]
    assert 2 in eng.tick_calls[-1] and 0 not in eng.tick_calls[-1]
    assert s.used == 0 and not s.live


def test_slots_limit_and_continuous_batching():
    eng = FakeEngine()
    s = Scheduler(eng, mem_budget_bytes=10 ** 9, max_slots=2, clock=_clock())
    # different targets: request 0 leaves early and request 2 takes its slot mid-run
    trace = [req(0, target=0.02), req(1, target=0.08), req(2, target=0.03)]
    s.run(trace, realtime=False)
    joined = [calls for calls in eng.tick_calls if 2 in calls]
    assert joined and 1 in joined[0]   # 2 runs alongside 1, which was already running
    for rid, target in ((0, 0.02), (1, 0.08), (2, 0.03)):
        r = s.results[rid]
        assert r.status == "done" and r.curve[-1][0] >= target - 1e-12


def test_invalid_and_oversized_requests_are_rejected():
    eng = FakeEngine()
    s = Scheduler(eng, mem_budget_bytes=1000 * 10 ** 3, clock=_clock())
    s.run([req(0, n=2), req(1, n=20), req(2)], realtime=False)
    assert s.results[0].status == "rejected" and "small" in s.results[0].error
    assert s.results[1].status == "rejected" and "budget" in s.results[1].error
    assert s.results[2].status == "done"


def test_out_of_memory_at_admission_retries():
    eng = FakeEngine(oom_once={1})
    s = Scheduler(eng, mem_budget_bytes=10 ** 9, clock=_clock())
    s.run([req(0), req(1)], realtime=False)
    assert s.results[0].status == "done" and s.results[1].status == "done"
    assert eng.created.count(1) == 1


def test_device_rejection_at_create():
    eng = FakeEngine(fail_create={1})
    s = Scheduler(eng, mem_budget_bytes=10 ** 9, clock=_clock())
    s.run([req(0), req(1), req(2)], realtime=False)
    assert s.results[1].status == "rejected"
    assert s.results[0].status == "done" and s.results[2].status == "done"


def test_failing_member_does_not_disturb_the_others():
    alone = Scheduler(FakeEngine(), mem_budget_bytes=10 ** 9, clock=_clock())
    alone.run([req(0, target=0.05)], realtime=False)
    eng = FakeEngine(fail_tick={1})
    s = Scheduler(eng, mem_budget_bytes=10 ** 9, clock=_clock())
    s.run([req(0, target=0.05), req(1, target=0.05)], realtime=False)
    assert s.results[1].status == "failed" and "simulated" in s.results[1].error
    assert 1 in eng.destroyed
    assert s.results[0].status == "done"
    assert s.results[0].curve == alone.results[0].curve


def test_recovered_member_repeats_its_tick_under_a_new_handle(tmp_path):
    from paper_2603_07321_gb300.metrics import JsonlLog
    alone = Scheduler(FakeEngine(), mem_budget_bytes=10 ** 9, clock=_clock())
    alone.run([req(1, target=0.05)], realtime=False)
    eng = FakeEngine(overflow_once={1})
    log = JsonlLog(str(tmp_path / "m.jsonl"))
    s = Scheduler(eng, mem_budget_bytes=10 ** 9, clock=_clock(), log=log)
    s.run([req(0, target=0.05), req(1, target=0.05)], realtime=False)
    log.close()
    # the recovered specimen finishes with the same curve as alone, one tick later
    assert s.results[1].status == "done" and s.results[0].status == "done"
    assert s.results[1].curve == alone.results[1].curve
    assert ("regrown", 1) in eng.destroyed and 1 in eng.destroyed
    assert s.used == 0 and not s.live
    recs = [json.loads(line) for line in open(tmp_path / "m.jsonl")]
    ev = [r for r in recs if r.get("kind") == "request_recovered"]
    assert len(ev) == 1 and ev[0]["tag"] == 1 and ev[0]["bytes"] == 2 * 1000 * 10 ** 3


def test_latency_statistics():
    s = Scheduler(FakeEngine(), mem_budget_bytes=10 ** 9, clock=_clock())
    s.run([req(i, target=0.03) for i in range(4)], realtime=False)
    st = s.stats()
    assert st["done"] == 4 and st["rejected"] == 0 and st["failed"] == 0
    assert st["coarse_step_latency_s"]["count"] > 0
    assert st["curve_latency_s"]["p50"] <= st["curve_latency_s"]["p99"]
    assert st["atom_steps"] > 0


def test_request_lanes_and_precision_reach_the_engine_parameters():
    # the parameters a request is created with depend on the request alone,
    # so its results are the same alone and in any mix
    from paper_2603_07321_gb300.serve import GPUEngine, Request
    eng = GPUEngine()
    r = Request(rid=1, n_cells=12, T0=300.0, seed=3, strain_rate=-2e-4, target_strain=0.05,
                burst_steps=500, precision=1, lanes=1)
    p = eng._p(r)
    assert (p.lanes, p.precision, p.burst_steps, p.strain_rate) == (1, 1, 500, -2e-4)
    assert eng._p(Request(rid=2, n_cells=12, T0=300.0, seed=3, strain_rate=1e-3,
                          target_strain=0.05)).lanes == 0
    assert eng.footprint(r) > 0


def test_bench_lanes_follow_the_workload_unless_overridden():
    import argparse
    import bench
    wl = bench.WORKLOADS["batched"]
    assert bench.lanes_of(argparse.Namespace(lanes=None), wl) == 1
    assert bench.lanes_of(argparse.Namespace(lanes=0), wl) == 0
    assert bench.lanes_of(argparse.Namespace(lanes=None), bench.WORKLOADS["large"]) == 0


def test_tune_cache_keys_and_round_trip(tmp_path, monkeypatch):
    monkeypatch.setenv("PTA_TUNE_CACHE", str(tmp_path / "t.json"))
    from paper_2603_07321_gb300 import tune
    assert tune.cache_key(32000, 1, 1) == "prec1:atoms32768:replicas1"
    assert tune.cache_key(470596, 64, 1) == "prec1:atoms524288:replicas64"
    assert tune.cache_key(470596, 40, 0) == "prec0:atoms524288:replicas64"
    assert tune.lookup(32000, 1, 1) is None
    tune.store(32000, 1, 1, {"lanes": 2, "skin": 1.5, "prune_margin": 0.3, "x": 9}, 1e9)
    assert tune.lookup(32000, 1, 1) == {"lanes": 2, "skin": 1.5, "prune_margin": 0.3}
    assert tune.lookup(31000, 1, 1) == {"lanes": 2, "skin": 1.5, "prune_margin": 0.3}
    assert tune.lookup(32000, 64, 1) is None
