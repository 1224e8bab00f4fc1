"""Serving on the GPU: each request's result is the same alone and in the
mix, and requests admitted while others run share the launches."""
import numpy as np
import pytest

from gpu_util import gpu_package
from paper_2603_07321_gb300.serve import GPUEngine, Request, Scheduler

pytestmark = pytest.mark.gpu


def _req(rid, n, rate, target, prec=1):
    return Request(rid=rid, n_cells=n, T0=300.0, seed=50 + rid, strain_rate=rate,
                   target_strain=target, burst_steps=40, precision=prec)


def _serve(reqs, slots):
    gpu_package()
    eng = GPUEngine()
    s = Scheduler(eng, mem_budget_bytes=8 << 30, max_slots=slots)
    res = s.run(reqs, realtime=False)
    eng.close()
    return s, res


def test_results_are_the_same_alone_and_in_the_mix():
    a = lambda: _req(0, 6, 1e-2, 0.025)
    b = lambda: _req(1, 5, -1e-2, 0.035)
    c = lambda: _req(2, 7, 2e-2, 0.05, prec=0)
    alone = {}
    for mk in (a, b, c):
        _, res = _serve([mk()], slots=1)
        r = list(res.values())[0]
        alone[r.rid] = r
    # two slots: c waits, then joins while b is still running
    s, mixed = _serve([a(), b(), c()], slots=2)
    for rid in (0, 1, 2):
        assert mixed[rid].status == "done"
        assert len(mixed[rid].curve) == len(alone[rid].curve) > 0
        for (s1, v1, src1), (s2, v2, src2) in zip(mixed[rid].curve, alone[rid].curve):
            assert s1 == s2 and v1 == v2 and src1 == src2   # bit-identical
    st = s.stats()
    assert st["done"] == 3 and st["coarse_step_latency_s"]["p99"] > 0


def test_batch_of_uneven_served_sizes_stays_finite():
    # sizes of a served trace (10..48 cells, mixed temperatures, tension and
    # compression); several have a last thread block whose trailing warps
    # hold no atom, which must write nothing beyond their lists
    import pta_inputs as PI
    P = gpu_package()
    trace = PI.served_trace(8, seed=7)
    ctxs = [P.Ctx(r.n_cells, T0=r.T0, seed=r.seed, precision=P.PREC_MIXED,
                  burst_steps=r.burst_steps, strain_rate=r.strain_rate) for r in trace]
    assert any((c.n % 128) and (c.n % 128) <= 96 for c in ctxs)
    b = P.Batch(ctxs)
    for _ in range(3):
        b.apply_strain([1e-5] * len(ctxs))
        res = b.fine_burst([200] * len(ctxs))
        assert all(a.status == 0 and a.nsteps == 200 for a in res)
    for c in ctxs:
        p, v = c.get_state()
        assert np.isfinite(p).all() and np.isfinite(v).all()
    b.close()
    for c in ctxs:
        c.close()


def test_neighbour_overflow_is_recovered_with_more_list_capacity():
    # request 1 asks for a list capacity (64 entries per atom) far below the
    # ~200 neighbours within the list radius: its first tick overflows; the
    # engine restores it from its state before that tick with twice the
    # capacity, until it fits.  Capacity changes where entries are stored,
    # not their order, so its curve is bit-identical to the same request at
    # the default capacity; request 0 in the same batch is undisturbed.
    def mk(rid, cap):
        r = _req(rid, 6, 1e-2, 0.025)
        r.seed = 70
        r.neigh_cap = cap
        return r
    _, ref = _serve([mk(0, 0)], slots=1)
    s, res = _serve([mk(0, 0), mk(1, 64)], slots=2)
    assert res[0].status == "done" and res[1].status == "done"
    for rid in (0, 1):
        assert len(res[rid].curve) == len(ref[0].curve) > 0
        for (s1, v1, src1), (s2, v2, src2) in zip(res[rid].curve, ref[0].curve):
            assert s1 == s2 and v1 == v2 and src1 == src2
    assert s.used == 0


def test_neighbour_overflow_without_recovery_fails_only_that_specimen():
    gpu_package()
    eng = GPUEngine(recover=False)
    s = Scheduler(eng, mem_budget_bytes=8 << 30, max_slots=2)
    ok, bad = _req(0, 6, 1e-2, 0.025), _req(1, 6, 1e-2, 0.025)
    bad.neigh_cap = 64
    res = s.run([ok, bad], realtime=False)
    eng.close()
    assert res[1].status == "failed" and "-4" in res[1].error
    assert res[0].status == "done" and len(res[0].curve) > 0
