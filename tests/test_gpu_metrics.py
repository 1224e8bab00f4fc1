"""The metrics log of a specimen and of a batch on the GPU: every burst and
coarse step appends one record holding what the call returned."""
import numpy as np
import pytest

from gpu_util import gpu_package

pytestmark = pytest.mark.gpu


def test_bursts_and_coarse_steps_are_logged(tmp_path):
    P = gpu_package()
    from paper_2603_07321_gb300.metrics import read
    path = tmp_path / "run.jsonl"
    ctx = P.Ctx((4, 4, 5), T0=300.0, seed=2, precision=P.PREC_MIXED, burst_steps=200,
                log=str(path), tag="cube")
    ctx.apply_strain(1e-3)
    a = ctx.fine_burst(150)
    r1 = ctx.coarse_step()          # the initial bursts, then the first coarse step
    r2 = ctx.coarse_step()
    ctx.close()
    recs = read(path)
    assert [r["kind"] for r in recs] == ["burst", "coarse", "coarse"]
    assert all(r["tag"] == "cube" for r in recs)
    assert recs[0]["mean"] == list(a.mean) and recs[0]["nsteps"] == 150
    for rec, r in zip(recs[1:], (r1, r2)):
        assert rec["t"] == r.t and rec["strain"] == r.strain and rec["v"] == list(r.v)
        assert rec["source"] == list(r.source) and rec["status"] == 0
        assert [b["mean"] for b in rec["burst"]] == [list(b.mean) for b in r.burst]
    # e2 is undefined at the first coarse step: null, not NaN, in the log
    if not np.all(np.isfinite(r1.e2)):
        assert None in recs[1]["e2"]


def test_batch_members_log_under_their_own_tags(tmp_path):
    P = gpu_package()
    from paper_2603_07321_gb300.metrics import JsonlLog, read
    path = tmp_path / "batch.jsonl"
    log = JsonlLog(str(path))
    cs = [P.Ctx((4, 4, 4), T0=100.0, seed=5 + i, precision=P.PREC_MIXED, burst_steps=100,
                log=log, tag="m%d" % i) for i in range(3)]
    b = P.Batch(cs)
    res = b.fine_burst([100, 120, 140])
    ticks = b.tick()
    b.close()
    for c in cs:
        c.close()
    log.close()
    recs = read(path)
    bursts = [r for r in recs if r["kind"] == "burst"]
    coarse = [r for r in recs if r["kind"] == "coarse"]
    assert [r["tag"] for r in bursts] == ["m0", "m1", "m2"]
    assert [r["nsteps"] for r in bursts] == [100, 120, 140]
    assert [r["mean"] for r in bursts] == [list(a.mean) for a in res]
    assert [r["tag"] for r in coarse] == ["m0", "m1", "m2"]
    assert [r["strain"] for r in coarse] == [t.strain for t in ticks]
