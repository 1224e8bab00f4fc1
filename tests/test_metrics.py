"""The JSONL metrics log (CPU): strict JSON per line, and the serving loop's
records agree with its own results."""
import io
import json
import math

import numpy as np

from paper_2603_07321_gb300.metrics import JsonlLog, read
from paper_2603_07321_gb300.serve import Scheduler
from test_serve import FakeEngine, _clock, req


def test_records_are_strict_json():
    buf = io.StringIO()
    log = JsonlLog(buf, clock=lambda: 12.5)
    log.write("coarse", tag="a", e2=[math.nan, 1.0, math.inf], v=np.array([1.0, 2.0]).tolist(),
              n=np.int64(3), x=np.float64(0.25))
    log.write("burst", tag="b", mean=[1, 2, 3])
    lines = buf.getvalue().splitlines()
    assert len(lines) == 2
    r0 = json.loads(lines[0])            # strict: NaN and inf became null
    assert r0 == {"kind": "coarse", "time": 12.5, "tag": "a", "e2": [None, 1.0, None],
                  "v": [1.0, 2.0], "n": 3, "x": 0.25}
    assert json.loads(lines[1])["mean"] == [1, 2, 3]


def test_serving_records_match_the_results(tmp_path):
    path = tmp_path / "serve.jsonl"
    eng = FakeEngine(fail_tick={3})
    s = Scheduler(eng, mem_budget_bytes=2 * 1000 * 10 ** 3, max_slots=8, clock=_clock(),
                  log=str(path))
    trace = [req(0), req(1, target=0.08), req(2, n=2), req(3), req(4, t=0.05)]
    res = s.run(trace, realtime=False)
    s.log.close()
    recs = read(path)
    kinds = [r["kind"] for r in recs]
    by = lambda k: [r for r in recs if r["kind"] == k]
    assert {r["tag"] for r in by("request_rejected")} == {2}
    assert {r["tag"] for r in by("request_queued")} == {0, 1, 3, 4}
    assert {r["tag"] for r in by("request_admitted")} == {0, 1, 3, 4}
    assert all(r["wait_s"] >= 0 for r in by("request_admitted"))
    assert {r["tag"] for r in by("request_done")} == {rid for rid, r in res.items()
                                                     if r.status == "done"}
    assert {r["tag"] for r in by("request_failed")} == {3}
    assert len(by("tick")) == s.ticks
    for r in by("request_done"):
        got = res[r["tag"]]
        assert r["coarse_steps"] == len(got.curve) and r["atom_steps"] == got.atom_steps
        assert math.isclose(r["curve_latency_s"], got.finished_s - got.arrival_s)
        steps = [c for c in by("coarse") if c["tag"] == r["tag"] and not c["initial"]]
        assert [c["strain"] for c in steps] == [c[0] for c in got.curve]
    # every request's admission precedes its coarse steps, which precede its end
    for rid in (0, 1, 4):
        order = [i for i, r in enumerate(recs) if r.get("tag") == rid]
        ks = [recs[i]["kind"] for i in order]
        assert ks[0] == "request_queued" and ks[1] == "request_admitted"
        assert ks[-1] == "request_done" and set(ks[2:-1]) == {"coarse"}
    assert kinds.count("request_done") + kinds.count("request_failed") == 4
