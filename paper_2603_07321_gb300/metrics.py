"""Metrics log: one JSON object per line (JSONL), appended as the run goes.

Records carry a "kind", the wall-clock "time" (s since the epoch) and the
kind's fields:

    burst          one fine burst of a specimen: means and block standard
                   errors of K, U, T, steps, list builds and prunings,
                   status, and with an adaptive length the convergence mask
                   and per-variable sample counts
    ramp_burst     the same for a continuously loaded burst
    relax          thermal relaxation: steps run, final stress, status
    coarse         one coarse step: t, strain, the accepted slow variables v,
                   v_pred, v_d, e_v, e1, e2, jump flags, accepted source per
                   variable, status and the three bursts
    request_*      serving: queued, rejected, admitted (with the queue wait),
                   done or failed (with the curve latency and atom-steps)
    tick           serving: one slow-time tick (live specimens, latency)

Non-finite numbers (e2 at the first coarse step) are written as null, so
every line is strict JSON.  `tag` names the specimen (a Ctx's tag, or the
request id in serving).
"""
from __future__ import annotations

import json
import math
import os
import threading
import time


def _clean(x):
    if isinstance(x, float):
        return x if math.isfinite(x) else None
    if isinstance(x, dict):
        return {k: _clean(v) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [_clean(v) for v in x]
    if hasattr(x, "item") and not isinstance(x, (str, bytes)):   # numpy scalars
        try:
            return _clean(x.item())
        except (TypeError, ValueError):
            return x
    return x


class JsonlLog:
    """Appends records to `dest` (a path, opened in append mode, or a text
    file object).  Thread-safe; each record is flushed when written."""

    def __init__(self, dest, clock=time.time):
        self._own = isinstance(dest, (str, os.PathLike))
        self._fh = open(dest, "a") if self._own else dest
        self._clock = clock
        self._mu = threading.Lock()

    def write(self, kind: str, **fields):
        rec = {"kind": kind, "time": self._clock()}
        rec.update(_clean(fields))
        line = json.dumps(rec, allow_nan=False, separators=(",", ":"))
        with self._mu:
            self._fh.write(line + "\n")
            self._fh.flush()

    def close(self):
        if self._own and self._fh is not None:
            self._fh.close()
        self._fh = None


def as_log(log):
    """None, a JsonlLog, or a path / file object to open one on."""
    if log is None or isinstance(log, JsonlLog):
        return log
    return JsonlLog(log)


def read(path):
    """The records of a JSONL log, in order."""
    with open(path) as fh:
        return [json.loads(line) for line in fh if line.strip()]
