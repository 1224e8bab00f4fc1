"""Continuous-batching request loop for PTA simulations.

Requests (a specimen size, temperature, seed, strain rate and target strain)
arrive over time.  Each is admitted as soon as a slot and enough device
memory (its pta_footprint_bytes) are free; all admitted specimens stay
resident on the device and advance together, one slow-time tick at a time
(pta_batch_tick: three grip increments and bursts, then the coarse-step
update; a newly admitted specimen's first tick runs its initial bursts).
A specimen leaves when its strain reaches the target; its slot and memory
go to the next waiting request at the next tick boundary.

The scheduler (admission, bookkeeping, latency statistics) is separate from
the engine that owns the device work, so that its logic can be exercised on
the CPU with a stand-in engine.  GPUEngine is the real one.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    n_cells: int
    T0: float
    seed: int
    strain_rate: float
    target_strain: float
    arrival_s: float = 0.0
    burst_steps: int = 2000
    precision: int = 1
    lanes: int = 0        # threads per atom (0: the library's per-specimen choice)
    neigh_cap: int = 0    # Verlet-list capacity per atom (0: the library's default)


@dataclass
class Result:
    rid: int
    status: str                      # "done", "rejected", "failed"
    arrival_s: float
    admitted_s: float = math.nan
    finished_s: float = math.nan
    curve: list = field(default_factory=list)   # per coarse step: (strain, v[3], source[3])
    tick_latency_s: list = field(default_factory=list)
    atom_steps: int = 0
    error: str = ""


class SchedulerError(RuntimeError):
    pass


class Scheduler:
    """Admission by slots and device-memory footprint, FIFO order."""

    def __init__(self, engine, mem_budget_bytes: int, max_slots: int = 64, clock=None, log=None):
        """log: a metrics.JsonlLog (or a path / text file) receiving one record
        per request event, per tick and per specimen coarse step."""
        from .metrics import as_log
        self.log = as_log(log)
        self.engine = engine
        self.budget = int(mem_budget_bytes)
        self.max_slots = int(max_slots)
        self.clock = clock or time.perf_counter
        self.t0 = None
        self.waiting: list[Request] = []
        self.live: dict[int, dict] = {}       # rid -> {"req", "handle", "bytes", "result"}
        self.results: dict[int, Result] = {}
        self.used = 0
        self.ticks = 0

    # ----------------------------------------------------------------- input
    def now(self) -> float:
        if self.t0 is None:
            self.t0 = self.clock()
        return self.clock() - self.t0

    def _event(self, kind, **fields):
        if self.log is not None:
            self.log.write(kind, **fields)

    def submit(self, req: Request):
        err = self.engine.validate(req)
        if not err and self.engine.footprint(req) > self.budget:
            err = "larger than the memory budget"
        if err:
            self.results[req.rid] = Result(req.rid, "rejected", req.arrival_s, error=err)
            self._event("request_rejected", tag=req.rid, error=err)
            return False
        self.waiting.append(req)
        self._event("request_queued", tag=req.rid, arrival_s=req.arrival_s, n_cells=req.n_cells,
                    T0=req.T0, strain_rate=req.strain_rate, target_strain=req.target_strain)
        return True

    # ------------------------------------------------------------- admission
    def admit(self, now: float) -> list[int]:
        admitted = []
        while self.waiting and len(self.live) < self.max_slots:
            req = self.waiting[0]
            if req.arrival_s > now:
                break
            need = self.engine.footprint(req)
            if self.used + need > self.budget:
                break                          # FIFO: the head waits for memory
            try:
                h = self.engine.create(req)
            except MemoryError:
                break                          # device could not place it now: retry later
            except Exception as e:             # invalid on the device: reject
                self.waiting.pop(0)
                self.results[req.rid] = Result(req.rid, "rejected", req.arrival_s, error=str(e))
                self._event("request_rejected", tag=req.rid, error=str(e))
                continue
            self.waiting.pop(0)
            res = Result(req.rid, "running", req.arrival_s, admitted_s=now)
            self.live[req.rid] = {"req": req, "handle": h, "bytes": need, "result": res}
            self.used += need
            admitted.append(req.rid)
            self._event("request_admitted", tag=req.rid, wait_s=now - req.arrival_s, bytes=need)
        return admitted

    def _retire(self, rid: int, status: str, now: float, error: str = ""):
        slot = self.live.pop(rid)
        self.engine.destroy(slot["handle"])
        self.used -= slot["bytes"]
        res = slot["result"]
        res.status = status
        res.finished_s = now
        res.error = error
        self.results[rid] = res
        self._event("request_" + status, tag=rid, curve_latency_s=now - res.arrival_s,
                    coarse_steps=len(res.curve), atom_steps=res.atom_steps, error=error)

    # ------------------------------------------------------------------ loop
    def tick(self) -> bool:
        """One slow-time tick of every live specimen.  Returns False when no
        specimen is live."""
        now = self.now()
        self.admit(now)
        if not self.live:
            return False
        rids = list(self.live)
        handles = [self.live[r]["handle"] for r in rids]
        t = self.clock()
        outs = self.engine.tick(handles)
        dt = self.clock() - t
        now = self.now()
        self.ticks += 1
        self._event("tick", live=len(rids), latency_s=dt)
        for rid, out in zip(rids, outs):
            slot = self.live[rid]
            res = slot["result"]
            if out.get("error"):
                self._retire(rid, "failed", now, out["error"])
                continue
            if out.get("recovered"):
                # the engine replaced the specimen (restored from its state
                # before this tick, with more list capacity): it repeats
                # the tick next time; its memory grew
                slot["handle"] = out["handle"]
                grow = int(out.get("bytes", slot["bytes"])) - slot["bytes"]
                slot["bytes"] += grow
                self.used += grow
                self._event("request_recovered", tag=rid, reason=out.get("reason", ""),
                            neigh_cap=out.get("neigh_cap"), bytes=slot["bytes"])
                continue
            res.tick_latency_s.append(dt)
            res.atom_steps += out["atom_steps"]
            if not out.get("initial"):
                res.curve.append((out["strain"], out["v"], out["source"]))
            self._event("coarse", tag=rid, initial=bool(out.get("initial")),
                        strain=out["strain"], v=list(out["v"]), source=list(out["source"]))
            req = slot["req"]
            if abs(out["strain"]) >= req.target_strain - 1e-12:
                self._retire(rid, "done", now)
        return True

    def run(self, trace: list[Request], max_ticks: int | None = None, realtime: bool = True):
        """Serve a trace.  With realtime=True requests become admissible at
        their arrival time on the wall clock; otherwise all are admissible
        at once (a closed-loop stress test)."""
        for r in sorted(trace, key=lambda r: r.arrival_s):
            if not realtime:
                r.arrival_s = 0.0
            self.submit(r)
        while (self.waiting or self.live) and (max_ticks is None or self.ticks < max_ticks):
            if not self.tick():
                # nothing live: wait for the next arrival
                nxt = self.waiting[0].arrival_s if self.waiting else None
                if nxt is None:
                    break
                wait = nxt - self.now()
                if wait > 0:
                    time.sleep(min(wait, 0.05))
        return self.results

    def stats(self) -> dict:
        ticks = [x for r in self.results.values() for x in r.tick_latency_s]
        ticks += [x for s in self.live.values() for x in s["result"].tick_latency_s]
        curves = [r.finished_s - r.arrival_s for r in self.results.values() if r.status == "done"]
        waits = [r.admitted_s - r.arrival_s for r in self.results.values()
                 if r.status in ("done", "failed") and math.isfinite(r.admitted_s)]
        waits += [s["result"].admitted_s - s["result"].arrival_s for s in self.live.values()]
        steps = sum(r.atom_steps for r in self.results.values())
        steps += sum(s["result"].atom_steps for s in self.live.values())
        pct = lambda a, q: float(np.percentile(a, q)) if a else None
        return {"coarse_step_latency_s": {"p50": pct(ticks, 50), "p99": pct(ticks, 99),
                                          "count": len(ticks)},
                "curve_latency_s": {"p50": pct(curves, 50), "p99": pct(curves, 99),
                                    "count": len(curves)},
                "queue_wait_s": {"p50": pct(waits, 50), "p99": pct(waits, 99),
                                 "count": len(waits)},
                "atom_steps": steps, "ticks": self.ticks,
                "done": sum(1 for r in self.results.values() if r.status == "done"),
                "rejected": sum(1 for r in self.results.values() if r.status == "rejected"),
                "failed": sum(1 for r in self.results.values() if r.status == "failed")}


PTA_ENEIGH_OVERFLOW = -4


class GPUEngine:
    """The device side: one pta_ctx per specimen, one pta_batch over the live
    set, rebuilt when the set changes.

    With `recover`, every live specimen's state is checkpointed (to host
    memory) before each tick; a specimen whose tick reports a neighbour-list
    overflow (an atom gathered more neighbours than its list holds, e.g.
    under strong compression) is recreated with twice the list capacity,
    restored from that checkpoint and handed back to the scheduler, which
    runs its tick again with the next one.  List capacity changes only where
    entries are stored, not their order, so the recovered specimen continues
    exactly as one created with the larger capacity would have.  At most
    `max_regrow` recoveries per specimen; after that the failure stands."""

    def __init__(self, stream=None, replicas_hint: int = 16, recover: bool = True,
                 max_regrow: int = 4):
        from . import (PTAError, Batch, Ctx, default_params, make_specimen,
                       pta_footprint_bytes)
        self._PTAError, self._Batch, self._Ctx = PTAError, Batch, Ctx
        self._params, self._spec, self._fp = default_params, make_specimen, pta_footprint_bytes
        self.batch = None
        self.batch_members: list = []
        self.stream = stream
        self.replicas_hint = replicas_hint
        self.recover = recover
        self.max_regrow = max_regrow
        self._info: dict = {}       # id(ctx) -> {"req", "neigh_cap", "regrow"}

    def validate(self, req: Request) -> str:
        if req.n_cells < 3 or req.n_cells > 126:
            return "n_cells out of range"
        if not (req.T0 >= 0) or not math.isfinite(req.strain_rate) or req.strain_rate == 0:
            return "bad temperature or strain rate"
        if not (req.target_strain > 0):
            return "target strain must be positive"
        return ""

    def _p(self, req, neigh_cap: int = 0):
        kw = dict(precision=req.precision, burst_steps=req.burst_steps,
                  strain_rate=req.strain_rate, lanes=req.lanes,
                  neigh_cap=neigh_cap or req.neigh_cap)
        if not req.lanes:
            # the autotuner's layout for this size among ~replicas_hint live specimens
            from .tune import lookup
            hit = lookup(4 * req.n_cells ** 3, self.replicas_hint, req.precision)
            if hit:
                kw.update(hit)
        return self._params(**kw)

    def footprint(self, req: Request, neigh_cap: int = 0) -> int:
        return int(self._fp(self._spec(req.n_cells), self._p(req, neigh_cap)))

    def create(self, req: Request, neigh_cap: int = 0):
        try:
            ctx = self._Ctx(req.n_cells, T0=req.T0, seed=req.seed,
                            params=self._p(req, neigh_cap), stream=self.stream)
        except self._PTAError as e:
            if e.status == -2:
                raise MemoryError(str(e))
            raise
        self._info[id(ctx)] = {"req": req, "regrow": 0}
        return ctx

    def destroy(self, ctx):
        if self.batch is not None and ctx in self.batch_members:
            self.batch.close()
            self.batch = None
            self.batch_members = []
        self._info.pop(id(ctx), None)
        ctx.close()

    def _regrow(self, ctx, blob):
        """A replacement for ctx with twice its list capacity, in the state
        `blob` (taken before the failed tick), or None."""
        info = self._info.get(id(ctx))
        if info is None or info["regrow"] >= self.max_regrow:
            return None
        req = info["req"]
        cap = 2 * int(ctx.layout()["neigh_cap"])
        try:
            new = self.create(req, neigh_cap=cap)
        except (MemoryError, self._PTAError):
            return None
        try:
            new.restore(blob)
        except self._PTAError:
            self.destroy(new)
            return None
        self._info[id(new)]["regrow"] = info["regrow"] + 1
        self.destroy(ctx)
        return {"recovered": True, "handle": new, "neigh_cap": cap, "atom_steps": 0,
                "bytes": self.footprint(req, cap), "reason": "neighbour-list overflow"}

    def tick(self, ctxs):
        if self.batch is None or self.batch_members != list(ctxs):
            if self.batch is not None:
                self.batch.close()
            self.batch = self._Batch(ctxs)
            self.batch_members = list(ctxs)
        blobs = [c.save() for c in ctxs] if self.recover else None
        try:
            res = self.batch.tick()
        except self._PTAError as e:
            return [{"error": str(e)} for _ in ctxs]
        out = []
        for i, (c, r) in enumerate(zip(ctxs, res)):
            if r.status == PTA_ENEIGH_OVERFLOW and self.recover:
                rec = self._regrow(c, blobs[i])
                if rec is not None:
                    out.append(rec)
                    continue
            if r.status != 0:
                out.append({"error": "status %d" % r.status})
                continue
            steps = sum(b.nsteps for b in r.burst)
            out.append({"strain": r.strain, "v": list(r.v), "source": list(r.source),
                        "initial": r.source[0] == -1, "atom_steps": int(steps) * c.n})
        return out

    def close(self):
        if self.batch is not None:
            self.batch.close()
            self.batch = None
