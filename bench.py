"""Benchmark of the PTA-MD fine-burst engine on GB300.

One bench step is one coarse step of the Practical Time Averaging protocol
on the single large specimen: a 49^3-cell FCC Al cube (470,596 atoms) at
300 K under tension at 1e-3 1/s with h = 1 s, i.e. three grip increments,
three fine bursts of 5,000 velocity-Verlet steps (FP32 pair arithmetic,
FP64 accumulators) and the coarse-step update.  The metric is atom-steps/s
(atoms x fine steps per second), whole job.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl pta|reference]
                    [--workload large|plain|batched|uneven|served|precision|profile|verify]

Under torchrun (N > 1) every rank advances its own specimen (independent
replicas, no collective on the data path); the time is the maximum over
ranks and the value counts the work of all ranks.  ``--impl reference``
times the FP64 CPU oracle on this machine's host cores on bounded samples of
the same workload (it is the reference arm: there is no other implementation
of the method to run).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import pta_inputs as PI  # noqa: E402

# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
WORKLOADS = {
    "large": dict(name="large_fp32_n49", n_cells=49, T0=300.0, rate=1e-3, burst=5000,
                  precision=1, count=1,
                  desc="49^3-cell FCC Al cube (470,596 atoms), 300 K, tension 1e-3/s, h=1 s, "
                       "3 bursts x 5,000 steps per coarse step, FP32 pair math, FP64 "
                       "accumulators"),
    "plain": dict(name="plain_fp64_n10", n_cells=10, T0=300.0, rate=1e-3, burst=2000,
                  precision=0, count=1,
                  desc="10^3-cell FCC Al cube (4,000 atoms), 300 K, tension 1e-3/s, "
                       "3 bursts x 2,000 steps per coarse step, FP64 throughout"),
    "batched": dict(name="batched_64x_n20", n_cells=20, T0=None, rate=None, burst=2000,
                    precision=1, count=64, lanes=1,
                    desc="64 replicas of a 20^3-cell cube (32,000 atoms each), T0 cycling "
                         "10/100/300 K, half tension half compression, rates log-uniform "
                         "1e-4..1e-3/s, 3 bursts x 2,000 steps per coarse step, one launch "
                         "set per fine step for all replicas"),
    "served": dict(name="served_poisson_realtime", n_cells=None, T0=None, rate=None, burst=2000,
                   precision=1, count=None, lanes=1,
                   desc="Poisson trace (cube side uniform 10..49 cells, T0 in 10/100/300 K, rate "
                        "log-uniform 1e-4..1e-3/s, tension or compression p=0.5, target strain "
                        "0.05..0.15 shortened to at most 4 coarse steps) replayed on the wall "
                        "clock at ~70% of the measured batched throughput; admission by memory "
                        "footprint and slots at tick boundaries (continuous batching), 3 x 2,000 "
                        "fine steps per coarse step"),
    "precision": dict(name="precision_by_size", n_cells=None, T0=300.0, rate=None, burst=1000,
                      precision=1, count=7,
                      desc="mixed precision vs FP64 per size (10..49 cells), same seed"),
    "verify": dict(name="verify_fine_dynamics_n20", n_cells=20, T0=300.0, rate=None, burst=2000,
                   precision=1, count=1,
                   desc="fine-dynamics verification: 20^3-cell cube (32,000 atoms, 8 nm), loaded "
                        "to 3.1% strain, then 5 slow jumps of h = 20,000 steps (Delta = 4,000) "
                        "at 2e-4 strain per jump: one uninterrupted ramped trajectory against "
                        "PTA with 2,000-step bursts, relative errors per jump"),
    "peaks": dict(name="op_rates", n_cells=None, T0=None, rate=None, burst=None, precision=1,
                  count=1,
                  desc="the probe's rates: FMA (FP32, packed FP32, FP64) and the operations "
                       "a pair pass evaluating each unordered pair once would add per pair for "
                       "deterministic 64-bit fixed-point j-side sums"),
    "profile": dict(name="profile_case", n_cells=None, T0=300.0, rate=None, burst=None,
                    precision=1, count=1,
                    desc="one specimen for Nsight Compute captures: --n-cells cube, "
                         "--precision, a 1e-3 strain step, a warm burst of --prof-warm steps "
                         "and a burst of --prof-steps steps"),
    "uneven": dict(name="uneven_28x_n10_49", n_cells=None, T0=300.0, rate=None, burst=2000,
                   precision=1, count=28, lanes=1,
                   desc="4 cubes each of 10,15,20,25,30,40,49 cells (3,786,384 atoms), "
                        "alternating tension/compression, 300 K, 3 bursts x 2,000 steps"),
}



PAIR_SOURCES = ("k_pair_f32.cu", "k_mixed.cuh", "k_pair_common.cuh", "pta_dev.cuh")


def pair_source_sha() -> str:
    """First 16 hex digits of the SHA-256 of the mixed-precision pair kernels'
    sources (concatenated in PAIR_SOURCES order)."""
    import hashlib
    h = hashlib.sha256()
    for name in PAIR_SOURCES:
        with open(os.path.join(ROOT, "paper_2603_07321_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def captured_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` from the committed Nsight Compute
    summary, or None when the summary is missing or the kernel's source has
    changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "%s_%s.md" % (kernel, workload))
    try:
        txt = open(path).read()
        vals = dict(line.split(": ", 1) for line in txt.splitlines()
                    if line.startswith(("dram_bytes_per_launch:", "kernel_source_sha256_16:")))
        cur = pair_source_sha()
        if vals.get("kernel_source_sha256_16", "").strip() != cur:
            return None
        return int(vals["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


def measure_fma_peaks(P, target_ms: float = 150.0):
    """FMA rates of this GPU (TFLOP/s) from the library's probe: scalar FP32,
    packed FP32 (two lanes per instruction) and FP64, each one launch of about
    target_ms after a calibration launch."""
    out = {}
    for kind, name in ((0, "fp32"), (1, "fp32x2"), (2, "fp64")):
        it = 2000 if kind < 2 else 200
        P.pta_measure_fma_rate(kind, it)
        fl, ms = P.pta_measure_fma_rate(kind, it)
        it = max(it, int(it * target_ms / max(ms, 1e-3)))
        fl, ms = P.pta_measure_fma_rate(kind, it)
        out[name] = fl / (ms / 1e3) / 1e12
    return out


def lanes_of(args, wl) -> int:
    """Threads per atom for the workload's specimens: --lanes if given, else
    the workload's setting (batched workloads run one lane per atom: the
    library's automatic choice sizes lanes for a specimen running alone, and a
    batch fills the device without them), else 0 (automatic)."""
    return args.lanes if args.lanes is not None else wl.get("lanes", 0)


def perfect_lattice_pairs(n_cells: int, rc_over_a0: float = 2.0) -> int:
    """Number of unordered atom pairs closer than rc in a perfect n^3-cell
    FCC cube (counted exactly over lattice vectors, r < rc strict)."""
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    R = int(np.ceil(rc_over_a0)) + 1
    total = 0
    n = n_cells
    for b1 in range(4):
        for b2 in range(4):
            d0 = basis[b2] - basis[b1]
            for i in range(-R, R + 1):
                for j in range(-R, R + 1):
                    for k in range(-R, R + 1):
                        d = d0 + np.array([i, j, k])
                        r2 = float(d @ d)
                        if r2 == 0.0 or not (r2 < rc_over_a0 ** 2):
                            continue
                        # cells c with c + (i,j,k) inside [0, n)^3
                        total += (n - abs(i)) * (n - abs(j)) * (n - abs(k)) if \
                            max(abs(i), abs(j), abs(k)) < n else 0
    return total // 2


# algorithmic floating-point operations (each add, multiply, divide, square
# root counted once, a fused multiply-add twice), from the oracle's formulas:
# per unordered pair within rc: density pass 19, force pass 41; per atom and
# step 33 (embedding, two half-kicks, drift, kinetic and potential energy)
FLOP_DENSITY_PAIR = 19
FLOP_FORCE_PAIR = 41
FLOP_ATOM = 33


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int = 0):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.dev = device_index

    def start(self):
        try:
            self.fh = open(self.path, "w")
            cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                   "-lms", "200"]
            uuid = os.environ.get("PTA_GPU_UUID")
            if uuid:
                cmd += ["-i", uuid]
            else:
                cmd += ["-i", str(self.dev)]
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out = {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                   "reasons": sorted(reasons), "samples": len(sm)}
        return out


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_requests(wl, rank):
    """The specimens one rank advances: every rank runs the whole workload
    on its own replicas (distinct seeds), so per-GPU work is fixed."""
    if wl["name"].startswith("batched"):
        reqs = PI.config_batched(64, 20)
    elif wl["name"].startswith("uneven"):
        reqs = PI.config_uneven()
    else:
        reqs = [PI.SpecimenRequest(n_cells=wl["n_cells"], T0=wl["T0"], seed=1,
                                   strain_rate=wl["rate"], burst_steps=wl["burst"])]
    for r in reqs:
        r.seed = r.seed + 100000 * rank
    return reqs


def max_over_ranks(x: float, device="cpu") -> float:
    """Maximum of x over the ranks of the default process group (x itself
    without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# own arm
# ---------------------------------------------------------------------------
def run_served(args, wl):
    """Served workload: the request loop of paper_2603_07321_gb300.serve on
    the Poisson trace replayed in real time at ~70% of the device's measured
    batched throughput (served_leg); one JSON line with the measured
    coarse-step, full-curve and queue-wait latencies."""
    import torch
    import paper_2603_07321_gb300 as P
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    P.build()
    sampler = ClockSampler(local)
    sampler.start()
    cap = batched_leg(P)["value"]
    res = served_leg(P, capacity=cap, n_requests=args.served_requests)
    clocks = sampler.stop()
    out = {"metric": "atom-steps/s", "value": res["value"], "unit": "atom-steps/s",
           "n_gpus": ws, "steps": res["ticks"], "warmup": 0,
           "ms_per_step": res["wall_s"] * 1e3 / max(res["ticks"], 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic (seeded Poisson request trace, replayed in real time)",
           "config": {"workload": wl["name"], "description": wl["desc"],
                      "parallelism": "continuous batching"},
           "served": res, "clocks": clocks}
    if rank == 0:
        print(json.dumps(out), flush=True)
    return out


def batched_leg(P, steps: int = 1, warmup: int = 1):
    """The batched ensemble (64 replicas of the 20^3-cell cube, one launch set
    per fine step for all of them) as a sub-result of the default run:
    atom-steps/s over `steps` coarse steps after `warmup`."""
    import torch
    reqs = PI.config_batched(64, 20)
    ctxs = [P.Ctx(r.n_cells, T0=r.T0, seed=r.seed, precision=1, burst_steps=r.burst_steps,
                  strain_rate=r.strain_rate, lanes=1) for r in reqs]
    b = P.Batch(ctxs)
    for _ in range(warmup):
        b.coarse_step()
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        b.coarse_step()
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    natoms = sum(c.n for c in ctxs)
    value = natoms * 3 * 2000 * steps / (ms / 1e3)
    b.close()
    for c in ctxs:
        c.close()
    # the same replica on the plain single-specimen path (alone on the GPU,
    # its automatic layout): what the replicas would get run one at a time
    r = reqs[0]
    solo = P.Ctx(r.n_cells, T0=r.T0, seed=r.seed, precision=1, burst_steps=r.burst_steps,
                 strain_rate=r.strain_rate)
    for _ in range(warmup):
        solo.coarse_step()
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(steps):
        solo.coarse_step()
    e1.record(st)
    torch.cuda.synchronize()
    ms_solo = e0.elapsed_time(e1)
    solo_value = solo.n * 3 * 2000 * steps / (ms_solo / 1e3)
    solo_lanes = solo.layout()["lanes"]
    solo.close()
    return {"workload": "batched_64x_n20", "value": value, "unit": "atom-steps/s",
            "atoms": natoms, "specimens": len(ctxs), "coarse_steps": steps, "warmup": warmup,
            "ms_per_coarse_step": ms / steps,
            "solo_replica": {"value": solo_value, "atoms": solo.n, "lanes": solo_lanes,
                             "ms_per_coarse_step": ms_solo / steps},
            "gain_over_solo_replicas": value / solo_value,
            "description": WORKLOADS["batched"]["desc"]}


def served_leg(P, capacity: float, n_requests: int = 28, utilisation: float = 0.7,
               max_coarse: int = 4, seed: int = 7, time_cap_s: float = 120.0):
    """The served workload in real time: the seeded Poisson trace (cube side
    10..49, T0, rate, sign, target as in the served config) replayed on the
    wall clock with its arrival rate scaled so that the offered load is
    `utilisation` of `capacity` (atom-steps/s); each request's curve is
    shortened to at most `max_coarse` coarse steps so that whole curves
    finish and their latencies are measured.  Requests are admitted by
    memory footprint and slots at tick boundaries (continuous batching)."""
    import torch
    from paper_2603_07321_gb300.serve import GPUEngine, Request, Scheduler
    trace = PI.served_trace(n_requests, seed=seed)
    h = 1.0
    work, reqs = 0.0, []
    for i, r in enumerate(trace):
        n_coarse = int(min(max_coarse, np.ceil(r.target_strain / (abs(r.strain_rate) * h))))
        target = n_coarse * abs(r.strain_rate) * h
        work += 4 * r.n_cells ** 3 * 3 * r.burst_steps * (n_coarse + 1)
        reqs.append(Request(rid=i, n_cells=r.n_cells, T0=r.T0, seed=r.seed,
                            strain_rate=r.strain_rate, target_strain=target,
                            arrival_s=r.arrival_s, burst_steps=r.burst_steps, precision=1,
                            lanes=1))
    # time-scale the arrivals: offered load = utilisation x capacity
    span = trace[-1].arrival_s
    offered_span = work / (utilisation * capacity)
    scale = offered_span / span
    for r in reqs:
        r.arrival_s *= scale
    eng = GPUEngine()
    free, _ = torch.cuda.mem_get_info()
    sched = Scheduler(eng, mem_budget_bytes=int(0.8 * free), max_slots=64)
    t0 = time.perf_counter()
    for r in sorted(reqs, key=lambda r: r.arrival_s):
        sched.submit(r)
    while (sched.waiting or sched.live) and time.perf_counter() - t0 < time_cap_s:
        if not sched.tick():
            nxt = sched.waiting[0].arrival_s if sched.waiting else None
            if nxt is None:
                break
            wait = nxt - sched.now()
            if wait > 0:
                time.sleep(min(wait, 0.05))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    stats = sched.stats()
    eng.close()
    for s in list(sched.live.values()):
        s["handle"].close()
    return {"workload": "served_poisson_realtime", "value": stats["atom_steps"] / wall,
            "unit": "atom-steps/s", "requests": n_requests, "utilisation_target": utilisation,
            "capacity_assumed": capacity, "arrival_time_scale": scale,
            "mean_arrival_rate_per_s": n_requests / (span * scale), "wall_s": wall,
            "max_coarse_steps_per_curve": max_coarse, **stats}


def run_precision(args, wl):
    """Mixed precision against FP64, per specimen size (both on the GPU from
    the same seed): relative differences of the burst means of K, U, T, the
    differences in units of their combined standard error, and the per-atom
    force error on identical positions."""
    import torch
    import paper_2603_07321_gb300 as P
    P.build()
    torch.cuda.set_device(0)
    rows = []
    for n in (10, 15, 20, 25, 30, 40, 49):
        c64 = P.Ctx(n, T0=300.0, seed=11, precision=P.PREC_FP64)
        c32 = P.Ctx(n, T0=300.0, seed=11, precision=P.PREC_MIXED)
        pos, vel = c64.get_state()
        c32.set_state(pos, vel)   # identical start
        f64, _, _ = c64.forces()
        f32, _, _ = c32.forces()
        scale = np.sqrt(np.mean(np.sum(f64 ** 2, axis=1)))
        ferr = float(np.max(np.linalg.norm(f32 - f64, axis=1)) / scale)
        for c in (c64, c32):
            c.apply_strain(1e-3)
        steps = args.prec_steps
        a64 = c64.fine_burst(steps)
        a32 = c32.fine_burst(steps)
        rel = [abs(a32.mean[q] - a64.mean[q]) / abs(a64.mean[q]) for q in range(3)]
        z = [abs(a32.mean[q] - a64.mean[q]) / max(np.hypot(a32.se[q], a64.se[q]), 1e-300)
             for q in range(3)]
        rows.append({"n_cells": n, "atoms": c64.n, "force_err_rel_rms": ferr,
                     "mean_rel_diff": {"K": rel[0], "U": rel[1], "T": rel[2]},
                     "diff_in_se": {"K": z[0], "U": z[1], "T": z[2]},
                     "fp64": list(a64.mean), "mixed": list(a32.mean)})
        c64.close()
        c32.close()
    out = {"metric": "mixed-vs-fp64 slow-variable error", "workload": "precision_by_size",
           "burst_steps": args.prec_steps, "rows": rows}
    print(json.dumps(out), flush=True)
    return out


def run_profile(args, wl):
    """A small, fixed case for profiler captures (run it under Nsight Compute
    with PTA_GRAPH_FLAT=1, graphs without conditional nodes, whose kernel
    nodes the profiler can capture); prints the second burst's throughput."""
    import torch
    import paper_2603_07321_gb300 as P
    P.build()
    torch.cuda.set_device(0)
    ctx = P.Ctx(args.n_cells, T0=300.0, seed=1, precision=args.precision,
                lanes=args.lanes or 0)
    ctx.apply_strain(1e-3)
    ctx.fine_burst(args.prof_warm)
    torch.cuda.synchronize()
    t = time.perf_counter()
    a = ctx.fine_burst(args.prof_steps)
    dt = time.perf_counter() - t
    out = {"workload": "profile_case", "n_cells": args.n_cells, "atoms": ctx.n,
           "precision": args.precision, "steps": args.prof_steps, "seconds": dt,
           "atom_steps_per_s": ctx.n * args.prof_steps / dt, "rebuilds": a.rebuilds,
           "prunes": a.prunes, "layout": ctx.layout()}
    print(json.dumps(out), flush=True)
    ctx.close()
    return out


def measure_op_rates(P, target_ms: float = 100.0):
    """Rates (G operations/s) of the probe's kinds 3-5: 64-bit integer
    reductions to global memory at scattered addresses, 64-bit shared-memory
    atomic adds, FP32 -> int64 conversions."""
    out = {}
    for kind, name in ((3, "red_global_u64"), (4, "atom_shared_u64"), (5, "cvt_f32_s64")):
        it = 64
        P.pta_measure_fma_rate(kind, it)
        ops, ms = P.pta_measure_fma_rate(kind, it)
        it = max(it, int(it * target_ms / max(ms, 1e-3)))
        ops, ms = P.pta_measure_fma_rate(kind, it)
        out[name] = ops / (ms / 1e3) / 1e9
    return out


def run_peaks(args, wl):
    """The probe's rates, and what they mean for a force pass that evaluates
    each unordered pair once with deterministic (64-bit fixed-point) j-side
    sums of F_x, F_y, F_z and the pair energy: four conversions and four
    reductions per pair, against the full-list pass's two evaluations."""
    import torch
    import paper_2603_07321_gb300 as P
    P.build()
    torch.cuda.set_device(0)
    fma = measure_fma_peaks(P)
    ops = measure_op_rates(P)
    pairs = perfect_lattice_pairs(49)
    per_pair = 4  # F_x, F_y, F_z, pair energy
    out = {"workload": wl["name"], "description": wl["desc"],
           "sm_count": torch.cuda.get_device_properties(0).multi_processor_count,
           "fma_tflops": fma, "ops_gops": ops,
           "newton3_force_pass_floor_us": {
               "pairs": pairs,
               "j_side_reductions_global": pairs * per_pair / (ops["red_global_u64"] * 1e9) * 1e6,
               "j_side_atomics_shared": pairs * per_pair / (ops["atom_shared_u64"] * 1e9) * 1e6,
               "conversions": pairs * per_pair / (ops["cvt_f32_s64"] * 1e9) * 1e6}}
    print(json.dumps(out), flush=True)
    return out


def run_verify(args, wl):
    """Sec. Verification with fine dynamics: relative errors of the PTA slow
    variables against the fine dynamics' measures, per slow jump."""
    import torch
    import paper_2603_07321_gb300 as P
    from paper_2603_07321_gb300.verify import fine_vs_pta
    P.build()
    torch.cuda.set_device(0)
    t = time.perf_counter()
    out = fine_vs_pta(wl["n_cells"], T0=wl["T0"], seed=1, strain0=0.031, prep_increments=10,
                      prep_steps=1000, h_steps=20000, delta_steps=4000, n_jumps=5,
                      burst_steps=wl["burst"], strain_per_jump=2e-4, precision=wl["precision"])
    dt = time.perf_counter() - t
    rows = [{"jump": k + 1, "fine_steps": (k + 1) * 20000 + 4000,
             "error_pct": {"K": 100 * out["errors"][k][0], "U": 100 * out["errors"][k][1],
                           "T": 100 * out["errors"][k][2]},
             "v_pta": out["v_pta"][k].tolist(), "v_fine": out["v_fine"][k + 1].tolist(),
             "source": out["sources"][k]} for k in range(len(out["errors"]))]
    res = {"workload": wl["name"], "description": wl["desc"], "seconds": dt,
           "fine_steps": out["fine_steps"], "pta_steps": out["pta_steps"],
           "v_fine_t0": out["v_fine"][0].tolist(), "rows": rows}
    print(json.dumps(res), flush=True)
    return res


def run_pta(args, wl):
    import torch
    import paper_2603_07321_gb300 as P

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    P.build()
    reqs = rank_requests(wl, rank)
    ctxs = []
    for r in reqs:
        ctxs.append(P.Ctx(r.n_cells, T0=r.T0, seed=r.seed, precision=wl["precision"],
                          burst_steps=r.burst_steps, strain_rate=r.strain_rate,
                          lanes=lanes_of(args, wl)))
    natoms = sum(c.n for c in ctxs)
    batch = P.Batch(ctxs) if len(ctxs) > 1 else None
    stepper = batch if batch is not None else ctxs[0]

    def one_step():
        if batch is not None:
            return batch.coarse_step()
        return [ctxs[0].coarse_step()]

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        one_step()
    barrier()
    # the FP32 / FP64 FMA peaks of this GPU, measured with its clocks sampled
    psampler = ClockSampler(local)
    psampler.start()
    peaks = measure_fma_peaks(P)
    peak_clocks = psampler.stop()
    barrier()
    # headline: the coarse steps alone, no per-kernel timing events
    sampler = ClockSampler(local)
    sampler.start()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(st)
    results = []
    for _ in range(args.steps):
        results.append(one_step())
    e1.record(st)
    barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    t_max = max_over_ranks(ms, "cuda")
    # per-kernel split, from a separate coarse step with CUDA events around
    # each part of every fine-step iteration (reported apart from the headline)
    stepper.set_timing(True)
    barrier()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(st)
    one_step()
    e3.record(st)
    barrier()
    split_ms = e2.elapsed_time(e3)
    kt = stepper.timing()
    stepper.set_timing(False)
    fine_per_step = 3 * max(r.burst_steps for r in reqs)
    atom_steps_rank = sum(c.n * 3 * r.burst_steps for c, r in zip(ctxs, reqs)) * args.steps
    value = atom_steps_rank * ws / (t_max / 1e3)

    # live roofline of the dominant kernel (the force pass): algorithmic flops
    # per launch / mean CUDA-event duration of the launch in the timed region
    pairs = sum(perfect_lattice_pairs(r.n_cells) for r in reqs)
    iters = max(kt.iterations, 1)
    force_ms = kt.force_ms / iters
    dens_ms = kt.density_ms / iters
    flops_force = pairs * FLOP_FORCE_PAIR + natoms * (FLOP_ATOM - 5)
    flops_dens = pairs * FLOP_DENSITY_PAIR + natoms * 5
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    # the peak of the arithmetic the pair passes run in: the larger measured
    # FP32 FMA rate (scalar or packed), or the FP64 FMA rate for FP64 specimens
    mixed = wl["precision"] == 1
    peak_tflops = max(peaks["fp32"], peaks["fp32x2"]) if mixed else peaks["fp64"]
    ach_force = flops_force / (force_ms / 1e3) / 1e12
    ach_dens = flops_dens / (dens_ms / 1e3) / 1e12
    dominant = ("force", ach_force, force_ms) if force_ms >= dens_ms else ("density", ach_dens,
                                                                           dens_ms)

    # launches of this library's kernels in the timed region: per fine-step
    # iteration the decide kernel and, per (precision, lanes) group, the
    # density and force passes; per list build 12 kernels; per pruning one
    # kernel per group and one bookkeeping kernel; per burst the grip
    # increment, burst start and burst end; per coarse step the update
    groups = len({(c.params.precision, c.layout()["lanes"]) for c in ctxs})
    builds = sum(b.rebuilds for step in results for r in step for b in r.burst)
    prunes = sum(b.prunes for step in results for r in step for b in r.burst)
    bursts = 3 * args.steps
    launches = int(kt.iterations * (1 + 2 * groups) + builds * 12 + prunes * (groups + 1)
                   + bursts * 3 + args.steps)

    # end to end through the public API with host buffers: per step the state
    # goes host -> device from pinned memory, the coarse step runs, and the
    # state and result come back to pinned host memory
    e2e = None
    if batch is None:
        c = ctxs[0]
        hpos = torch.empty((c.n, 3), dtype=torch.float64, pin_memory=True).numpy()
        hvel = torch.empty((c.n, 3), dtype=torch.float64, pin_memory=True).numpy()
        p, v = c.get_state()
        hpos[:] = p
        hvel[:] = v
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            c.set_state(hpos, hvel)
            c.coarse_step()
            p, v = c.get_state()
            hpos[:] = p
            hvel[:] = v
        barrier()
        dt = max_over_ranks(time.perf_counter() - t0, "cuda")
        nb = c.n * 6 * 8
        e2e = {"value": atom_steps_rank * ws / dt, "unit": "atom-steps/s",
               "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb + 3 * 416}

    layout_info = {"lanes": sorted({c.layout()["lanes"] for c in ctxs}),
                   "source": sorted({c.layout_source for c in ctxs}),
                   "skin": sorted({c.params.skin for c in ctxs}),
                   "prune_margin": sorted({c.params.prune_margin for c in ctxs})}
    # batched and served sub-results (single-GPU default run only)
    subs = {}
    if ws == 1 and not args.no_sub and wl["name"].startswith("large"):
        if batch is not None:
            batch.close()
            batch = None
        for c in ctxs:
            c.close()
        ctxs = []
        torch.cuda.synchronize()
        subs["batched"] = batched_leg(P)
        subs["batched"]["gain_over_plain"] = subs["batched"]["value"] / value
        subs["served"] = served_leg(P, capacity=subs["batched"]["value"])
        subs["served"]["gain_over_plain"] = subs["served"]["value"] / value

    out = None
    if rank == 0:
        cpu = cpu_baseline(wl, reqs[0].n_cells) if (ws == 1 and not args.no_cpu) else None
        out = {
            "metric": "atom-steps/s",
            "value": value,
            "unit": "atom-steps/s",
            "n_gpus": ws,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": t_max / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32" if wl["precision"] == 1 else "f64",
            "data": "synthetic (FCC lattice + seeded Maxwell-Boltzmann velocities)",
            "config": {"workload": wl["name"], "description": wl["desc"], "atoms": natoms,
                       "specimens": len(ctxs), "fine_steps_per_step": fine_per_step,
                       "lanes_per_atom": layout_info["lanes"],
                       "layout": layout_info,
                       "accumulators": "f64", "l2": "working set > 129 MB L2 (no flush)",
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "roofline": {"bound": "alu", "kernel": "k_%s_f32" % dominant[0]
                         if wl["precision"] == 1 else "k_%s_f64" % dominant[0],
                         "achieved": dominant[1], "peak": peak_tflops, "unit": "TFLOP/s",
                         "frac": dominant[1] / peak_tflops,
                         "traffic": captured_traffic("k_%s_f32" % dominant[0], wl["name"])
                         if wl["precision"] == 1 else None,
                         "peak_source": "measured: FMA-chain probe (pta_measure_fma_rate) "
                                        "on this GPU, %d SMs, median SM clock %s MHz; %s" % (
                                            n_sm, peak_clocks["sm_mhz"],
                                            "the larger of scalar and packed FP32" if mixed
                                            else "FP64"),
                         "peaks_measured_tflops": peaks,
                         "launch_ms": dominant[2],
                         "kernels_ms_per_iteration": {"rebuild": kt.rebuild_ms / iters,
                                                      "density": dens_ms, "force": force_ms},
                         "split_run": "one extra coarse step with per-iteration CUDA events "
                                      "(%d iterations, %.1f ms), not part of the headline" % (
                                          kt.iterations, split_ms)},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
            **subs,
        }
        print(json.dumps(out), flush=True)
    if batch is not None:
        batch.close()
    for c in ctxs:
        c.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return out


def cpu_baseline(wl, n_cells, target_s: float = 15.0):
    """The FP64 oracle timed on this machine's host cores on a bounded
    sample of the same workload (a few velocity-Verlet steps of one cube)."""
    import oracle as O
    O.build()
    spec = O.Specimen(n_cells)
    spec.thermalise(300.0, 1)
    spec.apply_strain(1e-3)
    t = time.perf_counter()
    spec.burst(1)
    one = time.perf_counter() - t
    steps = int(max(2, min(200, target_s / max(one, 1e-6))))
    t = time.perf_counter()
    spec.burst(steps)
    dt = time.perf_counter() - t
    return {"value": spec.n * steps / dt, "unit": "atom-steps/s",
            "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count())),
            "kind": "oracle",
            "sample": "%d velocity-Verlet steps of the %d-atom cube (FP64 oracle, OpenMP over "
                      "atoms, pairs found anew every step)" % (steps, spec.n)}


# ---------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------
def run_reference(args, wl):
    ws, rank, _ = _dist()
    if rank != 0:
        return None
    import oracle as O
    O.build()
    n_cells = wl["n_cells"] or 49
    spec = O.Specimen(n_cells)
    spec.thermalise(300.0, 1)
    spec.apply_strain(1e-3)
    sample_steps = args.ref_sample
    for _ in range(args.warmup):
        spec.burst(sample_steps)
    t = time.perf_counter()
    for _ in range(args.steps):
        spec.burst(sample_steps)
    dt = time.perf_counter() - t
    value = spec.n * sample_steps * args.steps / dt
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count()))
    sample = ("each step: %d velocity-Verlet steps of the %d-atom cube (FP64 oracle, OpenMP "
              "over atoms)" % (sample_steps, spec.n))
    out = {"impl": "reference", "metric": "atom-steps/s", "value": value,
           "unit": "atom-steps/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": wl["name"], "description": wl["desc"]},
           "cpu_baseline": {"kind": "oracle", "cores": cores, "sample": sample, "value": value,
                            "unit": "atom-steps/s"},
           "e2e": {"value": value, "unit": "atom-steps/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="pta", choices=["pta", "reference"])
    ap.add_argument("--workload", default="large", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--served-requests", type=int, default=40,
                    help="requests of the served workload's trace")
    ap.add_argument("--no-sub", action="store_true",
                    help="skip the batched and served sub-results of the default run")
    ap.add_argument("--lanes", type=int, default=None,
                    help="threads per atom of every specimen (default: the workload's choice; "
                         "0 = the library's per-specimen choice)")
    ap.add_argument("--prec-steps", type=int, default=1000,
                    help="burst length of the precision comparison")
    ap.add_argument("--ref-sample", type=int, default=4,
                    help="fine steps per reference-arm step")
    ap.add_argument("--n-cells", type=int, default=49, help="profile workload: cube side")
    ap.add_argument("--precision", type=int, default=1, help="profile workload: 0 FP64, 1 mixed")
    ap.add_argument("--prof-warm", type=int, default=5, help="profile workload: warm burst")
    ap.add_argument("--prof-steps", type=int, default=30, help="profile workload: timed burst")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, wl)
    elif args.workload == "served":
        run_served(args, wl)
    elif args.workload == "precision":
        run_precision(args, wl)
    elif args.workload == "profile":
        run_profile(args, wl)
    elif args.workload == "peaks":
        run_peaks(args, wl)
    elif args.workload == "verify":
        run_verify(args, wl)
    else:
        run_pta(args, wl)


if __name__ == "__main__":
    main()
