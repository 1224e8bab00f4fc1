"""Verification of PTA against the fine dynamics (Sec. Verification with
fine dynamics).

From one prepared state, two runs:

* fine: one uninterrupted trajectory under continuous loading (the right
  grip advances with every step, pta_ramp_burst), over the slow interval
  [-Delta, n_jumps h]; the slow variable at t_k = k h is Eq. (measure), the
  mean of the state functions over the Delta that ends at t_k -- no Simpson
  rule and no restart from guessed initial conditions;
* PTA: the same state advanced by n_jumps coarse steps of h (the same load
  rate), with bursts of burst_steps steps (Eqs. (dvdt_algo) - (jump_err)).

The error of each slow variable at each jump is |v^PTA - v^fine| / |v^fine|,
the quantity of the paper's Tables 2 and 3.  h and Delta are given in fine
steps; the library's h, Delta (s) and strain rate (1/s) follow from them.
All dynamics and averages run on the GPU through the C ABI; this module only
sequences the calls and forms the ratios.
"""
from __future__ import annotations

import numpy as np


def prepare(n_cells, T0: float, seed: int, strain: float, increments: int, settle_steps: int,
            precision: int, **kw):
    """A context loaded to `strain` in `increments` grip increments, each
    followed by a burst of settle_steps steps; returns (ctx, checkpoint)."""
    from . import Ctx
    ctx = Ctx(n_cells, T0=T0, seed=seed, precision=precision, **kw)
    for _ in range(increments):
        ctx.apply_strain(strain / increments)
        ctx.fine_burst(settle_steps)
    return ctx, ctx.save()


def fine_vs_pta(n_cells, *, T0=300.0, seed=1, strain0=0.0, prep_increments=1, prep_steps=0,
                h_steps=20000, delta_steps=4000, n_jumps=5, burst_steps=2000,
                strain_per_jump=2e-4, precision=1, dt_fs=1.0, **kw):
    """Run the verification; returns a dict with the fine measures v_fine
    [n_jumps + 1, 3] (t = 0..n_jumps h), the PTA results per jump and the
    relative errors [n_jumps, 3] (K, U, T)."""
    from . import Ctx
    ramp = strain_per_jump / h_steps          # strain per fine step
    dt_s = dt_fs * 1e-15
    src, blob = prepare(n_cells, T0, seed, strain0, prep_increments, prep_steps, precision,
                        dt_fs=dt_fs, **kw)
    src.close()
    # fine dynamics: one ramped trajectory from slow time -Delta
    fine = Ctx(n_cells, T0=T0, seed=seed, precision=precision, dt_fs=dt_fs, **kw)
    fine.restore(blob)
    v_fine = []
    for k in range(n_jumps + 1):
        if k > 0:
            fine.ramp_burst(h_steps - delta_steps, ramp)
        a = fine.ramp_burst(delta_steps, ramp)
        v_fine.append(list(a.mean))
    fine_strain = fine.strain
    fine.close()
    # PTA from the same state at the same load rate
    pta = Ctx(n_cells, T0=T0, seed=seed, precision=precision, dt_fs=dt_fs,
              h=h_steps * dt_s, Delta=delta_steps * dt_s, strain_rate=ramp / dt_s,
              burst_steps=burst_steps, **kw)
    pta.restore(blob)
    res = [pta.coarse_step() for _ in range(n_jumps)]
    pta.close()
    v_fine = np.array(v_fine)
    v_pta = np.array([list(r.v) for r in res])
    err = np.abs(v_pta - v_fine[1:]) / np.abs(v_fine[1:])
    return {"v_fine": v_fine, "v_pta": v_pta, "errors": err,
            "sources": [list(r.source) for r in res], "strain_fine_end": fine_strain,
            "strain_pta_end": res[-1].strain, "fine_steps": n_jumps * h_steps + delta_steps,
            "pta_steps": 3 * burst_steps * (n_jumps + 1)}
