"""The mixed-precision form against its own contract: FP32 pair terms with
FP64 (or exact hi/lo FP32) state and FP64 reductions must keep NVE energy
conserved over long bursts and the slow variables within the stated
tolerances of the FP64 oracle.

Bounds: velocity Verlet at dt = 1 fs conserves a shadow energy; E = K + U
fluctuates around it by O(dt^2) and does not drift in exact arithmetic.
Rounding adds a random walk; a systematic drift would show as a slope.  The
drift is measured as the least-squares slope of E over the burst times its
length, relative to |E| (about 1.26e4 eV here), and bounded by 1e-8 for both
forms (measured: |drift| ~ 5e-10 in either form, spread of E ~ 8e-7)."""
import numpy as np
import pytest

import pta_inputs as PI
from gpu_util import gpu_package, on_grid

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    return gpu_package()


def _drift(series):
    e = series[:, 0] + series[:, 1]
    t = np.arange(len(e), dtype=np.float64)
    slope = np.polyfit(t, e, 1)[0]
    return slope * len(e) / abs(e.mean()), (e.max() - e.min()) / abs(e.mean())


def test_nve_energy_drift_over_50000_steps(P):
    out = {}
    for prec in (P.PREC_FP64, P.PREC_MIXED):
        ctx = P.Ctx((10, 10, 10), T0=300.0, seed=21, precision=prec, burst_steps=50000)
        if prec == P.PREC_MIXED:  # the FP64 context's exact start
            ctx.set_state(*start)
        else:
            start = ctx.get_state()
            start = (on_grid(start[0]), start[1].astype(np.float32).astype(np.float64))
            ctx.set_state(*start)
        a = ctx.fine_burst(50000)
        assert a.status == 0 and a.nsteps == 50000
        out[prec] = _drift(ctx.series())
        ctx.close()
    print("NVE drift over 50,000 steps (relative): FP64 %.3e (spread %.3e), mixed %.3e "
          "(spread %.3e)" % (out[0][0], out[0][1], out[1][0], out[1][1]))
    for prec in out:
        assert abs(out[prec][0]) < 1e-8, out


@pytest.mark.parametrize("shape", [(4, 4, 4), (6, 6, 6), (8, 8, 8)])
def test_mixed_slow_variables_against_the_oracle(P, oracle, shape):
    ctx = P.Ctx(shape, T0=300.0, seed=12, precision=P.PREC_MIXED)
    spec = oracle.Specimen(shape)
    spec.thermalise(300.0, 12)
    pos = on_grid(spec.pos)
    vel = np.asarray(spec.vel, dtype=np.float32).astype(np.float64)
    spec.pos, spec.vel = pos.copy(), vel.copy()
    ctx.set_state(pos, vel)
    ctx.apply_strain(2e-3)
    spec.apply_strain(2e-3)
    a = ctx.fine_burst(200)
    s_gpu = ctx.series()
    s_ref = spec.burst(200)
    rel = np.max(np.abs(s_gpu[:, :2] - s_ref[:, :2]) / np.abs(s_ref[:, :2]), axis=0)
    dT = np.max(np.abs(s_gpu[:, 2] - s_ref[:, 2]))
    mean_rel = np.abs(np.array(a.mean[:2]) - s_ref[:, :2].mean(axis=0)) / np.abs(
        s_ref[:, :2].mean(axis=0))
    print("mixed vs oracle, %s, 200 steps: max per-step rel err K %.2e U %.2e, T %.2e GPa; "
          "burst means rel K %.2e U %.2e, T %.2e GPa" % (
              shape, rel[0], rel[1], dT, mean_rel[0], mean_rel[1],
              abs(a.mean[2] - s_ref[:, 2].mean())))
    assert rel[0] < 1e-5 and rel[1] < 1e-5 and dT < 1e-3
    ctx.close()
