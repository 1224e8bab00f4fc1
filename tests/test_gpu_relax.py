"""Thermal relaxation before loading on the GPU (right grip free along the
load axis), against the oracle's relaxation burst from the same state."""
import numpy as np
import pytest

from gpu_util import gpu_package, on_grid

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    return gpu_package()


@pytest.mark.parametrize("prec", [0, 1])
def test_relaxation_window_matches_the_oracle(P, oracle, prec):
    shape = (5, 5, 6)
    ctx = P.Ctx(shape, T0=300.0, seed=17, precision=prec)
    spec = oracle.Specimen(shape)
    spec.thermalise(300.0, 17)
    pos = on_grid(spec.pos)
    vel = np.asarray(spec.vel, dtype=np.float32).astype(np.float64) if prec else spec.vel.copy()
    spec.pos, spec.vel = pos.copy(), vel.copy()
    ctx.set_state(pos, vel)
    # tolerance 0 and max_steps = window: exactly one window
    a, steps = ctx.relax(window=200, max_steps=200, tol_gpa=0.0)
    s_ref = spec.burst(200, relax=True)
    p, v = ctx.get_state()
    assert steps == 200 and a.status == 0
    fl = ctx.flags()
    ax = 2
    other = [0, 1]
    right, left = fl == 2, fl == 1
    assert np.array_equal(p[left], pos[left])
    assert np.array_equal(p[right][:, other], pos[right][:, other])
    assert np.all(v[right][:, other] == 0)
    assert np.max(np.abs(p[right, ax] - pos[right, ax])) > 1e-3
    L_s = 6 * 4.05
    if prec == 0:
        assert np.max(np.abs(p - spec.pos)) < 1e-8
        assert np.allclose(ctx.series(), s_ref, rtol=1e-9, atol=1e-9)
    else:
        assert np.max(np.abs(p - spec.pos)) < 1e-4 * L_s
        assert np.allclose(ctx.series()[:, :2], s_ref[:, :2], rtol=1e-5)
    ctx.close()


def test_relaxation_stops_within_tolerance_and_the_grip_then_stays(P):
    ctx = P.Ctx((5, 5, 6), T0=300.0, seed=3, precision=P.PREC_MIXED)
    a0 = ctx.fine_burst(2000)            # grips fixed: the cut cube pulls on them
    a, steps = ctx.relax(window=2000, max_steps=20000, tol_gpa=0.5)
    assert a.status == 0 and 2000 <= steps <= 20000 and steps % 2000 == 0
    assert abs(a.mean[2]) < 0.5 or steps + 2000 > 20000
    assert abs(a.mean[2]) < abs(a0.mean[2])
    fl = ctx.flags()
    p1, _ = ctx.get_state()
    ctx.fine_burst(200)                  # the right grip is fixed again
    p2, v2 = ctx.get_state()
    assert np.array_equal(p2[fl != 0], p1[fl != 0])
    assert np.all(v2[fl != 0] == 0)
    ctx.close()


def test_relaxation_procedure_matches_the_oracle_in_fp64(P, oracle):
    shape = (5, 5, 6)
    for tol, expect in ((1e9, 100), (0.0, 400)):      # one window / runs to max_steps
        ctx = P.Ctx(shape, T0=300.0, seed=19, precision=P.PREC_FP64)
        spec = oracle.Specimen(shape)
        spec.thermalise(300.0, 19)
        ctx.set_state(spec.pos, spec.vel)
        a, steps = ctx.relax(window=100, max_steps=450, tol_gpa=tol)
        s_ref, steps_ref = spec.relax(100, 450, tol)
        assert steps == steps_ref == expect
        p, v = ctx.get_state()
        assert np.max(np.abs(p - spec.pos)) < 1e-7
        assert np.max(np.abs(v - spec.vel)) < 1e-9
        assert np.all(v[ctx.flags() == 2] == 0)
        assert a.mean[2] == pytest.approx(s_ref[:, 2].mean(), rel=1e-6, abs=1e-9)
        ctx.close()
