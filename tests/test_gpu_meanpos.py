"""Mean atomic positions over a burst (Eq. (mean_pos)) on the GPU, against
the oracle's step-by-step sums of the same trajectory."""
import numpy as np
import pytest

from gpu_util import gpu_package, on_grid

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    return gpu_package()


def _pair(P, oracle, shape, prec, seed):
    ctx = P.Ctx(shape, T0=300.0, seed=seed, precision=prec, mean_positions=1)
    spec = oracle.Specimen(shape)
    spec.thermalise(300.0, seed)
    pos = on_grid(spec.pos)
    vel = np.asarray(spec.vel, dtype=np.float32).astype(np.float64) if prec else spec.vel
    spec.pos, spec.vel = pos.copy(), vel.copy()
    ctx.set_state(pos, vel)
    return ctx, spec


@pytest.mark.parametrize("prec,tol", [(0, 1e-8), (1, 2e-4)])
def test_mean_positions_match_the_oracle(P, oracle, prec, tol):
    ctx, spec = _pair(P, oracle, (5, 5, 6), prec, seed=13)
    ctx.apply_strain(2e-3)
    spec.apply_strain(2e-3)
    a = ctx.fine_burst(120)
    m = ctx.mean_positions()
    s_ref, m_ref = spec.burst_mean_positions(120)
    assert a.status == 0
    assert np.max(np.abs(m - m_ref)) < tol
    # the grips do not move: their mean is their position
    fl = ctx.flags()
    p, _ = ctx.get_state()
    assert np.allclose(m[fl != 0], p[fl != 0], rtol=0, atol=1e-10)
    ctx.close()


def test_mean_positions_restart_with_every_burst_and_batch_equals_solo(P):
    kw = dict(T0=300.0, precision=P.PREC_MIXED, mean_positions=1)
    shapes = [(5, 5, 6), (6, 5, 5)]
    solo = []
    for i, sh in enumerate(shapes):
        c = P.Ctx(sh, seed=20 + i, **kw)
        c.fine_burst(50)
        c.fine_burst(80)           # the second burst's mean alone
        solo.append(c.mean_positions())
        c.close()
    ctxs = [P.Ctx(sh, seed=20 + i, **kw) for i, sh in enumerate(shapes)]
    b = P.Batch(ctxs)
    b.fine_burst([50, 50])
    b.fine_burst([80, 80])
    for c, ref in zip(ctxs, solo):
        assert np.array_equal(c.mean_positions(), ref)
    b.close()
    for c in ctxs:
        c.close()


def test_mean_positions_errors(P):
    c = P.Ctx((4, 4, 4), precision=P.PREC_MIXED)
    c.fine_burst(10)
    with pytest.raises(P.PTAError) as e:
        c.mean_positions()
    assert e.value.status == -8          # not asked for at creation
    c.close()
    c = P.Ctx((4, 4, 4), precision=P.PREC_MIXED, mean_positions=1)
    with pytest.raises(P.PTAError):
        c.mean_positions()               # no burst yet
    c.close()
