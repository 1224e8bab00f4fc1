"""Adaptive burst length (appendix, Eq. (R_m_conv)) on the GPU.

The device applies the running-average convergence test in the last block of
every fine step's reduction and ends a specimen's burst once K, U and T have
all converged.  The oracle's convergence function, applied to the samples the
device itself recorded, must reach the same decisions (steps of convergence,
which variables converged, where the burst stopped) and the same means: the
running sums are formed in step order on both sides, so these are exact.
"""
import numpy as np
import pytest

from gpu_util import gpu_package

pytestmark = pytest.mark.gpu

FLOOR = (1e-12, 1e-12, 0.05)


@pytest.fixture(scope="module")
def P():
    return gpu_package()


def _check_against_oracle(oracle, a, series, lag, tol, n_max, block=100):
    from oracle.pta_logic import converged_averages
    means, counts, mask, run = converged_averages(series, lag, tol, FLOOR, n_max=n_max)
    assert a.status == 0
    assert a.nsteps == run == len(series)
    assert a.converged == mask
    assert list(a.nsamples) == list(counts)
    assert np.array_equal(np.array(a.mean), means)
    for q in range(3):
        _, se = oracle.burst_averages(series[: counts[q]], block=block)
        if np.isfinite(se[q]):
            assert a.se[q] == pytest.approx(se[q], rel=1e-9)
    return mask, run


@pytest.mark.parametrize("prec", [0, 1])
def test_adaptive_burst_follows_the_convergence_rule(P, oracle, prec):
    lag, tol, n_max = 20, (0.002, 0.0005, 0.2), 3000
    ctx = P.Ctx((6, 6, 7), T0=300.0, seed=3, precision=prec, conv_lag=lag, conv_tol=tol,
                block_steps=20)
    ctx.apply_strain(1e-3)
    a = ctx.fine_burst(n_max)
    s = ctx.series()
    mask, run = _check_against_oracle(oracle, a, s, lag, tol, n_max, block=20)
    assert 2 * lag <= run < n_max and mask == 7   # these tolerances converge early
    ctx.close()


def test_unconverged_variables_run_to_the_burst_length(P, oracle):
    # a zero tolerance never passes: the burst runs to its length and every
    # mean is the average of all samples
    lag, tol, n_max = 10, (0.0, 0.0, 0.0), 400
    ctx = P.Ctx((5, 5, 6), T0=300.0, seed=4, precision=P.PREC_MIXED, conv_lag=lag, conv_tol=tol)
    a = ctx.fine_burst(n_max)
    s = ctx.series()
    mask, run = _check_against_oracle(oracle, a, s, lag, tol, n_max)
    assert mask == 0 and run == n_max
    ctx.close()


def test_fixed_length_when_the_lag_is_zero(P):
    ctx = P.Ctx((5, 5, 6), T0=300.0, seed=4, precision=P.PREC_MIXED)
    a = ctx.fine_burst(150)
    assert a.nsteps == 150 and a.converged == 0 and list(a.nsamples) == [150] * 3
    ctx.close()


def test_ragged_adaptive_ends_in_a_batch_equal_solo(P, oracle):
    kw = dict(precision=P.PREC_MIXED, conv_lag=25, conv_tol=(0.002, 0.0005, 0.2))
    specs = [((6, 6, 7), 300.0, 5), ((5, 6, 6), 100.0, 6), ((7, 6, 6), 10.0, 7)]
    solo = []
    for sh, T0, seed in specs:
        c = P.Ctx(sh, T0=T0, seed=seed, **kw)
        c.apply_strain(1e-3)
        a = c.fine_burst(2000)
        solo.append((a.nsteps, list(a.mean), c.get_state()[0]))
        c.close()
    ctxs = [P.Ctx(sh, T0=T0, seed=seed, **kw) for sh, T0, seed in specs]
    b = P.Batch(ctxs)
    b.apply_strain([1e-3] * 3)
    res = b.fine_burst([2000] * 3)
    assert len({r.nsteps for r in res}) > 1          # the members stop at different steps
    for c, r, (n, m, pos) in zip(ctxs, res, solo):
        assert r.nsteps == n and list(r.mean) == m
        assert np.array_equal(c.get_state()[0], pos)
    b.close()
    for c in ctxs:
        c.close()


def test_coarse_step_with_adaptive_bursts(P):
    ctx = P.Ctx((6, 6, 7), T0=300.0, seed=8, precision=P.PREC_MIXED, burst_steps=3000,
                conv_lag=25, conv_tol=(0.002, 0.0005, 0.2))
    r = ctx.coarse_step()
    assert r.status == 0
    assert all(0 < b.nsteps <= 3000 for b in r.burst)
    assert any(b.nsteps < 3000 for b in r.burst)
    ctx.close()
