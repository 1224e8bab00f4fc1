"""The layout autotuner on the GPU: it measures every candidate it can
create, ranks them by throughput, caches the winner, and contexts with an
automatic layout pick the cached one up."""
import numpy as np
import pytest

import pta_inputs as PI
from gpu_util import gpu_package

pytestmark = pytest.mark.gpu


@pytest.fixture()
def cache(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    monkeypatch.setenv("PTA_TUNE_CACHE", str(path))
    return path


def test_tuner_ranks_the_candidates_it_can_create(cache):
    P = gpu_package()
    from paper_2603_07321_gb300.tune import tune
    best, table = tune(8, precision=P.PREC_MIXED, lanes=(1, 2), skins=(1.0, 2.0),
                       steps=60, warm=20)
    assert len(table) == 4
    rates = [r for r, _ in table]
    assert rates == sorted(rates, reverse=True) and rates[-1] > 0
    assert best == table[0][1]
    assert cache.exists()
    ctx = P.Ctx(8, precision=P.PREC_MIXED)      # the winner is picked up
    assert ctx.layout_source == "tuned"
    assert ctx.layout()["lanes"] == best["lanes"]
    assert ctx.params.skin == best["skin"]
    ctx.close()


def test_tuned_layout_gives_the_same_results(cache):
    # the tuned layout computes the same physics: a pruning margin leaves
    # the summation order as it is (bit-identical, mixed precision); a skin
    # changes the cell edge h = rc + skin and with it the order of each
    # atom's list entries, so FP64 results agree to rounding
    P = gpu_package()
    from paper_2603_07321_gb300.tune import tune
    shape = 7
    pos = PI.gaussian_jitter_fcc((shape,) * 3, 0.1, seed=4)
    vel0 = PI.random_velocities(len(pos), 3e-3, seed=5)

    def run(**kw):
        c = P.Ctx(shape, **kw)
        vel = vel0.copy()
        vel[c.flags() != 0] = 0.0
        c.set_state(pos, vel)
        f, pe, _ = c.forces()
        c.fine_burst(100)
        r = (f, pe, c.series().copy(), c.get_state()[0], c.params.skin, c.layout_source)
        c.close()
        return r

    auto = P.Ctx(shape, precision=P.PREC_MIXED, tuned=False)
    L = auto.layout()["lanes"]
    skin = auto.params.skin
    auto.close()
    best, _ = tune(shape, precision=P.PREC_MIXED, lanes=(L,), skins=(skin,), margins=(0.2, 0.5),
                   steps=30, warm=10)
    a = run(precision=P.PREC_MIXED)
    b = run(precision=P.PREC_MIXED, tuned=False)
    assert a[5] == "tuned" and b[5] == "automatic"
    for x, y in zip(a[:4], b[:4]):
        assert np.array_equal(x, y)

    best, _ = tune(shape, precision=P.PREC_FP64, lanes=(L,), skins=(1.2, 2.4), margins=(0.3,),
                   steps=30, warm=10)
    a = run(precision=P.PREC_FP64)
    b = run(precision=P.PREC_FP64, tuned=False)
    assert a[5] == "tuned" and a[4] == best["skin"] and a[4] != b[4]
    np.testing.assert_allclose(a[0], b[0], rtol=0, atol=1e-12 * np.abs(b[0]).max())
    np.testing.assert_allclose(a[1], b[1], rtol=1e-12)
    np.testing.assert_allclose(a[2], b[2], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(a[3], b[3], rtol=0, atol=1e-9)


def test_tuner_for_a_batch_of_replicas(cache):
    P = gpu_package()
    from paper_2603_07321_gb300.tune import tune, lookup
    best, table = tune(6, replicas=4, lanes=(1, 4), skins=(2.0,), steps=40, warm=10)
    assert len(table) == 2 and best["lanes"] in (1, 4)
    assert lookup(4 * 6 ** 3, 4, 1)["lanes"] == best["lanes"]
    assert lookup(4 * 6 ** 3, 1, 1) is None      # another replica count, another entry
