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
    # candidates that differ only in skin and pruning margin: the tuned
    # layout must give bit-identical forces and trajectories in FP64
    P = gpu_package()
    from paper_2603_07321_gb300.tune import tune
    shape = 7
    auto = P.Ctx(shape, precision=P.PREC_FP64, tuned=False)
    L = auto.layout()["lanes"]
    auto.close()
    best, _ = tune(shape, precision=P.PREC_FP64, lanes=(L,), skins=(1.2, 2.4),
                   margins=(0.3,), steps=30, warm=10)
    pos = PI.gaussian_jitter_fcc((shape,) * 3, 0.1, seed=4)
    vel = PI.random_velocities(len(pos), 3e-3, seed=5)
    out = []
    for tuned in (True, False):
        c = P.Ctx(shape, precision=P.PREC_FP64, tuned=tuned)
        assert c.layout_source == ("tuned" if tuned else "automatic")
        vel[c.flags() != 0] = 0.0
        c.set_state(pos, vel)
        f, pe, _ = c.forces()
        c.fine_burst(100)
        out.append((f, pe, c.series().copy(), c.get_state()[0], c.params.skin))
        c.close()
    assert out[0][4] == best["skin"]
    for a, b in zip(out[0][:4], out[1][:4]):
        assert np.array_equal(a, b)


def test_tuner_for_a_batch_of_replicas(cache):
    P = gpu_package()
    from paper_2603_07321_gb300.tune import tune, lookup
    best, table = tune(6, replicas=4, lanes=(1, 4), skins=(2.0,), steps=40, warm=10)
    assert len(table) == 2 and best["lanes"] in (1, 4)
    assert lookup(4 * 6 ** 3, 4, 1)["lanes"] == best["lanes"]
    assert lookup(4 * 6 ** 3, 1, 1) is None      # another replica count, another entry
