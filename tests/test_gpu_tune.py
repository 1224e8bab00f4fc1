"""The layout autotuner on the GPU: it measures every candidate it can
create and ranks them by throughput."""
import pytest

from gpu_util import gpu_package

pytestmark = pytest.mark.gpu


def test_tuner_ranks_the_candidates_it_can_create():
    P = gpu_package()
    from paper_2603_07321_gb300.tune import tune
    best, table = tune(8, precision=P.PREC_MIXED, lanes=(1, 2), skins=(1.0, 2.0),
                       steps=60, warm=20)
    assert len(table) == 4
    rates = [r for r, _ in table]
    assert rates == sorted(rates, reverse=True) and rates[-1] > 0
    assert best == table[0][1]
    ctx = P.Ctx(8, **best)          # the winner is a valid creation
    ctx.close()


def test_tuner_for_a_batch_of_replicas():
    P = gpu_package()
    from paper_2603_07321_gb300.tune import tune
    best, table = tune(6, replicas=4, lanes=(1, 4), skins=(2.0,), steps=40, warm=10)
    assert len(table) == 2 and best["lanes"] in (1, 4)
