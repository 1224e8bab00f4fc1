"""Pins of the oracle's coarse-step logic (Eqs. dvdt_algo, pta_pred, simp,
rel_err, jump_err) on synthetic slow-variable sequences (CPU)."""
import numpy as np
import pytest

from oracle import pta_logic as L


def _vec(x):
    return np.array([x, x, x], dtype=float)


def _run_sequence(params, R):
    """Feed R(s) sampled at the protocol's slow times; return results."""
    h, D = params.h, params.Delta
    st = L.initial_state(params, _vec(R(-D)), _vec(R(-D / 2)), _vec(R(0.0)))
    out = []
    t = 0.0
    for _ in range(6):
        st, res = L.coarse_update(params, st, _vec(R(t + h - D)), _vec(R(t + h - D / 2)),
                                  _vec(R(t + h)))
        out.append((t + h, res, st))
        t += h
    return out


def test_linear_sequence_is_predicted_exactly():
    # R linear in slow time: v(t) = R(t - Delta/2), dv/dt exact, Euler exact
    p = L.PTAParams(h=1.0)
    a, b = 3.0, 0.25
    for t, res, st in _run_sequence(p, lambda s: a + b * s):
        assert np.allclose(res.v_pred, res.v_d, rtol=1e-14)
        assert np.allclose(res.v_d, a + b * (t - p.Delta / 2), rtol=1e-14)
        assert np.all(res.source == L.SRC_PREDICTED)


def test_simpson_exact_for_cubic():
    # v_d(t+h) approximates (1/Delta) int_{t+h-Delta}^{t+h} R ds: exact for cubics
    p = L.PTAParams(h=1.0)
    R = lambda s: 1.0 + 0.3 * s - 0.2 * s ** 2 + 0.05 * s ** 3
    Rint = lambda s: s + 0.15 * s ** 2 - 0.2 / 3 * s ** 3 + 0.0125 * s ** 4
    for t, res, st in _run_sequence(p, R):
        exact = (Rint(t) - Rint(t - p.Delta)) / p.Delta
        assert np.allclose(res.v_d, exact, rtol=1e-13)


def test_step_in_measure_is_a_jump():
    p = L.PTAParams(h=1.0)
    R = lambda s: 10.0 + 0.01 * s + (5.0 if s > 3.5 else 0.0)
    out = _run_sequence(p, R)
    srcs = [int(res.source[0]) for _, res, _ in out]
    # steps ending at t=1,2,3 are smooth; the one ending at t=4 contains the step
    assert srcs[:3] == [L.SRC_PREDICTED] * 3
    assert srcs[3] == L.SRC_MEASURE_JUMP
    assert out[3][2].jump[0]
    # accepted value is the measure
    assert out[3][1].v[0] == out[3][1].v_d[0]


def test_jump_flag_changes_the_test():
    p = L.PTAParams(h=1.0, tol_v=(1e-9,) * 3, tol_j=(0.05,) * 3)
    st = L.PTAState(t=0.0, v=_vec(1.0), R_t=_vec(1.0), R_tmD=_vec(1.0), R_tmh=_vec(1.0),
                    jump=np.array([True, False, False]))
    # e1 = 0.1 >= tol_j; e2 = 0 so the ratio test says "jump" only if e1 > 0
    st2, res = L.coarse_update(p, st, _vec(1.1), _vec(1.1), _vec(1.1))
    assert res.jump[0] and res.source[0] == L.SRC_MEASURE_JUMP
    assert res.jump[1] and res.jump[2]
    # small e1 with an earlier jump flagged -> no jump, mismatch
    st = L.PTAState(t=0.0, v=_vec(1.0), R_t=_vec(1.0), R_tmD=_vec(1.0), R_tmh=_vec(0.9),
                    jump=np.array([True, False, False]))
    st2, res = L.coarse_update(p, st, _vec(1.01), _vec(1.01), _vec(1.01))
    assert not res.jump[0] and res.source[0] == L.SRC_MEASURE_MISMATCH
    # same without the flag: e1 = 0.01, e2 = 0.111 -> |e1/e2 - 1| = 0.91 >= 0.05 -> jump
    assert res.jump[1] and res.source[1] == L.SRC_MEASURE_JUMP


@pytest.mark.parametrize("seed", range(4))
def test_acceptance_invariants(seed):
    rng = np.random.default_rng(seed)
    p = L.PTAParams(h=1.0)
    st = L.initial_state(p, rng.normal(5, 1, 3), rng.normal(5, 1, 3), rng.normal(5, 1, 3))
    for _ in range(50):
        Ra, Rb, Rc = rng.normal(5, 0.3, (3, 3))
        st_new, res = L.coarse_update(p, st, Ra, Rb, Rc)
        for m in range(3):
            if res.e_v[m] < p.tol_v[m]:
                assert res.v[m] == res.v_pred[m] and res.source[m] == L.SRC_PREDICTED
            else:
                assert res.v[m] == res.v_d[m] and res.source[m] != L.SRC_PREDICTED
            assert res.jump[m] == (res.source[m] == L.SRC_MEASURE_JUMP)
        # the chain: R_{t-Delta} <- R_{t+h-Delta}, R_t <- R_{t+h}, R_{t-h} <- R_t
        assert np.array_equal(st_new.R_tmD, Ra) and np.array_equal(st_new.R_t, Rc)
        assert np.array_equal(st_new.R_tmh, st.R_t)
        st = st_new


def test_protocol_increments_sum_to_rate_times_h():
    p = L.PTAParams(h=1.0, strain_rate=-3e-4)
    assert sum(p.step_increments()) == pytest.approx(-3e-4 * 1.0, rel=1e-15)
    assert sum(p.init_increments()) == pytest.approx(-3e-4 * p.Delta, rel=1e-15)
    assert p.Delta == pytest.approx(0.2)
