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


# ---------------------------------------------------------------------------
# adaptive burst length: the appendix's running-average convergence test
# ---------------------------------------------------------------------------
def _linear(n, a, b):
    i = np.arange(1, n + 1, dtype=np.float64)
    return a + b * i


def test_convergence_of_linear_series_at_the_closed_form_step():
    # m_i = a + b i has R^(i) = a + b (i + 1) / 2, so R^(i) - R^(i-k) = b k / 2 and
    # e(i) = (b k / 2) / (a + b (i + 1) / 2) < tol  <=>  i > k / tol - 2 a / b - 1
    from oracle.pta_logic import converged_averages
    k = 10
    cols = [(1.0, 1.0, 0.05), (100.0, 1.0, 0.05), (0.0, 1.0, 0.02)]
    s = np.stack([_linear(2000, a, b) for a, b, _ in cols], axis=1)
    tol = [t for _, _, t in cols]
    means, counts, mask, run = converged_averages(s, k, tol, (1e-12, 1e-12, 1e-12))
    expect = []
    for a, b, t in cols:
        bound = k / t - 2 * a / b - 1
        i = 2 * k
        while not i > bound:
            i += k
        expect.append(i)
    assert list(counts) == expect == [200, 20, 500]
    assert mask == 7 and run == 500
    for q, (a, b, _) in enumerate(cols):
        assert means[q] == pytest.approx(a + b * (expect[q] + 1) / 2, rel=1e-14)


def test_constant_and_periodic_series_converge_at_the_first_test():
    from oracle.pta_logic import converged_averages
    n, k = 400, 8
    i = np.arange(1, n + 1)
    s = np.stack([np.full(n, 3.5), 7.0 + 0.5 * (-1.0) ** i, -2.0 + np.cos(np.pi * i / 2)], axis=1)
    means, counts, mask, run = converged_averages(s, k, (1e-9,) * 3, (1e-12,) * 3)
    # k a multiple of the periods: R^(2k) = R^(k) exactly, e = 0
    assert mask == 7 and run == 2 * k and list(counts) == [2 * k] * 3
    assert np.allclose(means, [3.5, 7.0, -2.0], rtol=0, atol=1e-14)


def test_zero_tolerance_runs_to_n_max_with_the_full_average():
    from oracle.pta_logic import converged_averages
    rng = np.random.default_rng(3)
    s = 1.0 + rng.normal(0, 0.1, (300, 3))
    means, counts, mask, run = converged_averages(s, 10, (0.0,) * 3, (1e-12,) * 3, n_max=250)
    assert mask == 0 and run == 250 and list(counts) == [250] * 3
    assert np.allclose(means, s[:250].mean(axis=0), rtol=1e-13)


def test_floor_lets_a_near_zero_stress_converge():
    from oracle.pta_logic import converged_averages
    n, k = 2000, 7
    i = np.arange(1, n + 1)
    t = 1e-3 * (-1.0) ** i                 # a stress that averages to 0 GPa
    s = np.stack([np.full(n, 5.0), np.full(n, -9.0), t], axis=1)
    # with the 0.05 GPa floor: e(14) = |0 - (-1e-3 / 7)| / 0.05 < 0.05
    _, counts, mask, _ = converged_averages(s, k, (0.05,) * 3, (1e-12, 1e-12, 0.05))
    assert mask == 7 and counts[2] == 2 * k
    # relative to the running average itself (0 at even i, -1e-3 / i at odd
    # i, for an odd lag) e is 1 or unbounded: it never converges
    _, counts, mask, run = converged_averages(s, k, (0.05,) * 3, (1e-12, 1e-12, 1e-300))
    assert not mask & 4 and run == n and counts[2] == n


def test_convergence_against_brute_force_recomputation():
    from oracle.pta_logic import converged_averages
    rng = np.random.default_rng(11)
    for trial in range(20):
        n, k = int(rng.integers(50, 600)), int(rng.integers(1, 40))
        s = rng.normal([10.0, -50.0, 0.2], [1.0, 0.5, 0.3], (n, 3))
        tol = rng.uniform(0.001, 0.05, 3)
        means, counts, mask, run = converged_averages(s, k, tol, (1e-12, 1e-12, 0.05))
        # brute force: every candidate step checked from scratch
        for q in range(3):
            first = None
            for i in range(2 * k, n + 1, k):
                a = s[:i, q].sum() / i
                b = s[:i - k, q].sum() / (i - k)
                if abs(a - b) / max(abs(a), (1e-12, 1e-12, 0.05)[q]) < tol[q]:
                    first = i
                    break
            if first is not None and first <= run:
                assert mask & (1 << q) and counts[q] == first
                assert means[q] == pytest.approx(s[:first, q].mean(), rel=1e-12, abs=1e-12)
            else:
                assert not mask & (1 << q) and counts[q] == run
