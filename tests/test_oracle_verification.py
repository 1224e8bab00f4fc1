"""Pins of the oracle's fine-dynamics verification (Sec. Verification with
fine dynamics): the ramped-grip burst and the windowing of Eq. (measure)."""
import copy

import numpy as np
import pytest

from oracle import pta_logic as L


@pytest.fixture()
def spec(oracle):
    s = oracle.Specimen((3, 3, 4))
    s.thermalise(300.0, 5)
    return s


def test_ramp_zero_is_the_ordinary_burst(oracle, spec):
    a = copy.deepcopy(spec)
    s1 = spec.burst(15)
    s2 = a.burst(15, ramp=0.0)
    assert np.array_equal(s1, s2) and np.array_equal(spec.pos, a.pos)


def test_ramp_moves_only_the_right_grip_by_n_du(oracle, spec):
    p0 = spec.pos.copy()
    ramp = 3e-5
    spec.burst(20, ramp=ramp)
    du = ramp * spec.L_s
    right, left = spec.flags == 2, spec.flags == 1
    # every right-grip atom advanced by exactly 20 increments along z, nothing else
    assert np.allclose(spec.pos[right, 2] - p0[right, 2], 20 * du, rtol=0, atol=1e-12)
    assert np.array_equal(spec.pos[right, :2], p0[right, :2])
    assert np.array_equal(spec.pos[left], p0[left])
    assert spec.u == pytest.approx(20 * du, rel=1e-14)


def test_split_bursts_are_one_trajectory(oracle, spec):
    # a burst restarts from its starting positions' forces: windows of one
    # uninterrupted ramped trajectory are exactly its pieces
    a = copy.deepcopy(spec)
    whole = spec.burst(30, ramp=2e-5)
    parts = np.concatenate([a.burst(12, ramp=2e-5), a.burst(18, ramp=2e-5)])
    assert np.array_equal(whole, parts) and np.array_equal(spec.pos, a.pos)


def test_fine_measures_are_window_means_of_the_trajectory(oracle, spec):
    a = copy.deepcopy(spec)
    h, d, n = 20, 5, 3
    v = L.fine_dynamics_measures(spec, h, d, n, 2e-5)
    series = a.burst(n * h + d, ramp=2e-5)
    for k in range(n + 1):
        end = k * h + d
        assert np.allclose(v[k], series[end - d:end].mean(axis=0), rtol=1e-15, atol=0)
    assert v.shape == (n + 1, 3)


def test_verification_params_keep_the_protocol_consistent():
    p = L.verification_params(20000, 4000, 1e-8)
    # the PTA grip increments equal the ramp's displacement over the same steps
    inc = p.step_increments()
    assert inc[0] == pytest.approx(1e-8 * 16000, rel=1e-12)
    assert inc[1] == pytest.approx(1e-8 * 2000, rel=1e-12)
    assert p.Delta == pytest.approx(p.h / 5)


def test_verification_error_is_relative_to_the_fine_value():
    e = L.verification_errors([[1.1, -2.0, 0.0]], [[1.0, -2.5, 0.5]])
    assert np.allclose(e, [[0.1, 0.2, 1.0]])
