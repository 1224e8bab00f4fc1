"""Pins of the oracle's potential, forces and pair finder (CPU only).

Each test checks the oracle against something other than itself: published
parameters, crystallographic shell counts, calculus (finite differences),
symmetry (Newton's third law, zero net force on a perfect periodic lattice)
or brute force.
"""
import math

import numpy as np
import pytest

import pta_inputs as PI
from conftest import golden


def _sc_literature():
    return {row[0]: float(row[1]) for row in golden("sutton_chen_al.txt")}


def test_potential_literature_long_range(oracle):
    # With a long cutoff the shifted-force terms vanish and the equilibrium c
    # must reproduce Sutton-Chen's published c and cohesive energy for Al.
    lit = _sc_literature()
    p = oracle.Potential(eps=lit["eps"], a=lit["a"], rc=60.0, n=int(lit["n"]), m=int(lit["m"]))
    assert p.c == pytest.approx(lit["c"], rel=2e-4)
    e = oracle.cohesive_energy(p, lit["a"])
    assert -e == pytest.approx(lit["cohesive_energy_ev"], rel=2e-3)


def test_shifted_force_is_c1_at_cutoff(oracle):
    p = oracle.Potential()
    for k in (p.n, p.m):
        assert oracle.phi(p, k, p.rc) == 0.0
        below = np.nextafter(p.rc, 0.0)
        assert abs(oracle.phi(p, k, below)) < 1e-14
        assert abs(oracle.dphi(p, k, below)) < 1e-12
        # derivative consistent with the function (central difference)
        for r in (2.6, 2.86, 4.05, 6.0, 7.9):
            h = 1e-6
            fd = (oracle.phi(p, k, r + h) - oracle.phi(p, k, r - h)) / (2 * h)
            assert fd == pytest.approx(oracle.dphi(p, k, r), rel=1e-8, abs=1e-12)
        # and it reduces to (a/r)^k near r -> 0 in relative terms
        r = 1e-3
        assert oracle.phi(p, k, r) / (p.a / r) ** k == pytest.approx(1.0, rel=1e-9)


def _shell_sums(pot, oracle):
    S = {pot.n: 0.0, pot.m: 0.0}
    for d2, cnt in golden("fcc_shells.txt"):
        r = pot.a * math.sqrt(float(d2))
        for k in S:
            S[k] += int(cnt) * oracle.phi(pot, k, r)
    return S


def test_periodic_lattice_energy_equals_shell_sums(oracle):
    # N-body energy of the perfect periodic crystal vs the closed form
    # eps [ 1/2 S_n - c sqrt(S_m) ] over the textbook coordination shells.
    pot = oracle.Potential()
    ncell = 5
    pos = PI.fcc_sites(ncell, pot.a)
    f, pe, rho = oracle.eam_periodic(pos, ncell * pot.a, pot)
    S = _shell_sums(pot, oracle)
    e_closed = pot.eps * (0.5 * S[pot.n] - pot.c * math.sqrt(S[pot.m]))
    assert np.allclose(pe, e_closed, rtol=1e-12, atol=0)
    assert np.allclose(rho, S[pot.m], rtol=1e-12)
    assert e_closed == pytest.approx(oracle.cohesive_energy(pot, pot.a), rel=1e-12)
    # perfect lattice: zero net force on every atom
    assert np.max(np.abs(f)) < 1e-12


def test_equilibrium_lattice_constant(oracle):
    # c is chosen so that dE/da = 0 at a0: check with the N-body periodic energy.
    pot = oracle.Potential()
    ncell = 5

    def e_of(a):
        pos = PI.fcc_sites(ncell, a)
        _, pe, _ = oracle.eam_periodic(pos, ncell * a, pot)
        return pe.mean()

    # (the 8th shell sits exactly at rc = 2a and enters E(a - h) at O(h^2),
    # so the central difference carries an O(h) bias: keep h small)
    h = 1e-5
    dEda = (e_of(pot.a + h) - e_of(pot.a - h)) / (2 * h)
    off = (e_of(1.01 * pot.a + h) - e_of(1.01 * pot.a - h)) / (2 * h)
    assert abs(dEda) < 2e-8
    assert abs(off) > 1e5 * abs(dEda)
    assert off > 0.0  # energy rises on stretching: a minimum, not a maximum


def test_dimer_closed_form(oracle):
    # two atoms: U = eps[phi_n(r) - 2 c sqrt(phi_m(r))], F_2 = -dU/dr along the bond
    pot = oracle.Potential()
    for r in (2.5, 2.86, 3.5, 5.0, 8.0):
        pos = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
        f, pe, rho = oracle.eam(pos, pot)
        pn, pm = oracle.phi(pot, pot.n, r), oracle.phi(pot, pot.m, r)
        dn, dm = oracle.dphi(pot, pot.n, r), oracle.dphi(pot, pot.m, r)
        U = pot.eps * (pn - 2.0 * pot.c * math.sqrt(pm))
        dUdr = pot.eps * (dn - pot.c * dm / math.sqrt(pm))
        assert pe.sum() == pytest.approx(U, rel=1e-13)
        assert f[1, 0] == pytest.approx(-dUdr, rel=1e-12)
        assert f[0, 0] == pytest.approx(dUdr, rel=1e-12)
        assert np.all(f[:, 1:] == 0.0)
        assert rho[0] == rho[1] == pytest.approx(pm, rel=1e-15)


def test_forces_are_minus_energy_gradient(oracle):
    pot = oracle.Potential()
    pos = PI.gaussian_jitter_fcc(3, 0.12, seed=11)
    f, _, _ = oracle.eam(pos, pot)
    rng = np.random.default_rng(3)
    h = 1e-5
    fscale = np.sqrt(np.mean(f ** 2))
    for i in rng.choice(len(pos), 12, replace=False):
        for d in range(3):
            p1 = pos.copy(); p1[i, d] += h
            p2 = pos.copy(); p2[i, d] -= h
            e1 = oracle.eam(p1, pot)[1].sum()
            e2 = oracle.eam(p2, pot)[1].sum()
            fd = -(e1 - e2) / (2 * h)
            assert abs(fd - f[i, d]) <= 1e-7 * fscale + 1e-9


def test_newton_third_law(oracle):
    pot = oracle.Potential()
    pos = PI.gaussian_jitter_fcc((4, 3, 5), 0.15, seed=5)
    f, _, _ = oracle.eam(pos, pot)
    assert np.max(np.abs(f.sum(axis=0))) < 1e-11 * np.abs(f).max() * len(pos)


def test_isolated_atom_has_no_energy(oracle):
    pot = oracle.Potential()
    pos = np.array([[0.0, 0, 0], [3.0, 0, 0], [50.0, 0, 0]])
    f, pe, rho = oracle.eam(pos, pot)
    assert rho[2] == 0.0 and pe[2] == 0.0 and np.all(f[2] == 0.0)


@pytest.mark.parametrize("seed", [1, 2])
def test_cell_pairs_equal_brute_force(oracle, seed):
    pos = PI.jittered_fcc((5, 4, 6), 0.4, seed)
    for rcut in (8.1, 9.1, 5.0):
        c1, l1 = oracle.pairs(pos, rcut, cap=400, method="cells")
        c2, l2 = oracle.pairs(pos, rcut, cap=400, method="brute")
        assert np.array_equal(c1, c2)
        assert np.array_equal(l1, l2)


def test_pair_predicate_is_strict(oracle):
    pos = np.array([[0.0, 0, 0], [8.1, 0, 0], [0, 8.0999999, 0]])
    c, l = oracle.pairs(pos, 8.1, cap=8, method="brute")
    assert list(c) == [1, 0, 1]


def test_lattice_and_grips(oracle):
    n = 6
    pos = oracle.fcc_lattice(n, 4.05)
    assert len(pos) == 4 * n ** 3
    assert np.array_equal(pos, PI.fcc_sites(n, 4.05))
    for axis in range(3):
        fl = oracle.grip_flags(pos, axis, 4.05)
        # three atomic layers of 2 n^2 atoms on each side
        assert (fl == 1).sum() == 3 * 2 * n * n
        assert (fl == 2).sum() == 3 * 2 * n * n
        assert pos[fl == 1, axis].max() == pytest.approx(4.05)
        assert pos[fl == 2, axis].min() == pytest.approx((n - 1.5) * 4.05)
