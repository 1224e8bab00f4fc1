"""The lattice-stencil pair scheme of the mixed-precision form, against the
FP64 oracle and against the Verlet-list scheme.

The stencil visits, for every atom, the atoms at a fixed set of lattice
offsets; it must reach exactly the physics of Eqs. (pe) and (f_int): forces
on identical positions to the mixed-precision tolerance, 200-step
trajectories within 1e-4 L_s, and the same neighbour sets as the brute-force
search (tests/test_gpu_parity.py).  When the atoms no longer sit on their
lattice (swapped atoms), the specimen must move to lists and still be right.
"""
import numpy as np
import pytest

import pta_inputs as PI
from gpu_util import force_error, force_error_atom, gpu_package, on_grid

pytestmark = pytest.mark.gpu

LISTS, STENCIL = 2, 1


@pytest.fixture(scope="module")
def P():
    return gpu_package()


def _pot(oracle, ctx):
    p = ctx.potential
    return oracle.Potential(eps=p.eps, c=p.c, a=p.a, rc=p.rc, n=p.n, m=p.m)


def test_stencil_reports_its_keys(P):
    ctx = P.Ctx((8, 8, 8), T0=300.0, seed=3, precision=P.PREC_MIXED)
    ctx.apply_strain(1e-3)
    ctx.fine_burst(50)
    sc = ctx.scheme()
    # FCC offsets within rc + 1 A: shells 1-10 (200 offsets), a few more from
    # thermal motion, padded to a multiple of 4
    assert sc["scheme"] == "stencil"
    assert 176 <= sc["keys"] <= 320, sc
    assert sc["checks"] >= 2
    ctx.close()


@pytest.mark.parametrize("scheme", [STENCIL, LISTS])
def test_trajectory_matches_oracle_in_either_scheme(P, oracle, scheme):
    shape = (6, 5, 7)
    ctx = P.Ctx(shape, T0=300.0, seed=14, precision=P.PREC_MIXED, pair_scheme=scheme)
    spec = oracle.Specimen(shape)
    spec.thermalise(300.0, 14)
    pos = on_grid(spec.pos)
    vel = np.asarray(spec.vel, dtype=np.float32).astype(np.float64)
    spec.pos, spec.vel = pos.copy(), vel.copy()
    ctx.set_state(pos, vel)
    ctx.apply_strain(2e-3)
    spec.apply_strain(2e-3)
    ctx.fine_burst(200)
    s_gpu = ctx.series()
    s_ref = spec.burst(200)
    p_gpu, _ = ctx.get_state()
    assert np.max(np.abs(p_gpu - spec.pos)) < 1e-4 * 7 * 4.05
    assert np.allclose(s_gpu[:, :2], s_ref[:, :2], rtol=1e-5)
    assert np.max(np.abs(s_gpu[:, 2] - s_ref[:, 2])) < 1e-3
    assert ctx.scheme()["scheme"] == ("stencil" if scheme == STENCIL else "lists")
    ctx.close()


@pytest.mark.parametrize("strain", [(0.05, 0.0), (-0.08, 0.02)])
def test_forces_on_a_strained_lattice(P, oracle, strain):
    # an affinely strained, jittered crystal: the check refits the reference
    # lattice (its records stay small) and the stencil covers the new offsets
    shape = (7, 6, 8)
    ez, ex = strain
    pos = PI.gaussian_jitter_fcc(shape, 0.1, seed=77)
    pos[:, 2] *= 1.0 + ez
    pos[:, 0] *= 1.0 + ex
    pos[:, 1] *= 1.0 - 0.3 * ez
    pos = on_grid(pos)
    ctx = P.Ctx(shape, precision=P.PREC_MIXED)
    ctx.set_state(pos, np.zeros_like(pos))
    f, pe, _ = ctx.forces()
    f_ref, pe_ref, _ = oracle.eam(pos, _pot(oracle, ctx))
    assert force_error(f, f_ref) < 1e-5
    assert force_error_atom(f, f_ref) < 1e-5
    assert np.max(np.abs(pe - pe_ref) / np.abs(pe_ref)) < 1e-5
    assert ctx.scheme()["scheme"] == "stencil"
    ctx.close()


def _swapped(shape, seed):
    """A jittered lattice in which three mobile atoms of cell layer 2 along z
    have exchanged places with the atoms of the same sites in layer nz - 3:
    their lattice offsets to their new neighbours span nz - 5 cells (> 5
    cells, the stencil's reach, for nz >= 11)."""
    assert shape[2] >= 11
    pos = PI.gaussian_jitter_fcc(shape, 0.05, seed=seed)
    layer = 4 * shape[0] * shape[1]
    rng = np.random.default_rng(seed)
    a = 2 * layer + rng.choice(layer, 3, replace=False)
    b = a + (shape[2] - 5) * layer
    pos[a], pos[b] = pos[b].copy(), pos[a].copy()
    return on_grid(pos)


def test_lost_lattice_moves_the_specimen_to_lists(P, oracle):
    shape = (4, 5, 12)
    pos = _swapped(shape, 5)
    ctx = P.Ctx(shape, precision=P.PREC_MIXED)
    assert ctx.scheme()["scheme"] == "stencil"
    ctx.set_state(pos, np.zeros_like(pos))
    f, pe, _ = ctx.forces()
    f_ref, pe_ref, _ = oracle.eam(pos, _pot(oracle, ctx))
    assert ctx.scheme()["scheme"] == "lists"
    assert force_error(f, f_ref) < 1e-5
    assert np.max(np.abs(pe - pe_ref) / np.abs(pe_ref)) < 1e-5
    ctx.close()


def test_fallback_inside_a_burst_matches_oracle(P, oracle):
    # the check at the burst's first step finds the lost lattice; the list
    # build runs in the same step (inside the replayed graph) and the burst
    # goes on with lists
    shape = (4, 4, 11)
    pos = _swapped(shape, 9)
    vel = PI.random_velocities(len(pos), 3e-3, seed=4)
    ctx = P.Ctx(shape, precision=P.PREC_MIXED)
    spec = oracle.Specimen(shape)
    vel[spec.flags != 0] = 0.0
    vel = vel.astype(np.float32).astype(np.float64)
    ctx.set_state(pos, vel)
    spec.pos, spec.vel = pos.copy(), vel.copy()
    a = ctx.fine_burst(60)
    s_ref = spec.burst(60)
    assert a.status == 0 and a.nsteps == 60
    assert np.allclose(ctx.series()[:, :2], s_ref[:, :2], rtol=1e-5)
    assert ctx.scheme()["scheme"] == "lists"
    ctx.close()


def test_batch_with_a_fallen_back_member_equals_solo(P):
    shape = (4, 4, 11)
    pos = _swapped(shape, 21)
    runs = []
    for batched in (False, True):
        cs = [P.Ctx(shape, T0=300.0, seed=s, precision=P.PREC_MIXED) for s in (1, 2)]
        cs[1].set_state(pos, np.zeros_like(pos))
        if batched:
            b = P.Batch(cs)
            b.fine_burst([80, 80])
            b.close()
        else:
            for c in cs:
                c.fine_burst(80)
        runs.append([c.series().copy() for c in cs] + [cs[1].scheme()["scheme"]])
        for c in cs:
            c.close()
    assert runs[0][2] == runs[1][2] == "lists"
    assert np.array_equal(runs[0][0], runs[1][0])
    assert np.array_equal(runs[0][1], runs[1][1])


def test_checkpoint_moves_between_schemes(P):
    # checkpoints hold the state in creation order: a stencil context's state
    # loads into a list context and continues the same trajectory (to the
    # mixed-precision tolerance: the two schemes sum pairs in other orders)
    shape = (6, 6, 6)
    src = P.Ctx(shape, T0=300.0, seed=8, precision=P.PREC_MIXED)
    src.apply_strain(1e-3)
    src.fine_burst(40)
    blob = src.save()
    src.fine_burst(100)
    s_src = src.series().copy()
    dst = P.Ctx(shape, T0=10.0, seed=99, precision=P.PREC_MIXED, pair_scheme=LISTS)
    dst.restore(blob)
    dst.fine_burst(100)
    assert np.allclose(dst.series()[:, :2], s_src[:, :2], rtol=1e-5)
    assert np.array_equal(dst.flags(), src.flags())
    src.close()
    dst.close()
