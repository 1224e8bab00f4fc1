"""Cell tiles of the mixed-precision pair passes (one thread per atom).

A tile's atoms sum their neighbour lists in the same order and with the same
arithmetic whether the neighbour records come from the tile's shared-memory
copy, from global memory (a halo too dense for the copy), or from the
untiled kernels: forces, energies and trajectories are identical bit for
bit, and the neighbour sets equal the oracle's brute-force pairs.  The tiles'
shared-memory copy is sized for a 1 A Verlet skin, which these tests use.
"""
import numpy as np
import pytest

import pta_inputs as PI
from gpu_util import force_error_atom, gpu_package, on_grid, sorted_rows

pytestmark = pytest.mark.gpu
SKIN = 1.0


@pytest.fixture(scope="module")
def P():
    return gpu_package()


def _pot(oracle, ctx):
    p = ctx.potential
    return oracle.Potential(eps=p.eps, c=p.c, a=p.a, rc=p.rc, n=p.n, m=p.m)


def _forces(P, shape, pos, tiles, a0=4.05):
    ctx = P.Ctx(shape, precision=P.PREC_MIXED, lanes=1, cell_tiles=tiles, a0=a0, skin=SKIN)
    ctx.set_state(pos, np.zeros_like(pos))
    f, pe, obs = ctx.forces()
    info = ctx.tiling()
    ctx.close()
    return f, pe, obs, info


def test_tiled_forces_identical_to_untiled_and_match_oracle(P, oracle):
    shape = (8, 7, 9)
    pos = on_grid(PI.gaussian_jitter_fcc(shape, 0.1, seed=31))
    f1, pe1, obs1, info = _forces(P, shape, pos, 1)
    f0, pe0, obs0, info0 = _forces(P, shape, pos, -1)
    assert info["tiled"] and not info0["tiled"]
    assert info["tiles"] > 1 and info["staged_tiles"] == info["tiles"]
    assert np.array_equal(f1, f0) and np.array_equal(pe1, pe0)
    # U sums the same per-atom energies in other FP32 warp groups
    assert np.allclose(obs1, obs0, rtol=1e-6, atol=1e-9)
    f_ref, pe_ref, _ = oracle.eam(pos, oracle.Potential())
    assert force_error_atom(f1, f_ref) < 1e-5
    assert np.max(np.abs(pe1 - pe_ref) / np.abs(pe_ref)) < 1e-5


def test_dense_halo_reads_global_memory_with_identical_results(P, oracle):
    # at a0 = 3.6 A an interior tile's 4x4x4 cells hold ~4100 atoms, more
    # than the shared-memory copy takes; surface tiles still fit it
    shape = (12, 12, 12)
    a0 = 3.6
    pos = on_grid(PI.gaussian_jitter_fcc(shape, 0.05, seed=32, a0=a0))
    f1, pe1, _, info = _forces(P, shape, pos, 1, a0=a0)
    f0, pe0, _, _ = _forces(P, shape, pos, -1, a0=a0)
    assert 0 < info["staged_tiles"] < info["tiles"]
    assert np.array_equal(f1, f0) and np.array_equal(pe1, pe0)
    f_ref, _, _ = oracle.eam(pos, oracle.Potential())
    assert force_error_atom(f1, f_ref) < 1e-5


def test_tiled_trajectory_identical_to_untiled(P, oracle):
    out = []
    for tiles in (1, -1):
        ctx = P.Ctx((9, 8, 10), T0=300.0, seed=21, precision=P.PREC_MIXED, lanes=1,
                    cell_tiles=tiles, skin=SKIN)
        ctx.apply_strain(2e-3)
        a = ctx.fine_burst(300)
        out.append((ctx.series().copy(), ctx.get_state(), a.prunes, a.rebuilds))
        ctx.close()
    (s1, (p1, v1), pr1, rb1), (s0, (p0, v0), pr0, rb0) = out
    assert pr1 == pr0 and pr1 > 1 and rb1 == rb0
    assert np.array_equal(p1, p0) and np.array_equal(v1, v0)
    # K, U, T: the same per-atom terms summed in other FP32 warp groups
    assert np.allclose(s1, s0, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("shape", [(5, 4, 6), (7, 7, 7)])
def test_tiled_neighbour_sets_bit_exact(P, oracle, shape):
    ctx = P.Ctx(shape, T0=0.0, seed=1, precision=P.PREC_MIXED, cell_tiles=1, skin=SKIN)
    assert ctx.layout()["lanes"] == 1 and ctx.tiling()["tiled"]
    pos = on_grid(PI.jittered_fcc(shape, 0.35, seed=sum(shape) + 40))
    ctx.set_state(pos, np.zeros_like(pos))
    c_gpu, l_gpu = ctx.neighbours(cap=512)
    rl = ctx.potential.rc + ctx.params.skin
    c_ref, l_ref = oracle.pairs(pos, rl, cap=512, method="brute")
    assert np.array_equal(c_gpu, c_ref)
    assert sorted_rows(c_gpu, l_gpu) == sorted_rows(c_ref, l_ref)
    ctx.close()


def test_more_occupied_tiles_than_blocks(P, oracle):
    # a state spread to twice the specimen's size covers more tiles than the
    # pair passes have blocks: blocks then take several tiles each
    shape = (8, 8, 8)
    pos = on_grid(2.0 * PI.gaussian_jitter_fcc(shape, 0.05, seed=33))
    res = []
    for tiles in (1, -1):
        ctx = P.Ctx(shape, precision=P.PREC_MIXED, lanes=1, cell_tiles=tiles, skin=SKIN)
        ctx.set_state(pos, np.zeros_like(pos))
        f, pe, _ = ctx.forces()
        res.append((f, pe, ctx.tiling()))
        ctx.close()
    info = res[0][2]
    assert info["tiles"] > info["blocks"]
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])


def test_batch_of_tiled_and_untiled_specimens_equals_solo(P, oracle):
    kw = [dict(cell_tiles=1, lanes=1, skin=SKIN), dict(cell_tiles=-1, lanes=2, skin=SKIN),
          dict(cell_tiles=1, lanes=1, skin=SKIN)]
    shapes = [(7, 7, 8), (6, 6, 7), (8, 6, 7)]
    solo = []
    for sh, k in zip(shapes, kw):
        ctx = P.Ctx(sh, T0=300.0, seed=5, precision=P.PREC_MIXED, **k)
        ctx.apply_strain(1e-3)
        ctx.fine_burst(120)
        solo.append(ctx.get_state()[0])
        ctx.close()
    ctxs = [P.Ctx(sh, T0=300.0, seed=5, precision=P.PREC_MIXED, **k)
            for sh, k in zip(shapes, kw)]
    b = P.Batch(ctxs)
    b.apply_strain([1e-3] * 3)
    b.fine_burst([120] * 3)
    for c, ref in zip(ctxs, solo):
        assert np.array_equal(c.get_state()[0], ref)
    b.close()
    for c in ctxs:
        c.close()


def test_tile_parameter_validation(P):
    with pytest.raises(P.PTAError):
        P.Ctx((4, 4, 4), precision=P.PREC_FP64, cell_tiles=1)
    with pytest.raises(P.PTAError):
        P.Ctx((4, 4, 4), precision=P.PREC_MIXED, lanes=2, cell_tiles=1)
    with pytest.raises(P.PTAError):
        P.Ctx((4, 4, 4), precision=P.PREC_MIXED, cell_tiles=2)
    ctx = P.Ctx((4, 4, 4), precision=P.PREC_FP64)
    assert not ctx.tiling()["tiled"]
    ctx.close()
