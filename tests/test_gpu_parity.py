"""Parity of the CUDA path (through the C ABI) with the FP64 oracle."""
import numpy as np
import pytest

import pta_inputs as PI
from gpu_util import force_error, gpu_package, on_grid, sorted_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    return gpu_package()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape,axis", [((5, 5, 5), 2), ((4, 3, 6), 0), ((3, 4, 5), 1)])
def test_create_matches_oracle(P, oracle, prec, shape, axis):
    ctx = P.Ctx(shape, T0=300.0, seed=7, precision=prec, load_axis=axis)
    spec = oracle.Specimen(shape, axis=axis)
    spec.thermalise(300.0, 7)
    pos, vel = ctx.get_state()
    assert np.array_equal(ctx.flags(), spec.flags)
    if prec == P.PREC_FP64:
        assert np.array_equal(pos, spec.pos)
        assert np.allclose(vel, spec.vel, rtol=1e-12, atol=1e-16)
    else:
        assert np.max(np.abs(pos - spec.pos)) < 1e-10
        assert np.allclose(vel, spec.vel, rtol=2e-7, atol=1e-12)
    ctx.close()


@pytest.mark.parametrize("prec,lanes", [(0, 1), (0, 4), (0, 16), (1, 1), (1, 4), (1, 16)])
@pytest.mark.parametrize("shape", [(5, 4, 6), (7, 7, 7)])
def test_neighbour_sets_bit_exact(P, oracle, prec, lanes, shape):
    ctx = P.Ctx(shape, T0=0.0, seed=1, precision=prec, lanes=lanes)
    pos = on_grid(PI.jittered_fcc(shape, 0.35, seed=sum(shape) + lanes))
    ctx.set_state(pos, np.zeros_like(pos))
    c_gpu, l_gpu = ctx.neighbours(cap=512)
    rl = ctx.potential.rc + ctx.params.skin
    c_ref, l_ref = oracle.pairs(pos, rl, cap=512, method="brute")
    assert np.array_equal(c_gpu, c_ref)
    assert sorted_rows(c_gpu, l_gpu) == sorted_rows(c_ref, l_ref)
    ctx.close()


@pytest.mark.parametrize("lanes", [1, 2, 8, 16])
def test_forces_fp64(P, oracle, lanes):
    shape = (6, 5, 7)
    ctx = P.Ctx(shape, precision=P.PREC_FP64, lanes=lanes)
    pos = PI.gaussian_jitter_fcc(shape, 0.1, seed=lanes)
    vel = PI.random_velocities(len(pos), 3e-3, seed=2)
    ctx.set_state(pos, vel)
    f, pe, obs = ctx.forces()
    f_ref, pe_ref, _ = oracle.eam(pos, ctx_pot(oracle, ctx))
    assert force_error(f, f_ref) < 1e-10
    assert np.max(np.abs(pe - pe_ref)) < 1e-11
    ctx.close()


def ctx_pot(oracle, ctx):
    p = ctx.potential
    return oracle.Potential(eps=p.eps, c=p.c, a=p.a, rc=p.rc, n=p.n, m=p.m)


@pytest.mark.parametrize("margin", [0.0, -1.0])       # inner list (default margin) / none
@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16])
def test_forces_mixed(P, oracle, lanes, margin):
    # every lane's list (inner or Verlet) ends with sentinel entries up to a
    # multiple of four, whatever the lanes per atom
    shape = (6, 5, 7)
    ctx = P.Ctx(shape, precision=P.PREC_MIXED, lanes=lanes, prune_margin=margin)
    assert ctx.layout()["pruned_list"] == (margin == 0.0)
    pos = on_grid(PI.gaussian_jitter_fcc(shape, 0.1, seed=10 + lanes))
    ctx.set_state(pos, np.zeros_like(pos))
    f, pe, _ = ctx.forces()
    f_ref, pe_ref, _ = oracle.eam(pos, ctx_pot(oracle, ctx))
    err = force_error(f, f_ref)
    assert err < 1e-5, err
    assert np.max(np.abs(pe - pe_ref) / np.abs(pe_ref)) < 1e-5
    ctx.close()


def test_observables_of_a_state(P, oracle):
    shape = (5, 5, 5)
    ctx = P.Ctx(shape, precision=P.PREC_FP64)
    spec = oracle.Specimen(shape)
    pos = PI.gaussian_jitter_fcc(shape, 0.08, seed=4)
    vel = PI.random_velocities(len(pos), 3e-3, seed=5)
    vel[spec.flags != 0] = 0
    ctx.set_state(pos, vel)
    spec.pos, spec.vel = pos.copy(), vel.copy()
    _, _, obs = ctx.forces()
    assert np.allclose(obs, spec.observables(), rtol=1e-11, atol=1e-11)
    ctx.close()


def _pair(P, oracle, shape, prec, seed, T0=300.0, **kw):
    ctx = P.Ctx(shape, T0=T0, seed=seed, precision=prec, **kw)
    spec = oracle.Specimen(shape)
    spec.thermalise(T0, seed)
    if prec == P.PREC_MIXED:
        # start both from the same (exactly representable) state
        pos = on_grid(spec.pos)
        vel = np.asarray(spec.vel, dtype=np.float32).astype(np.float64)
        spec.pos, spec.vel = pos.copy(), vel.copy()
        ctx.set_state(pos, vel)
    return ctx, spec


def test_trajectory_fp64_200_steps(P, oracle):
    ctx, spec = _pair(P, oracle, (6, 6, 6), P.PREC_FP64, seed=11, block_steps=40)
    ctx.apply_strain(2e-3)
    spec.apply_strain(2e-3)
    a = ctx.fine_burst(200)
    s_gpu = ctx.series()
    s_ref = spec.burst(200)
    pos, vel = ctx.get_state()
    assert a.nsteps == 200 and a.status == 0
    assert np.max(np.abs(pos - spec.pos)) < 1e-8
    assert np.allclose(s_gpu, s_ref, rtol=1e-9, atol=1e-9)
    assert np.allclose(a.mean, s_ref.mean(axis=0), rtol=1e-12)
    # block standard errors (5 blocks of 40 steps), element by element: against
    # the oracle's estimator on the device's own samples (same numbers, so to
    # rounding) and on the oracle's trajectory (which agrees to ~1e-9)
    _, se_own = oracle.burst_averages(s_gpu, 40)
    _, se_ref = oracle.burst_averages(s_ref, 40)
    assert np.allclose(a.se, se_own, rtol=1e-10, atol=0)
    # |SE(x) - SE(y)| <= max |x - y| over the samples (the sample standard
    # deviation of block means is 1-Lipschitz in the largest sample difference)
    dmax = np.max(np.abs(s_gpu - s_ref), axis=0)
    assert np.all(np.abs(np.array(a.se) - se_ref) <= 1.01 * dmax + 1e-12)
    ctx.close()


def test_trajectory_mixed_200_steps(P, oracle):
    ctx, spec = _pair(P, oracle, (6, 6, 6), P.PREC_MIXED, seed=12)
    ctx.apply_strain(2e-3)
    spec.apply_strain(2e-3)
    ctx.fine_burst(200)
    s_gpu = ctx.series()
    s_ref = spec.burst(200)
    pos, _ = ctx.get_state()
    L_s = 6 * 4.05
    assert np.max(np.abs(pos - spec.pos)) < 1e-4 * L_s
    # per-step state functions: K and U to 1e-5 relative, T to 1e-3 GPa
    assert np.allclose(s_gpu[:, :2], s_ref[:, :2], rtol=1e-5)
    assert np.max(np.abs(s_gpu[:, 2] - s_ref[:, 2])) < 1e-3
    ctx.close()


def test_grips_fixed_and_strain_moves_right_grip(P, oracle):
    ctx = P.Ctx((5, 5, 5), T0=300.0, seed=2, precision=P.PREC_FP64)
    fl = ctx.flags()
    p0, _ = ctx.get_state()
    ctx.fine_burst(30)
    p1, v1 = ctx.get_state()
    assert np.array_equal(p1[fl != 0], p0[fl != 0])
    assert np.all(v1[fl != 0] == 0)
    ctx.apply_strain(1e-2)
    p2, _ = ctx.get_state()
    du = 1e-2 * 5 * 4.05
    assert np.allclose(p2[fl == 2, 2] - p1[fl == 2, 2], du, atol=1e-12)
    assert np.array_equal(p2[fl != 2], p1[fl != 2])
    assert ctx.strain == pytest.approx(1e-2)
    ctx.close()


def test_burst_means_within_two_se(P, oracle):
    """Plain FP64 workload: 10^3 cells, 300 K, seed 1, tension step 1e-3, 2,000 steps."""
    cfg = PI.config_plain()
    ctx, spec = _pair(P, oracle, cfg["n_cells"], P.PREC_FP64, seed=cfg["seed"], T0=cfg["T0"])
    ctx.apply_strain(cfg["d_eps"])
    spec.apply_strain(cfg["d_eps"])
    a = ctx.fine_burst(cfg["burst_steps"])
    m_ref, se_ref = oracle.burst_averages(spec.burst(cfg["burst_steps"]), 100)
    for q in range(3):
        bound = 2.0 * np.hypot(a.se[q], se_ref[q])
        assert abs(a.mean[q] - m_ref[q]) <= bound, (q, a.mean[q], m_ref[q], bound)
    ctx.close()


def test_checkpoint_round_trip_is_bit_exact(P, oracle):
    for prec in (P.PREC_FP64, P.PREC_MIXED):
        ctx = P.Ctx((5, 5, 5), T0=300.0, seed=3, precision=prec)
        ctx.fine_burst(20)
        blob = ctx.save()
        ctx.fine_burst(40)
        s1 = ctx.series().copy()
        p1, v1 = ctx.get_state()
        ctx.restore(blob)
        ctx.fine_burst(40)
        s2 = ctx.series()
        p2, v2 = ctx.get_state()
        assert np.array_equal(s1, s2)
        assert np.array_equal(p1, p2) and np.array_equal(v1, v2)
        ctx.close()


def test_runs_are_deterministic(P, oracle):
    out = []
    for _ in range(2):
        ctx = P.Ctx((6, 6, 6), T0=300.0, seed=9, precision=P.PREC_MIXED)
        ctx.apply_strain(1e-3)
        ctx.fine_burst(100)
        out.append(ctx.series().copy())
        ctx.close()
    assert np.array_equal(out[0], out[1])


def test_batch_equals_solo_bitwise(P, oracle):
    shapes = [(5, 5, 5), (6, 4, 7), (4, 4, 4)]
    precs = [P.PREC_MIXED, P.PREC_MIXED, P.PREC_FP64]
    solo = []
    for sh, pr in zip(shapes, precs):
        c = P.Ctx(sh, T0=300.0, seed=5, precision=pr, lanes=4)
        c.apply_strain(1e-3)
        c.fine_burst(120)
        solo.append(c.series().copy())
        c.close()
    members = [P.Ctx(sh, T0=300.0, seed=5, precision=pr, lanes=4) for sh, pr in zip(shapes, precs)]
    b = P.Batch(members)
    b.apply_strain([1e-3] * 3)
    res = b.fine_burst([120, 120, 120])
    for m, s, r in zip(members, solo, res):
        assert r.nsteps == 120
        assert np.array_equal(m.series(), s)
    # ragged burst lengths: a member with 0 steps stays idle
    p_before, _ = members[2].get_state()
    b.fine_burst([10, 30, 0])
    p_after, _ = members[2].get_state()
    assert np.array_equal(p_before, p_after)
    assert len(members[0].series()) == 10 and len(members[1].series()) == 30
    b.close()
    for m in members:
        m.close()


def test_coarse_steps_match_oracle_protocol(P, oracle):
    from oracle import pta_logic as L
    shape = (4, 4, 5)
    nb = 40
    ctx, spec = _pair(P, oracle, shape, P.PREC_FP64, seed=21)
    ctx.close()
    ctx = P.Ctx(shape, T0=300.0, seed=21, precision=P.PREC_FP64, burst_steps=nb,
                strain_rate=2e-2)
    params = L.PTAParams(h=1.0, strain_rate=2e-2)
    res_ref, _ = L.run(spec, params, nb, 3)
    res_gpu = [ctx.coarse_step() for _ in range(3)]
    for (strain, r), g in zip(res_ref, res_gpu):
        assert g.strain == pytest.approx(strain, rel=1e-12)
        assert np.allclose(g.v_d, r.v_d, rtol=1e-7)
        assert np.allclose(g.v_pred, r.v_pred, rtol=1e-7)
        assert np.allclose(g.v, r.v, rtol=1e-7)
        assert list(g.source) == list(r.source)
    ctx.close()


def test_neighbour_overflow_is_reported(P, oracle):
    ctx = P.Ctx((5, 5, 5), precision=P.PREC_FP64, neigh_cap=32)
    with pytest.raises(P.PTAError) as e:
        ctx.fine_burst(5)
    assert e.value.status == -4
    ctx.close()


def test_invalid_arguments(P):
    with pytest.raises(P.PTAError):
        P.Ctx((2, 2, 2))  # fewer than 3 cells along the load axis
    with pytest.raises(P.PTAError):
        P.Ctx((4, 4, 4), lanes=3)
    with pytest.raises(P.PTAError):
        P.Ctx((4, 4, 4), precision=P.PREC_FP64, atoms_per_thread=2)
    ctx = P.Ctx((4, 4, 4))
    with pytest.raises(P.PTAError):
        ctx.fine_burst(0)
    with pytest.raises(P.PTAError):
        ctx.set_state(np.full((ctx.n, 3), np.nan), np.zeros((ctx.n, 3)))
    ctx.close()


def test_kernel_timing_records_every_iteration(P, oracle):
    ctx = P.Ctx((6, 6, 6), T0=300.0, seed=4, precision=P.PREC_MIXED)
    ctx.fine_burst(10)
    s_ref = ctx.series().copy()
    ctx.set_timing(True)
    ctx.fine_burst(100)
    t = ctx.timing()
    assert t.iterations == 101  # one force refresh + 100 steps
    assert t.force_ms > 0 and t.density_ms > 0 and t.rebuild_ms > 0
    ctx.set_timing(False)
    # timing changes nothing in the results
    ctx2 = P.Ctx((6, 6, 6), T0=300.0, seed=4, precision=P.PREC_MIXED)
    ctx2.fine_burst(10)
    ctx2.fine_burst(100)
    assert np.array_equal(ctx.series(), ctx2.series())
    ctx.close()
    ctx2.close()


def test_pruned_inner_list_changes_no_result(P, oracle):
    # the inner list holds every pair within rc in the same per-lane order:
    # trajectories with and without it are bit-identical
    out = []
    for margin in (0.3, -1.0):
        ctx = P.Ctx((8, 7, 9), T0=300.0, seed=12, precision=P.PREC_MIXED, lanes=2,
                    prune_margin=margin)
        ctx.apply_strain(2e-3)
        a = ctx.fine_burst(300)
        out.append((ctx.series().copy(), ctx.get_state(), a.prunes))
        ctx.close()
    assert out[0][2] > 1 and out[1][2] == 0
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1][0], out[1][1][0])


def test_batch_members_match_the_oracle(P, oracle):
    # uneven sizes and both precisions in one batch; each member against its
    # own oracle trajectory of 200 steps (not only against a solo GPU run)
    cases = [((5, 5, 5), P.PREC_MIXED, 31), ((6, 4, 7), P.PREC_FP64, 32),
             ((4, 6, 5), P.PREC_MIXED, 33), ((3, 3, 4), P.PREC_FP64, 34)]
    pairs = [_pair(P, oracle, sh, pr, seed) for sh, pr, seed in cases]
    members = [c for c, _ in pairs]
    b = P.Batch(members)
    d_eps = [1e-3, 2e-3, -1e-3, 3e-3]
    b.apply_strain(d_eps)
    res = b.fine_burst([200, 200, 200, 200])
    for (ctx, spec), (sh, pr, _), de, r in zip(pairs, cases, d_eps, res):
        spec.apply_strain(de)
        s_ref = spec.burst(200)
        s_gpu = ctx.series()
        pos, _ = ctx.get_state()
        assert r.nsteps == 200 and r.status == 0
        if pr == P.PREC_FP64:
            assert np.max(np.abs(pos - spec.pos)) < 1e-8
            assert np.allclose(s_gpu, s_ref, rtol=1e-9, atol=1e-9)
        else:
            assert np.max(np.abs(pos - spec.pos)) < 1e-4 * 4.05 * sh[2]
            assert np.allclose(s_gpu[:, :2], s_ref[:, :2], rtol=1e-5)
            assert np.max(np.abs(s_gpu[:, 2] - s_ref[:, 2])) < 1e-3
    b.close()
    for m in members:
        m.close()


def test_atom_beyond_the_cell_grid_is_reported(P, oracle):
    # the cell grid extends a quarter of the specimen's span beyond the
    # lattice; an atom placed far outside it (still inside the coordinate
    # range of the mixed form) makes the burst report PTA_ERANGE
    for prec in (P.PREC_FP64, P.PREC_MIXED):
        shape = (5, 5, 5)
        pos = PI.jittered_fcc(shape, 0.05, seed=3)
        ctx = P.Ctx(shape, T0=0.0, precision=prec)
        flags = ctx.flags()
        i = int(np.flatnonzero(flags == 0)[0])
        pos[i] = [-150.0, 5.0, 5.0]
        ctx.set_state(pos, np.zeros_like(pos))
        with pytest.raises(P.PTAError) as e:
            ctx.fine_burst(5)
        assert e.value.status == -7
        ctx.close()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape", [(1, 1, 3), (1, 2, 5), (2, 1, 9), (8, 8, 4)])
def test_thinnest_specimens_match_the_oracle(P, oracle, prec, shape):
    # the smallest specimens the boundary accepts (one or two cells across,
    # three or more along the load axis, a plate): fewer atoms than a warp or
    # a block, cell grids of one or two cells, lists shorter than the loops'
    # four-entry groups; in the 1 x 1 x 3 cube every atom is a grip atom, so
    # no velocity is drawn and nothing moves
    ctx = P.Ctx(shape, T0=0.0, seed=1, precision=prec)
    pos = on_grid(PI.jittered_fcc(shape, 0.2, seed=sum(shape)))
    ctx.set_state(pos, np.zeros_like(pos))
    c_gpu, l_gpu = ctx.neighbours(cap=512)
    rl = ctx.potential.rc + ctx.params.skin
    c_ref, l_ref = oracle.pairs(pos, rl, cap=512, method="brute")
    assert np.array_equal(c_gpu, c_ref)
    assert sorted_rows(c_gpu, l_gpu) == sorted_rows(c_ref, l_ref)
    f, pe, _ = ctx.forces()
    f_ref, pe_ref, _ = oracle.eam(pos, ctx_pot(oracle, ctx))
    assert force_error(f, f_ref) < (1e-10 if prec == 0 else 1e-5)
    assert np.max(np.abs(pe - pe_ref) / np.abs(pe_ref)) < (1e-11 if prec == 0 else 1e-5)
    ctx.close()
    # 100 steps at 300 K after a tension step, against the oracle's burst
    ctx, spec = _pair(P, oracle, shape, prec, seed=5)
    ctx.apply_strain(2e-3)
    spec.apply_strain(2e-3)
    a = ctx.fine_burst(100)
    s_gpu = ctx.series()
    s_ref = spec.burst(100)
    p_gpu, _ = ctx.get_state()
    assert a.status == 0 and a.nsteps == 100
    if prec == 0:
        assert np.max(np.abs(p_gpu - spec.pos)) < 1e-8
        assert np.allclose(s_gpu, s_ref, rtol=1e-9, atol=1e-9)
    else:
        assert np.max(np.abs(p_gpu - spec.pos)) < 1e-4 * 4.05 * max(shape)
        assert np.all(np.abs(s_gpu[:, :2] - s_ref[:, :2]) <= 1e-5 * np.abs(s_ref[:, :2]) + 1e-9)
        assert np.max(np.abs(s_gpu[:, 2] - s_ref[:, 2])) < 1e-3
    ctx.close()
