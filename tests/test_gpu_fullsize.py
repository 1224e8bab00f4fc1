"""Parity at the full benchmark size, in the launch configuration bench.py
times: the 49^3-cell cube (470,596 atoms), mixed precision, automatic lanes.
The oracle evaluates the forces of sampled atoms one by one."""
import numpy as np
import pytest

import pta_inputs as PI
from gpu_util import gpu_package, on_grid

pytestmark = pytest.mark.gpu


def test_sampled_forces_on_the_470596_atom_cube(oracle):
    P = gpu_package()
    n = 49
    pos = on_grid(PI.gaussian_jitter_fcc(n, 0.1, seed=49))
    ctx = P.Ctx(n, T0=0.0, seed=1, precision=P.PREC_MIXED)
    assert ctx.n == 470596
    ctx.set_state(pos, np.zeros_like(pos))
    f, pe, _ = ctx.forces()
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(ctx.n, 256, replace=False))
    # include grip atoms and surface atoms explicitly
    fl = ctx.flags()
    idx = np.unique(np.concatenate([idx, np.flatnonzero(fl == 2)[:16], np.flatnonzero(fl == 1)[:16],
                                    [0, ctx.n - 1]]))
    p = ctx.potential
    pot = oracle.Potential(eps=p.eps, c=p.c, a=p.a, rc=p.rc, n=p.n, m=p.m)
    f_ref, pe_ref = oracle.eam_sampled(pos, pot, idx)
    scale = np.sqrt(np.mean(np.sum(f_ref ** 2, axis=1)))
    err = np.max(np.linalg.norm(f[idx] - f_ref, axis=1)) / scale
    assert err < 1e-5, err
    assert np.max(np.abs(pe[idx] - pe_ref) / np.abs(pe_ref)) < 1e-5
    ctx.close()


def test_full_size_burst_is_stable_and_conserves_grips():
    P = gpu_package()
    ctx = P.Ctx(49, T0=300.0, seed=3, precision=P.PREC_MIXED, burst_steps=200)
    fl = ctx.flags()
    p0, _ = ctx.get_state()
    ctx.apply_strain(1e-3)
    a = ctx.fine_burst(200)
    p1, v1 = ctx.get_state()
    assert a.status == 0 and a.nsteps == 200 and a.rebuilds >= 1
    right = fl == 2
    assert np.allclose(p1[right, 2] - p0[right, 2], 1e-3 * 49 * 4.05, atol=1e-9)
    assert np.array_equal(p1[fl == 1], p0[fl == 1])
    assert np.all(v1[fl != 0] == 0)
    # the kinetic energy stays near its 300 K value (energy drains into potential)
    K = a.mean[0]
    mob = int((fl == 0).sum())
    assert 0.3 < K / (1.5 * mob * 8.617333262e-5 * 300.0) < 0.8
    ctx.close()
