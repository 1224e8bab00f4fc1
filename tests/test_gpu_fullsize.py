"""Parity at the full benchmark size, in the launch configuration bench.py
times: the 49^3-cell cube (470,596 atoms), mixed precision, automatic lanes.
The oracle evaluates the forces of every atom."""
import numpy as np
import pytest

import pta_inputs as PI
from gpu_util import force_error, force_error_atom, force_error_rms, gpu_package, on_grid

pytestmark = pytest.mark.gpu


def test_forces_of_every_atom_of_the_470596_atom_cube(oracle):
    P = gpu_package()
    n = 49
    pos = on_grid(PI.gaussian_jitter_fcc(n, 0.1, seed=49))
    ctx = P.Ctx(n, T0=0.0, seed=1, precision=P.PREC_MIXED)
    assert ctx.n == 470596
    ctx.set_state(pos, np.zeros_like(pos))
    f, pe, _ = ctx.forces()
    p = ctx.potential
    pot = oracle.Potential(eps=p.eps, c=p.c, a=p.a, rc=p.rc, n=p.n, m=p.m)
    f_ref, pe_ref, _ = oracle.eam(pos, pot)
    # every atom's force to 1e-5 of itself (floored at the rms force), the
    # rms error to 3e-6; atoms pushed into close pairs carry forces of ~5x
    # the rms, and their absolute errors reach ~1.5e-5 of the rms force
    e_pe = np.max(np.abs(pe - pe_ref) / np.abs(pe_ref))
    print("\n470,596-atom cube vs oracle: per-atom force error %.2e, rms %.2e, max/rms %.2e, "
          "per-atom energy %.2e" % (force_error_atom(f, f_ref), force_error_rms(f, f_ref),
                                    force_error(f, f_ref), e_pe))
    assert force_error_atom(f, f_ref) < 1e-5
    assert force_error_rms(f, f_ref) < 3e-6
    assert force_error(f, f_ref) < 3e-5
    assert np.max(np.abs(pe - pe_ref) / np.abs(pe_ref)) < 1e-5
    # the sampled one-by-one evaluation agrees with the full one
    idx = np.unique(np.concatenate([np.random.default_rng(5).choice(ctx.n, 64, replace=False),
                                    np.flatnonzero(ctx.flags() == 2)[:8], [0, ctx.n - 1]]))
    fs, pes = oracle.eam_sampled(pos, pot, idx)
    assert np.allclose(fs, f_ref[idx], rtol=1e-12, atol=1e-12)
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
