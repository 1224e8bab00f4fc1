"""Every branch of the coarse-step update (Eqs. (dvdt_algo), (pta_pred),
(simp), (rel_err), (jump_err) and the readings where the paper is silent),
driven through the CUDA kernel by pta_coarse_update and compared element by
element with the oracle's pta_logic on the same burst means.

The scripted sequence mixes smooth continuations, steps, repeated values
(which make e2 exactly 0) and returns after a jump; a CPU test checks with the
oracle alone that it reaches all eight paths of the acceptance rule."""
import numpy as np
import pytest

from oracle import pta_logic as L

PATHS = ("predicted", "first_step", "flagged_jump", "flagged_no_jump", "ratio_jump",
         "ratio_no_jump", "e2_zero_jump", "e2_zero_no_jump")


def scripted_means(n_steps=60, seed=3):
    """(n_steps + 1) x 3 x 3 burst means: the initial triple, then one triple
    per coarse step, per variable one of: smooth drift, a step, a repeat of
    the previous burst values (e1 = 0 or e2 = 0) or noise."""
    rng = np.random.default_rng(seed)
    base = np.array([150.0, -3000.0, 1.5])
    slope = np.array([0.2, -0.5, 0.01])
    out = np.zeros((n_steps + 1, 3, 3))
    cur = base.copy()
    out[0] = [cur - 2 * slope * 0.1, cur - slope * 0.1, cur]
    prev_c = cur.copy()
    last_rate = np.zeros(3)
    for s in range(1, n_steps + 1):
        for m in range(3):
            kind = rng.choice(["smooth", "step", "repeat", "noise", "smooth", "same_rate"])
            if s <= 2:
                kind = ["noise", "smooth"][s - 1] if m != 1 else "smooth"
            if kind == "smooth":
                c = prev_c[m] + slope[m]
                tri = [c - 0.2 * slope[m], c - 0.1 * slope[m], c]
            elif kind == "step":
                c = prev_c[m] * (1.0 + rng.choice([-1, 1]) * rng.uniform(0.05, 0.3))
                tri = [c, c, c]
            elif kind == "repeat":
                c = prev_c[m]
                tri = [c * (1 + rng.uniform(-0.2, 0.2)), c * (1 + rng.uniform(-0.2, 0.2)), c]
            elif kind == "same_rate":
                # the same relative change as the step before (e1 close to
                # e2), with scattered earlier bursts (e_v large)
                c = prev_c[m] * (1.0 + last_rate[m])
                tri = [c * (1 + rng.uniform(-0.2, 0.2)), c * (1 + rng.uniform(-0.2, 0.2)), c]
            else:
                c = prev_c[m] * (1.0 + rng.uniform(-0.04, 0.04))
                tri = [c * (1 + rng.uniform(-0.03, 0.03)), c * (1 + rng.uniform(-0.03, 0.03)), c]
            out[s, :, m] = tri
            last_rate[m] = (c - prev_c[m]) / prev_c[m]
            prev_c[m] = c
    return out


def oracle_run(means, params):
    """Run the oracle's coarse logic; per step the result and, per variable,
    the path the acceptance rule took (classified from the state before the
    step)."""
    st = L.initial_state(params, *means[0])
    results, paths = [], []
    for s in range(1, len(means)):
        before = st
        st, r = L.coarse_update(params, st, *means[s])
        pth = []
        for m in range(3):
            if r.e_v[m] < params.tol_v[m]:
                pth.append("predicted")
            elif before.jump[m]:
                pth.append("flagged_jump" if r.jump[m] else "flagged_no_jump")
            elif before.R_tmh is None:
                pth.append("first_step")
            elif r.e2[m] > 0.0:
                pth.append("ratio_jump" if r.jump[m] else "ratio_no_jump")
            else:
                pth.append("e2_zero_jump" if r.jump[m] else "e2_zero_no_jump")
        results.append(r)
        paths.append(pth)
    return results, paths


def test_script_reaches_every_branch():
    params = L.PTAParams()
    _, paths = oracle_run(scripted_means(), params)
    seen = {p for row in paths for p in row}
    assert seen == set(PATHS), sorted(set(PATHS) - seen)


@pytest.mark.gpu
def test_coarse_update_kernel_matches_oracle_on_every_branch():
    from gpu_util import gpu_package
    P = gpu_package()
    params = L.PTAParams()
    means = scripted_means()
    ref, paths = oracle_run(means, params)
    ctx = P.Ctx((4, 4, 4), precision=P.PREC_FP64)
    r0 = ctx.coarse_update(means[0])
    assert list(r0.source) == [-1, -1, -1]
    assert np.array_equal(np.array(r0.v), L.simpson(*means[0]))
    t = 0.0
    for s, (r, pth) in enumerate(zip(ref, paths), start=1):
        g = ctx.coarse_update(means[s])
        t += params.h
        assert g.t == t
        for name in ("v", "v_pred", "v_d", "e_v", "e1", "e2"):
            a, b = np.array(getattr(g, name)), np.asarray(getattr(r, name), dtype=float)
            assert np.array_equal(np.isnan(a), np.isnan(b)), (s, name, a, b)
            assert np.array_equal(a[~np.isnan(a)], b[~np.isnan(b)]), (s, name, pth, a, b)
        assert list(g.jump) == [int(x) for x in r.jump], (s, pth)
        assert list(g.source) == [int(x) for x in r.source], (s, pth)
    ctx.close()
