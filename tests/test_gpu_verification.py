"""The fine-dynamics verification workload (Sec. Verification with fine
dynamics) on the GPU against the oracle's restatement of the same
procedure: same start, the same ramped fine trajectory windows (Eq.
(measure)), the same PTA coarse steps, the same relative errors."""
import numpy as np
import pytest

from gpu_util import gpu_package
from oracle import pta_logic as L

pytestmark = pytest.mark.gpu


def test_fine_vs_pta_matches_the_oracle(oracle):
    P = gpu_package()
    from paper_2603_07321_gb300.verify import fine_vs_pta
    shape, T0, seed = (4, 4, 5), 300.0, 3
    cfg = dict(h_steps=40, delta_steps=8, n_jumps=3, burst_steps=8, strain_per_jump=4e-4)
    prep = dict(strain0=0.01, prep_increments=2, prep_steps=20)
    out = fine_vs_pta(shape, T0=T0, seed=seed, precision=P.PREC_FP64, **prep, **cfg)

    # the oracle from the GPU context's own start (the same seed)
    c = P.Ctx(shape, T0=T0, seed=seed, precision=P.PREC_FP64)
    pos, vel = c.get_state()
    c.close()
    spec = oracle.Specimen(shape)
    spec.pos, spec.vel = pos.copy(), vel.copy()
    for _ in range(prep["prep_increments"]):
        spec.apply_strain(prep["strain0"] / prep["prep_increments"])
        spec.burst(prep["prep_steps"])
    import copy
    spec_pta = copy.deepcopy(spec)
    ramp = cfg["strain_per_jump"] / cfg["h_steps"]
    v_fine = L.fine_dynamics_measures(spec, cfg["h_steps"], cfg["delta_steps"], cfg["n_jumps"],
                                      ramp)
    params = L.verification_params(cfg["h_steps"], cfg["delta_steps"], ramp)
    res, _ = L.run(spec_pta, params, cfg["burst_steps"], cfg["n_jumps"])
    v_pta = np.array([r.v for _, r in res])
    err = L.verification_errors(v_pta, v_fine[1:])

    assert np.allclose(out["v_fine"], v_fine, rtol=1e-9, atol=1e-9)
    assert np.allclose(out["v_pta"], v_pta, rtol=1e-7, atol=1e-9)
    assert np.allclose(out["errors"], err, rtol=1e-4, atol=1e-8)
    assert out["sources"] == [[int(x) for x in r.source] for _, r in res]
    # both runs end at the same load
    assert out["strain_fine_end"] == pytest.approx(out["strain_pta_end"], rel=1e-9)
