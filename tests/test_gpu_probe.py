"""The rate probe behind the roofline's peak: every kind returns the count
its launch performed and a positive time, and the FP32 rate is in the range
the GPU's FMA units allow (SM count x 128 lanes x 2 flop x clock)."""
import pytest

from gpu_util import gpu_package

pytestmark = pytest.mark.gpu


def test_probe_kinds_report_their_counts():
    P = gpu_package()
    import torch
    props = torch.cuda.get_device_properties(0)
    for kind in range(6):
        a, ms_a = P.pta_measure_fma_rate(kind, 8)
        b, ms_b = P.pta_measure_fma_rate(kind, 16)
        assert a > 0 and ms_a > 0 and ms_b > 0
        assert b == 2 * a                      # counts scale with the iterations
    fl, ms = P.pta_measure_fma_rate(0, 2000)
    tflops = fl / (ms * 1e-3) / 1e12
    # at most the units' rate at 2.2 GHz, at least a tenth of it at 1 GHz
    upper = props.multi_processor_count * 128 * 2 * 2.2e9 / 1e12
    lower = props.multi_processor_count * 128 * 2 * 1.0e9 / 1e12 / 10
    assert lower < tflops < upper


def test_probe_rejects_an_unknown_kind():
    P = gpu_package()
    for kind, iters in ((6, 8), (-1, 8), (0, 0)):
        with pytest.raises(P.PTAError):
            P.pta_measure_fma_rate(kind, iters)
