"""The FP64 rate self-test (dqmc_selftest_fp64_rate): the roofline denominator.

GB300 issues one FP64 warp instruction per 64 cycles on each SM sub-partition,
i.e. 2 DFMA lanes (4 flop) per clock per SM: at most 152 x 4 x 2.07 GHz =
1.259 TFLOP/s.  The loop kernels must land below that bound (they do the work
they count) and well above a tenth of it (they are not latency bound)."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2003_05286_gb300 as m
    m.lib()
    return m


@pytest.mark.parametrize("kind", ["dfma", "dmma_m8n8k4", "dmma_m16n8k8"])
def test_fp64_rate_in_range(dq, kind):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    clk_ghz = 2.07
    bound = sms * 4 * clk_ghz * 1e9 / 1e12
    tf, ms = dq.selftest_fp64_rate(kind, 2000 if kind != "dmma_m16n8k8" else 500)
    assert ms > 0
    assert 0.1 * bound < tf <= 1.05 * bound, (kind, tf, bound)
