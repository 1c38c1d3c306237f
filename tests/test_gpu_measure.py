"""The float64 rate probe behind the edge-cost roofline: the fused multiply-add
rate is near the GPU's float64 FMA units x clock, and a division or square
root costs several FMA slots (they are instruction sequences)."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


def test_fp64_rates_are_plausible():
    import paper_2509_05595_gb300 as pamo
    r = pamo.pamo_measure_fp64()
    props = torch.cuda.get_device_properties(0)
    assert r["fma_per_s"] > 1e10
    # no more than 64 float64 FMA lanes per SM at 3 GHz on any current part
    assert r["fma_per_s"] < props.multi_processor_count * 64 * 3.0e9
    for k in ("div_per_s", "sqrt_per_s"):
        assert 0 < r[k] < r["fma_per_s"]
