"""The arithmetic-throughput probe behind the sweep kernels' roofline."""
import pytest

torch = pytest.importorskip("torch")

import paper_2204_07921_gb300 as cm  # noqa: E402


@pytest.mark.gpu
def test_alu_probe_rates_are_plausible():
    """FP32 FMA and rsqrtf rates of the whole GPU.  Bounds from the unit
    counts: per SM 128 FP32 lanes and 16 MUFU lanes per clock, 152 SMs,
    clocks from ~1 to 2.07 GHz; the probe must land within a factor of two
    below those nominal rates and never above them by more than 5%."""
    r = cm.cm_probe_alu(0)
    torch.cuda.synchronize()
    props = torch.cuda.get_device_properties(0)
    nsm = props.multi_processor_count
    fma_nom = nsm * 128 * 2.07e9
    rsq_nom = nsm * 16 * 2.07e9
    assert 0.5 * fma_nom < r["fma_per_s"] < 1.05 * fma_nom, r
    assert 0.5 * rsq_nom < r["rsqrt_per_s"] < 1.05 * rsq_nom, r
