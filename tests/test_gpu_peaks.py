"""The roofline microbenchmarks (FP64 FMA, FP32 FMA and special-function throughput)
return plausible rates through the C ABI."""
import pytest

pytestmark = pytest.mark.gpu


def test_pipe_peaks_are_plausible():
    import torch
    from paper_1608_07058_gb300 import build, matleap as ml
    assert torch.cuda.is_available()
    build.build()
    pk = ml.ml_measure_pipe_peaks()
    assert pk["fp64_fma_flops"] > 1e11 and pk["fp32_fma_flops"] > 10 * pk["fp64_fma_flops"]
    assert pk["mufu_lg2_ops"] > 1e11
