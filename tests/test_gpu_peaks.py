"""The ALU issue-rate probes (the FP32 FMA, MUFU ex2 and FP64 FMA roofs the
cell kernels are placed against) give plausible, correctly ordered rates."""
import pytest

pytestmark = pytest.mark.gpu


def test_alu_peaks_plausible():
    import torch
    assert torch.cuda.is_available()
    from paper_2112_12854_b300 import ep
    ctx = ep.Context()
    p = ep.alu_peaks(ctx)
    ctx.close()
    print(p)
    assert 10e12 < p["fp32_fma_flops"] < 400e12
    assert 0.3e12 < p["mufu_ex2_ops"] < 100e12
    assert 0.0 < p["fp64_fma_flops"] < p["fp32_fma_flops"]
    assert p["mufu_ex2_ops"] < p["fp32_fma_flops"]
