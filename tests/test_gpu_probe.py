"""The pipe probe behind the ALU roofline peaks reports plausible rates."""
import pytest

pytestmark = pytest.mark.gpu

ok = pytest.importorskip("paper_2604_15765_gb300.orkan")
torch = pytest.importorskip("torch")


def test_probe_pipes_rates_are_plausible():
    scratch = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    r = ok.orkan_probe_pipes(scratch.data_ptr(), scratch.numel())
    assert all(v > 0 for v in r.values())
    assert r["fp32_fma_per_s"] > 8 * r["fp64_fma_per_s"]     # FP64 is a small fraction of FP32 on this part
    assert 100.0 < r["copy_GBps"] < 20000.0
    # paired FMA does the same lane work per instruction pair; on GB300 its lane rate equals the scalar one
    assert 0.5 * r["fp32_fma_per_s"] < r["fp32x2_fma_lanes_per_s"] < 2.5 * r["fp32_fma_per_s"]
    with pytest.raises(ok.OrkanError):
        ok.orkan_probe_pipes(scratch.data_ptr(), 1 << 20)      # below the 32 MiB minimum
