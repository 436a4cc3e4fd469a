"""klr_probe_peaks on the device: every measured rate positive and inside
what the GB300's unit counts and clocks allow (152 SMs at up to 2.07 GHz: 128
FP32 lanes, 16 reciprocal units per SM; FP64 far below FP32)."""
import pytest

pytestmark = pytest.mark.gpu


def test_probe_peaks_are_plausible():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1911_02373_gb300 as klr
    ctx = klr.Context(0)
    pk = ctx.probe_peaks()
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    ghz = 2.2   # above any clock of the part
    fp32_bound = n_sm * 128 * 2 * ghz * 1e-3          # TFLOP/s, scalar FFMA
    assert 0.3 * fp32_bound < pk["fp32_fma_tflops"] <= fp32_bound
    assert 0.3 * fp32_bound < pk["fp32x2_fma_tflops"] <= 2.0 * fp32_bound
    assert 0.0 < pk["fp64_fma_tflops"] < 0.5 * pk["fp32_fma_tflops"]
    assert 0.0 < pk["mufu_rcp_tops"] <= n_sm * 32 * ghz * 1e-3
    assert pk["tf32_mma_sync_tflops"] > pk["fp32_fma_tflops"] / 4
    ctx.close()
