"""The throughput probes that give the evaluation kernels their roofline denominators."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_01844_gb300 import binding, build

    build.build()
    return binding


def test_probe_rates_are_plausible(B):
    import bench

    dev = torch.device("cuda")
    p = bench.alu_peaks(dev, blocks_per_sm=4, iters=512)
    sms = p["sms"]
    # per SM per clock at no more than 2.2 GHz and no less than 0.5 GHz: the SFU does a few to a
    # few tens of ex2, the FP32 pipes on the order of a hundred fma
    for key, lo, hi in (("ex2_per_s", 4, 64), ("fma_per_s", 32, 512)):
        per_clk_hi = p[key] / (sms * 0.5e9)
        per_clk_lo = p[key] / (sms * 2.2e9)
        assert per_clk_lo < hi and per_clk_hi > lo, (key, per_clk_lo, per_clk_hi)
    assert p["fma_per_s"] > 2 * p["ex2_per_s"]


def test_probe_rejects_bad_arguments(B):
    sink = torch.empty(256, device="cuda")
    L = B.lib()
    s = B.stream_handle()
    assert L.gs_probe_rate(2, 1, 1, B.ptr(sink), s) == B.GS_ERR_ARG
    assert L.gs_probe_rate(0, 0, 1, B.ptr(sink), s) == B.GS_ERR_ARG
    assert L.gs_probe_rate(0, 1, 1, None, s) == B.GS_ERR_ARG
