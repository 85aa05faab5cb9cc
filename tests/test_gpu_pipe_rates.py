"""The measured pipe rates behind the per-pipe generation roofline
(mf_pipe_rates): every class reports a positive finite rate, the FP32 FMA
chain lands near the unit count (152 SMs x 128 lanes, one FMA per lane and
clock, at no more than the maximum clock), GB300's FP64 pipe is far
slower than its FP32 pipe, and the tensor-core MMA rates are plausible."""
import math

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_pipe_rates_are_plausible():
    import paper_2606_31598_gb300 as mf
    r = mf.mf_pipe_rates(0)
    assert set(r) == set(mf.PIPES)
    assert all(math.isfinite(v) and v > 0 for v in r.values()), r
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    unit = sms * 128 * 2.07e9
    assert 0.5 * unit < r["ffma"] < 1.05 * unit, r
    assert r["dfma"] < r["ffma"] / 16, r
    assert r["imad_hi"] <= 1.05 * r["ffma"] and r["mufu"] <= 1.05 * r["ffma"], r
    # tensor cores: N = 256 MMAs at no more than the nominal dense BF16 rate
    # (2.25 PFLOP/s), and an N = 128 instruction no faster than an N = 256 one
    flop256 = 2.0 * 128 * 256 * 16
    assert 0.3e15 < r["mma256"] * flop256 < 2.3e15, r
    assert r["mma128"] < 1.2 * r["mma256"], r
