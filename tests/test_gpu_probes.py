"""The FMA throughput probe reported beside the ALU rooflines
(claw_fma_peak): the clock it reports is a plausible SM clock, and its rate
per SM per clock lies between 75 % and 110 % of the unit count of the GB300
FMA pipes (FP64: 2 FMA lanes = 4 FLOP per SM per clock; FP32: 128 lanes =
256 FLOP).  Boxes differ: FP64 probes at the same clock have given 3.4 and
4.0 FLOP per SM per clock."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("prec,per_sm_clk", [("fp64", 4.0), ("fp32", 256.0)])
def test_fma_probe_rate_per_clock(prec, per_sm_clk):
    import torch
    from paper_1111_6583_gb300 import claw
    tf, mhz = claw.fma_peak(prec, with_clock=True)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert 300.0 < mhz < 2500.0, mhz
    per = tf * 1e12 / (mhz * 1e6) / sms
    assert 0.75 <= per / per_sm_clk <= 1.10, (tf, mhz, per)
