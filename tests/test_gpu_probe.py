"""The unit-rate probes behind the ALU rooflines (FP64 FMA, FP32 FMA, MUFU
ex2): each returns a rate in the range the unit counts and clocks allow."""

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ny():
    from paper_2110_02820_gb300 import build, nyspcg
    build.build()
    nyspcg.lib()
    return nyspcg


def test_unit_peaks_are_plausible(ny):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    clk = 2.1e9  # above the maximum SM clock of the part
    fp32 = ny.nys_unit_peak(ny.UNIT_FP32_FMA)
    fp64 = ny.nys_unit_peak(ny.UNIT_FP64_FMA)
    ex2 = ny.nys_unit_peak(ny.UNIT_MUFU_EX2)
    # FP32: at most 128 FMA lanes per SM per clock (2 FLOP each), at least a tenth
    assert 0.1 * sms * 128 * 2 * clk < fp32 <= sms * 128 * 2 * clk
    # FP64 and ex2 run far below the FP32 pipe on this part
    assert 0 < fp64 < fp32 / 4
    assert 0 < ex2 <= sms * 32 * clk
    assert ex2 > 0.01 * fp32 / 2
