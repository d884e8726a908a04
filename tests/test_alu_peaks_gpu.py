"""The arithmetic throughput probes (srfmg_alu_peaks) that give the measured
denominators of the arithmetic rooflines: positive, repeatable within timing
noise, and ordered as the hardware is built (FP32 far above FP64 on this
part; a 64-bit add at least as fast as the add-add-shift step)."""
import pytest

from paper_1207_6720_gb300 import srfmg

pytestmark = pytest.mark.gpu


def test_alu_peaks_are_plausible_and_repeatable():
    pytest.importorskip("torch")
    p1 = srfmg.alu_peaks(0)
    p2 = srfmg.alu_peaks(0)
    for k in p1:
        assert p1[k] > 1e11, k
        assert 0.5 < p1[k] / p2[k] < 2.0, k
    assert p1["fp32_flops"] > 8 * p1["fp64_flops"]
    assert p1["i64_add_per_s"] > p1["fp64_flops"] / 2
