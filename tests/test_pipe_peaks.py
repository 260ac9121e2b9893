"""Device throughput of the pipes that bound the operators (the roofline denominators that the
benchmark measures beside the ones derived from unit counts and the clock)."""
import pytest

from paper_2602_03893_gb300 import _lib

pytestmark = pytest.mark.gpu


def test_pipe_peaks_are_plausible():
    """FFMA and ex2 throughput microbenchmarks (the operators' roofline denominators) lie between
    half of and just above the unit counts: 152 SMs x 128 FP32 / 32 MUFU lanes x 2.07 GHz =
    40.3 / 10.1 T lane-ops/s."""
    fp32 = _lib.gpair_pipe_peak(_lib.PIPE_FP32) / 1e12
    mufu = _lib.gpair_pipe_peak(_lib.PIPE_MUFU) / 1e12
    print("measured T lane-ops/s: fp32", fp32, "mufu", mufu)
    assert 20.0 < fp32 < 45.0
    assert 5.0 < mufu < 11.5
