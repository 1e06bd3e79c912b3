"""The FP64 rate probe behind the tetrahedral roofline (fe_measure_fp64_rate).

GB300's FP64 units issue 2 instructions per SM per clock: 152 SMs at up to 2.07 GHz give about
6.3e11 FP64 instructions per second. The probe must land in a broad band around that figure (clocks
vary on a shared GPU, and the band only has to rule out a probe that measures nothing or double
counts), and repeated calls must agree.
"""
from __future__ import annotations

import pytest

from paper_1305_3122_gb300 import feasm

pytestmark = pytest.mark.gpu

NOMINAL = 2 * 152 * 2.07e9


def test_fp64_rate_probe():
    rates = [feasm.measure_fp64_rate() for _ in range(3)]
    for r in rates:
        assert 0.25 * NOMINAL <= r <= 1.3 * NOMINAL, rates
    assert max(rates) <= 1.5 * min(rates), rates
