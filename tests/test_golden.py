"""The oracle still reproduces the stored values in tests/golden/ (CPU only)."""
import os

import numpy as np

from oracle import templates, thresholds

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_threshold_golden():
    ta = thresholds.threshold_array(16, 1, sigma=6.0)
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "thresholds_sigma6.txt")) if not ln.startswith("#")]
    assert len(rows) == 16
    for k, bits, _ in rows:
        assert ta[int(k) - 1, 0].view(np.uint32) == int(bits, 16)


def test_template_golden(bank):
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "template_taps.txt")) if not ln.startswith("#")]
    assert len(rows) == 85 * 4
    for z, q, re, im in rows:
        v = bank[int(z) + 42, 210 + int(q)]
        assert abs(v - complex(float(re), float(im))) < 1e-15
