"""Writes the stored expected values under tests/golden/ from the oracle alone.

Run from the repository root:  python tests/golden/make_golden.py
The paper prints no worked numerical example, so every stored value here is an oracle value.
Each one is also pinned by a closed form or a library routine in tests/test_oracle_*.py.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import templates, thresholds  # noqa: E402


def main():
    ta = thresholds.threshold_array(16, 1, sigma=6.0)
    with open(os.path.join(HERE, "thresholds_sigma6.txt"), "w") as f:
        f.write("# TA(k) for Algorithm 1: S_k(x) = Q(6), Gamma(k,1) survival, float32 bits and value\n")
        for k in range(16):
            f.write(f"{k + 1} 0x{ta[k, 0].view(np.uint32):08x} {float(ta[k, 0]):.9g}\n")
    bank = templates.template_bank()
    with open(os.path.join(HERE, "template_taps.txt"), "w") as f:
        f.write("# A_z(q) of the 85 x 421 template bank at q in {0, 1, 7, 210}: z re im (FP64)\n")
        for t, z in enumerate(templates.TemplateGrid().z()):
            for q in (0, 1, 7, 210):
                v = bank[t, 210 + q]
                f.write(f"{int(z)} {q} {v.real:.17e} {v.imag:.17e}\n")


if __name__ == "__main__":
    main()
