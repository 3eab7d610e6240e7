"""FP64 CPU oracle for the FDAS hot path.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product path (the CUDA library and its Python
binding) never imports, links or runs it, and it shares no code with that path. The only
common module is ``synth``, which makes seeded inputs and holds none of the method's arithmetic.

The oracle is plain and slow on purpose. Each function states the passage of the paper
(Wang, Thiagaraj and Sinnen, "Combining Multiple Optimized FPGA-based Pulsar Search Modules
Using OpenCL") that it follows:

* ``templates``  - the 85 acceleration templates (FIR coefficients, Sec. 2.1, Table "FDAS Module
  Parameters": N_temp = 85, N_tap = 421). The paper does not define the correlation kernel,
  so the module states the reading it uses.
* ``fft``        - the oracle's own radix-2 FFT, used by the overlap-save check.
* ``correlate``  - the FT convolution: direct correlation (Eq. 1 in correlation form) and the
  overlap-save FDFIR of Sec. 2.1 (chunks overlapping by N_tap-1, first chunk zero padded, first
  N_tap-1 outputs of each chunk discarded). Power |y|^2 as in AOLS-2048-P.
* ``harmonic``   - harmonic summing with threshold detection (Algorithm 1, Sec. 2.2), in float32
  with a fixed summation order so that candidates can be compared bit for bit.
* ``thresholds`` - the threshold array TA(k, i) of Algorithm 1. The paper gives no values; this
  module uses the false-alarm reading.

Every function here is pinned by tests in ``tests/test_oracle_*.py`` against closed forms,
an independent library routine, brute force on tiny inputs, or the physics of an injected
signal. None of them is "parity unpinned".
"""
from . import correlate, fft, harmonic, templates, thresholds  # noqa: F401

__all__ = ["correlate", "fft", "harmonic", "templates", "thresholds"]
