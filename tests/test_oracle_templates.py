"""Pins for the oracle's acceleration templates (CPU only).

The paper prints no template values. The templates are pinned by properties that follow from
the definition A_z(q) = int_0^1 exp(2 pi i (-(q + z/2) tau + z tau^2/2)) d tau, by a second
closed form (Fresnel integrals from scipy), and by the physics they model: the DFT of a sampled
drifting tone, computed by numpy's FFT.
"""
import numpy as np
import pytest
import scipy.special as sp

import synth
from oracle import templates

H = 210
Q = np.arange(-H, H + 1)


def fresnel_closed_form(z: float, q: np.ndarray) -> np.ndarray:
    """A_z(q) for z > 0 by completing the square (independent of the quadrature route).

    pi z tau^2 - 2 pi (q + z/2) tau = (pi/2) u^2 - pi (q + z/2)^2 / z with
    u = sqrt(2z) (tau - (q + z/2)/z). So A = exp(-i pi (q+z/2)^2/z) / sqrt(2z) *
    [C(u) + i S(u)] evaluated between u0 = -sqrt(2z)(q/z + 1/2) and u1 = sqrt(2z)(1/2 - q/z).
    scipy.special.fresnel returns (S, C) with the pi/2 convention used here.
    """
    s = np.sqrt(2.0 * z)
    u0 = -s * (q / z + 0.5)
    u1 = s * (0.5 - q / z)
    s1, c1 = sp.fresnel(u1)
    s0, c0 = sp.fresnel(u0)
    return np.exp(-1j * np.pi * (q + z / 2.0) ** 2 / z) / s * ((c1 - c0) + 1j * (s1 - s0))


def test_zero_drift_template_is_unit_impulse(bank):
    # A_0(q) = int_0^1 exp(-2 pi i q tau) d tau = delta_{q,0} for integer q.
    row = bank[42]
    assert row[H] == 1.0
    assert np.all(row[np.arange(len(row)) != H] == 0.0)


def test_time_reversal_and_conjugate_symmetry(bank):
    # tau -> 1 - tau maps A_z(q) to A_z(-q); z -> -z conjugates the integrand for integer q.
    assert np.max(np.abs(bank - bank[:, ::-1])) < 1e-13
    assert np.max(np.abs(bank - np.conj(bank[::-1]))) < 1e-13


def test_parseval_truncation(bank):
    # sum over all integer q of |A_z(q)|^2 = int_0^1 |.|^2 = 1. Truncation to |q| <= 210 must lose < 1e-2.
    energy = np.sum(np.abs(bank) ** 2, axis=1)
    shortfall = 1.0 - energy
    assert np.all(shortfall >= -1e-12)
    assert np.max(shortfall) < 1e-2
    # The shortfall grows with |z| and is about 3.2e-6 at |z| = 42 (stated in the design notes).
    assert 1e-6 < shortfall[0] < 1e-5
    assert shortfall[42] == 0.0


@pytest.mark.parametrize("z", [1, 2, 7, 20, 33, 42])
def test_quadrature_matches_fresnel_closed_form(z):
    got = templates.response(float(z), Q)
    want = fresnel_closed_form(float(z), Q.astype(np.float64))
    assert np.max(np.abs(got - want)) < 2e-13


def test_negative_drift_matches_conjugated_closed_form():
    got = templates.response(-13.0, Q)
    want = np.conj(fresnel_closed_form(13.0, Q.astype(np.float64)))
    assert np.max(np.abs(got - want)) < 2e-13


@pytest.mark.parametrize("z,mean", [(20, 12000), (-33, 5000), (7, 30001), (1, 777)])
def test_template_is_the_dft_of_a_sampled_drifting_tone(bank, z, mean):
    # A noise-free tone with drift z and mean bin r_bar has X[r_bar + q] = amp * A_z(q) + O(1/N).
    # numpy's FFT of the sampled chirp is independent of the quadrature. This pins sign, centring
    # and the mean-frequency convention of the templates, not just their magnitudes.
    n = 1 << 16
    x = synth.tone_spectrum(n, [synth.Tone(mean, z, 1.0, 1)])
    got = x[mean + Q]
    want = bank[42 + z]
    assert np.max(np.abs(got - want)) < 1e-6


def test_frequency_templates_against_numpy_fft(bank):
    # Wrapped placement (q >= 0 -> q, q < 0 -> F + q), then T = conj(DFT_F). numpy.fft is the check.
    f = 2048
    tf = templates.frequency_templates(bank[::21], f)
    wrapped = np.zeros((tf.shape[0], f), dtype=np.complex128)
    wrapped[:, : H + 1] = bank[::21, H:]
    wrapped[:, f - H :] = bank[::21, :H]
    want = np.conj(np.fft.fft(wrapped, axis=1))
    assert np.max(np.abs(tf - want)) < 1e-11


def test_frequency_templates_zero_drift_is_flat(bank):
    # The unit impulse at q = 0 has a flat spectrum of ones.
    tf = templates.frequency_templates(bank[42:43], 1024)
    assert np.max(np.abs(tf - 1.0)) < 1e-15
