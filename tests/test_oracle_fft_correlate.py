"""Pins for the oracle's FFT and FT convolution (CPU only).

The overlap-save route and the direct route are two computations of one definition. Each is
also pinned on its own: the FFT against numpy and the DFT sum, the direct correlation against
a pure-Python double loop, and the whole plane against the physics of an injected tone.
"""
import numpy as np
import pytest

import synth
from oracle import correlate, fft


@pytest.mark.parametrize("n", [2, 4, 8, 32, 256, 4096])
def test_own_fft_matches_numpy(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))
    assert np.max(np.abs(fft.fft(x) - np.fft.fft(x, axis=1))) < 1e-11 * n
    assert np.max(np.abs(fft.fft(x, inverse=True) - np.fft.ifft(x, axis=1))) < 1e-13 * n


def test_own_fft_matches_dft_sum():
    n = 16
    rng = np.random.default_rng(7)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    k = np.arange(n)
    want = np.array([np.sum(x * np.exp(-2j * np.pi * kk * k / n)) for kk in k])
    assert np.max(np.abs(fft.fft(x) - want)) < 1e-13


def _random_bank(rng, n_temp, n_tap):
    return rng.standard_normal((n_temp, n_tap)) + 1j * rng.standard_normal((n_temp, n_tap))


def test_direct_correlation_matches_brute_force_loop():
    rng = np.random.default_rng(1)
    n, n_tap = 37, 5
    h = (n_tap - 1) // 2
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    bank = _random_bank(rng, 3, n_tap)
    got = correlate.correlate_direct(x, bank)
    for t in range(3):
        for j in range(n):
            acc = 0j
            for q in range(-h, h + 1):
                if 0 <= j + q < n:
                    acc += x[j + q] * np.conj(bank[t][q + h])
            assert abs(got[t][j] - acc) < 1e-13
    # power_at evaluates single points by the same definition
    rows, cols = np.array([0, 1, 2, 2]), np.array([0, 5, 36, 18])
    p = correlate.power_at(x, bank, rows, cols)
    assert np.allclose(p, np.abs(got[rows, cols]) ** 2, rtol=1e-13, atol=0)


@pytest.mark.parametrize("n", [64, 1000])
@pytest.mark.parametrize("n_tap", [5, 21])
@pytest.mark.parametrize("f", [32, 64])
def test_overlap_save_equals_direct(n, n_tap, f):
    rng = np.random.default_rng(n + n_tap + f)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    bank = _random_bank(rng, 4, n_tap)
    d = correlate.correlate_direct(x, bank)
    o = correlate.correlate_ols(x, bank, f)
    assert np.max(np.abs(d - o)) <= 1e-12 * np.max(np.abs(d))


def test_overlap_save_real_templates_small_n(bank):
    # The real 421-tap templates at F = 2048 on a spectrum shorter than one chunk and on a ragged one.
    rng = np.random.default_rng(3)
    for n in (300, 5000):
        x = synth.complex_noise(rng, n)
        d = correlate.plane_direct(x, bank[::12])
        o = correlate.plane_ols(x, bank[::12], 2048)
        assert np.max(np.abs(d - o)) <= 1e-12 * np.max(d)


def test_zero_drift_row_reproduces_input_power(bank):
    rng = np.random.default_rng(4)
    x = synth.complex_noise(rng, 4096).astype(np.complex64)
    p = correlate.plane_direct(x, bank[40:45])
    xd = x.astype(np.complex128)
    assert np.array_equal(p[2], xd.real**2 + xd.imag**2)


def test_injected_tone_peaks_at_its_bin_and_drift(bank):
    wl = synth.small_workload()
    plane = correlate.plane_ols(wl.spectrum, bank, 2048)
    t, j = np.unravel_index(np.argmax(plane), plane.shape)
    assert (t, j) == (62, 12000)
    s = np.sum(np.abs(bank[62]) ** 2)
    # Noise-free the peak is amp^2 s^2 to O(1/N); unit noise moves |y| by less than 4 (|n| < 4 w.p. 1 - e^-16).
    assert abs(np.sqrt(plane[t, j]) - 20.0 * s) < 4.0
    clean = synth.tone_spectrum(wl.n, wl.tones)
    p = correlate.power_at(clean, bank, np.array([62]), np.array([12000]))[0]
    assert abs(p / (400.0 * s * s) - 1.0) < 1e-6


def test_noise_row_mean_is_template_energy(bank):
    # For unit-power white noise, E P[t][j] = sum_q |a_t[q]|^2 away from the edges.
    rng = np.random.default_rng(5)
    x = synth.complex_noise(rng, 1 << 15)
    rows = bank[[0, 42, 84]]
    p = correlate.plane_ols(x, rows, 2048)[:, 300:-300]
    want = np.sum(np.abs(rows) ** 2, axis=1)
    assert np.all(np.abs(p.mean(axis=1) / want - 1.0) < 0.03)
