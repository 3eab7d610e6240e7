"""Seeded synthetic inputs for the FDAS hot path.

This module is shared by the oracle-side tests, the CUDA-side tests and the benchmark. It holds
none of the method's arithmetic (no templates, no correlation, no harmonic summing, no thresholds).
It only makes the signals that stand in for one dedispersed, Fourier-transformed time series.
That is the "input array" of the FDAS module (Sec. 2, Table "FDAS Module Parameters": N_chan
complex single-precision points).

Signal model (the paper cites it but does not spell it out, Sec. 1): a pulsar in a binary orbit
gives a tone whose frequency drifts linearly during the observation. Over normalised time
tau = m / n in [0, 1) the phase, in cycles, is  r0*tau + z*tau**2/2. The frequency then runs from
r0 to r0 + z Fourier bins, and its mean is r0 + z/2. The spectrum handed to FDAS is
X = FFT(x) / n, so a steady tone of amplitude a gives |X| = a at its bin. Noise is complex
Gaussian with E|X|^2 = 1: real and imaginary parts are each N(0, 1/2).

numpy's FFT is used here only to synthesise data. All arrays returned are complex64, which is
the precision of the input array in the paper (Eq. 1: complex single-precision signals).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Tone",
    "Workload",
    "complex_noise",
    "chirp_time_series",
    "tone_spectrum",
    "pulse_train_spectrum",
    "exponential_plane",
    "small_workload",
    "ska_workload",
    "batch_lengths",
    "batch_workloads",
]


@dataclass(frozen=True)
class Tone:
    """One injected drifting tone.

    mean_bin: mean frequency r_bar in Fourier bins (the fundamental column j it should land on).
    z: total frequency drift in bins over the observation.
    amp: amplitude of the fundamental; |X| of a steady tone of this amplitude would be ``amp``.
    n_harm: number of harmonics. Harmonic l (1-based) has mean frequency l*mean_bin, drift l*z
        and amplitude amp/l.
    """

    mean_bin: float
    z: float
    amp: float
    n_harm: int = 1


@dataclass
class Workload:
    """A named synthetic spectrum with the tones that were injected into it."""

    name: str
    n: int
    seed: int
    spectrum: np.ndarray  # complex64[n]
    tones: list[Tone] = field(default_factory=list)


def complex_noise(rng: np.random.Generator, n: int) -> np.ndarray:
    """Unit-power circular complex Gaussian noise, complex128[n], E|X|^2 = 1."""
    re = rng.standard_normal(n)
    im = rng.standard_normal(n)
    return (re + 1j * im) * np.sqrt(0.5)


def chirp_time_series(n: int, r0: float, z: float, amp: float) -> np.ndarray:
    """amp * exp(2 pi i (r0 tau + z tau^2 / 2)), tau = m / n, m = 0..n-1, complex128[n].

    The phase is formed in cycles and reduced mod 1 before the exponential. That keeps FP64
    phase error near 1e-16 cycles even for bins near 2^22.
    """
    m = np.arange(n, dtype=np.float64)
    tau = m / n
    cycles = r0 * tau + 0.5 * z * tau * tau
    cycles -= np.floor(cycles)
    return amp * np.exp(2j * np.pi * cycles)


def tone_spectrum(n: int, tones: list[Tone]) -> np.ndarray:
    """Noise-free spectrum X = FFT(sum of chirps) / n of the given tones, complex128[n]."""
    x = np.zeros(n, dtype=np.complex128)
    for t in tones:
        for l in range(1, t.n_harm + 1):
            mean = l * t.mean_bin
            z = l * t.z
            x += chirp_time_series(n, mean - 0.5 * z, z, t.amp / l)
    return np.fft.fft(x) / n


def pulse_train_spectrum(n: int, f0: int) -> np.ndarray:
    """Noise-free spectrum of f0 unit pulses spaced n/f0 samples apart, complex64[n].

    x[m] = 1 for m = 0, n/f0, 2n/f0, ..., so X = FFT(x)/n is f0/n at every multiple of f0 and
    exactly 0 elsewhere (n must be a multiple of f0).
    """
    if n % f0:
        raise ValueError("n must be a multiple of f0")
    x = np.zeros(n, dtype=np.complex128)
    x[:: n // f0] = 1.0
    return (np.fft.fft(x) / n).astype(np.complex64)


def exponential_plane(rng: np.random.Generator, n_temp: int, n: int) -> np.ndarray:
    """A float32[n_temp][n] plane of unit-mean exponential values.

    This is the distribution of |y|^2 for unit-power Gaussian input. It is used to feed the
    harmonic-sum stage on its own.
    """
    return rng.exponential(1.0, size=(n_temp, n)).astype(np.float32)


def _finish(name: str, n: int, seed: int, noise: np.ndarray, tones: list[Tone]) -> Workload:
    spec = noise + tone_spectrum(n, tones) if tones else noise
    return Workload(name, n, seed, spec.astype(np.complex64), tones)


def small_workload(n: int = 1 << 16, seed: int = 0) -> Workload:
    """One spectrum of n bins: unit noise (seed) plus one tone, z=+20, mean bin 12000, amp 20.

    The tone's mean bin is 12000 for the default n and scales as n/2^16 * 12000 otherwise.
    """
    rng = np.random.default_rng(seed)
    noise = complex_noise(rng, n)
    mean = 12000 if n == 1 << 16 else max(64, int(12000 * n / (1 << 16)))
    return _finish("small", n, seed, noise, [Tone(mean, 20.0, 20.0, 1)])


def ska_workload(n: int = 1 << 21, seed: int = 1, n_tones: int = 4, amp: float = 20.0) -> Workload:
    """SKA-sized spectrum: unit noise plus n_tones tones with 8 harmonics each.

    Draw order from default_rng(seed): mean bins (integers, uniform in [2^10, n/8 - 2^10]), then
    drifts (integers, uniform in [-40, 40]), then the noise (real parts, then imaginary parts).
    The harmonic amplitudes are amp * (1, 1/2, ..., 1/8).
    """
    rng = np.random.default_rng(seed)
    lo, hi = 1 << 10, max((1 << 10) + 1, n // 8 - (1 << 10))
    means = rng.integers(lo, hi, size=n_tones, endpoint=True)
    zs = rng.integers(-40, 40, size=n_tones, endpoint=True)
    noise = complex_noise(rng, n)
    tones = [Tone(float(m), float(z), amp, 8) for m, z in zip(means, zs)]
    return _finish("ska", n, seed, noise, tones)


def batch_lengths(count: int = 64, seed: int = 3, lo_log2: float = 18.0, hi_log2: float = 22.0) -> list[int]:
    """Uneven spectrum lengths floor(2^U), U ~ Uniform(lo_log2, hi_log2), for batched runs."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(lo_log2, hi_log2, size=count)
    return [int(np.floor(2.0 ** v)) for v in u]


def batch_workloads(count: int = 64, seed: int = 3, amp: float = 20.0) -> list[Workload]:
    """Dedispersion-trial spectra of uneven length for batched runs.

    Lengths are ``batch_lengths(count, seed)``. Spectrum b then draws from default_rng([seed, b]):
    the number of tones (0..3), their mean bins (uniform in [2^10, n/8 - 2^10]) and drifts
    (uniform in [-40, 40]), then its noise. Each tone has 8 harmonics with amplitudes amp/l.
    """
    out = []
    for b, n in enumerate(batch_lengths(count, seed)):
        rng = np.random.default_rng([seed, b])
        k = int(rng.integers(0, 4))
        lo, hi = 1 << 10, max((1 << 10) + 1, n // 8 - (1 << 10))
        means = rng.integers(lo, hi, size=k, endpoint=True)
        zs = rng.integers(-40, 40, size=k, endpoint=True)
        noise = complex_noise(rng, n)
        tones = [Tone(float(m), float(z), amp, 8) for m, z in zip(means, zs)]
        out.append(_finish(f"trial{b}", n, seed, noise, tones))
    return out
