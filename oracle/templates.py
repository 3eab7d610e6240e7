"""Acceleration templates (oracle, FP64). Test infrastructure only.

The paper says the FT convolution applies N_temp = 85 FIR filters with N_tap = 421 taps
(Sec. 2.1; Table "FDAS Module Parameters"). These filters remove the smearing of an
accelerated pulsar by correlation (Sec. 1). The coefficients themselves are not printed.

Reading used here. This is the standard Fourier-domain response of a linearly drifting tone
(the correlation technique the paper cites in Sec. 1). Take a tone whose phase, in cycles, is
r0*tau + z*tau^2/2 over normalised time tau in [0, 1). It drifts by z bins and has mean
frequency r_bar = r0 + z/2. Its normalised DFT at bin r_bar + q is

    A_z(q) = integral_0^1 exp(2 pi i (-(q + z/2) tau + z tau^2 / 2)) d tau.

Template t has drift z_t = z_min + t*z_step. Its coefficients are a_t[q] = A_{z_t}(q) for the
integer offsets q = -h..h, with h = (N_tap - 1)/2. The F-A plane is then the correlation
y_t[j] = sum_q X[j+q] conj(a_t[q]) (see ``correlate``).

The integral is evaluated by composite Gauss-Legendre quadrature, 16 nodes per panel. The
panel count keeps every panel under one cycle of the integrand. The 16-point rule's error on
one cycle is below 1e-28, so the result is exact to FP64 rounding.
"""
from __future__ import annotations

import functools
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class TemplateGrid:
    """The template parameters: z_t = z_min + t*z_step for t = 0..n_temp-1, and n_tap taps."""

    n_temp: int = 85
    z_min: float = -42.0
    z_step: float = 1.0
    n_tap: int = 421

    @property
    def half_width(self) -> int:
        return (self.n_tap - 1) // 2

    def z(self) -> np.ndarray:
        return self.z_min + self.z_step * np.arange(self.n_temp, dtype=np.float64)


def _panel_count(max_cycles: float) -> int:
    return 16 + int(np.ceil(max_cycles))


def response(z: float, q: np.ndarray) -> np.ndarray:
    """A_z(q) for integer offsets q (complex128), by composite 16-point Gauss-Legendre quadrature.

    The phase in cycles is c(tau) = -(q + z/2) tau + z tau^2 / 2. Its rate |dc/dtau| is at most
    |q| + |z|/2. With at least that many panels, each panel holds under one cycle.
    """
    q = np.atleast_1d(np.asarray(q, dtype=np.float64))
    if z == 0.0:
        return np.where(q == 0.0, 1.0 + 0.0j, 0.0 + 0.0j)
    n_panel = _panel_count(np.max(np.abs(q)) + abs(z) / 2.0)
    x, w = np.polynomial.legendre.leggauss(16)
    left = np.arange(n_panel, dtype=np.float64) / n_panel
    tau = (left[:, None] + (x[None, :] + 1.0) / (2.0 * n_panel)).ravel()
    wt = np.tile(w / (2.0 * n_panel), n_panel)
    out = np.empty(q.shape, dtype=np.complex128)
    for start in range(0, q.size, 64):
        qq = q[start : start + 64]
        cycles = -(qq[:, None] + z / 2.0) * tau[None, :] + 0.5 * z * tau[None, :] ** 2
        cycles -= np.floor(cycles)
        out[start : start + 64] = np.exp(2j * np.pi * cycles) @ wt
    return out


@functools.lru_cache(maxsize=8)
def _bank_cached(grid: TemplateGrid) -> np.ndarray:
    h = grid.half_width
    q = np.arange(-h, h + 1, dtype=np.float64)
    bank = np.empty((grid.n_temp, grid.n_tap), dtype=np.complex128)
    for t, z in enumerate(grid.z()):
        bank[t] = response(float(z), q)
    bank.setflags(write=False)
    return bank


def template_bank(grid: TemplateGrid = TemplateGrid()) -> np.ndarray:
    """a[t][q + h] = A_{z_t}(q) for q = -h..h: complex128[n_temp][n_tap], time-domain taps."""
    return _bank_cached(grid)


def frequency_templates(bank: np.ndarray, fft_len: int) -> np.ndarray:
    """The templates as the overlap-save kernel consumes them: complex128[n_temp][fft_len].

    This follows the convolution theorem, Eq. 2 (x * h = F^-1{F{x} . F{h}}). It is written for
    the centred correlation that is used here. Each template is placed wrapped in a length-F
    array: offset q >= 0 goes to index q and q < 0 goes to F + q. Then

        T_t[m] = conj( sum_q a_t[q] exp(-2 pi i m q / F) ),

    so that IDFT(DFT(w) * T_t)[p] = sum_q w[(p + q) mod F] conj(a_t[q]), the circular
    correlation. The sum is the plain DFT definition, with the exponent reduced exactly in
    integers as (m*q) mod F.
    """
    n_temp, n_tap = bank.shape
    h = (n_tap - 1) // 2
    if n_tap >= fft_len:
        raise ValueError("n_tap must be below fft_len")
    m = np.arange(fft_len, dtype=np.int64)
    q = np.arange(-h, h + 1, dtype=np.int64)
    k = np.mod(m[:, None] * q[None, :], fft_len).astype(np.float64)
    dft = np.exp(-2j * np.pi * k / fft_len)  # [F][n_tap]
    return np.conj(bank @ dft.T)
