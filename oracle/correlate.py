"""FT convolution producing the F-A power plane (oracle, FP64). Test infrastructure only.

Paper, Sec. 2.1. The FT convolution filters the N_chan-point input array with N_temp FIR filters
(Eq. 1: y[i] = sum_{j<N_tap} x[i-j] h[j]). With AOLS-2048-P it also takes the power |y|^2 of
the complex outputs. The result is the filter-output plane (FOP) of Sec. 2.2: one row per
template, one column per channel.

Correlation form used here. Template t has taps a_t[q] (q = -h..h, see ``templates``). Its
plane row is

    y_t[j] = sum_{q=-h}^{h} X[j+q] conj(a_t[q]),   X[m] = 0 outside [0, N),
    P[t][j] = |y_t[j]|^2,                            j = 0..N-1.

This is Eq. 1 with the causal filter g_t[m] = conj(a_t[h-m]), m = 0..N_tap-1, read h samples
later: y_t[j] = y_causal[j + h].

Two routes are given. ``plane_direct`` is the definition as written. ``plane_ols`` follows the
overlap-save FDFIR of Sec. 2.1 step by step, on the causal filter:
  1. Split the input into chunks of F points. Neighbouring chunks overlap by N_tap-1, and the
     first chunk has N_tap-1 zeros at its start.
  2. Transform each chunk and the zero-padded filter, multiply, and transform back (Eq. 2).
  3. Discard the first N_tap-1 outputs of each chunk. The remaining L = F - N_tap + 1 outputs
     are exact linear-convolution outputs.
The two routes must agree to rounding (tests). ``plane_ols`` uses the oracle's own FFT.
"""
from __future__ import annotations

import numpy as np

from .fft import fft


def correlate_direct(spectrum: np.ndarray, bank: np.ndarray) -> np.ndarray:
    """y[t][j] = sum_q X[j+q] conj(a_t[q]), complex128[n_temp][N], by the definition."""
    x = np.asarray(spectrum, dtype=np.complex128)
    n = x.shape[0]
    n_temp, n_tap = bank.shape
    h = (n_tap - 1) // 2
    padded = np.concatenate([np.zeros(h, np.complex128), x, np.zeros(h, np.complex128)])
    y = np.zeros((n_temp, n), dtype=np.complex128)
    cb = np.conj(bank)
    for qi in range(n_tap):  # q = qi - h; X[j+q] = padded[j + qi]
        y += cb[:, qi : qi + 1] * padded[None, qi : qi + n]
    return y


def plane_direct(spectrum: np.ndarray, bank: np.ndarray) -> np.ndarray:
    """P[t][j] = |y_t[j]|^2 from the direct correlation, float64[n_temp][N]."""
    y = correlate_direct(spectrum, bank)
    return y.real**2 + y.imag**2


def power_at(spectrum: np.ndarray, bank: np.ndarray, rows: np.ndarray, cols: np.ndarray) -> np.ndarray:
    """P[rows[k]][cols[k]] one point at a time from the definition (for sampled checks at scale)."""
    x = np.asarray(spectrum, dtype=np.complex128)
    n = x.shape[0]
    h = (bank.shape[1] - 1) // 2
    out = np.empty(len(rows), dtype=np.float64)
    q = np.arange(-h, h + 1)
    for k, (t, j) in enumerate(zip(np.asarray(rows), np.asarray(cols))):
        idx = j + q
        ok = (idx >= 0) & (idx < n)
        y = np.sum(x[idx[ok]] * np.conj(bank[t][ok]))
        out[k] = y.real**2 + y.imag**2
    return out


def _ols_rows(spectrum: np.ndarray, bank: np.ndarray, fft_len: int):
    """Yield (t, y_t) by overlap-save (Sec. 2.1) on the causal filter, with the oracle's own FFT."""
    x = np.asarray(spectrum, dtype=np.complex128)
    n = x.shape[0]
    n_temp, n_tap = bank.shape
    h = (n_tap - 1) // 2
    f = fft_len
    keep = f - (n_tap - 1)  # L valid outputs per chunk
    if keep <= 0:
        raise ValueError("fft_len must exceed n_tap - 1")
    # Causal outputs needed: i = j + h for j = 0..N-1, i.e. i in [h, N + h).
    n_causal = n + h
    n_chunk = -(-n_causal // keep)
    # Step 1: chunk c holds the inputs of causal outputs i in [c*L, c*L + L), starting N_tap-1 earlier.
    padded = np.concatenate(
        [np.zeros(n_tap - 1, np.complex128), x, np.zeros(n_chunk * keep + f, np.complex128)]
    )
    starts = np.arange(n_chunk) * keep
    chunks = padded[starts[:, None] + np.arange(f)[None, :]]  # [n_chunk][F]
    spec_chunks = fft(chunks)
    # Causal filter g_t[m] = conj(a_t[h - m]) zero padded to F.
    g = np.zeros((n_temp, f), dtype=np.complex128)
    g[:, :n_tap] = np.conj(bank[:, ::-1])
    spec_g = fft(g)
    for t in range(n_temp):
        # Step 2: multiply and transform back.
        out = fft(spec_chunks * spec_g[t][None, :], inverse=True)
        # Step 3: discard the first N_tap - 1 outputs of every chunk.
        causal = out[:, n_tap - 1 :].reshape(-1)[:n_causal]
        yield t, causal[h : h + n]


def correlate_ols(spectrum: np.ndarray, bank: np.ndarray, fft_len: int) -> np.ndarray:
    """y[t][j] by overlap-save (Sec. 2.1), complex128[n_temp][N]."""
    y = np.empty((bank.shape[0], len(spectrum)), dtype=np.complex128)
    for t, row in _ols_rows(spectrum, bank, fft_len):
        y[t] = row
    return y


def plane_ols(spectrum: np.ndarray, bank: np.ndarray, fft_len: int) -> np.ndarray:
    """P[t][j] = |y_t[j]|^2 from the overlap-save route, float64[n_temp][N]."""
    p = np.empty((bank.shape[0], len(spectrum)), dtype=np.float64)
    for t, row in _ols_rows(spectrum, bank, fft_len):
        p[t] = row.real**2 + row.imag**2
    return p
