"""The oracle's own FFT (FP64). Test infrastructure only.

This is a textbook iterative radix-2 Cooley-Tukey transform: bit-reversal permutation, then
log2(n) stages of butterflies. Each stage merges pairs of length-s/2 DFTs into length-s DFTs
with twiddles exp(-+2 pi i k / s). It works along the last axis of a batch.

The overlap-save check in ``correlate`` uses it, so that it does not rest on numpy's FFT.
Tests pin it against numpy.fft and the DFT definition.
"""
from __future__ import annotations

import numpy as np


def _bit_reverse(n: int) -> np.ndarray:
    bits = n.bit_length() - 1
    idx = np.arange(n)
    rev = np.zeros(n, dtype=np.int64)
    for b in range(bits):
        rev |= ((idx >> b) & 1) << (bits - 1 - b)
    return rev


def fft(x: np.ndarray, inverse: bool = False) -> np.ndarray:
    """DFT along the last axis: X[k] = sum_n x[n] exp(-2 pi i k n / n_len).

    With inverse=True the exponent sign is + and the result is divided by n_len.
    n_len must be a power of two.
    """
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[-1]
    if n & (n - 1):
        raise ValueError("length must be a power of two")
    sign = 1.0 if inverse else -1.0
    lead = x.shape[:-1]
    a = x[..., _bit_reverse(n)].reshape(-1, n)
    size = 2
    while size <= n:
        half = size // 2
        w = np.exp(sign * 2j * np.pi * np.arange(half) / size)
        blocks = a.reshape(a.shape[0], n // size, size)
        even = blocks[:, :, :half]
        odd = blocks[:, :, half:] * w
        a = np.concatenate([even + odd, even - odd], axis=2).reshape(a.shape[0], n)
        size *= 2
    if inverse:
        a = a / n
    return a.reshape(*lead, n)
