"""Threshold array TA(k, i) for Algorithm 1 (oracle, FP64). Test infrastructure only.

Algorithm 1 compares every harmonic-plane value HP_k(i, j) with TA(k, i). The paper gives no
values for TA. Reading used here: a fixed false-alarm probability per plane value. For
unit-power Gaussian input, each plane point |y|^2 is close to a unit-mean exponential. So HP_k,
a sum of k such points, follows Gamma(k, 1), whose survival function for integer k is the
Poisson sum

    S_k(x) = P(Gamma(k,1) > x) = exp(-x) * sum_{m=0}^{k-1} x^m / m!.

A "sigma" threshold matches the one-sided Gaussian tail p = Q(sigma) = erfc(sigma/sqrt 2)/2, so
TA(k, i) solves S_k(x) = p. It is the same for every row i, and is computed in FP64 then
rounded to float32. The literal alternative, mean + sigma*sd = k + sigma*sqrt(k), is given too.
"""
from __future__ import annotations

import math

import numpy as np


def gaussian_tail(sigma: float) -> float:
    """Q(sigma) = P(N(0,1) > sigma)."""
    return 0.5 * math.erfc(sigma / math.sqrt(2.0))


def gamma_survival(k: int, x: float) -> float:
    """S_k(x) = exp(-x) * sum_{m<k} x^m / m! for integer k >= 1."""
    term, total = 1.0, 1.0
    for m in range(1, k):
        term *= x / m
        total += term
    return math.exp(-x) * total


def gamma_threshold(k: int, p: float) -> float:
    """The x with S_k(x) = p, by bisection in FP64 (S_k is strictly decreasing on x > 0)."""
    lo, hi = 0.0, 1.0
    while gamma_survival(k, hi) > p:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if gamma_survival(k, mid) > p:
            lo = mid
        else:
            hi = mid
        if hi - lo <= 1e-15 * hi:
            break
    return 0.5 * (lo + hi)


def threshold_array(n_harm: int, n_temp: int, sigma: float = 6.0, kind: str = "gamma") -> np.ndarray:
    """TA as float32[n_harm][n_temp]; row k-1 holds the threshold for HP_k."""
    out = np.empty((n_harm, n_temp), dtype=np.float32)
    for k in range(1, n_harm + 1):
        if kind == "gamma":
            v = gamma_threshold(k, gaussian_tail(sigma))
        elif kind == "meansd":
            v = k + sigma * math.sqrt(k)
        else:
            raise ValueError(kind)
        out[k - 1, :] = np.float32(v)
    return out
