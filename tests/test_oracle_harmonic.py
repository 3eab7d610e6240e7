"""Pins for the oracle's harmonic sum, detection and thresholds (CPU only).

Algorithm 1 is checked against a pure-Python brute force on tiny planes and against the closed
form of a pulse train. The thresholds are checked against scipy's inverse incomplete gamma
function.
"""
import math

import numpy as np
import pytest
import scipy.special as sp

import synth
from oracle import correlate, harmonic, thresholds


def brute_force(plane, ta, n_harm, mask, cap):
    """Algorithm 1 with explicit loops and float32 running sums (fundamental-indexed stretch)."""
    n_temp, n = plane.shape
    c = (n_temp - 1) // 2
    hp_all, cands, counts, peaks = {}, [], [], []
    for k in range(1, n_harm + 1):
        found, best = [], None
        for i in range(-c, c + 1):
            if abs(k * i) > c:
                continue
            for j in range(0, n):
                if k * j > n - 1:
                    continue
                acc = np.float32(0.0)
                for l in range(1, k + 1):
                    acc = np.float32(acc + np.float32(plane[c + l * i, l * j]))
                hp_all[(k, i, j)] = acc
                if best is None or acc > best[0]:
                    best = (acc, i, j)
                if (mask >> (k - 1)) & 1 and acc > ta[k - 1, c + i]:
                    found.append((acc, i, j))
        found.sort(key=lambda r: (-float(r[0]), r[1], r[2]))
        counts.append(len(found))
        cands.append(found[:cap])
        peaks.append(best)
    return hp_all, cands, counts, peaks


def _compare(res, bf_cands, bf_counts, bf_peaks):
    assert list(res.counts) == bf_counts
    for k, (got, want) in enumerate(zip(res.cands, bf_cands), start=1):
        assert len(got) == len(want)
        for g, w in zip(got, want):
            assert (g["power"], int(g["i"]), int(g["j"]), int(g["k"])) == (w[0], w[1], w[2], k)
    for g, w in zip(res.peaks, bf_peaks):
        assert (np.float32(g[0]), g[1], g[2]) == w


@pytest.mark.parametrize("shape,n_harm,mask", [((5, 64), 3, 0b111), ((9, 50), 4, 0b1010), ((7, 33), 5, 0b11111)])
def test_harmonic_sum_matches_brute_force(shape, n_harm, mask):
    rng = np.random.default_rng(shape[1])
    plane = synth.exponential_plane(rng, *shape)
    ta = np.array([[k + 1.5 * math.sqrt(k)] * shape[0] for k in range(1, n_harm + 1)], dtype=np.float32)
    hp_all, bf_cands, bf_counts, bf_peaks = brute_force(plane, ta, n_harm, mask, cap=7)
    for k, i, hp in harmonic.harmonic_planes(plane, n_harm):
        for j, v in enumerate(hp):
            assert v == hp_all[(k, i, j)]
    assert sum(1 for key in hp_all if key[0] == 1) == shape[0] * shape[1]
    res = harmonic.detect(plane, ta, n_harm, mask, cand_cap=7)
    _compare(res, bf_cands, bf_counts, bf_peaks)


def test_candidate_order_breaks_ties_by_row_then_column():
    plane = np.ones((5, 16), dtype=np.float32)
    plane[2, 3] = plane[0, 9] = plane[4, 1] = plane[0, 2] = 4.0
    ta = np.full((1, 5), 2.0, dtype=np.float32)
    res = harmonic.detect(plane, ta, 1, 1, cand_cap=3)
    got = [(int(r["i"]), int(r["j"])) for r in res.cands[0]]
    assert got == [(-2, 2), (-2, 9), (0, 3)]
    assert res.counts[0] == 4
    assert res.peaks[0][1:] == (-2, 2)


def test_pulse_train_closed_form(bank):
    # f0 unit pulses over N samples: X = f0/N at multiples of f0, 0 elsewhere. With f0 > 2h no two
    # harmonics share a template window, so P[t][l f0] = (f0/N)^2 |A_{z_t}(0)|^2 and
    # HP_k(i, f0) = (f0/N)^2 sum_{l<=k} |A_{l i}(0)|^2; on the zero-drift row that is k (f0/N)^2.
    n, f0 = 1 << 14, 512
    x = synth.pulse_train_spectrum(n, f0)
    plane = correlate.plane_direct(x, bank).astype(np.float32)
    unit = (f0 / n) ** 2

    def a0_sq(z):  # |A_z(0)|^2 from the Fresnel closed form (scipy), independent of the quadrature
        if z == 0:
            return 1.0
        s = math.sqrt(2.0 * abs(z))
        sv, cv = sp.fresnel(s * 0.5)
        return (2.0 * cv) ** 2 / (2 * abs(z)) + (2.0 * sv) ** 2 / (2 * abs(z))

    for k, i, hp in harmonic.harmonic_planes(plane, 8):
        want = unit * sum(a0_sq(l * i) for l in range(1, k + 1))
        assert abs(hp[f0] / want - 1.0) < 2e-6
        if i == 0:
            assert abs(hp[f0] / (k * unit) - 1.0) < 1e-6
        if k == 1:  # column f0 + 211 is more than h bins from every multiple of f0
            assert hp[f0 + 211] < 1e-12 * unit


def test_threshold_matches_scipy_inverse_gamma():
    p = thresholds.gaussian_tail(6.0)
    assert abs(p / sp.ndtr(-6.0) - 1.0) < 1e-12
    for k in range(1, 17):
        got = thresholds.gamma_threshold(k, p)
        want = sp.gammainccinv(k, p)
        assert abs(got / want - 1.0) < 1e-12
    ta = thresholds.threshold_array(16, 85)
    want32 = np.array([np.float32(sp.gammainccinv(k, p)) for k in range(1, 17)])
    assert np.all(np.abs(ta[:, 0].view(np.int32) - want32.view(np.int32)) <= 1)
    assert np.all(ta == ta[:, :1])
    # -ln(Q(6)) for k = 1, since S_1(x) = exp(-x)
    assert abs(ta[0, 0] - (-math.log(p))) < 1e-5


def test_meansd_threshold_is_literal():
    ta = thresholds.threshold_array(4, 3, sigma=6.0, kind="meansd")
    assert np.allclose(ta[:, 0], [1 + 6, 2 + 6 * math.sqrt(2), 3 + 6 * math.sqrt(3), 4 + 12], rtol=1e-7)


# ---------------------------------------------------------------- highest-harmonic indexing


def _rd(a, b):
    """round(a/b), halves away from zero, by exact rational arithmetic (independent of round_div)."""
    from fractions import Fraction

    x = Fraction(a, b)
    f = abs(x)
    n = int(f)
    if f - n >= Fraction(1, 2):
        n += 1
    return n if x >= 0 else -n


def test_round_div_matches_exact_rounding():
    for a in range(-60, 61):
        for b in range(1, 17):
            assert int(harmonic.round_div(a, b)) == _rd(a, b), (a, b)


def test_highest_harmonic_brute_force():
    """Every HP_k value on a 7 x 41 plane against a pure-Python sum with exact rounding."""
    rng = np.random.default_rng(21)
    plane = rng.exponential(1.0, size=(7, 41)).astype(np.float32)
    c = 3
    got = {(k, i): hp for k, i, hp in harmonic.harmonic_planes_highest(plane, 4)}
    for k in range(1, 5):
        for i in range(-c, c + 1):
            for j in range(41):
                s = np.float32(0)
                for l in range(1, k + 1):
                    v = plane[c + _rd(l * i, k), _rd(l * j, k)]
                    s = v if l == 1 else np.float32(s + v)
                assert got[(k, i)][j] == s, (k, i, j)


def test_highest_harmonic_equals_fundamental_where_k_divides():
    """Where k divides i and j, the highest-harmonic point (i, j) has the terms of the fundamental
    point (i/k, j/k): the values agree bit for bit."""
    rng = np.random.default_rng(22)
    plane = rng.exponential(1.0, size=(17, 300)).astype(np.float32)
    c = 8
    hh = {(k, i): hp for k, i, hp in harmonic.harmonic_planes_highest(plane, 4)}
    fu = {(k, i): hp for k, i, hp in harmonic.harmonic_planes(plane, 4)}
    for k in range(1, 5):
        for i in range(-c, c + 1):
            if i % k or abs(i) > c:
                continue
            f = fu[(k, i // k)]
            for j in range(0, 300, k):
                if j // k < f.size:
                    assert hh[(k, i)][j] == f[j // k], (k, i, j)


def test_highest_harmonic_pulse_train_closed_form(bank):
    """A pulse train (harmonics at multiples of f0, f0 > 2h): at the k-th harmonic position
    j = k f0 of the zero-drift row, HP_k = k (f0/N)^2, as in the fundamental reading."""
    n, f0 = 1 << 14, 512
    spec = synth.pulse_train_spectrum(n, f0)
    plane = correlate.plane_direct(spec, bank).astype(np.float32)
    c = (plane.shape[0] - 1) // 2
    unit = (f0 / n) ** 2
    for k, i, hp in harmonic.harmonic_planes_highest(plane, 8):
        if i != 0 or k * f0 >= n:
            continue
        assert abs(float(hp[k * f0]) / (k * unit) - 1.0) < 1e-6, k
        # Between harmonics (211 bins past the k-th) every term is zero.
        if k * f0 + 211 < n:
            assert hp[k * f0 + 211] < 1e-12 * unit


def test_detect_highest_index_counts_and_order():
    rng = np.random.default_rng(23)
    plane = rng.exponential(1.0, size=(9, 500)).astype(np.float32)
    ta = np.full((4, 9), 6.0, dtype=np.float32)
    res = harmonic.detect(plane, ta, 4, 0xF, 50, index="highest")
    allv = {(k, i): hp for k, i, hp in harmonic.harmonic_planes_highest(plane, 4)}
    for k in range(1, 5):
        total = sum(int((allv[(k, i)] > ta[k - 1, 0]).sum()) for i in range(-4, 5))
        assert res.counts[k - 1] == total
        c = res.cands[k - 1]
        assert np.all(np.diff(c["power"].astype(np.float64)) <= 0)
