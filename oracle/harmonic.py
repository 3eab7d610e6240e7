"""Harmonic summing and threshold detection (oracle). Test infrastructure only.

Paper, Sec. 2.2, Algorithm 1. The FOP is stretched by a group of integers into stretch planes
SP_k. Then HP_k = HP_{k-1} + SP_k for k = 1..N_hp, and every HP_k(i, j) is tested against
TA(k, i) to collect candidates. Sec. 2.2 and the parameter table give N_hp = 8 planes and
N_cand = 200 candidates per plane.

The paper leaves ``stretch`` undefined, and Algorithm 1 writes SP_1 <- FOP but then
stretch(SP_0, ...). The reading used here indexes by the fundamental:

    SP_k(i, j) = FOP(k*i, k*j),   HP_0 = 0,   HP_k = HP_{k-1} + SP_k,

with exact integer indices. Row index i is the template offset from the zero-drift row,
|i| <= c = (N_temp-1)/2, so FOP(r, j) means plane row c + r. HP_k is defined on the domain
D_k = {|k*i| <= c, k*j <= N-1}. Points outside D_k are not evaluated.

A second reading, offered as an option (``index="highest"``), indexes every harmonic plane by
the position of its highest harmonic, as pulsar searches commonly do. The point (i, j) of HP_k is
taken as the k-th harmonic of a signal, and the lower harmonics l = 1..k sit at l/k of its row
offset and column, rounded to the nearest integer (halves away from zero):

    HP_k(i, j) = sum_{l=1..k} FOP(rd(l*i, k), rd(l*j, k)),   rd(a, b) = round(a / b),

on the whole plane (|i| <= c, 0 <= j <= N-1), as float32 running sums in the order l = 1..k. It
is not incremental in k, because the positions change with k. Where k divides both i and j the
terms are those of the fundamental reading at (i/k, j/k).

Detection emits (k, i, j, HP_k(i, j)) when HP_k(i, j) > TA(k, i), for the harmonics k
selected by ``harm_mask`` (bit k-1). The test is strict and done in float32. The sums are
float32 running sums in the order l = 1, 2, ..., k, so a device implementation that adds in
the same order gets the same bits. For each k, the top ``cand_cap`` crossings are kept in the
canonical order (power descending, then i ascending, then j ascending), and the total number
of crossings is reported.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class HarmonicResult:
    """Candidates per harmonic plane, in canonical order, plus totals and per-plane peaks.

    cands[k-1]: structured array with fields power (float32), i (int16), j (uint32), k (uint8).
    counts[k-1]: total number of crossings in HP_k (0 for unreported k).
    peaks[k-1]: (power, i, j), the first point of HP_k over D_k in canonical order.
    """

    cands: list
    counts: np.ndarray
    peaks: list


CAND_DTYPE = np.dtype([("power", np.float32), ("i", np.int16), ("j", np.uint32), ("k", np.uint8)])


def _canonical(power: np.ndarray, i: np.ndarray, j: np.ndarray) -> np.ndarray:
    """Indices that sort by (power desc, i asc, j asc)."""
    return np.lexsort((j, i, -power.astype(np.float64)))


def harmonic_planes(plane32: np.ndarray, n_harm: int):
    """Yield (k, i, HP_k(i, :)) for k = 1..n_harm and every i with |k*i| <= c, in float32.

    HP_k(i, j) for j = 0..(N-1)//k is the running float32 sum of plane[c + l*i][l*j],
    l = 1..k (Algorithm 1 with the fundamental-indexed stretch).
    """
    p = np.asarray(plane32, dtype=np.float32)
    n_temp, n = p.shape
    c = (n_temp - 1) // 2
    prev = {}
    for k in range(1, n_harm + 1):
        jmax = (n - 1) // k  # k*j <= N-1
        cols = k * np.arange(jmax + 1)
        for i in range(-c, c + 1):
            if abs(k * i) > c:
                continue
            sp = p[c + k * i, cols]
            hp = sp.copy() if k == 1 else (prev[i][: jmax + 1] + sp).astype(np.float32)
            prev[i] = hp
            yield k, i, hp


def round_div(a, b: int):
    """round(a / b) for integers a (scalar or array) and b > 0, halves away from zero, exactly."""
    a = np.asarray(a, dtype=np.int64)
    return np.sign(a) * ((2 * np.abs(a) + b) // (2 * b))


def harmonic_planes_highest(plane32: np.ndarray, n_harm: int):
    """Yield (k, i, HP_k(i, :)) for k = 1..n_harm and every |i| <= c, indexed by the highest harmonic.

    HP_k(i, j) for j = 0..N-1 is the running float32 sum over l = 1..k of
    plane[c + rd(l*i, k)][rd(l*j, k)].
    """
    p = np.asarray(plane32, dtype=np.float32)
    n_temp, n = p.shape
    c = (n_temp - 1) // 2
    j = np.arange(n, dtype=np.int64)
    for k in range(1, n_harm + 1):
        cols = [round_div(l * j, k) for l in range(1, k + 1)]
        for i in range(-c, c + 1):
            hp = None
            for l in range(1, k + 1):
                v = p[c + int(round_div(l * i, k)), cols[l - 1]]
                hp = v.copy() if hp is None else (hp + v).astype(np.float32)
            yield k, i, hp


def detect(
    plane32: np.ndarray,
    thresh: np.ndarray,
    n_harm: int,
    harm_mask: int,
    cand_cap: int,
    index: str = "fundamental",
) -> HarmonicResult:
    """Algorithm 1 over a float32 plane with float32 thresholds TA[k-1][c + i].

    index: "fundamental" (SP_k(i, j) = FOP(k i, k j)) or "highest" (harmonic_planes_highest).
    """
    p = np.asarray(plane32, dtype=np.float32)
    ta = np.asarray(thresh, dtype=np.float32)
    c = (p.shape[0] - 1) // 2
    found = {k: ([], [], []) for k in range(1, n_harm + 1)}
    best = {}
    planes = harmonic_planes(p, n_harm) if index == "fundamental" else harmonic_planes_highest(p, n_harm)
    for k, i, hp in planes:
        # Per-plane peak: the largest value, earliest (i, j) on ties (i is visited ascending).
        jbest = int(np.argmax(hp))
        cur = (hp[jbest], i, jbest)
        if k not in best or cur[0] > best[k][0]:
            best[k] = cur
        if not (harm_mask >> (k - 1)) & 1:
            continue
        hit = np.nonzero(hp > ta[k - 1, c + i])[0]
        if hit.size:
            found[k][0].append(hp[hit])
            found[k][1].append(np.full(hit.size, i, dtype=np.int16))
            found[k][2].append(hit.astype(np.uint32))
    cands, counts, peaks = [], np.zeros(n_harm, dtype=np.int64), []
    for k in range(1, n_harm + 1):
        pw, ii, jj = found[k]
        if pw:
            pw, ii, jj = np.concatenate(pw), np.concatenate(ii), np.concatenate(jj)
        else:
            pw, ii, jj = (np.zeros(0, np.float32), np.zeros(0, np.int16), np.zeros(0, np.uint32))
        counts[k - 1] = pw.size
        order = _canonical(pw, ii, jj)[:cand_cap]
        rec = np.zeros(order.size, dtype=CAND_DTYPE)
        rec["power"], rec["i"], rec["j"], rec["k"] = pw[order], ii[order], jj[order], k
        cands.append(rec)
        peaks.append(best[k])
    return HarmonicResult(cands, counts, peaks)
