"""Comparisons of GPU results with the FP64 oracle, shared by the GPU test files.

* Planes: rel = |P_gpu - P_ref| / max(P_ref, mean P_ref) (the floored relative error), bar 1e-4.
* Candidates of a search (the GPU computed its own plane): the GPU plane differs from the oracle's
  by up to 1e-4 (floored), so a harmonic sum of k terms differs by up to about 1e-4 (HP + k mean).
  Every GPU candidate must carry the oracle's HP_k(i, j) within 2 k 1e-4 relative, and the two lists
  may differ only by points that lie within that tolerance of the threshold.
"""
import numpy as np

from oracle import harmonic

REL_TOL = 1e-4


def plane_rel(gpu, ref):
    rel = np.abs(gpu.astype(np.float64) - ref) / np.maximum(ref, ref.mean())
    return rel.max(), np.sqrt(np.mean(rel**2))


def assert_candidates_within_tolerance(cands, counts, ref_plane, ta, n_harm, mask, cap, rel_tol=REL_TOL):
    """cands/counts: the GPU's per-plane lists (canonical order) and totals, for a search whose plane
    matched ref_plane (FP64 oracle) within rel_tol. Every list must be complete (counts < cap)."""
    ref32 = np.asarray(ref_plane, dtype=np.float32)
    ref = harmonic.detect(ref32, ta, n_harm, mask, cap)
    c = (ref32.shape[0] - 1) // 2
    hp = {(k, i): v for k, i, v in harmonic.harmonic_planes(ref32, n_harm)}
    checked = 0
    for k in range(1, n_harm + 1):
        if not (mask >> (k - 1)) & 1:
            assert counts[k - 1] == 0
            continue
        assert counts[k - 1] < cap and ref.counts[k - 1] < cap, (k, counts[k - 1], ref.counts[k - 1])
        assert len(cands[k - 1]) == counts[k - 1]
        tol = 2 * k * rel_tol
        g = {(int(r["i"]), int(r["j"])): float(r["power"]) for r in cands[k - 1]}
        r = {(int(x["i"]), int(x["j"])): float(x["power"]) for x in ref.cands[k - 1]}
        for (i, j), v in g.items():
            want = float(hp[(k, i)][j])
            assert abs(v - want) <= tol * want, (k, i, j, v, want)
            if (i, j) not in r:
                assert want >= ta[k - 1, c + i] * (1 - tol), (k, i, j, want)
        for (i, j) in set(r) - set(g):
            assert r[(i, j)] <= ta[k - 1, c + i] * (1 + tol), (k, i, j, r[(i, j)])
        # the canonical order of the GPU list
        pw = np.array([float(x["power"]) for x in cands[k - 1]])
        assert np.all(np.diff(pw) <= 0)
        checked += len(g)
    return checked


def assert_same_candidates(got_cands, got_counts, got_peaks, ref, mask):
    """Bit-for-bit equality with the oracle's Algorithm 1 on the same float32 plane: counts, every
    kept candidate (power bits, i, j, k) in canonical order, and every plane's peak."""
    assert [int(c) for c in got_counts] == [int(c) for c in ref.counts]
    for k, (g, r) in enumerate(zip(got_cands, ref.cands), start=1):
        assert len(g) == len(r), k
        assert np.array_equal(g["power"].view(np.uint32), r["power"].view(np.uint32)), k
        assert np.array_equal(g["i"], r["i"]) and np.array_equal(g["j"], r["j"]), k
        assert np.all(g["k"] == k)
    for k, (g, r) in enumerate(zip(got_peaks, ref.peaks), start=1):
        assert (np.float32(g["power"]).view(np.uint32), int(g["i"]), int(g["j"])) == (
            np.float32(r[0]).view(np.uint32), r[1], r[2]), k
