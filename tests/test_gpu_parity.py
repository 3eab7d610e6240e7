"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances:
* Template bank: max |T_gpu - T_ref| <= 1e-6 * max |T_ref| (one float32 rounding of FP64 values).
* F-A plane: rel = |P_gpu - P_ref| / max(P_ref, mean P_ref) <= 1e-4, the bar for the float32 path.
  The max and RMS are printed for every case.
* Harmonic sum fed the oracle's float32 plane: candidates, counts and peaks bit for bit.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import correlate, harmonic, templates, thresholds

from parity_helpers import REL_TOL, assert_candidates_within_tolerance, assert_same_candidates, plane_rel

pytestmark = pytest.mark.gpu


def run_convolve(fd, p, spec, ld=None, fill=np.nan):
    n = len(spec)
    ld = n if ld is None else ld
    tmpl = torch.empty(fd.fdas_templates_bytes(p), dtype=torch.uint8, device="cuda")
    fd.fdas_make_templates(p, tmpl)
    d_spec = torch.from_numpy(np.ascontiguousarray(spec, dtype=np.complex64)).cuda()
    plane = torch.full((p.n_temp, ld), fill, dtype=torch.float32, device="cuda")
    fd.fdas_convolve(p, d_spec, n, tmpl, plane, ld)
    torch.cuda.synchronize()
    return plane.cpu().numpy(), tmpl


def run_harmonic(fd, p, plane32, thresh, ld=None):
    n_temp, n = plane32.shape
    ld = n if ld is None else ld
    d_plane = torch.full((n_temp, ld), 1e30, dtype=torch.float32, device="cuda")
    d_plane[:, :n] = torch.from_numpy(np.ascontiguousarray(plane32)).cuda()
    d_ta = torch.from_numpy(np.ascontiguousarray(thresh, dtype=np.float32)).cuda()
    ws_bytes = fd.fdas_workspace_bytes(p, n)
    ws = torch.full((ws_bytes,), 0xAB, dtype=torch.uint8, device="cuda")  # contents need no initialisation
    cands = torch.zeros(p.n_harm * p.cand_cap * 12, dtype=torch.uint8, device="cuda")
    counts = torch.zeros(p.n_harm, dtype=torch.int32, device="cuda")
    peaks = torch.zeros(p.n_harm * 12, dtype=torch.uint8, device="cuda")
    fd.fdas_harmonic_sum(p, d_plane, n, ld, d_ta, cands, counts, peaks, ws, ws_bytes)
    torch.cuda.synchronize()
    counts = counts.cpu().numpy().astype(np.uint32)
    return fd.decode_cands(cands.cpu().numpy(), counts, p.cand_cap), counts, peaks.cpu().numpy().view(fd.CAND_DTYPE)


# ---------------------------------------------------------------- templates


@pytest.mark.parametrize(
    "kw", [dict(), dict(n_temp=9, z_min=-8, z_step=2, n_tap=101), dict(n_temp=3, z_min=-1, n_tap=1023)]
)
def test_templates_match_oracle(fd, kw):
    p = fd.Params(**kw)
    grid = templates.TemplateGrid(p.n_temp, float(p.z_min), float(p.z_step), p.n_tap)
    ref = templates.frequency_templates(templates.template_bank(grid), p.fft_len)
    tmpl = torch.empty(fd.fdas_templates_bytes(p), dtype=torch.uint8, device="cuda")
    fd.fdas_make_templates(p, tmpl)
    torch.cuda.synchronize()
    got = tmpl.cpu().numpy().view(np.complex64).reshape(p.n_temp + 1, p.fft_len)
    err = np.max(np.abs(got[: p.n_temp] - ref))
    print(f"templates {kw}: max abs err {err:.3e} (max |T| {np.max(np.abs(ref)):.3f})")
    assert err <= 1e-6 * np.max(np.abs(ref))
    twiddle = np.exp(-2j * np.pi * np.arange(p.fft_len) / p.fft_len)
    assert np.max(np.abs(got[p.n_temp] - twiddle)) < 1.2e-7


# ---------------------------------------------------------------- convolution


@pytest.mark.parametrize("n", [1, 2, 211, 1628, 1629, 3257, 5000, 20000])
def test_plane_small_and_ragged(fd, bank, n):
    p = fd.Params()
    rng = np.random.default_rng(n)
    spec = synth.complex_noise(rng, n) + synth.tone_spectrum(n, [synth.Tone(n // 2, 11, 15.0, 1)])
    spec = spec.astype(np.complex64)
    got, _ = run_convolve(fd, p, spec)
    ref = correlate.plane_direct(spec, bank)
    mx, rms = plane_rel(got, ref)
    print(f"N={n}: plane rel max {mx:.2e} rms {rms:.2e}")
    assert mx <= REL_TOL


def test_plane_leaves_padding_columns_untouched(fd, bank):
    p = fd.Params()
    n, ld = 3000, 3072
    spec = synth.complex_noise(np.random.default_rng(2), n).astype(np.complex64)
    got, _ = run_convolve(fd, p, spec, ld=ld, fill=-7.0)
    assert np.all(got[:, n:] == -7.0)
    mx, _ = plane_rel(got[:, :n], correlate.plane_direct(spec, bank))
    assert mx <= REL_TOL


def test_plane_small_workload(fd, small_case):
    wl, ref = small_case
    got, _ = run_convolve(fd, fd.Params(), wl.spectrum)
    mx, rms = plane_rel(got, ref)
    print(f"N=2^16 small workload: plane rel max {mx:.2e} rms {rms:.2e}, max|dP|/maxP "
          f"{np.max(np.abs(got - ref)) / ref.max():.2e}")
    assert mx <= REL_TOL
    assert np.unravel_index(np.argmax(got), got.shape) == (62, 12000)
    # zero-drift row is |X|^2 up to float32 FFT rounding
    x = wl.spectrum.astype(np.complex128)
    assert np.max(np.abs(got[42] - np.abs(x) ** 2) / np.maximum(np.abs(x) ** 2, 1.0)) < 1e-5


def test_plane_other_template_grid(fd):
    p = fd.Params(n_temp=9, z_min=-8, z_step=2, n_tap=101)
    grid = templates.TemplateGrid(9, -8.0, 2.0, 101)
    bank = templates.template_bank(grid)
    n = 9000
    spec = synth.complex_noise(np.random.default_rng(5), n).astype(np.complex64)
    got, _ = run_convolve(fd, p, spec)
    mx, _ = plane_rel(got, correlate.plane_ols(spec, bank, 2048))
    assert mx <= REL_TOL


def test_plane_full_size(fd, ska_case):
    """N = 2^21, 85 templates: the whole plane against the oracle, in the bench's launch configuration."""
    wl, ref = ska_case
    p = fd.Params()
    s = fd.Searcher(p, wl.n)
    d_spec = torch.from_numpy(wl.spectrum).cuda()
    s.search(d_spec, wl.n)
    torch.cuda.synchronize()
    got = s.plane[:, : wl.n].cpu().numpy()
    mx, rms = plane_rel(got, ref)
    print(f"N=2^21: plane rel max {mx:.2e} rms {rms:.2e}")
    assert mx <= REL_TOL
    # Spot points from the direct definition too (independent of the oracle's overlap-save route).
    rng = np.random.default_rng(9)
    rows = rng.integers(0, 85, 64)
    cols = np.concatenate([rng.integers(0, wl.n, 56), [0, 1, 1627, 1628, wl.n - 2, wl.n - 1, 1628 * 1288, 2047]])
    direct = correlate.power_at(wl.spectrum, templates.template_bank(), rows, cols)
    rel = np.abs(got[rows, cols] - direct) / np.maximum(direct, 1.0)
    assert rel.max() <= REL_TOL
    # Every injected fundamental with |z| <= 42 peaks in its own row and column.
    for t in wl.tones:
        row = 42 + int(t.z)
        col = int(t.mean_bin)
        assert got[row, col] == got[row, col - 3 : col + 4].max()


# ---------------------------------------------------------------- harmonic sum


@pytest.mark.parametrize(
    "kw,sigma",
    [
        (dict(n_harm=8, harm_mask=0b10001011), 6.0),
        (dict(n_harm=8, harm_mask=0xFF), 3.0),
        (dict(n_harm=16, harm_mask=0xFFFF, cand_cap=50), 3.5),
        (dict(n_harm=4, harm_mask=0b0101, cand_cap=1), 3.0),
    ],
)
def test_harmonic_bit_exact_small(fd, small_case, kw, sigma):
    wl, ref_plane = small_case
    p = fd.Params(**kw)
    plane32 = ref_plane.astype(np.float32)
    ta = thresholds.threshold_array(p.n_harm, 85, sigma=sigma)
    got = run_harmonic(fd, p, plane32, ta)
    ref = harmonic.detect(plane32, ta, p.n_harm, p.harm_mask, p.cand_cap)
    print(f"{kw} sigma {sigma}: counts {list(ref.counts)}")
    assert_same_candidates(*got, ref, p.harm_mask)


@pytest.mark.parametrize("n,ld", [(1, 1), (7, 16), (1000, 1000), (4099, 4160)])
def test_harmonic_bit_exact_edges(fd, n, ld):
    p = fd.Params(n_temp=17, z_min=-8, n_harm=8, harm_mask=0xFF, cand_cap=64)
    plane = synth.exponential_plane(np.random.default_rng(n), 17, n)
    ta = thresholds.threshold_array(8, 17, sigma=1.5)
    got = run_harmonic(fd, p, plane, ta, ld=ld)
    ref = harmonic.detect(plane, ta, 8, 0xFF, 64)
    assert_same_candidates(*got, ref, 0xFF)


def test_harmonic_many_crossings_top_cap(fd):
    # Hundreds to thousands of crossings per plane, all above cand_cap: the top 200 must be exact.
    p = fd.Params()
    plane = synth.exponential_plane(np.random.default_rng(21), 85, 1 << 15)
    ta = np.concatenate(
        [thresholds.threshold_array(8, 85, sigma=3.2 - 1.0 * k / 7)[k : k + 1] for k in range(8)]
    )
    got = run_harmonic(fd, p, plane, ta)
    ref = harmonic.detect(plane, ta, 8, 0xFF, 200)
    assert min(ref.counts) > 200 and max(ref.counts) < 16384, ref.counts
    assert_same_candidates(*got, ref, 0xFF)


def test_harmonic_raw_overflow_counts_everything(fd):
    # More crossings than the raw buffer holds: counts stay exact and every record is a true crossing.
    p = fd.Params(n_harm=2, harm_mask=0b11)
    plane = synth.exponential_plane(np.random.default_rng(22), 85, 1 << 15)
    ta = thresholds.threshold_array(2, 85, sigma=1.0)
    cands, counts, _ = run_harmonic(fd, p, plane, ta)
    ref = harmonic.detect(plane, ta, 2, 0b11, 200)
    assert [int(c) for c in counts] == [int(c) for c in ref.counts]
    assert min(ref.counts) > 16384
    hp = {(k, i): v for k, i, v in harmonic.harmonic_planes(plane, 2)}
    for k, rec in enumerate(cands, start=1):
        assert len(rec) == 200
        assert np.all(np.diff(rec["power"]) <= 0)
        for r in rec:
            assert hp[(k, int(r["i"]))][int(r["j"])] == r["power"] > ta[k - 1, 42 + int(r["i"])]


def test_harmonic_bit_exact_full_size(fd, ska_case):
    """N = 2^21: the harmonic sum fed the oracle's float32 plane returns the oracle's candidates."""
    wl, ref_plane = ska_case
    p = fd.Params()
    plane32 = ref_plane.astype(np.float32)
    ta = thresholds.threshold_array(8, 85, sigma=6.0)
    got = run_harmonic(fd, p, plane32, ta, ld=wl.n + 64)
    ref = harmonic.detect(plane32, ta, 8, 0xFF, 200)
    print(f"N=2^21 counts {list(ref.counts)}")
    assert_same_candidates(*got, ref, 0xFF)
    assert sum(ref.counts) > 0


# ---------------------------------------------------------------- whole search


def test_search_host_equals_device_and_repeats(fd, small_case):
    wl, _ = small_case
    p = fd.Params(harm_mask=0b10001011)
    s = fd.Searcher(p, wl.n)
    d_spec = torch.from_numpy(wl.spectrum).cuda()
    s.search(d_spec, wl.n)
    torch.cuda.synchronize()
    a = s.results()
    h_spec = torch.from_numpy(wl.spectrum).pin_memory()
    for _ in range(2):
        s.search_host(h_spec, wl.n)
        b = s.results(host=True)
        assert np.array_equal(a[1], b[1])
        for x, y in zip(a[0], b[0]):
            assert x.tobytes() == y.tobytes()
        assert a[2].tobytes() == b[2].tobytes()
    # the injected tone is the loudest HP_1 point, at (i = +20, j = 12000)
    top = a[0][0][0]
    assert (int(top["i"]), int(top["j"])) == (20, 12000)


def test_search_candidates_match_oracle_within_tolerance(fd, small_case):
    """fdas_search on the GPU plane against Algorithm 1 on the oracle plane.

    Where they differ, the point must lie within the plane tolerance of the threshold.
    """
    wl, ref_plane = small_case
    p = fd.Params(harm_mask=0b10001011, cand_cap=1000)  # the tone's sidelobes give ~330 crossings
    ta = thresholds.threshold_array(8, 85, sigma=6.0)
    s = fd.Searcher(p, wl.n, thresh=ta)
    s.search(torch.from_numpy(wl.spectrum).cuda(), wl.n)
    torch.cuda.synchronize()
    cands, counts, _ = s.results()
    ref32 = ref_plane.astype(np.float32)
    ref = harmonic.detect(ref32, ta, 8, p.harm_mask, 1000)
    hp = {(k, i): v for k, i, v in harmonic.harmonic_planes(ref32, 8)}
    tol = 2 * 8 * REL_TOL
    for k in (1, 2, 4, 8):
        assert counts[k - 1] < 1000 and ref.counts[k - 1] < 1000
        g = {(int(r["i"]), int(r["j"])): float(r["power"]) for r in cands[k - 1]}
        r = {(int(x["i"]), int(x["j"])): float(x["power"]) for x in ref.cands[k - 1]}
        for q, v in g.items():
            want = float(hp[(k, q[0])][q[1]])
            assert abs(v - want) <= tol * want
            if q not in r:
                assert want >= ta[k - 1, 0] * (1 - tol)
        for q in set(r) - set(g):
            assert r[q] <= ta[k - 1, 0] * (1 + tol)
    assert (int(cands[0][0]["i"]), int(cands[0][0]["j"])) == (20, 12000)


def test_search_candidates_match_oracle_at_full_size(fd, ska_case):
    """fdas_search at N = 2^21 in the bench's configuration (FP32, HP_1 of the single-plane rows taken
    inside the convolution, row groups concurrent): every candidate of all 8 planes at the 6-sigma
    thresholds against Algorithm 1 on the oracle plane, within the plane tolerance."""
    wl, ref = ska_case
    p = fd.Params(cand_cap=4096)
    ta = thresholds.threshold_array(8, 85, sigma=6.0)
    s = fd.Searcher(p, wl.n, thresh=ta)
    s.search(torch.from_numpy(wl.spectrum).cuda(), wl.n)
    torch.cuda.synchronize()
    cands, counts, _ = s.results()
    checked = assert_candidates_within_tolerance(cands, counts, ref, ta, 8, 0xFF, p.cand_cap)
    print(f"N=2^21: {checked} candidates checked, counts {list(counts)}")
    assert counts[0] > 100 and counts[7] > 10


def test_no_bounded_wait_gave_up(fd, small_case):
    """The convolution's bounded waits on its template copies all completed in every launch so far."""
    wl, _ = small_case
    p = fd.Params()
    s = fd.Searcher(p, wl.n)
    s.search(torch.from_numpy(wl.spectrum).cuda(), wl.n)
    torch.cuda.synchronize()
    assert fd.fdas_device_status(clear=True) == 0
    assert fd.fdas_device_status() == 0


def test_bounded_wait_gives_up_and_the_context_stays_usable(fd, small_case):
    """A wait on an mbarrier nothing completes ends after about a second with the status bit set;
    the next convolution runs normally and leaves the status clear."""
    import time

    t0 = time.perf_counter()
    flags = fd.fdas_check_wait_timeout()
    dt = time.perf_counter() - t0
    assert flags & 1
    assert 0.2 < dt < 30.0
    assert fd.fdas_device_status() == 0  # cleared by the diagnostic
    wl, ref = small_case
    p = fd.Params()
    s = fd.Searcher(p, wl.n)
    s.search(torch.from_numpy(wl.spectrum).cuda(), wl.n)
    torch.cuda.synchronize()
    got = s.plane[:, : wl.n].cpu().numpy()
    mx, _ = plane_rel(got, ref)
    assert mx <= REL_TOL
    assert fd.fdas_device_status() == 0


def _search_both_ways(fd, p, spec, thresh, ld=None):
    """fdas_search (HP_1 taken by the convolution) and fdas_convolve + fdas_harmonic_sum."""
    n = len(spec)
    ld = n if ld is None else ld
    tmpl = torch.empty(fd.fdas_templates_bytes(p), dtype=torch.uint8, device="cuda")
    fd.fdas_make_templates(p, tmpl)
    d_spec = torch.from_numpy(np.ascontiguousarray(spec, dtype=np.complex64)).cuda()
    d_ta = torch.from_numpy(np.ascontiguousarray(thresh, dtype=np.float32)).cuda()
    ws_bytes = fd.fdas_workspace_bytes(p, n)
    out = []
    for fused in (True, False):
        plane = torch.full((p.n_temp, ld), np.nan, dtype=torch.float32, device="cuda")
        ws = torch.full((ws_bytes,), 0xCD, dtype=torch.uint8, device="cuda")
        cands = torch.zeros(p.n_harm * p.cand_cap * 12, dtype=torch.uint8, device="cuda")
        counts = torch.zeros(p.n_harm, dtype=torch.int32, device="cuda")
        peaks = torch.zeros(p.n_harm * 12, dtype=torch.uint8, device="cuda")
        if fused:
            fd.fdas_search(p, d_spec, n, tmpl, plane, ld, d_ta, cands, counts, peaks, ws, ws_bytes)
        else:
            fd.fdas_convolve(p, d_spec, n, tmpl, plane, ld)
            fd.fdas_harmonic_sum(p, plane, n, ld, d_ta, cands, counts, peaks, ws, ws_bytes)
        torch.cuda.synchronize()
        cnt = counts.cpu().numpy().astype(np.uint32)
        out.append((plane.cpu().numpy(), fd.decode_cands(cands.cpu().numpy(), cnt, p.cand_cap), cnt,
                    peaks.cpu().numpy().view(fd.CAND_DTYPE)))
    return out


@pytest.mark.parametrize(
    "n,kw,sigma",
    [
        (1, {}, 6.0),
        (211, {}, 3.0),
        (5000, {}, 3.0),
        (40000, dict(cand_cap=1000), 3.5),
        (40000, dict(harm_mask=0b11111110), 3.5),
        (40000, dict(n_harm=1, harm_mask=1, cand_cap=1000), 3.5),
        (40000, dict(n_harm=16, harm_mask=0xFFFF), 3.5),
        (30000, dict(n_temp=9, z_min=-8, z_step=2, n_tap=129, n_harm=4, harm_mask=0xF), 3.0),
        (30000, dict(harm_index=1), 3.5),
        (1628 * 7 + 5, dict(n_harm=16, harm_mask=0xFFFF, cand_cap=500), 3.0),
        (65536, dict(n_harm=5, harm_mask=0b10110), 3.5),
        (99991, dict(n_temp=255, z_min=-127, n_harm=12, harm_mask=0xFFF), 4.0),
    ],
)
def test_search_with_fused_hp1_equals_separate_calls(fd, n, kw, sigma):
    """fdas_search takes HP_1 inside the convolution; its plane, candidates, counts and peaks equal
    those of fdas_convolve followed by fdas_harmonic_sum, bit for bit (below FDAS_RAW_CAP)."""
    p = fd.Params(**kw)
    wl = synth.small_workload(n=max(n, 64))
    spec = wl.spectrum[:n].copy()
    ta = thresholds.threshold_array(p.n_harm, p.n_temp, sigma=sigma)
    (pa, ca, na, ka), (pb, cb, nb, kb) = _search_both_ways(fd, p, spec, ta, ld=n + 3 * (n % 2 == 0))
    assert np.array_equal(pa.view(np.uint32)[:, :n], pb.view(np.uint32)[:, :n])
    assert np.array_equal(na, nb) and int(na.max()) < 16384
    for k in range(p.n_harm):
        assert np.array_equal(ca[k], cb[k]), k
    assert np.array_equal(ka, kb)
    if p.harm_mask & 1:
        assert int(na[0]) > 0 or n < 64


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("n_tap", [257, 129])
def test_plane_reduced_taps(fd, prec, n_tap):
    """The paper's reduced-tap variants (256 and 128 taps, Sec. 4, run as 257 and 129 so that every
    template stays centred) on the full 85-template grid, every convolution form."""
    p = fd.Params(n_tap=n_tap, precision=prec)
    grid = templates.TemplateGrid(n_tap=n_tap)
    bank = templates.template_bank(grid)
    spec = synth.small_workload(n=20000).spectrum
    got, _ = run_convolve(fd, p, spec)
    mx, rms = plane_rel(got, correlate.plane_ols(spec, bank, 2048))
    print(f"n_tap={n_tap} precision={prec}: rel max {mx:.2e} rms {rms:.2e}")
    assert mx <= REL_TOL


# ---------------------------------------------------------------- highest-harmonic indexing


@pytest.mark.parametrize(
    "n,kw,sigma,aligned",
    [
        (7, dict(n_harm=3, harm_mask=0b101), 1.5, False),
        (1000, dict(n_harm=4, harm_mask=0xF), 3.0, False),
        (4099, {}, 3.5, False),
        (4099, {}, 3.5, True),
        (20000, dict(n_harm=16, harm_mask=0xFFFF), 4.0, False),
        (20000, dict(n_harm=16, harm_mask=0xFFFF), 4.0, True),
        (3001, dict(n_harm=11, harm_mask=0x7FF), 3.0, True),
        (20000, dict(n_temp=9, z_min=-8, z_step=2, n_harm=8, harm_mask=0b10010110), 3.0, False),
    ],
)
def test_harmonic_highest_index_bit_exact(fd, n, kw, sigma, aligned):
    """FDAS_INDEX_HIGHEST against the oracle's highest-harmonic planes: candidates, counts and peaks
    bit for bit on unit-exponential planes; with a row stride that allows 16-byte loads and one that
    does not."""
    p = fd.Params(harm_index=1, cand_cap=1000, **kw)
    plane = synth.exponential_plane(np.random.default_rng(100 + n), p.n_temp, n)
    ta = thresholds.threshold_array(p.n_harm, p.n_temp, sigma=sigma)
    got = run_harmonic(fd, p, plane, ta, ld=(n + 63) // 64 * 64 if aligned else n + 5)
    ref = harmonic.detect(plane, ta, p.n_harm, p.harm_mask, p.cand_cap, index="highest")
    assert_same_candidates(*got, ref, p.harm_mask)


def test_harmonic_highest_index_large(fd):
    """N = 2^18 with the default 85 x 8 planes: counts and candidates against the oracle."""
    p = fd.Params(harm_index=1, cand_cap=500)
    n = 1 << 18
    plane = synth.exponential_plane(np.random.default_rng(7), p.n_temp, n)
    ta = thresholds.threshold_array(p.n_harm, p.n_temp, sigma=4.5)
    got = run_harmonic(fd, p, plane, ta)
    ref = harmonic.detect(plane, ta, p.n_harm, p.harm_mask, p.cand_cap, index="highest")
    assert_same_candidates(*got, ref, p.harm_mask)


# ---------------------------------------------------------------- graph capture of a whole search


@pytest.mark.parametrize("precision", [0, 1])
def test_search_captured_in_a_cuda_graph_equals_eager(fd, small_case, precision):
    """fdas_search captured into a CUDA graph from a user stream (its harmonic-sum launches fork into
    the library's auxiliary streams and join back) replays to the eager results, bit for bit."""
    wl, _ = small_case
    p = fd.Params(precision=precision)
    s = fd.Searcher(p, wl.n, thresh=thresholds.threshold_array(p.n_harm, p.n_temp, sigma=3.0))
    d_spec = torch.from_numpy(wl.spectrum).cuda()
    s.search(d_spec, wl.n)
    torch.cuda.synchronize()
    want_c, want_n, want_p = s.results()
    assert want_n.sum() > 0
    for t in (s.cands, s.counts, s.peaks, s.plane):
        t.zero_()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.graph(g, stream=side, capture_error_mode="thread_local"):
        s.search(d_spec, wl.n)  # enqueued on the capturing stream
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    got_c, got_n, got_p = s.results()
    assert np.array_equal(got_n, want_n)
    for a, b in zip(got_c, want_c):
        assert a.tobytes() == b.tobytes()
    assert got_p.tobytes() == want_p.tobytes()
    assert fd.fdas_device_status() == 0


@pytest.mark.parametrize("m", [2, 3])
def test_search_host_async_on_several_streams_equals_the_synchronous_call(fd, small_case, m):
    """fdas_search_host_async on m searchers and streams in turn (copies of one spectrum overlapping
    the others' searches; three is the pattern bench.py times) leaves the same host results as
    fdas_search_host."""
    wl, _ = small_case
    p = fd.Params()
    ta = thresholds.threshold_array(p.n_harm, p.n_temp, sigma=3.0)
    h = torch.from_numpy(wl.spectrum).pin_memory()
    ref = fd.Searcher(p, wl.n, thresh=ta)
    ref.search_host(h, wl.n)
    want_c, want_n, want_p = ref.results(host=True)
    assert want_n.sum() > 0
    pair = [fd.Searcher(p, wl.n, thresh=ta) for _ in range(m)]
    streams = [torch.cuda.Stream() for _ in range(m)]
    for k in range(2 * m + 1):
        pair[k % m].search_host_async(h, wl.n, streams[k % m])
    torch.cuda.synchronize()
    for s in pair:
        got_c, got_n, got_p = s.results(host=True)
        assert np.array_equal(got_n, want_n)
        for a, b in zip(got_c, want_c):
            assert a.tobytes() == b.tobytes()
        assert got_p.tobytes() == want_p.tobytes()


def test_searches_from_two_host_threads_equal_one_thread(fd, small_case):
    """Two host threads searching at the same time, each on its own searcher and stream (the
    library's auxiliary streams are shared, its fork and join events are per thread), get the same
    results as one thread alone."""
    import threading

    wl, _ = small_case
    p = fd.Params()
    ta = thresholds.threshold_array(p.n_harm, p.n_temp, sigma=3.0)
    d_spec = torch.from_numpy(wl.spectrum).cuda()
    ref = fd.Searcher(p, wl.n, thresh=ta)
    ref.search(d_spec, wl.n)
    torch.cuda.synchronize()
    want_c, want_n, want_p = ref.results()
    workers = [fd.Searcher(p, wl.n, thresh=ta) for _ in range(2)]
    errors = []

    def run(s):
        try:
            torch.cuda.set_device(0)
            st = torch.cuda.Stream()
            for _ in range(6):
                s.search(d_spec, wl.n, stream=st)
            st.synchronize()
        except Exception as exc:  # reported below, in the test's own thread
            errors.append(exc)

    threads = [threading.Thread(target=run, args=(s,)) for s in workers]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for s in workers:
        got_c, got_n, got_p = s.results()
        assert np.array_equal(got_n, want_n)
        for a, b in zip(got_c, want_c):
            assert a.tobytes() == b.tobytes()
        assert got_p.tobytes() == want_p.tobytes()


# ---------------------------------------------------------------- maximum size


def test_search_at_the_maximum_length(fd):
    """N = FDAS_MAX_N = 2^24 (a 5.7 GB plane), with a drifting tone near the last bin, so that
    candidate columns use all 24 bits of the key. The oracle cannot build this plane in seconds, so
    the check uses properties that hold at any size:
    - sampled plane points, including the last columns, against the direct definition;
    - every reported candidate's HP_k recomputed from the GPU plane (float32, l = 1..k) bit for
      bit, above its threshold, in canonical order, its count at least the listed number;
    - each plane's peak no smaller than its best candidate."""
    n = 1 << 24
    p = fd.Params(harm_mask=0b10001011)
    rng = np.random.default_rng(24)
    x = synth.complex_noise(rng, n) + synth.tone_spectrum(n, [synth.Tone(n - 3000, 5, 25.0, 1)])
    spec = x.astype(np.complex64)
    s = fd.Searcher(p, n)
    s.search(torch.from_numpy(spec).cuda(), n)
    torch.cuda.synchronize()
    assert fd.fdas_device_status() == 0
    cands, counts, peaks = s.results()
    c = (p.n_temp - 1) // 2

    rows = np.concatenate([rng.integers(0, 85, 24), [0, 84, 42, 47, 42, 84]])
    cols = np.concatenate([rng.integers(0, n, 24), [n - 1, n - 1, 0, n - 3000, n - 2, 1 << 23]])
    got = s.plane[torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()].cpu().numpy()
    direct = correlate.power_at(spec, templates.template_bank(), rows, cols)
    assert (np.abs(got - direct) / np.maximum(direct, 1.0)).max() <= REL_TOL

    ta = fd.fdas_default_thresholds(p)
    plane = s.plane
    for k in range(1, p.n_harm + 1):
        rec = cands[k - 1]
        if not (p.harm_mask >> (k - 1)) & 1:
            assert len(rec) == 0
            continue
        assert int(counts[k - 1]) >= len(rec)
        keys = [(-float(r["power"]), int(r["i"]), int(r["j"])) for r in rec]
        assert keys == sorted(keys)
        for r in rec[:50]:
            i, j = int(r["i"]), int(r["j"])
            idx_r = torch.tensor([c + l * i for l in range(1, k + 1)], device="cuda")
            idx_c = torch.tensor([l * j for l in range(1, k + 1)], device="cuda")
            terms = plane[idx_r, idx_c].cpu().numpy().astype(np.float32)
            hp = np.float32(terms[0])
            for v in terms[1:]:
                hp = np.float32(hp + v)
            assert hp == np.float32(r["power"])
            assert hp > ta[k - 1, c + i]
        if len(rec):
            assert float(peaks[k - 1]["power"]) >= float(rec[0]["power"])
    # the tone (z = +5, mean bin n - 3000) is the loudest HP_1 point, in row +5 near its bin
    top = cands[0][0]
    assert int(top["i"]) == 5 and abs(int(top["j"]) - (n - 3000)) <= 2


# ---------------------------------------------------------------- largest template grid


@pytest.fixture(scope="module")
def grid255():
    """255 templates (z = -127..127, the most fdas_params allows), 421 taps, N = 5000: spectrum and
    FP64 oracle plane."""
    grid = templates.TemplateGrid(n_temp=255, z_min=-127.0, z_step=1.0, n_tap=421)
    bank = templates.template_bank(grid)
    rng = np.random.default_rng(255)
    n = 5000
    spec = (synth.complex_noise(rng, n) + synth.tone_spectrum(n, [synth.Tone(2500, 100, 20.0, 2)])).astype(
        np.complex64)
    return spec, correlate.plane_ols(spec, bank, 2048)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_largest_template_grid(fd, grid255, prec):
    """Every convolution form on 255 templates (rows up to 254 in the candidate keys) against the
    oracle plane, and the harmonic sum fed the oracle plane bit for bit."""
    spec, ref = grid255
    p = fd.Params(n_temp=255, z_min=-127, n_harm=8, harm_mask=0xFF, cand_cap=500, precision=prec)
    got, _ = run_convolve(fd, p, spec)
    mx, _ = plane_rel(got, ref)
    assert mx <= REL_TOL
    if prec == 0:
        plane32 = ref.astype(np.float32)
        ta = thresholds.threshold_array(8, 255, sigma=3.5)
        res = run_harmonic(fd, p, plane32, ta)
        want = harmonic.detect(plane32, ta, 8, 0xFF, 500)
        assert sum(want.counts) > 0
        assert_same_candidates(*res, want, 0xFF)
