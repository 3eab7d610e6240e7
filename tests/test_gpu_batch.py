"""GPU: the batched form (fdas_search_batch, fdas_harmonic_sum_batch, the graph-replayed plan, the
autotuner).

Against the FP64 oracle (the paper's Sec. 3.5, many input arrays through one device):
* every spectrum's plane of an uneven batch, elementwise, at the 1e-4 floored bar;
* its candidates from the batched search within the plane tolerance of Algorithm 1 on the oracle plane;
* the batched harmonic-sum kernels fed the oracle's float32 planes: candidates, counts and peaks bit
  for bit.
Against fdas_search on each spectrum alone: every output identical (same arithmetic).
"""
import numpy as np
import pytest
import torch

import synth
from oracle import correlate, harmonic, thresholds
from parity_helpers import REL_TOL, assert_candidates_within_tolerance, assert_same_candidates, plane_rel

pytestmark = pytest.mark.gpu

LENGTHS = [1, 3000, 20011, 65536, 100003, 1629]


def _fill(batch, seed=5):
    rng = np.random.default_rng(seed)
    for b, n in enumerate(batch.lengths):
        x = synth.complex_noise(rng, n)
        if n > 5000:
            x = x + synth.tone_spectrum(n, [synth.Tone(n // 7, int(rng.integers(-5, 6)), 15.0, 8)])
        batch.specs[b].copy_(torch.from_numpy(x.astype(np.complex64)))


def _single(fd, batch, b):
    s = fd.Searcher(batch.p, batch.lengths[b], thresh=batch.thresh.cpu().numpy())
    s.search(batch.specs[b], batch.lengths[b])
    torch.cuda.synchronize()
    return s


def _same(fd, batch, b, s):
    n = batch.lengths[b]
    assert torch.equal(batch.planes[b][:, :n], s.plane[:, :n])
    assert torch.equal(batch.counts[b], s.counts)
    got, want = batch.results(b), s.results()
    for x, y in zip(got[0], want[0]):
        assert x.tobytes() == y.tobytes()
    assert got[2].tobytes() == want[2].tobytes()


@pytest.mark.parametrize("shape", [(0, 0), (2, 17), (3, 43)])
def test_batch_equals_single_spectrum_search(fd, shape):
    p = fd.Params(harm_mask=0b10001011)
    batch = fd.Batch(p, LENGTHS, thresh=thresholds.threshold_array(8, 85, sigma=3.5))
    _fill(batch)
    batch.search(*shape)
    torch.cuda.synchronize()
    for b in range(len(LENGTHS)):
        _same(fd, batch, b, _single(fd, batch, b))


def test_batch_sixteen_planes(fd):
    p = fd.Params(n_harm=16, harm_mask=0xFFFF, cand_cap=40)
    batch = fd.Batch(p, [40000, 7000], thresh=thresholds.threshold_array(16, 85, sigma=3.0))
    _fill(batch, seed=6)
    batch.search()
    torch.cuda.synchronize()
    for b in range(2):
        _same(fd, batch, b, _single(fd, batch, b))


def _written(batch, b):
    """What the search writes for spectrum b: decoded candidates (up to the counts), counts, peaks, plane columns < n."""
    cands, counts, peaks = batch.results(b)
    n = batch.lengths[b]
    return [c.tobytes() for c in cands], counts.tobytes(), peaks.tobytes(), batch.planes[b][:, :n].clone()


def _same_written(a, b):
    return a[0] == b[0] and a[1] == b[1] and a[2] == b[2] and torch.equal(a[3], b[3])


def test_plan_graph_replay_and_tuning_keep_results(fd):
    p = fd.Params()
    batch = fd.Batch(p, LENGTHS, thresh=thresholds.threshold_array(8, 85, sigma=3.5))
    _fill(batch, seed=7)
    batch.search()
    torch.cuda.synchronize()
    ref = [_written(batch, b) for b in range(len(LENGTHS))]
    plan = batch.plan()
    for _ in range(2):  # first launch captures the graph, the second replays it
        for t in batch.cands + batch.planes + batch.counts + batch.peaks:
            t.zero_()
        plan.launch()
        torch.cuda.synchronize()
        for b in range(len(LENGTHS)):
            assert _same_written(ref[b], _written(batch, b)), b
    (ctas, tpi), ms = plan.tune()
    assert ctas in (0, 2) and tpi in (0, 43, 29, 17) and ms > 0
    for t in batch.cands + batch.planes:
        t.zero_()
    plan.launch()
    torch.cuda.synchronize()
    for b in range(len(LENGTHS)):
        assert _same_written(ref[b], _written(batch, b)), b
    plan.close()


@pytest.mark.parametrize("lengths", [[70001], [5000, 1, 90000, 300, 40000]])
def test_batch_groupings_equal_single_spectrum_search(fd, lengths):
    """A batch of one spectrum, and five of very uneven lengths (down to a single bin), give the same
    results as fdas_search on each spectrum alone."""
    p = fd.Params()
    batch = fd.Batch(p, lengths, thresh=thresholds.threshold_array(8, 85, sigma=3.5))
    _fill(batch, seed=8)
    batch.search()
    torch.cuda.synchronize()
    for b in range(len(lengths)):
        _same(fd, batch, b, _single(fd, batch, b))


def test_batch_of_the_maximum_count(fd):
    """FDAS_MAX_BATCH = 256 spectra of 1 to 5000 bins in one call (the job tables are kernel
    parameters at their largest) and through the graph plan: a sample of spectra against
    fdas_search alone."""
    rng = np.random.default_rng(256)
    lengths = [int(v) for v in rng.integers(1, 5001, 256)]
    lengths[0], lengths[255] = 1, 5000
    p = fd.Params(harm_mask=0b10001011)
    batch = fd.Batch(p, lengths, thresh=thresholds.threshold_array(8, 85, sigma=3.0))
    _fill(batch, seed=9)
    batch.search()
    torch.cuda.synchronize()
    sample = [0, 1, 77, 128, 200, 255]
    for b in sample:
        _same(fd, batch, b, _single(fd, batch, b))
    ref = [_written(batch, b) for b in sample]
    plan = batch.plan()
    for t in batch.cands + batch.planes + batch.counts + batch.peaks:
        t.zero_()
    plan.launch()
    torch.cuda.synchronize()
    for b, r in zip(sample, ref):
        assert _same_written(r, _written(batch, b)), b
    plan.close()


# Lengths on both sides of segment boundaries (L = 1628 kept outputs per segment), a single bin, and
# one spectrum near 2^18 bins.
ORACLE_LENGTHS = [1, 1628, 1629, 3256, 3257, 20011, 262139]


@pytest.fixture(scope="module")
def oracle_batch(bank):
    rng = np.random.default_rng(13)
    specs, planes = [], []
    for n in ORACLE_LENGTHS:
        x = synth.complex_noise(rng, n)
        if n > 5000:
            x = x + synth.tone_spectrum(n, [synth.Tone(n // 7, int(rng.integers(-5, 6)), 15.0, 8)])
        x = x.astype(np.complex64)
        specs.append(x)
        planes.append(correlate.plane_ols(x, bank, 2048))
    return specs, planes


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_batch_against_the_oracle(fd, oracle_batch, precision):
    """fdas_search_batch on an uneven batch: each plane against the oracle, and each spectrum's
    candidates (8 planes, 6 sigma) against Algorithm 1 on the oracle plane, within tolerance."""
    specs, planes = oracle_batch
    p = fd.Params(precision=precision, cand_cap=4096)
    ta = thresholds.threshold_array(8, 85, sigma=6.0)
    batch = fd.Batch(p, ORACLE_LENGTHS, thresh=ta)
    for b, x in enumerate(specs):
        batch.specs[b].copy_(torch.from_numpy(x))
    batch.search()
    torch.cuda.synchronize()
    checked = 0
    for b, n in enumerate(ORACLE_LENGTHS):
        mx, rms = plane_rel(batch.planes[b][:, :n].cpu().numpy(), planes[b])
        print(f"precision {precision} n={n}: plane rel max {mx:.2e} rms {rms:.2e}")
        assert mx <= REL_TOL
        cands, counts, _ = batch.results(b)
        checked += assert_candidates_within_tolerance(cands, counts, planes[b], ta, 8, p.harm_mask, p.cand_cap)
    assert checked > 50
    assert fd.fdas_device_status() == 0


@pytest.mark.parametrize(
    "kw,sigma",
    [(dict(), 6.0), (dict(harm_mask=0b10001011, cand_cap=300), 4.0), (dict(n_harm=16, harm_mask=0xFFFF, cand_cap=64), 3.5)],
)
def test_batched_harmonic_sum_on_oracle_planes_is_bit_exact(fd, oracle_batch, kw, sigma):
    """fdas_harmonic_sum_batch (the batched kernels: job lookup by binary search, per-spectrum CTA
    tables, the single-plane launch, per-(plane, spectrum) finalize) fed the oracle's float32 planes
    returns Algorithm 1's candidates, counts and peaks bit for bit, for every spectrum."""
    _, planes = oracle_batch
    p = fd.Params(**kw)
    ta = thresholds.threshold_array(p.n_harm, 85, sigma=sigma)
    batch = fd.Batch(p, ORACLE_LENGTHS, thresh=ta)
    for b, n in enumerate(ORACLE_LENGTHS):
        batch.planes[b].fill_(1e30)  # the columns past n must never be read
        batch.planes[b][:, :n] = torch.from_numpy(planes[b].astype(np.float32)).cuda()
    batch.harmonic_sum()
    torch.cuda.synchronize()
    for b in range(len(ORACLE_LENGTHS)):
        ref = harmonic.detect(planes[b].astype(np.float32), ta, p.n_harm, p.harm_mask, p.cand_cap)
        cands, counts, peaks = batch.results(b)
        assert_same_candidates(cands, counts, peaks, ref, p.harm_mask)
