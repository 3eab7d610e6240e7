"""GPU: the batched form (fdas_search_batch, the graph-replayed plan, the autotuner) against
fdas_search on each spectrum alone. Same kernels, same arithmetic: every output must be identical."""
import numpy as np
import pytest
import torch

import synth
from oracle import thresholds

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
