"""GPU: the serving form. Requests of mixed sizes are submitted in a burst to a server whose device
arena holds only about two of them at a time. They must all complete, their work must overlap on the
GPU, and each result must equal fdas_search on that spectrum alone, bit for bit."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

SIZES = [1 << 16, 3000, 1 << 17, 50000, 1 << 16, 777, 1 << 17, 20011]


def _spectra(seed):
    rng = np.random.default_rng(seed)
    out = []
    for n in SIZES:
        x = synth.complex_noise(rng, n)
        if n > 10000:
            x = x + synth.tone_spectrum(n, [synth.Tone(n // 5, int(rng.integers(-6, 7)), 15.0, 8)])
        out.append(torch.from_numpy(x.astype(np.complex64)).pin_memory())
    return out


def _alone(fd, p, spec):
    s = fd.Searcher(p, spec.numel())
    s.search(spec.cuda(), spec.numel())
    torch.cuda.synchronize()
    return s.results()


def _drain(server, count):
    done = []
    while len(done) < count:
        done += server.poll(64, wait_ms=200)
    return done


@pytest.mark.parametrize("kw", [dict(), dict(n_harm=16, harm_mask=0xFFFF, cand_cap=64), dict(precision=1),
                                dict(precision=2, n_harm=16, harm_mask=0xFFFF, cand_cap=64)])
def test_server_results_equal_standalone_search(fd, kw):
    p = fd.Params(**kw)
    specs = _spectra(11)
    big = fd.Server.request_bytes(p, max(SIZES))
    server = fd.Server(p, device_bytes=2 * big + (1 << 20), max_inflight=3)
    for k, x in enumerate(specs):
        server.submit(x, k)
    done = sorted(_drain(server, len(specs)), key=lambda r: r["id"])
    server.close()
    assert [r["id"] for r in done] == list(range(len(specs)))
    for r, x in zip(done, specs):
        assert r["status"] == 0 and r["n"] == x.numel()
        cands, counts, peaks = _alone(fd, p, x)
        assert np.array_equal(r["counts"], counts)
        for a, b in zip(r["cands"], cands):
            assert a.tobytes() == b.tobytes()
        assert r["peaks"].tobytes() == peaks.tobytes()
        assert r["submit_s"] <= r["admit_s"] <= r["done_s"]
    # continuous batching: some request was admitted while another was still in flight
    spans = [(r["admit_s"], r["done_s"]) for r in done]
    assert any(a2 < d1 and a1 < d2 for i, (a1, d1) in enumerate(spans) for (a2, d2) in spans[i + 1:])


def test_server_rejects_requests_that_never_fit(fd):
    p = fd.Params()
    server = fd.Server(p, device_bytes=fd.Server.request_bytes(p, 4096) + 4096, max_inflight=1)
    with pytest.raises(fd.FdasError) as err:
        server.submit(np.zeros(1 << 16, dtype=np.complex64), 1)
    assert err.value.status == -3
    x = _spectra(12)[5]  # 777 bins: fits
    server.submit(x, 2)
    (r,) = _drain(server, 1)
    server.close()
    cands, counts, _ = _alone(fd, p, x)
    assert r["id"] == 2 and np.array_equal(r["counts"], counts)
