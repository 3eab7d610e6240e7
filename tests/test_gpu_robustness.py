"""GPU: how failures and concurrency reach the caller.

* FDAS_ERR_TIMEOUT: the calls that wait on the device (fdas_search_host, fdas_batch_plan_tune, the
  request loop's per-request status) report a bounded wait that gave up. The condition is made on
  the host: the test sets the device status word with fdas_set_device_status, so no kernel waits
  for anything that does not come.
* A batch plan captured into a CUDA graph in one host thread while another thread runs eager
  searches: both get their own results (each thread has its own auxiliary streams, and the capture
  is thread-local). And within one thread: an eager search on one stream while a capture on another
  stream is open does not use the auxiliary streams that joined the capture.
* The FP32 peak diagnostic returns a plausible rate.
"""
import threading

import numpy as np
import pytest
import torch

import synth
from oracle import thresholds

pytestmark = pytest.mark.gpu


def _same_results(got, want):
    gc, gn, gp = got
    wc, wn, wp = want
    assert np.array_equal(gn, wn)
    for a, b in zip(gc, wc):
        assert a.tobytes() == b.tobytes()
    assert gp.tobytes() == wp.tobytes()


def test_search_host_reports_a_timeout_from_the_device_status(fd, small_case):
    wl, _ = small_case
    p = fd.Params()
    s = fd.Searcher(p, wl.n)
    h = torch.from_numpy(wl.spectrum).pin_memory()
    s.search_host(h, wl.n)  # clean status: FDAS_OK
    assert fd.fdas_device_status() == 0
    fd.fdas_set_device_status(fd._lib.FDAS_DEV_WAIT_TIMEOUT)
    try:
        with pytest.raises(fd.FdasError) as err:
            s.search_host(h, wl.n)
        assert err.value.status == fd._lib.FDAS_ERR_TIMEOUT
        assert fd.fdas_device_status() == fd._lib.FDAS_DEV_WAIT_TIMEOUT  # left as it was
    finally:
        fd.fdas_device_status(clear=True)
    assert fd.fdas_device_status() == 0
    s.search_host(h, wl.n)  # OK again once the word is cleared


def test_server_and_plan_tune_report_a_timeout(fd):
    p = fd.Params()
    rng = np.random.default_rng(21)
    x = torch.from_numpy(synth.complex_noise(rng, 20000).astype(np.complex64)).pin_memory()
    server = fd.Server(p, device_bytes=2 * fd.Server.request_bytes(p, 20000) + (1 << 20), max_inflight=2)
    batch = fd.Batch(p, [5000, 3000])
    plan = batch.plan()
    try:
        server.submit(x, 1)
        got = []
        while not got:
            got = server.poll(4, wait_ms=200)
        assert got[0]["status"] == 0
        fd.fdas_set_device_status(fd._lib.FDAS_DEV_WAIT_TIMEOUT)
        server.submit(x, 2)
        got = []
        while not got:
            got = server.poll(4, wait_ms=200)
        assert got[0]["id"] == 2 and got[0]["status"] == fd._lib.FDAS_ERR_TIMEOUT
        with pytest.raises(fd.FdasError) as err:
            plan.tune()
        assert err.value.status == fd._lib.FDAS_ERR_TIMEOUT
        fd.fdas_device_status(clear=True)
        (ctas, tpi), ms = plan.tune()
        assert ms > 0
        server.submit(x, 3)
        got = []
        while not got:
            got = server.poll(4, wait_ms=200)
        assert got[0]["id"] == 3 and got[0]["status"] == 0
    finally:
        fd.fdas_device_status(clear=True)
        plan.close()
        server.close()


def test_plan_capture_in_one_thread_while_another_searches(fd, small_case):
    """Thread A captures batch plans into CUDA graphs (a fresh plan, so a fresh capture, each time)
    and replays them; thread B runs eager fdas_search calls on its own stream meanwhile. Both keep
    getting exactly the results each gets alone."""
    wl, _ = small_case
    p = fd.Params()
    ta = thresholds.threshold_array(p.n_harm, p.n_temp, sigma=3.5)
    d_spec = torch.from_numpy(wl.spectrum).cuda()
    ref = fd.Searcher(p, wl.n, thresh=ta)
    ref.search(d_spec, wl.n)
    torch.cuda.synchronize()
    want_search = ref.results()
    lengths = [30000, 4097, 70001]
    batch = fd.Batch(p, lengths, thresh=ta)
    rng = np.random.default_rng(41)
    for b, n in enumerate(lengths):
        batch.specs[b].copy_(torch.from_numpy(synth.complex_noise(rng, n).astype(np.complex64)))
    batch.search()
    torch.cuda.synchronize()
    want_batch = [batch.results(b) for b in range(len(lengths))]
    errors = []
    go = threading.Event()
    stop = threading.Event()

    def searcher():
        try:
            torch.cuda.set_device(0)
            s = fd.Searcher(p, wl.n, thresh=ta)
            st = torch.cuda.Stream()
            go.wait()
            rounds = 0
            while not stop.is_set() or rounds < 3:
                for t in (s.cands, s.counts, s.peaks):
                    t.zero_()
                s.search(d_spec, wl.n, stream=st)
                st.synchronize()
                _same_results(s.results(), want_search)
                rounds += 1
        except Exception as exc:
            errors.append(exc)

    def capturer():
        try:
            torch.cuda.set_device(0)
            st = torch.cuda.Stream()
            go.wait()
            for _ in range(4):
                plan = batch.plan()
                for t in batch.cands + batch.counts + batch.peaks:
                    t.zero_()
                torch.cuda.synchronize()
                plan.launch(st)  # captures on the plan's private stream, then replays on st
                plan.launch(st)
                st.synchronize()
                for b in range(len(lengths)):
                    _same_results(batch.results(b), want_batch[b])
                plan.close()
        except Exception as exc:
            errors.append(exc)
        finally:
            stop.set()

    threads = [threading.Thread(target=searcher), threading.Thread(target=capturer)]
    for t in threads:
        t.start()
    go.set()
    for t in threads:
        t.join(timeout=300)
    assert not any(t.is_alive() for t in threads)
    assert not errors, errors
    assert fd.fdas_device_status() == 0


def test_fp32_peak_diagnostic(fd):
    """FFMA chains on every SM: the rate lies below the nominal 152 SMs x 128 lanes x 2 flop x 2.07 GHz
    (80.5 TFLOP/s, with a little headroom for a higher clock) and well above a third of it."""
    tflops, ms = fd.fdas_measure_fp32_peak(50.0)
    assert 10.0 < ms < 1000.0
    assert 25.0 < tflops < 90.0, tflops


def test_eager_search_beside_a_capture_in_the_same_thread(fd, small_case):
    """One thread captures fdas_search on stream X and, while that capture is open, runs an eager
    fdas_search on stream Y. The thread's auxiliary streams join X's capture, so the eager call must
    take another pair: the eager results are right at once, and the graph replays to the same results."""
    wl, _ = small_case
    p = fd.Params()
    ta = thresholds.threshold_array(p.n_harm, p.n_temp, sigma=3.0)
    d_spec = torch.from_numpy(wl.spectrum).cuda()
    ref = fd.Searcher(p, wl.n, thresh=ta)
    ref.search(d_spec, wl.n)
    torch.cuda.synchronize()
    want = ref.results()
    cap_s, eager_s = fd.Searcher(p, wl.n, thresh=ta), fd.Searcher(p, wl.n, thresh=ta)
    x, y = torch.cuda.Stream(), torch.cuda.Stream()
    cap_s.search(d_spec, wl.n, stream=x)  # eager warm-up on x
    torch.cuda.synchronize()
    for t in (cap_s.cands, cap_s.counts, cap_s.peaks):
        t.zero_()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=x, capture_error_mode="thread_local"):
        cap_s.search(d_spec, wl.n)  # captured on x
        eager_s.search(d_spec, wl.n, stream=y)  # eager on y, while x's capture is open
    y.synchronize()
    _same_results(eager_s.results(), want)
    g.replay()
    torch.cuda.synchronize()
    _same_results(cap_s.results(), want)
    assert fd.fdas_device_status() == 0
