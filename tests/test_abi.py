"""The C ABI library loads, exports every symbol include/fdas.h declares, and checks its
arguments on the host (CPU only: no call here reaches a kernel)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fdas.h")


@pytest.fixture(scope="module")
def fd():
    from paper_1806_01556_gb300 import build

    build.build()
    import paper_1806_01556_gb300 as fdas

    fdas.lib()
    return fdas


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fdas_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported_and_bound(fd):
    from paper_1806_01556_gb300 import _lib

    names = declared_functions()
    assert len(names) >= 12
    lib = fd.lib()
    for name in names:
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"{name} has no ctypes signature"
    assert set(_lib.SIGNATURES) == set(names)


def test_struct_layouts_match_header(fd):
    from paper_1806_01556_gb300 import _lib

    assert C.sizeof(_lib.fdas_params) == 40
    assert C.sizeof(_lib.fdas_cand) == 12
    assert fd.CAND_DTYPE.itemsize == 12


def test_defaults_and_sizes(fd):
    from paper_1806_01556_gb300 import _lib

    p = _lib.fdas_params()
    fd.lib().fdas_default_params(C.byref(p))
    assert (p.n_temp, p.z_min, p.z_step, p.n_tap, p.fft_len, p.n_harm, p.harm_mask, p.cand_cap) == (
        85, -42, 1, 421, 2048, 8, 0xFF, 200)
    q = fd.Params()
    assert fd.fdas_check_params(q) == 0
    assert fd.fdas_templates_bytes(q) == 86 * 2048 * 8
    assert fd.fdas_plane_bytes(q, 1 << 21, 1 << 21) == 85 * (1 << 21) * 4
    assert fd.fdas_workspace_bytes(q, 1 << 21) == 8 * 8 * (16384 + 4)


@pytest.mark.parametrize(
    "change,code",
    [
        (dict(n_temp=84), -1),
        (dict(n_temp=1, z_min=0), -1),
        (dict(z_min=-41), -1),
        (dict(n_tap=420), -1),
        (dict(n_tap=1025), -1),
        (dict(fft_len=3000), -1),
        (dict(n_harm=17), -1),
        (dict(harm_mask=0), -1),
        (dict(harm_mask=0x100), -1),
        (dict(cand_cap=0), -1),
        (dict(cand_cap=5000), -1),
        (dict(precision=7), -1),
        (dict(fft_len=4096), -2),
        (dict(precision=1, fft_len=4096), -2),
        (dict(precision=1), 0),
        (dict(precision=2), 0),
        (dict(harm_index=1), 0),
        (dict(harm_index=2), -1),
        (dict(n_temp=9, z_min=-8, z_step=2), 0),
        (dict(n_harm=16, harm_mask=0xFFFF), 0),
    ],
)
def test_param_validation(fd, change, code):
    p = fd.Params(**change)
    assert fd.fdas_check_params(p) == code


def test_thresholds_match_oracle(fd):
    from oracle import thresholds

    for kind, name in ((0, "gamma"), (1, "meansd")):
        for sigma in (6.0, 3.0):
            p = fd.Params(n_harm=16, harm_mask=0xFFFF)
            got = fd.fdas_default_thresholds(p, sigma, kind)
            want = thresholds.threshold_array(16, 85, sigma=sigma, kind=name)
            assert np.all(np.abs(got.view(np.int32) - want.view(np.int32)) <= 1)


def test_bad_pointers_are_rejected_before_any_launch(fd):
    lib = fd.lib()
    p = fd.Params().c()
    null = C.c_void_p(0)
    fake = C.c_void_p(0x10000)  # never dereferenced: argument checks fail first
    odd = C.c_void_p(0x10004)
    assert lib.fdas_make_templates(C.byref(p), null, null) == -1
    assert lib.fdas_make_templates(C.byref(p), odd, null) == -1
    assert lib.fdas_convolve(C.byref(p), null, 100, fake, fake, 100, null) == -1
    assert lib.fdas_convolve(C.byref(p), fake, 0, fake, fake, 100, null) == -1
    assert lib.fdas_convolve(C.byref(p), fake, 100, fake, fake, 99, null) == -1
    assert lib.fdas_convolve(C.byref(p), fake, (1 << 24) + 1, fake, fake, 1 << 25, null) == -1
    assert lib.fdas_convolve(C.byref(p), odd, 100, fake, fake, 100, null) == -1
    ws = fd.fdas_workspace_bytes(fd.Params(), 100)
    assert lib.fdas_harmonic_sum(C.byref(p), fake, 100, 100, fake, fake, fake, null, fake, ws - 8, null) == -3
    assert lib.fdas_harmonic_sum(C.byref(p), fake, 100, 100, null, fake, fake, null, fake, ws, null) == -1
    assert lib.fdas_search(C.byref(p), fake, 100, fake, fake, 100, fake, fake, fake, null, fake, 16, null) == -3
    bad = fd.Params(fft_len=4096).c()
    assert lib.fdas_search(C.byref(bad), fake, 100, fake, fake, 100, fake, fake, fake, null, fake, ws, null) == -2
    assert lib.fdas_search_host(C.byref(p), null, 100, fake, fake, fake, 100, fake, fake, fake, null, fake, fake,
                                null, fake, ws, null) == -1
    assert lib.fdas_search_host_async(C.byref(p), null, 100, fake, fake, fake, 100, fake, fake, fake, null, fake,
                                      fake, null, fake, ws, null) == -1
    assert lib.fdas_search_host_async(C.byref(p), fake, 100, odd, fake, fake, 100, fake, fake, fake, null, fake,
                                      fake, null, fake, ws, null) == -1
    assert lib.fdas_default_thresholds(C.byref(p), 6.0, 2, fake) == -1
    assert lib.fdas_status_string(-3) == b"workspace too small"
    assert lib.fdas_device_status(None, 0) == -1
    assert lib.fdas_check_wait_timeout(None) == -1
    tf, el = C.c_double(), C.c_float()
    assert lib.fdas_measure_fp32_peak(50.0, None, C.byref(el)) == -1
    assert lib.fdas_measure_fp32_peak(5.0, C.byref(tf), C.byref(el)) == -1
    assert lib.fdas_measure_fp32_peak(5000.0, C.byref(tf), C.byref(el)) == -1


def test_timeout_status_code(fd):
    """FDAS_ERR_TIMEOUT (-5) is declared in the header, bound, and has its own message."""
    from paper_1806_01556_gb300 import _lib

    text = open(HEADER).read()
    assert re.search(r"#define FDAS_ERR_TIMEOUT \(-5\)", text)
    assert _lib.FDAS_ERR_TIMEOUT == -5
    assert fd.lib().fdas_status_string(-5) == b"a kernel gave up on a bounded device wait"
    assert fd.lib().fdas_status_string(-6) == b"unknown status"
    assert fd.lib().fdas_last_error() == b""  # no CUDA call has failed on this thread


class _NullStream:
    cuda_stream = 0


def test_python_wrappers_marshal_and_raise_on_rejected_arguments(fd):
    """Every binding wrapper reaches its C entry point; n = 0 is rejected before any CUDA call."""
    import numpy as np

    p = fd.Params()
    buf = np.zeros(64, dtype=np.float32)
    st = _NullStream()
    calls = [
        lambda: fd.fdas_convolve(p, buf, 0, buf, buf, 0, st),
        lambda: fd.fdas_search_convolve(p, buf, 0, buf, buf, 0, buf, buf, 1 << 20, st),
        lambda: fd.fdas_search_harmonic(p, buf, 0, 0, buf, buf, buf, buf, buf, 1 << 20, st),
        lambda: fd.fdas_convolve_cfg(p, buf, 0, buf, buf, 0, 2, 17, st),
        lambda: fd.fdas_harmonic_sum(p, buf, 0, 0, buf, buf, buf, None, buf, 1 << 30, st),
        lambda: fd.fdas_search(p, buf, 0, buf, buf, 0, buf, buf, buf, None, buf, 1 << 30, st),
        lambda: fd.fdas_search_host(p, buf, 0, buf, buf, buf, 0, buf, buf, buf, None, buf, buf, None, buf, 1 << 30, st),
        lambda: fd.fdas_harmonic_sum_noalloc(p, buf, 0, 0, buf, buf, buf, None, st),
        lambda: fd.fdas_make_templates(fd.Params(n_temp=4), buf, st),
    ]
    for call in calls:
        with pytest.raises(fd.FdasError) as err:
            call()
        assert err.value.status == -1
    bad = fd.Params(n_temp=84)
    assert fd.fdas_templates_bytes(bad) == 0 and fd.fdas_workspace_bytes(bad, 10) == 0


def test_batch_arguments_are_checked_on_the_host(fd):
    from paper_1806_01556_gb300 import _lib

    lib = fd.lib()
    p = fd.Params().c()
    assert fd.fdas_batch_workspace_bytes(fd.Params(), 4) == 4 * ((8 * 8 * (16384 + 4) + 255) // 256 * 256)
    assert fd.fdas_batch_workspace_bytes(fd.Params(), 0) == 0
    assert fd.fdas_batch_workspace_bytes(fd.Params(), 257) == 0
    fake = 0x10000
    good = _lib.fdas_batch_item(fake, 100, fake, 128, fake, fake, 0)
    items = (_lib.fdas_batch_item * 2)(good, good)
    ws = fd.fdas_batch_workspace_bytes(fd.Params(), 2)
    vp = C.c_void_p
    args = (vp(fake), vp(fake), vp(fake))
    assert lib.fdas_search_batch(C.byref(p), C.cast(items, vp), 0, *args, ws, None, None) == -1
    assert lib.fdas_search_batch(C.byref(p), C.cast(items, vp), 2, *args, ws - 1, None, None) == -3
    items[1].n = 0
    assert lib.fdas_search_batch(C.byref(p), C.cast(items, vp), 2, *args, ws, None, None) == -1
    items[1].n, items[1].ld = 100, 99
    assert lib.fdas_search_batch(C.byref(p), C.cast(items, vp), 2, *args, ws, None, None) == -1
    items[1].ld, items[1].d_plane = 128, fake + 4
    assert lib.fdas_search_batch(C.byref(p), C.cast(items, vp), 2, *args, ws, None, None) == -1
    h = C.c_void_p()
    assert lib.fdas_batch_plan_create(C.byref(p), C.cast(items, vp), 2, *args, ws, C.byref(h)) == -1
    assert not h.value
    assert lib.fdas_batch_plan_launch(None, None) == -1
    lib.fdas_batch_plan_destroy(None)
    items[1].d_plane = fake
    hh = fd.Params(harm_index=1).c()  # the batched launches index by fundamental only
    assert lib.fdas_search_batch(C.byref(hh), C.cast(items, vp), 2, *args, ws, None, None) == -2
    # The batched harmonic sum reads planes only: a NULL spectrum is fine, everything else is checked.
    items[0].d_spec = items[1].d_spec = 0
    hs = (vp(fake), vp(fake))  # d_thresh, d_ws
    assert lib.fdas_harmonic_sum_batch(C.byref(hh), C.cast(items, vp), 2, *hs, ws, None) == -2
    assert lib.fdas_harmonic_sum_batch(C.byref(p), C.cast(items, vp), 0, *hs, ws, None) == -1
    assert lib.fdas_harmonic_sum_batch(C.byref(p), C.cast(items, vp), 2, *hs, ws - 1, None) == -3
    assert lib.fdas_harmonic_sum_batch(C.byref(p), C.cast(items, vp), 2, vp(0), vp(fake), ws, None) == -1
    items[1].d_plane = fake + 4
    assert lib.fdas_harmonic_sum_batch(C.byref(p), C.cast(items, vp), 2, *hs, ws, None) == -1
    items[1].d_plane = fake
    items[1].d_counts = 0
    assert lib.fdas_harmonic_sum_batch(C.byref(p), C.cast(items, vp), 2, *hs, ws, None) == -1


def test_server_arguments_are_checked_on_the_host(fd):
    lib = fd.lib()
    p = fd.Params().c()
    h = C.c_void_p()
    assert lib.fdas_server_create(C.byref(p), 1 << 30, 0, C.byref(h)) == -1
    assert lib.fdas_server_create(C.byref(p), 1 << 30, 17, C.byref(h)) == -1
    assert lib.fdas_server_create(C.byref(p), 1000, 3, C.byref(h)) == -1
    assert lib.fdas_server_create(C.byref(p), 1 << 30, 3, None) == -1
    assert lib.fdas_server_create(C.byref(fd.Params(n_temp=4).c()), 1 << 30, 3, C.byref(h)) == -1
    assert not h.value
    assert lib.fdas_server_submit(None, C.c_void_p(0x10000), 100, 1, None) == -1
    n_out = C.c_int()
    assert lib.fdas_server_poll(None, C.c_void_p(0x10000), 1, C.byref(n_out), 0) == -1
    lib.fdas_server_destroy(None)
    lib.fdas_server_stats(None, None, None)
    # footprint: spectrum + plane (ld rounded to 64) + workspace + results, each rounded to 256 bytes
    q = fd.Params()
    n = 100000
    up = lambda x: (x + 255) // 256 * 256
    want = up(8 * n) + up(85 * ((n + 63) // 64 * 64) * 4) + up(fd.fdas_workspace_bytes(q, n)) + up(8 * 200 * 12) \
        + up(8 * 4) + up(8 * 12)
    assert fd.Server.request_bytes(q, n) == want


def test_bench_launch_count_follows_the_row_groups():
    """bench.py counts the harmonic-sum launches: reset, one per non-empty row group, single-plane rows, finalize."""
    import bench

    assert bench.hs_launches(8, 85) == 6
    assert bench.hs_launches(16, 85) == 6
    assert bench.hs_launches(2, 85) == 4
    assert bench.hs_launches(1, 85) == 3


def test_clock_sampler_keeps_the_timed_window():
    """bench.py's clock summary uses the nvidia-smi samples taken inside the timed region."""
    import datetime

    import bench

    cs = bench.ClockSampler(0)
    t0 = datetime.datetime(2026, 1, 1, 12, 0, 0).timestamp()

    def line(dt, mhz, power_cap="Not Active"):
        ts = datetime.datetime.fromtimestamp(t0 + dt).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return f"{ts}, 0, {mhz}, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, {power_cap}"

    cs.lines = [line(0.0, 1000), line(1.0, 2070), line(1.02, 2070, "Active"), line(1.04, 2070), line(3.0, 1200)]
    cs.t_begin, cs.t_end = t0 + 0.9, t0 + 1.5
    s = cs.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2070.0 and s["reasons"] == ["sw_power_cap"]
    assert s["window"] == "timed region"
    cs.t_begin, cs.t_end = t0 + 5.0, t0 + 5.01  # nothing inside: the whole run is reported
    assert cs.summary()["window"] == "whole run"


def test_bench_path_roofline_is_the_slower_floor():
    """bench.py's whole-path roofline: FFT flops at the FP32 peak against the plane's bytes (written
    once, read once, plus the spectrum segments) at HBM bandwidth; the slower one bounds the step."""
    import bench

    n = 1 << 21
    alg = bench.algorithmic(n)
    r = bench.path_roofline(n, 421, 1.0, 6800.0, "test")
    plane = 85 * n * 4
    assert r["bytes"] == alg["conv_bytes"] + plane == 1289 * 2048 * 8 + 2 * plane
    assert abs(r["ms_bytes"] - r["bytes"] / 6800e9 * 1e3) < 1e-12
    assert abs(r["ms_flop"] - alg["conv_flop"] / (bench.FP32_PEAK_TFLOPS * 1e12) * 1e3) < 1e-12
    assert r["bound"] == "hbm" and r["ms_at_roofline"] == r["ms_bytes"] and r["frac"] == r["ms_bytes"] / 1.0
    fast = bench.path_roofline(n, 421, 1.0, 1e9, "test")  # absurd bandwidth: the flops bound
    assert fast["bound"] == "alu" and fast["ms_at_roofline"] == fast["ms_flop"]


def test_bench_algorithmic_work_at_2_21():
    """bench.py's algorithmic work per 2^21-bin spectrum, against the counts of the method: 1289
    segments of L = 2048 - 420 = 1628 outputs; one forward and 85 inverse 2048-point FFTs per
    segment at 5 F log2 F = 112,640 flop each; 85 complex products of 2048 points per segment at 6
    flop; |y|^2 at 3 flop per plane point; 2048 complex64 read per segment and the 713 MB plane
    written. The FP32 search's harmonic stage reads the 43 rows with |i| <= 21 again, the split forms
    all 85."""
    import bench

    n = 1 << 21
    alg = bench.algorithmic(n)
    assert alg["n_seg"] == 1289 and (1289 - 1) * 1628 < n <= 1289 * 1628
    fft = 112_640
    want = 1289 * fft + 85 * 1289 * fft + 85 * 1289 * 2048 * 6 + 85 * n * 3
    assert alg["conv_flop"] == want and abs(want - 1.4368e10) < 1e7
    assert alg["conv_bytes"] == 1289 * 2048 * 8 + 85 * n * 4
    assert alg["hs_bytes"] == 85 * n * 4 == 713_031_680
    assert bench.hs_rows("fp32") == 43 and bench.hs_rows("bf16x3") == 85 and bench.hs_rows("fp16s") == 85
    assert bench.algorithmic(n, rows_read=43)["hs_bytes"] == 43 * n * 4


def test_bench_oracle_pool_equals_the_oracle():
    """The CPU baseline's split of the oracle plane over worker processes (column blocks computed from
    bins widened by the half width) equals the oracle's plane_ols on the whole spectrum, and the
    harmonic sum after it equals Algorithm 1 on that plane."""
    import bench
    import synth
    from oracle import correlate, harmonic

    n = 9000
    rng = np.random.default_rng(3)
    x = synth.complex_noise(rng, n) + synth.tone_spectrum(n, [synth.Tone(1500, 4, 15.0, 4)])
    pool = bench.OraclePool(n, workers=3)
    try:
        _, _, res = pool.run(x)
        got = np.ndarray((85, n), dtype=np.float32, buffer=pool._shm[1].buf).copy()
        ref = correlate.plane_ols(x, pool.bank, 2048).astype(np.float32)
        want = harmonic.detect(ref, pool.ta, 8, 0xFF, 200)
    finally:
        pool.close()
    assert np.allclose(got, ref, rtol=2e-7, atol=0)
    assert list(res.counts) == list(want.counts) and res.counts[0] > 0
