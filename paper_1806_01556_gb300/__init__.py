"""Python binding of libfdas, the FDAS hot path on one GB300 (sm_103a).

The functions here have the names of the C entry points in include/fdas.h and only marshal
arguments: torch tensors are passed as device pointers, and the current torch CUDA stream as the
cudaStream_t. Every step of the path runs in the library's CUDA kernels. PyTorch only provides
device memory and streams. If libfdas.so is missing, the first call raises ImportError;
nothing falls back to the CPU.

``Searcher`` bundles the buffers one spectrum length needs (template bank, plane, workspace,
thresholds, candidate outputs) and runs ``fdas_search`` or ``fdas_search_host`` on them.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import asdict, dataclass

import numpy as np

from . import _lib

__all__ = [
    "FdasError",
    "Params",
    "CAND_DTYPE",
    "lib",
    "fdas_check_params",
    "fdas_device_status",
    "fdas_check_wait_timeout",
    "fdas_set_device_status",
    "fdas_measure_fp32_peak",
    "fdas_templates_bytes",
    "fdas_plane_bytes",
    "fdas_workspace_bytes",
    "fdas_default_thresholds",
    "fdas_make_templates",
    "fdas_convolve",
    "fdas_convolve_cfg",
    "fdas_harmonic_sum",
    "fdas_search",
    "fdas_search_host",
    "fdas_search_host_async",
    "fdas_search_convolve",
    "fdas_search_harmonic",
    "fdas_harmonic_sum_noalloc",
    "decode_cands",
    "Searcher",
    "fdas_batch_workspace_bytes",
    "fdas_search_batch",
    "fdas_harmonic_sum_batch",
    "BatchPlan",
    "Batch",
    "Server",
]

# Host view of fdas_cand (12 bytes): power, j, i, k, pad.
CAND_DTYPE = np.dtype([("power", "<f4"), ("j", "<u4"), ("i", "<i2"), ("k", "u1"), ("pad", "u1")])
assert CAND_DTYPE.itemsize == C.sizeof(_lib.fdas_cand)


class FdasError(RuntimeError):
    def __init__(self, status: int, what: str):
        msg = lib().fdas_status_string(status).decode()
        if status == _lib.FDAS_ERR_CUDA:
            detail = lib().fdas_last_error().decode()
            if detail:
                msg += f": {detail}"
        super().__init__(f"{what}: {msg} ({status})")
        self.status = status


def lib() -> C.CDLL:
    return _lib.load()


@dataclass
class Params:
    """Search parameters; the fields of fdas_params (see include/fdas.h)."""

    n_temp: int = 85
    z_min: int = -42
    z_step: int = 1
    n_tap: int = 421
    fft_len: int = 2048
    n_harm: int = 8
    harm_mask: int = 0xFF
    cand_cap: int = 200
    precision: int = _lib.FDAS_FP32
    harm_index: int = _lib.FDAS_INDEX_FUNDAMENTAL

    def c(self) -> _lib.fdas_params:
        return _lib.fdas_params(**asdict(self))


def _ptr(t) -> C.c_void_p:
    if t is None:
        return C.c_void_p(0)
    if isinstance(t, np.ndarray):
        return C.c_void_p(t.ctypes.data)
    return C.c_void_p(t.data_ptr())


def _stream(stream) -> C.c_void_p:
    if stream is None:
        import torch

        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _check(status: int, what: str) -> None:
    if status != _lib.FDAS_OK:
        raise FdasError(status, what)


def fdas_check_params(p: Params) -> int:
    return lib().fdas_check_params(C.byref(p.c()))


def fdas_device_status(clear: bool = False) -> int:
    """Device status bits of the current device (FDAS_DEV_WAIT_TIMEOUT: a bounded wait gave up)."""
    flags = C.c_uint32(0)
    _check(lib().fdas_device_status(C.byref(flags), int(clear)), "fdas_device_status")
    return flags.value


def fdas_set_device_status(flags: int) -> None:
    """Sets the current device's status word (a diagnostic for testing FDAS_ERR_TIMEOUT handling)."""
    _check(lib().fdas_set_device_status(flags), "fdas_set_device_status")


def fdas_measure_fp32_peak(ms: float = 50.0) -> tuple[float, float]:
    """FFMA-chain FP32 throughput of the current device: (TFLOP/s, timed milliseconds)."""
    tf, el = C.c_double(), C.c_float()
    _check(lib().fdas_measure_fp32_peak(ms, C.byref(tf), C.byref(el)), "fdas_measure_fp32_peak")
    return tf.value, el.value


def fdas_check_wait_timeout() -> int:
    """Runs the bounded-wait diagnostic (about one second); returns the status bits it left."""
    flags = C.c_uint32(0)
    _check(lib().fdas_check_wait_timeout(C.byref(flags)), "fdas_check_wait_timeout")
    return flags.value


def fdas_templates_bytes(p: Params) -> int:
    return lib().fdas_templates_bytes(C.byref(p.c()))


def fdas_plane_bytes(p: Params, n: int, ld: int) -> int:
    return lib().fdas_plane_bytes(C.byref(p.c()), n, ld)


def fdas_workspace_bytes(p: Params, n: int) -> int:
    return lib().fdas_workspace_bytes(C.byref(p.c()), n)


def fdas_default_thresholds(p: Params, sigma: float = 6.0, kind: int = 0) -> np.ndarray:
    """TA as float32[n_harm][n_temp], computed by the library on the host."""
    out = np.empty((p.n_harm, p.n_temp), dtype=np.float32)
    _check(lib().fdas_default_thresholds(C.byref(p.c()), sigma, kind, _ptr(out)), "fdas_default_thresholds")
    return out


def fdas_make_templates(p: Params, d_tmpl, stream=None) -> None:
    _check(lib().fdas_make_templates(C.byref(p.c()), _ptr(d_tmpl), _stream(stream)), "fdas_make_templates")


def fdas_convolve(p: Params, d_spec, n: int, d_tmpl, d_plane, ld: int, stream=None) -> None:
    _check(
        lib().fdas_convolve(C.byref(p.c()), _ptr(d_spec), n, _ptr(d_tmpl), _ptr(d_plane), ld, _stream(stream)),
        "fdas_convolve",
    )


def fdas_convolve_cfg(p: Params, d_spec, n: int, d_tmpl, d_plane, ld: int, ctas_per_sm: int = 0,
                      templates_per_item: int = 0, stream=None) -> None:
    cfg = _lib.fdas_launch_config(ctas_per_sm, templates_per_item)
    _check(
        lib().fdas_convolve_cfg(C.byref(p.c()), _ptr(d_spec), n, _ptr(d_tmpl), _ptr(d_plane), ld, C.byref(cfg),
                                _stream(stream)),
        "fdas_convolve_cfg",
    )


def fdas_harmonic_sum(p: Params, d_plane, n, ld, d_thresh, d_cands, d_counts, d_peaks, d_ws, ws_bytes, stream=None):
    _check(
        lib().fdas_harmonic_sum(
            C.byref(p.c()), _ptr(d_plane), n, ld, _ptr(d_thresh), _ptr(d_cands), _ptr(d_counts), _ptr(d_peaks),
            _ptr(d_ws), ws_bytes, _stream(stream),
        ),
        "fdas_harmonic_sum",
    )


def fdas_search(p: Params, d_spec, n, d_tmpl, d_plane, ld, d_thresh, d_cands, d_counts, d_peaks, d_ws, ws_bytes,
                stream=None):
    _check(
        lib().fdas_search(
            C.byref(p.c()), _ptr(d_spec), n, _ptr(d_tmpl), _ptr(d_plane), ld, _ptr(d_thresh), _ptr(d_cands),
            _ptr(d_counts), _ptr(d_peaks), _ptr(d_ws), ws_bytes, _stream(stream),
        ),
        "fdas_search",
    )


def fdas_search_convolve(p: Params, d_spec, n, d_tmpl, d_plane, ld, d_thresh, d_ws, ws_bytes, stream=None):
    """First stage of fdas_search: workspace reset, convolution (and HP_1 detection for FP32)."""
    _check(
        lib().fdas_search_convolve(C.byref(p.c()), _ptr(d_spec), n, _ptr(d_tmpl), _ptr(d_plane), ld, _ptr(d_thresh),
                                   _ptr(d_ws), ws_bytes, _stream(stream)),
        "fdas_search_convolve",
    )


def fdas_search_harmonic(p: Params, d_plane, n, ld, d_thresh, d_cands, d_counts, d_peaks, d_ws, ws_bytes,
                         stream=None):
    """Second stage of fdas_search: the remaining harmonic planes and the candidate lists."""
    _check(
        lib().fdas_search_harmonic(C.byref(p.c()), _ptr(d_plane), n, ld, _ptr(d_thresh), _ptr(d_cands),
                                   _ptr(d_counts), _ptr(d_peaks), _ptr(d_ws), ws_bytes, _stream(stream)),
        "fdas_search_harmonic",
    )


def fdas_search_host(p: Params, h_spec, n, d_spec, d_tmpl, d_plane, ld, d_thresh, d_cands, d_counts, d_peaks,
                     h_cands, h_counts, h_peaks, d_ws, ws_bytes, stream=None):
    _check(
        lib().fdas_search_host(
            C.byref(p.c()), _ptr(h_spec), n, _ptr(d_spec), _ptr(d_tmpl), _ptr(d_plane), ld, _ptr(d_thresh),
            _ptr(d_cands), _ptr(d_counts), _ptr(d_peaks), _ptr(h_cands), _ptr(h_counts), _ptr(h_peaks), _ptr(d_ws),
            ws_bytes, _stream(stream),
        ),
        "fdas_search_host",
    )


def fdas_search_host_async(p: Params, h_spec, n, d_spec, d_tmpl, d_plane, ld, d_thresh, d_cands, d_counts, d_peaks,
                           h_cands, h_counts, h_peaks, d_ws, ws_bytes, stream=None):
    """fdas_search_host without the final wait: the host results are valid once `stream` gets there."""
    _check(
        lib().fdas_search_host_async(
            C.byref(p.c()), _ptr(h_spec), n, _ptr(d_spec), _ptr(d_tmpl), _ptr(d_plane), ld, _ptr(d_thresh),
            _ptr(d_cands), _ptr(d_counts), _ptr(d_peaks), _ptr(h_cands), _ptr(h_counts), _ptr(h_peaks), _ptr(d_ws),
            ws_bytes, _stream(stream),
        ),
        "fdas_search_host_async",
    )


def fdas_harmonic_sum_noalloc(p: Params, d_plane, n, ld, d_thresh, d_cands, d_counts, d_peaks, stream=None):
    """fdas_harmonic_sum with the library's static scratch array instead of a workspace (n_harm <= 8)."""
    _check(
        lib().fdas_harmonic_sum_noalloc(
            C.byref(p.c()), _ptr(d_plane), n, ld, _ptr(d_thresh), _ptr(d_cands), _ptr(d_counts), _ptr(d_peaks),
            _stream(stream),
        ),
        "fdas_harmonic_sum_noalloc",
    )


def fdas_batch_workspace_bytes(p: Params, count: int) -> int:
    return lib().fdas_batch_workspace_bytes(C.byref(p.c()), count)


def _items(entries) -> "C.Array":
    """entries: (d_spec, n, d_plane, ld, d_cands, d_counts, d_peaks) tuples -> fdas_batch_item[count]."""
    arr = (_lib.fdas_batch_item * len(entries))()
    for k, (spec, n, plane, ld, cands, counts, peaks) in enumerate(entries):
        arr[k] = _lib.fdas_batch_item(_ptr(spec).value, n, _ptr(plane).value, ld, _ptr(cands).value,
                                      _ptr(counts).value, _ptr(peaks).value)
    return arr


def fdas_search_batch(p: Params, entries, d_tmpl, d_thresh, d_ws, ws_bytes, ctas_per_sm=0, templates_per_item=0,
                      stream=None) -> None:
    arr = _items(entries)
    cfg = _lib.fdas_launch_config(ctas_per_sm, templates_per_item)
    _check(
        lib().fdas_search_batch(C.byref(p.c()), C.cast(arr, C.c_void_p), len(entries), _ptr(d_tmpl), _ptr(d_thresh),
                                _ptr(d_ws), ws_bytes, C.byref(cfg), _stream(stream)),
        "fdas_search_batch",
    )


def fdas_harmonic_sum_batch(p: Params, entries, d_thresh, d_ws, ws_bytes, stream=None) -> None:
    """Harmonic sum of every entry's plane (the d_spec of an entry may be None)."""
    arr = _items(entries)
    _check(
        lib().fdas_harmonic_sum_batch(C.byref(p.c()), C.cast(arr, C.c_void_p), len(entries), _ptr(d_thresh),
                                      _ptr(d_ws), ws_bytes, _stream(stream)),
        "fdas_harmonic_sum_batch",
    )


class BatchPlan:
    """fdas_batch_plan: a batch with fixed buffers, replayed as a CUDA graph; tune() picks the launch shape."""

    def __init__(self, p: Params, entries, d_tmpl, d_thresh, d_ws, ws_bytes):
        arr = _items(entries)
        self._h = C.c_void_p()
        self._keep = (entries, d_tmpl, d_thresh, d_ws)
        _check(
            lib().fdas_batch_plan_create(C.byref(p.c()), C.cast(arr, C.c_void_p), len(entries), _ptr(d_tmpl),
                                         _ptr(d_thresh), _ptr(d_ws), ws_bytes, C.byref(self._h)),
            "fdas_batch_plan_create",
        )

    def tune(self, stream=None):
        cfg = _lib.fdas_launch_config()
        ms = C.c_float()
        _check(lib().fdas_batch_plan_tune(self._h, _stream(stream), C.byref(cfg), C.byref(ms)), "fdas_batch_plan_tune")
        return (cfg.ctas_per_sm, cfg.templates_per_item), ms.value

    def launch(self, stream=None) -> None:
        _check(lib().fdas_batch_plan_launch(self._h, _stream(stream)), "fdas_batch_plan_launch")

    def close(self) -> None:
        if self._h:
            lib().fdas_batch_plan_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Device buffers for a batch of spectra of the given lengths, allocated once with torch."""

    def __init__(self, params: Params, lengths, thresh: np.ndarray | None = None, device: str = "cuda:0"):
        import torch

        st = fdas_check_params(params)
        if st != _lib.FDAS_OK:
            raise FdasError(st, "params")
        self.p = params
        self.lengths = [int(n) for n in lengths]
        self.device = torch.device(device)
        u8 = dict(dtype=torch.uint8, device=self.device)
        self.tmpl = torch.empty(fdas_templates_bytes(params), **u8)
        ta = fdas_default_thresholds(params) if thresh is None else np.ascontiguousarray(thresh, dtype=np.float32)
        self.thresh = torch.from_numpy(ta).to(self.device)
        self.ws_bytes = fdas_batch_workspace_bytes(params, len(self.lengths))
        self.ws = torch.empty(self.ws_bytes, **u8)
        nrec = params.n_harm * params.cand_cap * CAND_DTYPE.itemsize
        self.specs, self.planes, self.cands, self.counts, self.peaks, self.ld = [], [], [], [], [], []
        for n in self.lengths:
            ld = round_up(n, 64)
            self.ld.append(ld)
            self.specs.append(torch.empty(n, dtype=torch.complex64, device=self.device))
            self.planes.append(torch.empty((params.n_temp, ld), dtype=torch.float32, device=self.device))
            self.cands.append(torch.empty(nrec, **u8))
            self.counts.append(torch.empty(params.n_harm, dtype=torch.int32, device=self.device))
            self.peaks.append(torch.empty(params.n_harm * CAND_DTYPE.itemsize, **u8))
        with torch.cuda.device(self.device):
            fdas_make_templates(params, self.tmpl)
            # The bank and thresholds are ready before any search, on whichever stream it runs.
            torch.cuda.current_stream(self.device).synchronize()

    def entries(self):
        return [(self.specs[b], n, self.planes[b], self.ld[b], self.cands[b], self.counts[b], self.peaks[b])
                for b, n in enumerate(self.lengths)]

    def search(self, ctas_per_sm=0, templates_per_item=0, stream=None) -> None:
        fdas_search_batch(self.p, self.entries(), self.tmpl, self.thresh, self.ws, self.ws_bytes, ctas_per_sm,
                          templates_per_item, stream)

    def harmonic_sum(self, stream=None) -> None:
        """fdas_harmonic_sum_batch on the batch's planes as they stand (e.g. planes written by the caller)."""
        fdas_harmonic_sum_batch(self.p, self.entries(), self.thresh, self.ws, self.ws_bytes, stream)

    def plan(self) -> BatchPlan:
        return BatchPlan(self.p, self.entries(), self.tmpl, self.thresh, self.ws, self.ws_bytes)

    def results(self, b: int):
        counts = self.counts[b].cpu().numpy().astype(np.uint32)
        return (decode_cands(self.cands[b].cpu().numpy(), counts, self.p.cand_cap), counts,
                self.peaks[b].cpu().numpy().view(CAND_DTYPE).copy())


class Server:
    """fdas_server: a request loop (native worker thread) with admission by device-memory footprint.

    submit() takes a host complex64 array (keep it alive until its result is polled) and returns at
    once; poll() returns finished requests as dicts with the candidates, counts, peaks and times.
    """

    def __init__(self, params: Params, device_bytes: int, max_inflight: int = 3):
        self.p = params
        self._h = C.c_void_p()
        self._keep = {}
        _check(lib().fdas_server_create(C.byref(params.c()), device_bytes, max_inflight, C.byref(self._h)),
               "fdas_server_create")

    @staticmethod
    def request_bytes(params: Params, n: int) -> int:
        return lib().fdas_server_request_bytes(C.byref(params.c()), n)

    def submit(self, h_spec, request_id: int) -> None:
        n = h_spec.numel() if hasattr(h_spec, "numel") else h_spec.size
        cands = np.zeros(self.p.n_harm * self.p.cand_cap, dtype=CAND_DTYPE)
        self._keep[request_id] = (h_spec, cands)
        _check(lib().fdas_server_submit(self._h, _ptr(h_spec), n, request_id, _ptr(cands)), "fdas_server_submit")

    def poll(self, max_results: int = 64, wait_ms: int = 0) -> list[dict]:
        out = (_lib.fdas_result * max_results)()
        got = C.c_int()
        _check(lib().fdas_server_poll(self._h, C.cast(out, C.c_void_p), max_results, C.byref(got), wait_ms),
               "fdas_server_poll")
        res = []
        for r in out[: got.value]:
            _, cands = self._keep.pop(r.id)
            nh = self.p.n_harm
            counts = np.array(r.counts[:nh], dtype=np.uint32)
            per = [cands[k * self.p.cand_cap: k * self.p.cand_cap + min(int(counts[k]), self.p.cand_cap)]
                   for k in range(nh)]
            peaks = np.frombuffer(bytes(r.peaks), dtype=CAND_DTYPE)[:nh].copy()
            res.append(dict(id=r.id, n=r.n, status=r.status, submit_s=r.submit_s, admit_s=r.admit_s,
                            done_s=r.done_s, counts=counts, cands=per, peaks=peaks))
        return res

    def stats(self):
        pend, infl = C.c_int(), C.c_int()
        lib().fdas_server_stats(self._h, C.byref(pend), C.byref(infl))
        return pend.value, infl.value

    def close(self) -> None:
        if self._h:
            lib().fdas_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def decode_cands(raw: np.ndarray, counts: np.ndarray, cand_cap: int) -> list[np.ndarray]:
    """Split the cand buffer (n_harm * cand_cap records) into per-plane arrays of the written length."""
    rec = np.ascontiguousarray(raw).view(CAND_DTYPE).reshape(len(counts), cand_cap)
    return [rec[k, : min(int(counts[k]), cand_cap)].copy() for k in range(len(counts))]


def round_up(x: int, m: int) -> int:
    return (x + m - 1) // m * m


class Searcher:
    """Device buffers for spectra of up to ``n_max`` bins, allocated once with torch.

    The template bank is generated on the device at construction (fdas_make_templates). The
    thresholds default to the library's 6-sigma table, or an explicit float32[n_harm][n_temp]
    array can be given.
    """

    def __init__(self, params: Params, n_max: int, thresh: np.ndarray | None = None, device: str = "cuda:0"):
        import torch

        st = fdas_check_params(params)
        if st != _lib.FDAS_OK:
            raise FdasError(st, "params")
        self.p = params
        self.n_max = n_max
        self.ld = round_up(n_max, 64)
        self.device = torch.device(device)
        u8 = dict(dtype=torch.uint8, device=self.device)
        self.tmpl = torch.empty(fdas_templates_bytes(params), **u8)
        self.plane = torch.empty((params.n_temp, self.ld), dtype=torch.float32, device=self.device)
        self.ws_bytes = fdas_workspace_bytes(params, n_max)
        self.ws = torch.empty(self.ws_bytes, **u8)
        self.spec = torch.empty(n_max, dtype=torch.complex64, device=self.device)
        ta = fdas_default_thresholds(params) if thresh is None else np.ascontiguousarray(thresh, dtype=np.float32)
        self.thresh_host = ta
        self.thresh = torch.from_numpy(ta).to(self.device)
        nrec = params.n_harm * params.cand_cap
        self.cands = torch.empty(nrec * CAND_DTYPE.itemsize, **u8)
        self.counts = torch.empty(params.n_harm, dtype=torch.int32, device=self.device)
        self.peaks = torch.empty(params.n_harm * CAND_DTYPE.itemsize, **u8)
        self.h_cands = torch.empty(nrec * CAND_DTYPE.itemsize, dtype=torch.uint8, pin_memory=True)
        self.h_counts = torch.empty(params.n_harm, dtype=torch.int32, pin_memory=True)
        self.h_peaks = torch.empty(params.n_harm * CAND_DTYPE.itemsize, dtype=torch.uint8, pin_memory=True)
        with torch.cuda.device(self.device):
            fdas_make_templates(params, self.tmpl)
            # The bank and thresholds are ready before any search, on whichever stream it runs.
            torch.cuda.current_stream(self.device).synchronize()

    def search(self, spec, n: int | None = None, stream=None) -> None:
        """Run fdas_search on a device complex64 tensor (results stay on the device)."""
        n = spec.numel() if n is None else n
        fdas_search(self.p, spec, n, self.tmpl, self.plane, self.ld, self.thresh, self.cands, self.counts,
                    self.peaks, self.ws, self.ws_bytes, stream)

    def search_host(self, h_spec, n: int | None = None, stream=None) -> None:
        """Run fdas_search_host on a host complex64 buffer (pinned torch tensor or numpy array)."""
        n = (h_spec.numel() if hasattr(h_spec, "numel") else h_spec.size) if n is None else n
        fdas_search_host(self.p, h_spec, n, self.spec, self.tmpl, self.plane, self.ld, self.thresh, self.cands,
                         self.counts, self.peaks, self.h_cands, self.h_counts, self.h_peaks, self.ws, self.ws_bytes,
                         stream)

    def search_host_async(self, h_spec, n: int | None = None, stream=None) -> None:
        """fdas_search_host_async: enqueue copy in, search and copies out on `stream` and return. The
        host results (results(host=True)) are valid once the stream has completed them."""
        n = (h_spec.numel() if hasattr(h_spec, "numel") else h_spec.size) if n is None else n
        fdas_search_host_async(self.p, h_spec, n, self.spec, self.tmpl, self.plane, self.ld, self.thresh, self.cands,
                               self.counts, self.peaks, self.h_cands, self.h_counts, self.h_peaks, self.ws,
                               self.ws_bytes, stream)

    def results(self, host: bool = False):
        """(per-plane candidate arrays, counts, peaks) as numpy, from the device or host buffers."""
        if host:
            raw, counts, peaks = self.h_cands.numpy(), self.h_counts.numpy(), self.h_peaks.numpy()
        else:
            raw, counts, peaks = self.cands.cpu().numpy(), self.counts.cpu().numpy(), self.peaks.cpu().numpy()
        counts = counts.astype(np.uint32)
        return decode_cands(raw, counts, self.p.cand_cap), counts, peaks.view(CAND_DTYPE).copy()
