"""Benchmark of the FDAS hot path: spectra/s at N = 2^21, 85 templates, 8 harmonic planes.

One step is one pass of the whole path over one spectrum: fdas_convolve (overlap-save FT
convolution into the 85 x 2^21 F-A plane) then fdas_harmonic_sum (harmonic summing, detection,
compaction). The spectrum is the seeded SKA-sized synthetic workload (4 drifting tones with 8
harmonics in unit noise). Each rank of a multi-GPU run searches its own spectrum (independent DM
trials, weak scaling, no collective on the data path).

Prints one JSON line (rank 0). --impl reference times the FP64 CPU oracle instead, as the
reference arm.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FDAS spectra/s, N=2^21, 85 templates, 8 harm: split-BF16 vs FP32; % roofline"
N_DEFAULT = 1 << 21
SM_COUNT = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
# Nominal FP32 CUDA-core peak: 152 SMs x 128 lanes x 2 flop (FMA) x 2.07 GHz. Reported beside the
# measured one (fdas_measure_fp32_peak, FFMA chains on every SM), which is the roofline denominator.
FP32_PEAK_TFLOPS = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from the last ncu capture of
# each kernel at N = 2^21, valid only while the sources it was built from are unchanged:
# kernel file -> (sha256[:12] of its sources, bytes per fdas_convolve / fdas_harmonic_sum call).
KERNEL_SOURCES = {
    "convolve.cu": ("convolve.cu", "ols_common.cuh", "hs_keys.cuh"),
    "convolve_tc.cu": ("convolve_tc.cu", "ols_common.cuh", "tc_ops.cuh"),
    "harmonic.cu": ("harmonic.cu", "hs_keys.cuh"),
    "harmonic.cu+k1": ("harmonic.cu", "hs_keys.cuh"),
}
# "harmonic.cu": the harmonic stage of an FP32 search (no single-plane launch); "harmonic.cu+k1":
# the full harmonic sum, as the tensor-core forms run it.
NCU_TRAFFIC = {
    "convolve.cu": ("9be72b55dc87", 682.1e6),
    "convolve_tc.cu": ("f72553a64fe0", 670.0e6),
    "harmonic.cu": ("a419de2895ad", 1262.2e6),
    "harmonic.cu+k1": ("a419de2895ad", 1612.7e6),
}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def bf16_peak():
    """Dense BF16 tensor peak in TFLOP/s (measured cuBLAS burst figure), and its source."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def src_hash(kernel_file):
    d = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel_file]:
        with open(os.path.join(ROOT, "paper_1806_01556_gb300", "csrc", name), "rb") as f:
            d.update(f.read())
    return d.hexdigest()[:12]


def traffic_for(kernel_file):
    entry = NCU_TRAFFIC.get(kernel_file)
    if entry and entry[0] == src_hash(kernel_file):
        return entry[1]
    return None


# Convolution forms (fdas_params.precision). The plane error of each against the FP64 oracle is
# checked by the GPU tests (bar: 1e-4 relative everywhere); this file times them.
FORMS = {"fp32": 0, "bf16x3": 1, "fp16s": 2}
TC_TEMPLATES_PER_ITEM = 44  # default work-item size of the tensor-core form (pairs of templates)


def hs_launches(n_harm=8, n_temp=85):
    """Kernel launches of one fdas_harmonic_sum: reset, one per non-empty group of rows (plane
    counts 5-16, 3-4, 2), the single-plane rows, finalize."""
    c = (n_temp - 1) // 2
    groups = 0
    for kmin, kmax in ((5, 16), (3, 4), (2, 2)):
        if kmin > n_harm:
            continue
        lo = 0 if kmax >= n_harm else c // (kmax + 1) + 1
        if c // kmin >= lo:
            groups += 1
    k1 = 1 if (n_harm < 2 or c // 2 + 1 <= c) else 0
    return 2 + groups + k1


def search_launches(precision, n_harm=8, n_temp=85, harm_index=0):
    """Kernel launches of one fdas_search (its two stages). FP32 takes HP_1 in the convolution, so
    its launches are reset, convolution, the row groups and finalize: as many as a harmonic sum
    alone. The tensor-core forms: reset, convolution, then the whole harmonic sum."""
    if harm_index:
        return 5  # reset, convolution, reset, the highest-harmonic launch, finalize
    return hs_launches(n_harm, n_temp) + (0 if precision == "fp32" else 2)


def hs_rows(precision, n_harm=8, n_temp=85):
    """Plane rows the harmonic stage of fdas_search reads: with FP32 the single-plane rows are done
    in the convolution, so only the rows with two or more planes (|i| <= c/2) are read again."""
    c = (n_temp - 1) // 2
    if precision == "fp32" and n_harm >= 2:
        return 2 * (c // 2) + 1
    return n_temp if precision != "fp32" else 0


def tc_executed_flop(n, n_temp=85, n_tap=421, fft_len=2048):
    """Tensor-core flops the split forms execute per spectrum: 24 MMAs (M=128, N=64, K=16) per
    pair of templates per segment, with templates chunked 44 per work item."""
    keep = fft_len - n_tap + 1
    n_seg = -(-n // keep)
    pairs = 0
    for t0 in range(0, n_temp, TC_TEMPLATES_PER_ITEM):
        pairs += -(-min(TC_TEMPLATES_PER_ITEM, n_temp - t0) // 2)
    return n_seg * pairs * 24 * 2 * 128 * 64 * 16


def algorithmic(n, n_temp=85, n_tap=421, fft_len=2048, n_harm=8, rows_read=None):
    """Algorithmic work of one spectrum (nominal FFT count 5 F log2 F per transform). The harmonic
    stage reads each plane point of its rows once (rows_read, all rows by default)."""
    keep = fft_len - n_tap + 1
    n_seg = -(-n // keep)
    fft_flop = 5 * fft_len * int(np.log2(fft_len))
    conv_flop = fft_flop * n_seg * (1 + n_temp) + 6 * fft_len * n_seg * n_temp + 3 * n_temp * n
    conv_bytes = n_seg * fft_len * 8 + n_temp * n * 4  # segment reads (with overlap) + plane write
    hs_bytes = (n_temp if rows_read is None else rows_read) * n * 4
    return dict(conv_flop=conv_flop, conv_bytes=conv_bytes, hs_bytes=hs_bytes, n_seg=n_seg)


def path_roofline(n, n_tap, ms_per_step, hbm_gbs, hbm_kind, n_temp=85, fp32_tflops=FP32_PEAK_TFLOPS,
                  fp32_kind="unit counts x clock"):
    """The whole search against the slower of its two floors: the FFT flops at the FP32 ALU peak, and
    the plane's bytes at the measured HBM bandwidth (written once by the convolution, read once by
    the harmonic sum, plus the spectrum read with the segment overlap)."""
    alg = algorithmic(n, n_temp=n_temp, n_tap=n_tap)
    t_flop = alg["conv_flop"] / (fp32_tflops * 1e12) * 1e3
    plane = n_temp * n * 4
    t_bytes = (alg["conv_bytes"] + plane) / (hbm_gbs * 1e9) * 1e3
    t_roof = max(t_flop, t_bytes)
    return {"bound": "hbm" if t_bytes >= t_flop else "alu", "ms_at_roofline": t_roof, "ms_flop": t_flop,
            "ms_bytes": t_bytes, "achieved_ms": ms_per_step, "frac": t_roof / ms_per_step,
            "bytes": alg["conv_bytes"] + plane, "flop": alg["conv_flop"],
            "peaks": f"FP32 {fp32_tflops:.1f} TFLOP/s ({fp32_kind}), HBM {hbm_gbs:.0f} GB/s ({hbm_kind})"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 20 ms from __enter__ to __exit__.

    begin()/end() mark the timed region; summary() keeps the samples taken in it, widened by
    0.1 s on each side when the region is shorter than a few sampling periods."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.t_begin = self.t_end = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.3)  # let it start sampling before the timed region
        except Exception:
            self.proc = None
        return self

    def begin(self):
        self.t_begin = time.time()

    def end(self):
        self.t_end = time.time()

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        import datetime

        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(f[2]), float(f[3]), f[6:10]))
            except ValueError:
                continue
        lo, hi = self.t_begin, self.t_end
        window = None
        if lo is not None and hi is not None:
            pad = 0.1 if hi - lo < 0.1 else 0.0
            window = [r for r in rows if lo - pad <= r[0] <= hi + pad]
        sel = window if window else rows
        if not sel:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        reasons = set()
        for r in sel:
            for name, v in zip(names, r[3]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r[1] for r in sel), "sm_max_mhz": sel[-1][2], "reasons": sorted(reasons),
                "samples": len(sel), "window": "timed region" if window else "whole run"}


class _Null:
    def __enter__(self):
        return self

    def begin(self):
        pass

    def end(self):
        pass

    def __exit__(self, *exc):
        return False


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_seed(rank: int) -> int:
    """Each rank searches its own spectrum (an independent DM trial): seed 1 + rank."""
    return 1 + rank


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The slowest rank's time (all_reduce MAX); the identity on one rank."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, steps: int, seconds: float) -> float:
    """Whole-job spectra/s: every rank processes `steps` spectra in the (max-over-ranks) time."""
    return world * steps / seconds


# ---- the FP64 oracle on the host's cores (CPU baseline and reference arm) ---------------------------
# The oracle's plane_ols runs unmodified on contiguous column blocks of the spectrum, one block per
# task, in a pool of worker processes (one per core). Column j of the plane depends only on bins
# j-h..j+h, so a block [j0, j1) is computed from bins [j0-h, j1+h) (clipped to the spectrum, where the
# zero padding is the oracle's own) and its columns [j0, j1) are exact. The workers write float32 rows
# into shared memory; the main process then runs the oracle's Algorithm 1 (harmonic.detect) on the
# whole plane, single-threaded, as it stands.
_W = {}


def _oracle_worker_init(spec_name, plane_name, n, n_temp, bank, h, fft_len):
    from multiprocessing import shared_memory

    _W["shm"] = [shared_memory.SharedMemory(name=spec_name), shared_memory.SharedMemory(name=plane_name)]
    _W["spec"] = np.ndarray((n,), dtype=np.complex128, buffer=_W["shm"][0].buf)
    _W["plane"] = np.ndarray((n_temp, n), dtype=np.float32, buffer=_W["shm"][1].buf)
    _W["bank"], _W["h"], _W["fft_len"] = bank, h, fft_len


def _oracle_block(task):
    from oracle import correlate

    j0, j1, n = task
    h = _W["h"]
    a, b = max(0, j0 - h), min(n, j1 + h)
    p = correlate.plane_ols(_W["spec"][a:b], _W["bank"], _W["fft_len"])
    _W["plane"][:, j0:j1] = p[:, j0 - a : j1 - a]
    return j1 - j0


class OraclePool:
    """The oracle's plane (all host cores) and harmonic sum for spectra of up to n_max bins."""

    def __init__(self, n_max, n_temp=85, n_tap=421, fft_len=2048, workers=None):
        import multiprocessing as mp
        from multiprocessing import shared_memory

        from oracle import templates, thresholds

        self.cores = workers or len(os.sched_getaffinity(0))
        self.n_max, self.n_temp, self.fft_len = n_max, n_temp, fft_len
        grid = templates.TemplateGrid(n_temp=n_temp, z_min=-float((n_temp - 1) // 2), z_step=1.0, n_tap=n_tap)
        self.bank = templates.template_bank(grid)
        self.ta = thresholds.threshold_array(8, n_temp)
        self._shm = [shared_memory.SharedMemory(create=True, size=n_max * 16),
                     shared_memory.SharedMemory(create=True, size=n_temp * n_max * 4)]
        self.spec = np.ndarray((n_max,), dtype=np.complex128, buffer=self._shm[0].buf)
        # spawn: the workers start clean, whatever CUDA state this process has or will have
        ctx = mp.get_context("spawn")
        env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in env:
            os.environ[k] = "1"
        try:
            self.pool = ctx.Pool(self.cores, initializer=_oracle_worker_init,
                                 initargs=(self._shm[0].name, self._shm[1].name, n_max, n_temp, self.bank,
                                           (n_tap - 1) // 2, fft_len))
        finally:
            for k, v in env.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self.pool.map(_oracle_block, [(0, 1, 1)] * self.cores)  # every worker imported the oracle

    def run(self, spectrum):
        """One search of `spectrum` (its first n bins): seconds for the plane and for Algorithm 1."""
        from oracle import harmonic

        n = len(spectrum)
        self.spec[:n] = spectrum
        self.spec[n:] = 0
        blocks = 4 * self.cores
        edges = np.linspace(0, n, blocks + 1).astype(np.int64)
        tasks = [(int(a), int(b), n) for a, b in zip(edges[:-1], edges[1:]) if b > a]
        t0 = time.perf_counter()
        self.pool.map(_oracle_block, tasks, chunksize=1)
        t1 = time.perf_counter()
        plane = np.ndarray((self.n_temp, self.n_max), dtype=np.float32, buffer=self._shm[1].buf)
        res = harmonic.detect(np.ascontiguousarray(plane[:, :n]) if n < self.n_max else plane, self.ta, 8, 0xFF,
                              200)
        t2 = time.perf_counter()
        return t1 - t0, t2 - t1, res

    def close(self):
        self.pool.terminate()
        self.pool.join()
        self.spec = None
        for m in self._shm:
            m.close()
            m.unlink()


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def cpu_baseline(wl, runs=3):
    """The oracle on one whole spectrum on all host cores, median of `runs` (spectra/s)."""
    pool = OraclePool(wl.n)
    try:
        times = [pool.run(wl.spectrum)[:2] for _ in range(runs)]
    finally:
        pool.close()
    tot = [a + b for a, b in times]
    med = float(np.median(tot))
    return {"value": 1.0 / med, "unit": "spectra/s", "cores": pool.cores, "kind": "oracle",
            "cpu": cpu_model(), "median_of": runs, "s_per_spectrum": med,
            "s_plane": float(np.median([a for a, _ in times])), "s_harmonic": float(np.median([b for _, b in times])),
            "sample": f"the whole spectrum ({wl.n} bins, 85 templates, 8 planes): oracle plane_ols on "
                      f"{pool.cores} worker processes over column blocks, then harmonic.detect (1 thread)"}


def run_reference(args):
    """The reference arm: the FP64 oracle, as it stands, on the host's cores (rank 0 only). Each step
    searches the whole spectrum, unless the run has more than 40 steps in all, in which case each
    step searches a contiguous sample of ~N*40/(steps+warmup) bins, so that the run stays within
    about two minutes; value is spectra/s either way and ms_per_step the measured time of a step."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import synth

    wl = synth.ska_workload(n=args.n, seed=1)
    total = args.steps + args.warmup
    bins = wl.n if total <= 40 else max(1 << 16, int(wl.n * 40 / total))
    pool = OraclePool(bins)
    try:
        for _ in range(args.warmup):
            pool.run(wl.spectrum[:bins])
        times = []
        for _ in range(args.steps):
            a, b, _ = pool.run(wl.spectrum[:bins])
            times.append(a + b)
    finally:
        pool.close()
    sec = float(np.mean(times))
    frac = bins / wl.n
    value = frac / sec
    sample = (f"{'the whole spectrum' if bins == wl.n else f'the first {bins} of {wl.n} bins'} per step "
              f"({frac:g} spectrum), 85 templates, 8 planes: oracle plane_ols on {pool.cores} worker processes "
              "over column blocks, then harmonic.detect (1 thread)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "spectra/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.n, args.n_tap, args.harm_index, "fp32"),
        "spectra_per_step": frac,
        "cpu_baseline": {"value": value, "unit": "spectra/s", "cores": pool.cores, "kind": "oracle",
                         "cpu": cpu_model(), "sample": sample},
        "e2e": {"value": value, "unit": "spectra/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(n, n_tap=421, harm_index=0, precision="fp32"):
    """The workload both arms report. precision is the convolution form in value (the reference arm
    computes in FP64 and reports the FP32 form it stands beside)."""
    return {
        "workload": f"SKA-sized spectrum N={n} (2^{int(np.log2(n))}), 4 drifting tones x 8 harmonics in unit "
                    f"complex Gaussian noise (seed 1, rank r uses seed 1+r); 85 templates z=-42..42, {n_tap} taps, "
                    "overlap-save F=2048; 8 harmonic planes, 6-sigma thresholds, 200 candidates per plane",
        "n": n, "n_temp": 85, "n_tap": n_tap, "fft_len": 2048, "n_harm": 8,
        "l2": "inputs larger than L2: the 713 MB plane is written and read every step",
        "parallelism": "replicas (one spectrum per GPU, no collective)",
        "harm_index": "highest" if harm_index else "fundamental",
        "precision": precision,
    }


def run_fdas(args):
    import torch

    import paper_1806_01556_gb300 as fdas
    import synth

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    wl = synth.ska_workload(n=args.n, seed=rank_seed(rank))
    # The CPU baseline runs before any timed GPU work (rank 0, N = 1 only).
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl)

    d_spec = torch.from_numpy(wl.spectrum).to(dev)
    stream = torch.cuda.current_stream(dev)
    searchers = {name: fdas.Searcher(fdas.Params(precision=code, n_tap=args.n_tap, harm_index=args.harm_index),
                                     args.n, device=f"cuda:{local}")
                 for name, code in FORMS.items() if name in args.forms}

    def step(s, ev=None):
        """One fdas_search, through its two stages so that each can be timed."""
        p = s.p
        if ev is not None:
            ev[0].record(stream)
        fdas.fdas_search_convolve(p, d_spec, args.n, s.tmpl, s.plane, s.ld, s.thresh, s.ws, s.ws_bytes, stream)
        if ev is not None:
            ev[1].record(stream)
        fdas.fdas_search_harmonic(p, s.plane, args.n, s.ld, s.thresh, s.cands, s.counts, s.peaks, s.ws, s.ws_bytes,
                                  stream)
        if ev is not None:
            ev[2].record(stream)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def timed(s, sampler=None):
        """K steps of one form, bracketed by barrier + synchronize; per-step stage events."""
        for _ in range(args.warmup):
            step(s)
        torch.cuda.synchronize(dev)
        events = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ctx = sampler if sampler is not None else _Null()
        with ctx:
            barrier()
            torch.cuda.synchronize(dev)
            ctx.begin()
            start.record(stream)
            for k in range(args.steps):
                step(s, events[k])
            end.record(stream)
            torch.cuda.synchronize(dev)
            ctx.end()
            barrier()
        total_ms = max_over_ranks(start.elapsed_time(end), world, dev)
        return {"total_ms": total_ms,
                "conv_ms": float(np.mean([e[0].elapsed_time(e[1]) for e in events])),
                "hs_ms": float(np.mean([e[1].elapsed_time(e[2]) for e in events]))}

    # The FP32 CUDA-core peak of this GPU, measured (FFMA chains on every SM for about 200 ms), with the
    # clocks it ran at: the denominator of the FP32 convolution's roofline.
    fp32_sampler = ClockSampler(local)
    with fp32_sampler:
        fp32_sampler.begin()
        fp32_tflops, fp32_ms = fdas.fdas_measure_fp32_peak(200.0)
        fp32_sampler.end()
    fp32_peak = {"value": fp32_tflops, "unit": "TFLOP/s", "timed_ms": fp32_ms, "clocks": fp32_sampler.summary(),
                 "nominal": FP32_PEAK_TFLOPS,
                 "how": "fdas_measure_fp32_peak: 8 independent FFMA chains per thread, 4 CTAs of 256 threads per "
                        "SM, 2 flop per FFMA, CUDA events"}
    fp32_src = "measured (fdas_measure_fp32_peak, FFMA chains on every SM)"

    # The form that goes in "value" is timed with the clock sampler; the others are timed the same way.
    results, samplers = {}, {}
    for name, s in searchers.items():
        samplers[name] = ClockSampler(local)
        results[name] = timed(s, samplers[name])
    head = min(results, key=lambda k: results[k]["total_ms"]) if args.headline == "best" else args.headline
    s = searchers[head]
    p = s.p
    ms_per_step = results[head]["total_ms"] / args.steps
    value = job_throughput(world, args.steps, results[head]["total_ms"] / 1e3)

    # A longer run of the same steps (about one second, untimed for value) for a fuller clock record
    # under load, with its own per-step time as a consistency check.
    soak_sampler = ClockSampler(local)
    soak_steps = max(args.steps, int(1000.0 / max(ms_per_step, 1e-3)))
    with soak_sampler:
        barrier()
        torch.cuda.synchronize(dev)
        soak_sampler.begin()
        sa, sb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sa.record(stream)
        for _ in range(soak_steps):
            step(s)
        sb.record(stream)
        torch.cuda.synchronize(dev)
        soak_sampler.end()
    soak = {"steps": soak_steps, "ms_per_step": sa.elapsed_time(sb) / soak_steps, "clocks": soak_sampler.summary()}

    # A stream of spectra: the plain convolution and the full harmonic sum of each spectrum, spectra
    # taking three streams and planes in turn, so that one spectrum's harmonic sum (HBM-bound) runs
    # beside the next one's convolution (ALU-bound). Reported beside the one-stream value.
    pipelined = None
    if "fp32" in searchers:
        pair = [searchers["fp32"]] + [fdas.Searcher(searchers["fp32"].p, args.n, device=f"cuda:{local}")
                                      for _ in range(2)]
        streams = [torch.cuda.Stream(dev) for _ in range(3)]

        def pstep(k):
            s2, st = pair[k % 3], streams[k % 3]
            fdas.fdas_convolve(s2.p, d_spec, args.n, s2.tmpl, s2.plane, s2.ld, st)
            fdas.fdas_harmonic_sum(s2.p, s2.plane, args.n, s2.ld, s2.thresh, s2.cands, s2.counts, s2.peaks, s2.ws,
                                   s2.ws_bytes, st)

        for k in range(args.warmup):
            pstep(k)
        torch.cuda.synchronize(dev)
        barrier()
        pa, pb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        pa.record(stream)
        for st in streams:
            st.wait_event(pa)
        for k in range(args.steps):
            pstep(k)
        for st in streams:
            ev = torch.cuda.Event()
            ev.record(st)
            stream.wait_event(ev)
        pb.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        p_ms = max_over_ranks(pa.elapsed_time(pb), world, dev)
        pipelined = {"spectra_per_s": job_throughput(world, args.steps, p_ms / 1e3), "streams": 3,
                     "ms_per_spectrum": p_ms / args.steps, "precision": "fp32",
                     "path": "fdas_convolve + fdas_harmonic_sum per spectrum, spectra taking three streams and "
                             "planes in turn (a convolution overlaps the harmonic sums of the others)"}
        del pair

    # End to end from host memory, every step: the pinned spectrum in, the candidates, counts and
    # peaks out. Headline: fdas_search_host_async on three searchers and streams in turn. A stream's
    # copy in waits for that stream's previous search, which is then two spectra back and finished,
    # so every copy overlaps the searches of the other two streams (with two streams about half of
    # each 82 us copy stayed exposed). Beside it, fdas_search_host one call at a time.
    h_spec = torch.from_numpy(wl.spectrum).pin_memory()
    trio = [s] + [fdas.Searcher(s.p, args.n, device=f"cuda:{local}") for _ in range(2)]
    trio_streams = [torch.cuda.Stream(dev) for _ in range(3)]
    for k in range(6):
        trio[k % 3].search_host_async(h_spec, args.n, trio_streams[k % 3])
    torch.cuda.synchronize(dev)
    barrier()
    t0 = time.perf_counter()
    for k in range(args.steps):
        trio[k % 3].search_host_async(h_spec, args.n, trio_streams[k % 3])
    for st in trio_streams:
        st.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    del trio[1:]
    for _ in range(2):
        s.search_host(h_spec, args.n)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.search_host(h_spec, args.n)
    e2e_sync_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    cands, counts, _ = s.results(host=True)

    if rank == 0:
        hbm, hbm_kind = peaks()
        tc_peak, tc_kind = bf16_peak()
        forms = {}
        for name, r in results.items():
            alg = algorithmic(args.n, n_tap=args.n_tap, rows_read=85 if args.harm_index else hs_rows(name))
            conv_s, hs_s = r["conv_ms"] / 1e3, r["hs_ms"] / 1e3
            conv_tflops = alg["conv_flop"] / conv_s / 1e12
            hs_gbs = alg["hs_bytes"] / hs_s / 1e9
            conv = {"ms": r["conv_ms"], "bound": "alu", "achieved": conv_tflops, "unit": "TFLOP/s",
                    "peak": fp32_tflops, "frac": conv_tflops / fp32_tflops, "peak_source": fp32_src,
                    "frac_of_nominal": conv_tflops / FP32_PEAK_TFLOPS,
                    "hbm_gbs": alg["conv_bytes"] / conv_s / 1e9,
                    "traffic": traffic_for("convolve.cu" if name == "fp32" else "convolve_tc.cu")}
            if name != "fp32":
                executed = tc_executed_flop(args.n, n_tap=args.n_tap)
                conv["tensor"] = {"executed_tflops": executed / conv_s / 1e12, "peak": tc_peak,
                                  "frac": executed / conv_s / 1e12 / tc_peak,
                                  "peak_source": f"MEASURED_PEAKS.json bf16_tflops ({tc_kind})",
                                  "note": "MMA flops executed (3 split products, real form) over the kernel time"}
            forms[name] = {
                "spectra_per_s": job_throughput(world, args.steps, r["total_ms"] / 1e3),
                "ms_per_step": r["total_ms"] / args.steps,
                "stages": {
                    "convolve": conv,
                    "harmonic_sum": {"ms": r["hs_ms"], "bound": "hbm", "achieved": hs_gbs, "unit": "GB/s",
                                     "peak": hbm, "frac": hs_gbs / hbm,
                                     "traffic": traffic_for("harmonic.cu" if name == "fp32" else "harmonic.cu+k1"),
                                     "rows_read": hs_rows(name),
                                     "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({hbm_kind})"},
                },
                "clocks": samplers[name].summary(),
            }
        st = forms[head]["stages"]
        dom = "convolve" if st["convolve"]["ms"] >= st["harmonic_sum"]["ms"] else "harmonic_sum"
        d = st[dom]
        roof = {"kernel": dom, "bound": d["bound"], "achieved": d["achieved"], "peak": d["peak"], "unit": d["unit"],
                "frac": d["frac"], "traffic": d["traffic"], "peak_source": d["peak_source"]}
        d2h = p.n_harm * p.cand_cap * 12 + p.n_harm * 4 + p.n_harm * 12
        cfg = workload_config(args.n, args.n_tap, args.harm_index, head)
        line = {
            "metric": METRIC, "value": value, "unit": "spectra/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
            "fa_points_per_s": value * 85 * args.n,
            "clocks": forms[head]["clocks"],
            "e2e": {"value": job_throughput(world, args.steps, e2e_s), "unit": "spectra/s",
                    "h2d_bytes_per_step": args.n * 8, "d2h_bytes_per_step": d2h,
                    "api": "fdas_search_host_async, three searchers and streams in turn",
                    "one_call_at_a_time": job_throughput(world, args.steps, e2e_sync_s)},
            "gpu_launches": search_launches(head, p.n_harm, p.n_temp, args.harm_index) * args.steps,
            "roofline": roof,
            "path_roofline": path_roofline(args.n, args.n_tap, ms_per_step, hbm, hbm_kind, fp32_tflops=fp32_tflops,
                                           fp32_kind="measured"),
            "fp32_peak": fp32_peak,
            "clocks_soak": soak,
            "stages": st,
            "forms": forms,
            "cpu_baseline": cpu,
            "pipelined": pipelined,
            "candidates_per_plane": [int(c) for c in counts],
        }
        if "fp32" in forms and "bf16x3" in forms:
            line["split_bf16_vs_fp32"] = forms["bf16x3"]["spectra_per_s"] / forms["fp32"]["spectra_per_s"]
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_batch(args):
    """Batched form: 64 uneven spectra (2^18..2^22 bins), one plan replayed as a CUDA graph, for each
    convolution form in --forms; the fastest goes in value."""
    import torch

    import paper_1806_01556_gb300 as fdas
    import synth

    torch.cuda.set_device(0)
    wls = synth.batch_workloads(args.batch, seed=3)
    bins = sum(w.n for w in wls)
    stream = torch.cuda.current_stream()
    forms = {}
    for name in args.forms:
        p = fdas.Params(precision=FORMS[name])
        batch = fdas.Batch(p, [w.n for w in wls])
        for b, w in enumerate(wls):
            batch.specs[b].copy_(torch.from_numpy(w.spectrum))
        plan = batch.plan()
        (ctas, tpi), conv_ms = plan.tune()
        for _ in range(args.warmup):
            plan.launch()
        torch.cuda.synchronize()
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sampler = ClockSampler(0)
        with sampler:
            sampler.begin()
            start.record(stream)
            for _ in range(args.steps):
                plan.launch()
            end.record(stream)
            torch.cuda.synchronize()
            sampler.end()
        ms = start.elapsed_time(end) / args.steps
        forms[name] = {"spectra_per_s": len(wls) / (ms / 1e3), "ms_per_step": ms,
                       "tuned": {"ctas_per_sm": ctas, "templates_per_item": tpi, "conv_ms": conv_ms},
                       "clocks": sampler.summary(), "gpu_launches_per_step": 1 + hs_launches(p.n_harm, p.n_temp) - (1 if name == "fp32" else 0)}
        plan.close()
        del batch
    head = max(forms, key=lambda k: forms[k]["spectra_per_s"])
    f = forms[head]
    line = {
        "metric": "FDAS spectra/s, batched uneven spectra", "value": f["spectra_per_s"], "unit": "spectra/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": f["ms_per_step"],
        "higher_is_better": True, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{len(wls)} dedispersion-trial spectra, lengths floor(2^U), U~Uniform(18,22), seed 3, "
                               "0-3 drifting tones x 8 harmonics each; 85 templates, 421 taps, F=2048, 8 planes",
                   "total_bins": bins, "launch": "fdas_batch_plan (CUDA graph replay)", "precision": head},
        "fa_points_per_s": 85 * bins / (f["ms_per_step"] / 1e3),
        "clocks": f["clocks"],
        "gpu_launches": f["gpu_launches_per_step"] * args.steps,
        "forms": forms,
    }
    print(json.dumps(line), flush=True)


def run_serve(args):
    """Serving form: Poisson arrivals (mean 200 spectra/s, seed 4) of spectra of 2^19..2^22 bins, 16
    harmonic planes, through the native request loop; throughput and p50/p99 latency."""
    import torch

    import paper_1806_01556_gb300 as fdas
    import synth

    torch.cuda.set_device(0)
    p = fdas.Params(n_harm=16, harm_mask=0xFFFF)
    sizes = [1 << 19, 1 << 20, 1 << 21, 1 << 22]
    pool = {n: [torch.from_numpy(synth.ska_workload(n=n, seed=40 + k).spectrum).pin_memory() for k in range(2)]
            for n in sizes}
    rng = np.random.default_rng(4)
    n_req = int(args.rate * args.duration)
    gaps = rng.exponential(1.0 / args.rate, size=n_req)
    which = rng.integers(0, len(sizes), size=n_req)
    server = fdas.Server(p, device_bytes=args.serve_gb << 30, max_inflight=3)
    # warm-up: one request of each size, not timed
    for k, n in enumerate(sizes):
        server.submit(pool[n][0], 10**9 + k)
    got = 0
    while got < len(sizes):
        got += len(server.poll(64, wait_ms=100))
    sampler = ClockSampler(0)
    done = []
    with sampler:
        sampler.begin()
        t0 = time.perf_counter()
        t_next = t0
        for k in range(n_req):
            t_next += gaps[k]
            while True:
                now = time.perf_counter()
                if now >= t_next:
                    break
                done += server.poll(256, wait_ms=0)
                time.sleep(min(2e-4, t_next - now))
            n = sizes[which[k]]
            server.submit(pool[n][k % 2], k)
        while len(done) < n_req:
            done += server.poll(256, wait_ms=50)
        t1 = time.perf_counter()
        sampler.end()
    server.close()
    lat = np.array([r["done_s"] - r["submit_s"] for r in done]) * 1e3
    wait = np.array([r["admit_s"] - r["submit_s"] for r in done]) * 1e3
    bins = sum(int(r["n"]) for r in done)
    line = {
        "metric": "FDAS serving: spectra/s and latency under Poisson arrivals", "value": n_req / (t1 - t0),
        "unit": "spectra/s", "n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"Poisson arrivals, mean {args.rate:g}/s (seed 4), {n_req} requests, lengths uniform in "
                               "{2^19, 2^20, 2^21, 2^22}; 85 templates, 421 taps, F=2048, 16 harmonic planes",
                   "max_inflight": 3, "arena_gb": args.serve_gb},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "mean": float(lat.mean()), "max": float(lat.max())},
        "queue_wait_ms": {"p50": float(np.percentile(wait, 50)), "p99": float(np.percentile(wait, 99))},
        "fa_points_per_s": 85 * bins / (t1 - t0),
        "failed": int(sum(1 for r in done if r["status"] != 0)),
        "clocks": sampler.summary(),
    }
    print(json.dumps(line), flush=True)


def run_profile(args):
    """Untimed searches for profiler captures: --steps searches of the SKA workload (args.n bins) with
    each form in --forms, one after the other. Prints nothing but a status line."""
    import torch

    import paper_1806_01556_gb300 as fdas
    import synth

    torch.cuda.set_device(0)
    wl = synth.ska_workload(n=args.n, seed=1)
    d_spec = torch.from_numpy(wl.spectrum).cuda()
    for name in args.forms:
        s = fdas.Searcher(fdas.Params(precision=FORMS[name], n_tap=args.n_tap, harm_index=args.harm_index), args.n)
        for _ in range(args.steps):
            s.search(d_spec, args.n)
        torch.cuda.synchronize()
    print(json.dumps({"mode": "profile", "n": args.n, "forms": args.forms, "searches_per_form": args.steps,
                      "device_status": fdas.fdas_device_status()}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="fdas", choices=["fdas", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--harm-index", type=int, default=0, choices=[0, 1],
                    help="harmonic-plane indexing: 0 by fundamental (default), 1 by highest harmonic")
    ap.add_argument("--n-tap", type=int, default=421, help="taps per template (odd; the paper's reduced variants "
                    "256 and 128 are run as 257 and 129)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", default="single", choices=["single", "batch", "serve", "profile"])
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--duration", type=float, default=5.0)
    ap.add_argument("--serve-gb", type=int, default=8)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--forms", default="fp32,bf16x3,fp16s",
                    help="convolution forms to time (comma list of fp32, bf16x3, fp16s)")
    ap.add_argument("--headline", default="best",
                    help="form reported in value: best (fastest measured) or one of the forms")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    args.forms = [f for f in args.forms.split(",") if f in FORMS] or ["fp32"]
    if args.headline != "best" and args.headline not in args.forms:
        args.forms.append(args.headline)
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "batch":
        run_batch(args)
    elif args.mode == "serve":
        run_serve(args)
    elif args.mode == "profile":
        run_profile(args)
    else:
        run_fdas(args)


if __name__ == "__main__":
    main()
