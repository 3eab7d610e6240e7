"""fdas_harmonic_sum_noalloc, the harmonic sum for callers that cannot allocate device memory.

Such a caller cannot provide the workspace fdas_harmonic_sum needs, so this entry point uses a
static scratch array inside the library instead. The test calls it through the C ABI and checks
that it returns exactly what fdas_harmonic_sum returns with a caller workspace, on two calls in
a row with different inputs. The second call also shows that the first call's leftovers in the
shared array do not leak into it. The harmonic sum is exact, so the comparison is bit for bit,
as in the other harmonic-sum tests. This file is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import synth
from oracle import thresholds

pytestmark = pytest.mark.gpu


def _buffers(p, n):
    cands = torch.zeros(p.n_harm * p.cand_cap * 12, dtype=torch.uint8, device="cuda")
    counts = torch.zeros(p.n_harm, dtype=torch.int32, device="cuda")
    peaks = torch.zeros(p.n_harm * 12, dtype=torch.uint8, device="cuda")
    return cands, counts, peaks


def _host(bufs):
    return tuple(b.cpu().numpy().tobytes() for b in bufs)


@pytest.mark.parametrize("kw", [dict(), dict(harm_index=1), dict(harm_mask=0b10100100)],
                         ids=["fundamental", "highest", "sparse-mask"])
def test_noalloc_matches_workspace_entry_point_on_two_calls(fd, kw):
    """Both indexings of the harmonic planes, and a mask that reports only planes 3, 6 and 8."""
    p = fd.Params(**kw)  # 8 harmonic planes, the most the static scratch holds
    n = 1 << 15
    ta = torch.from_numpy(thresholds.threshold_array(8, 85, sigma=3.0)).cuda()
    free = []
    for seed in (31, 32):  # two calls in a row, different planes
        plane = torch.from_numpy(synth.exponential_plane(np.random.default_rng(seed), 85, n)).cuda()
        ws_bytes = fd.fdas_workspace_bytes(p, n)
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
        ref = _buffers(p, n)
        fd.fdas_harmonic_sum(p, plane, n, n, ta, *ref, ws, ws_bytes)
        got = _buffers(p, n)
        torch.cuda.synchronize()
        before = torch.cuda.mem_get_info()[0]
        fd.fdas_harmonic_sum_noalloc(p, plane, n, n, ta, *got)
        torch.cuda.synchronize()
        free.append((before, torch.cuda.mem_get_info()[0]))
        r, g = _host(ref), _host(got)
        counts = np.frombuffer(r[1], np.int32)
        reported = [k for k in range(8) if (p.harm_mask >> k) & 1]
        assert max(counts[k] for k in reported) > 200  # many crossings: the top-200 selection is exercised
        assert all(counts[k] == 0 for k in range(8) if k not in reported)
        assert g == r
    # The second call takes no device memory at all (the first one may load the library's scratch
    # array, with CUDA's lazy module loading).
    assert free[1][0] == free[1][1]


def test_noalloc_rejects_more_planes_than_its_scratch_holds(fd):
    p = fd.Params(n_harm=16, harm_mask=0xFFFF)
    null = C.c_void_p(0)
    fake = C.c_void_p(0x10000)  # rejected before any pointer is used
    st = fd.lib().fdas_harmonic_sum_noalloc(C.byref(p.c()), fake, 100, 100, fake, fake, fake, null, null)
    assert st == -3  # FDAS_ERR_WORKSPACE
