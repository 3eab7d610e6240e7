"""Tensor-core convolution (precisions FDAS_BF16X3 and FDAS_FP16S) against the FP64 oracle.

The plane bar is the same as for the FP32 kernel: rel = |P_gpu - P_ref| / max(P_ref, mean P_ref)
at most 1e-4 everywhere. Every test prints the measured max and RMS so that the accuracy of each
split is on record.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import correlate, harmonic, templates, thresholds

pytestmark = pytest.mark.gpu

REL_TOL = 1e-4
PRECISIONS = {"bf16x3": 1, "fp16s": 2}


def plane_rel(gpu, ref):
    rel = np.abs(gpu.astype(np.float64) - ref) / np.maximum(ref, ref.mean())
    return rel.max(), np.sqrt(np.mean(rel**2))


def run_convolve(fd, p, spec, ld=None, fill=np.nan, cfg=None):
    n = len(spec)
    ld = n if ld is None else ld
    tmpl = torch.empty(fd.fdas_templates_bytes(p), dtype=torch.uint8, device="cuda")
    fd.fdas_make_templates(p, tmpl)
    d_spec = torch.from_numpy(np.ascontiguousarray(spec, dtype=np.complex64)).cuda()
    plane = torch.full((p.n_temp, ld), fill, dtype=torch.float32, device="cuda")
    if cfg is None:
        fd.fdas_convolve(p, d_spec, n, tmpl, plane, ld)
    else:
        fd.fdas_convolve_cfg(p, d_spec, n, tmpl, plane, ld, *cfg)
    torch.cuda.synchronize()
    return plane.cpu().numpy()


@pytest.mark.parametrize("prec", sorted(PRECISIONS))
@pytest.mark.parametrize("n", [1, 211, 1628, 1629, 5000, 20000])
def test_tc_plane_small_and_ragged(fd, bank, prec, n):
    p = fd.Params(precision=PRECISIONS[prec])
    spec = synth.complex_noise(np.random.default_rng(n), n).astype(np.complex64)
    got = run_convolve(fd, p, spec)
    ref = correlate.plane_ols(spec, bank, 2048)
    mx, rms = plane_rel(got, ref)
    print(f"{prec} n={n}: rel max {mx:.2e} rms {rms:.2e}")
    assert mx <= REL_TOL


@pytest.mark.parametrize("prec", sorted(PRECISIONS))
def test_tc_plane_small_workload(fd, small_case, prec):
    wl, ref = small_case
    p = fd.Params(precision=PRECISIONS[prec])
    got = run_convolve(fd, p, wl.spectrum, ld=wl.n + 64)
    assert np.isnan(got[:, wl.n:]).all()  # padding columns untouched
    got = got[:, : wl.n]
    mx, rms = plane_rel(got, ref)
    print(f"{prec} N=2^16: rel max {mx:.2e} rms {rms:.2e}")
    assert mx <= REL_TOL
    assert np.unravel_index(np.argmax(got), got.shape) == (62, 12000)


@pytest.mark.parametrize("prec", sorted(PRECISIONS))
@pytest.mark.parametrize("cfg", [(1, 0), (2, 2), (2, 7), (0, 85)])
def test_tc_launch_shapes_agree(fd, prec, cfg):
    """Every CTA count and template chunking gives the same plane, bit for bit."""
    p = fd.Params(precision=PRECISIONS[prec])
    spec = synth.complex_noise(np.random.default_rng(11), 30000).astype(np.complex64)
    base = run_convolve(fd, p, spec)
    got = run_convolve(fd, p, spec, cfg=cfg)
    assert np.array_equal(got.view(np.uint32), base.view(np.uint32))


@pytest.mark.parametrize("prec", sorted(PRECISIONS))
def test_tc_plane_other_template_grid(fd, prec):
    """9 templates with z_step 2 and 129 taps: a grid the kernel was not shaped around."""
    p = fd.Params(n_temp=9, z_min=-8, z_step=2, n_tap=129, precision=PRECISIONS[prec])
    grid = templates.TemplateGrid(n_temp=9, z_min=-8, z_step=2, n_tap=129)
    bank = templates.template_bank(grid)
    spec = synth.complex_noise(np.random.default_rng(5), 9000).astype(np.complex64)
    got = run_convolve(fd, p, spec)
    mx, rms = plane_rel(got, correlate.plane_ols(spec, bank, 2048))
    print(f"{prec} 9x129: rel max {mx:.2e} rms {rms:.2e}")
    assert mx <= REL_TOL


@pytest.mark.parametrize("prec", sorted(PRECISIONS))
def test_tc_plane_full_size(fd, ska_case, prec):
    """N = 2^21, 85 templates: the whole plane against the oracle in the bench's launch shape."""
    wl, ref = ska_case
    p = fd.Params(precision=PRECISIONS[prec])
    s = fd.Searcher(p, wl.n)
    s.search(torch.from_numpy(wl.spectrum).cuda(), wl.n)
    torch.cuda.synchronize()
    got = s.plane[:, : wl.n].cpu().numpy()
    mx, rms = plane_rel(got, ref)
    print(f"{prec} N=2^21: plane rel max {mx:.2e} rms {rms:.2e}")
    assert mx <= REL_TOL
    assert fd.fdas_device_status(clear=True) == 0


@pytest.mark.parametrize("prec", sorted(PRECISIONS))
def test_tc_large_dynamic_range(fd, bank, prec):
    """Spectra scaled by 2^-30 and 2^+30: FP16's range is handled by the per-segment scaling."""
    p = fd.Params(precision=PRECISIONS[prec])
    wl = synth.small_workload(n=1 << 14)
    for scale in (2.0**-30, 2.0**30):
        spec = (wl.spectrum.astype(np.complex128) * scale).astype(np.complex64)
        got = run_convolve(fd, p, spec)
        ref = correlate.plane_ols(spec, bank, 2048)
        mx, rms = plane_rel(got, ref)
        print(f"{prec} scale {scale:.0e}: rel max {mx:.2e} rms {rms:.2e}")
        assert mx <= REL_TOL


@pytest.mark.parametrize("prec", sorted(PRECISIONS))
def test_tc_search_candidates_match_oracle_within_tolerance(fd, small_case, prec):
    """Candidates of the tensor-core search against Algorithm 1 on the oracle plane.

    A point may differ only when its harmonic sum lies within the plane tolerance of the threshold.
    """
    wl, ref_plane = small_case
    p = fd.Params(harm_mask=0b10001011, cand_cap=1000, precision=PRECISIONS[prec])
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


@pytest.mark.parametrize("prec", sorted(PRECISIONS))
def test_tc_batch_equals_single(fd, prec):
    """The batched tensor-core form gives the same planes and candidates as one search per spectrum."""
    p = fd.Params(precision=PRECISIONS[prec])
    wls = synth.batch_workloads(count=5, seed=3)
    b = fd.Batch(p, [w.n for w in wls])
    for i, w in enumerate(wls):
        b.specs[i].copy_(torch.from_numpy(w.spectrum))
    b.search()
    torch.cuda.synchronize()
    for i, w in enumerate(wls):
        s = fd.Searcher(p, w.n)
        s.search(b.specs[i], w.n)
        torch.cuda.synchronize()
        assert torch.equal(b.planes[i][:, : w.n], s.plane[:, : w.n])
        got, want = b.results(i), s.results()
        for k in range(p.n_harm):
            assert np.array_equal(got[0][k], want[0][k])
        assert np.array_equal(got[1], want[1])
