"""Projection on the tensor cores (split precision, proj_engine "tensor") against the FP64
oracle's projection.

The tensor-core projection splits the frame and the basis into FP16 hi and lo parts (uint16
counts exactly), so its coefficients carry FP32-level error: each is held to 2e-6 relative L2
over a batch, the level of the SIMT FP32 projection.  Shapes cover full and partial 32-column
chunks and detector heights above and below one 128-row tile.
"""
import dataclasses

import numpy as np
import pytest

import oracle.wdd_oracle as W
import synth
from wdd_harness import gpu_plan, oracle_params, rel_l2, to_source

pytestmark = pytest.mark.gpu

COEFF_TOL = 2e-6


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def _acq(det, dtype, dose, seed, scan=(6, 7)):
    c1, _ = synth.config("c1")
    return dataclasses.replace(c1, scan_y=scan[0], scan_x=scan[1], obj_y=2 * scan[0] + det // 2,
                               obj_x=2 * scan[1] + det // 2, det=det, defocus_m=3e-9,
                               dtype=dtype, dose=dose, seed_noise=seed)


CASES = [
    # name, detector, frame type, dose (None: noise-free intensities), basis, K
    ("u16_n128_hg64", 128, "u16", 1e4, "hg_tensor", 64),
    ("f32_n96_noisefree_hg49", 96, "f32", None, "hg_tensor", 49),
    ("u16_n144_energy100", 144, "u16", 3e3, "hg_energy", 100),
    ("f32_n48_counts_energy30", 48, "f32", 5e2, "hg_energy", 30),
    ("u16_n256_hg256", 256, "u16", 1e3, "hg_tensor", 256),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
@pytest.mark.parametrize("source", ["device", "pinned"])
def test_tensor_projection_matches_oracle(torch_cuda, case, source):
    name, det, dtype, dose, basis, k = case
    acq = _acq(det, dtype, dose, seed=len(name))
    F = synth.all_frames(acq)
    idx = synth.raster_indices(acq)
    ref = W.coefficients(F, W.build_plan(oracle_params(acq, basis, k)))
    with gpu_plan(acq, basis, k, precision="split", max_batch=len(idx),
                  accum_depth=len(idx), proj_engine="tensor") as g:
        assert g.info()["proj_tensor"] == 1
        g.push(to_source(F, source), idx)
        g.check_device()
        c = g.copy_array("coeff")
    assert c.shape == ref.shape
    assert rel_l2(c, ref) < COEFF_TOL


def test_sources_give_identical_coefficients(torch_cuda):
    acq = _acq(128, "u16", 1e4, seed=5)
    F = synth.all_frames(acq)
    idx = synth.raster_indices(acq)
    out = []
    for source in ("device", "pinned", "pageable"):
        with gpu_plan(acq, "hg_tensor", 64, precision="split", max_batch=len(idx),
                      accum_depth=len(idx), proj_engine="tensor") as g:
            g.push(to_source(F, source), idx)
            g.check_device()
            out.append(g.copy_array("coeff"))
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


def test_path_selection(torch_cuda):
    """Split plans project with the streaming FP32 kernel where it applies, on the tensor cores
    when asked (and applicable); the plain FP32 path keeps the staged SIMT kernel."""
    from paper_2212_01309_gb300 import wdd
    E = wdd.PROJ_ENGINE
    a = _acq(128, "u16", 1e4, seed=6)
    with gpu_plan(a, "hg_tensor", 64, precision="split") as g:
        assert g.info()["proj_engine"] == E["stream"] and g.info()["proj_tensor"] == 0
    with gpu_plan(a, "hg_tensor", 64, precision="split", proj_engine="tensor") as g:
        assert g.info()["proj_engine"] == E["tensor"] and g.info()["proj_tensor"] == 1
    with gpu_plan(a, "hg_tensor", 64, precision="split", proj_engine="simt") as g:
        assert g.info()["proj_engine"] == E["simt"]
    with gpu_plan(a, "hg_tensor", 64, precision="fp32") as g:
        assert g.info()["proj_engine"] == E["simt"]  # the plain path stays on the staged kernel
    b = _acq(40, "u16", 1e4, seed=7)
    with gpu_plan(b, "hg_tensor", 16, precision="split", proj_engine="tensor") as g:
        # detector width not a multiple of 16: no tensor-core projection, streaming instead
        assert g.info()["proj_engine"] == E["stream"]
    c = _acq(32, "f64", None, seed=8)
    with gpu_plan(c, "hg_tensor", 16, precision="split") as g:
        assert g.info()["proj_engine"] == E["simt"]  # float64 frames


def test_out_of_range_float_frame_is_reported(torch_cuda):
    """A float32 value beyond the FP16 split range sets the device status word: the check
    reports it as unsupported, clears it, and the plan keeps working."""
    from paper_2212_01309_gb300 import wdd
    acq = _acq(64, "f32", 1e3, seed=9)
    F = synth.all_frames(acq)
    idx = synth.raster_indices(acq)
    bad = F[:4].copy()
    bad[2, 10, 20] = 1.0e5
    with gpu_plan(acq, "hg_tensor", 16, precision="split", max_batch=64,
                  proj_engine="tensor") as g:
        g.push(to_source(bad, "device"), idx[:4])
        with pytest.raises(wdd.WddError) as ei:
            g.check_device()
        assert ei.value.status == wdd.ERR_UNSUPPORTED
        g.check_device()                             # cleared
        g.reset()
        g.push(to_source(F, "device"), idx)
        g.check_device()


def _run(acq, F, idx, pushes, source_of=None, depth=1024, engine="tensor", **kw):
    # the device copy stays alive for the whole run: gathered pushes are read when launched
    d = to_source(F, "device")
    with gpu_plan(acq, "hg_tensor", 64, precision="split", max_batch=256, accum_depth=depth,
                  proj_engine=engine, **kw) as g:
        pos = 0
        pending_seen = 0
        for i, n in enumerate(pushes):
            src = source_of(i) if source_of else "device"
            g.push(d[pos:pos + n] if src == "device" else F[pos:pos + n], idx[pos:pos + n])
            pending_seen = max(pending_seen, g.info()["pending"])
            pos += n
        _, ph, _, _ = g.finalize()
        g.check_device()
        return g.copy_array("accum"), ph.cpu().numpy(), pending_seen


@pytest.mark.parametrize("engine", ["tensor", "stream"])
def test_coalesced_pushes_match_immediate(torch_cuda, engine):
    """Pushes gathered into shared launches (many small ones, more than 16 per launch, some
    crossing the 256-frame launch size) give bit-identical results to projecting every push
    when it is made, as long as the accumulation sees the same groups of frames (one flush at
    the end); with a 300-frame staging depth the flush points move and only rounding changes."""
    acq = _acq(128, "u16", 1e4, seed=15, scan=(24, 25))
    F = synth.all_frames(acq)
    idx = synth.raster_indices(acq)
    rng = np.random.default_rng(3)
    pushes = []
    left = len(idx)
    while left:
        n = int(min(left, rng.choice([1, 3, 7, 16, 64, 200, 256])))
        pushes.append(n)
        left -= n
    H0, ph0, p0 = _run(acq, F, idx, pushes, engine=engine)
    H1, ph1, p1 = _run(acq, F, idx, pushes, engine=engine, coalesce_frames=256)
    assert p0 == 0 and p1 > 0
    assert np.array_equal(H0, H1) and np.array_equal(ph0, ph1)
    # pageable pushes bypass the gathering (and launch what is pending first)
    H2, ph2, _ = _run(acq, F, idx, pushes, source_of=lambda i: "pageable" if i % 3 == 0 else "device",
                      engine=engine, coalesce_frames=128)
    assert np.array_equal(H0, H2) and np.array_equal(ph0, ph2)
    H3, ph3, _ = _run(acq, F, idx, pushes, depth=300, engine=engine, coalesce_frames=256)
    assert rel_l2(H3, H0) < 3e-6
    assert W.phase_rel_l2(ph3.astype(np.float64), ph0.astype(np.float64)) < 1e-5
