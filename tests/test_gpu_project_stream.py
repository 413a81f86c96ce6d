"""The streaming FP32 projection (proj_engine "stream", the split path's default where it
applies) against the FP64 oracle's projection.

Every product and sum is FP32 on FP32-rounded bases, so each batch's coefficients are held to
1e-6 relative L2.  Shapes cover detector widths whose four-column groups fill a warp exactly
(128), leave lanes of the warp idle (36, 48, 96), fold two row phases into a warp (64), take
teams of two and four warps per frame (144, 256, 512) and sixteen Hermite-Gauss functions per
axis (the register-heavy instance), with uint16 counts and float32 intensities,
from device, pinned and pageable memory; a float32 value far outside the FP16 range (which the
tensor-core projection must refuse) is projected like any other.
"""
import dataclasses

import numpy as np
import pytest

import oracle.wdd_oracle as W
import synth
from wdd_harness import gpu_plan, oracle_params, rel_l2, to_source

pytestmark = pytest.mark.gpu

COEFF_TOL = 1e-6


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
    ("f32_n128_energy128", 128, "f32", 1e4, "hg_energy", 128),
    ("u16_n36_energy20", 36, "u16", 2e3, "hg_energy", 20),
    ("u16_n64_hg36", 64, "u16", 1e3, "hg_tensor", 36),
    ("u16_n512_hg64", 512, "u16", 1e3, "hg_tensor", 64),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
@pytest.mark.parametrize("source", ["device", "pinned"])
def test_stream_projection_matches_oracle(torch_cuda, case, source):
    from paper_2212_01309_gb300 import wdd
    name, det, dtype, dose, basis, k = case
    acq = _acq(det, dtype, dose, seed=len(name))
    F = synth.all_frames(acq)
    idx = synth.raster_indices(acq)
    ref = W.coefficients(F, W.build_plan(oracle_params(acq, basis, k)))
    with gpu_plan(acq, basis, k, precision="split", max_batch=len(idx),
                  accum_depth=len(idx)) as g:
        assert g.info()["proj_engine"] == wdd.PROJ_ENGINE["stream"]
        g.push(to_source(F, source), idx)
        g.check_device()
        c = g.copy_array("coeff")
    assert c.shape == ref.shape
    assert rel_l2(c, ref) < COEFF_TOL


def test_sources_give_identical_coefficients(torch_cuda):
    acq = _acq(128, "f32", 1e4, seed=5)
    F = synth.all_frames(acq)
    idx = synth.raster_indices(acq)
    out = []
    for source in ("device", "pinned", "pageable"):
        with gpu_plan(acq, "hg_tensor", 64, precision="split", max_batch=len(idx),
                      accum_depth=len(idx)) as g:
            g.push(to_source(F, source), idx)
            g.check_device()
            out.append(g.copy_array("coeff"))
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


def test_large_float_values(torch_cuda):
    acq = _acq(64, "f32", 1e3, seed=9)
    F = synth.all_frames(acq)[:4].copy()
    F[2, 10, 20] = 1.0e5
    idx = synth.raster_indices(acq)[:4]
    ref = W.coefficients(F, W.build_plan(oracle_params(acq, "hg_tensor", 16)))
    with gpu_plan(acq, "hg_tensor", 16, precision="split", max_batch=64, accum_depth=64) as g:
        g.push(to_source(F, "device"), idx)
        g.check_device()
        c = g.copy_array("coeff")
    assert rel_l2(c, ref) < COEFF_TOL
