"""Scan rotation and the data-estimated detector centre on the GPU against the FP64 oracle.

The rotation turns the scan-frequency shift inside the probe autocorrelation (reading R15); the
chi tables are built in FP64 on both sides and held to the same 1e-11 relative L2 as without a
rotation, the reconstruction to the FP32 path's phase bound.  A quarter turn of every detector
image with a +90 degree rotation must reproduce the unrotated reconstruction.  The centre of mass
(the centre of the basis sampling grid, Sect. 5) is a plain FP64 sum: held to 1e-12 pixels
against the oracle on every frame type and source, bit-reproducible between calls, and fed into
a plan whose reconstruction must match the oracle using the oracle's centre.
"""
import ctypes
import dataclasses
import math

import numpy as np
import pytest

import oracle.wdd_oracle as W
import synth
from wdd_harness import gpu_plan, oracle_params, phase_err, push_all, rel_l2, small_cases, to_source

pytestmark = pytest.mark.gpu

PHASE_TOL = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def _oracle(acq, basis, k, F, idx, **kw):
    p = oracle_params(acq, basis, k, **kw)
    plan = W.build_plan(p)
    H = W.accumulate(W.coefficients(F, plan), idx, p)
    _, ph = W.finalize(W.deconvolve(H, plan), p)
    return plan, ph


def _gpu(acq, basis, k, F, idx, precision="fp32", **kw):
    with gpu_plan(acq, basis, k, precision=precision, max_batch=64, **kw) as g:
        chi = g.copy_array("chi")
        Wg = g.copy_array("weights")
        push_all(g, F, idx, 64)
        _, ph, _, _ = g.finalize()
        g.check_device()
        return chi, Wg, ph.cpu().numpy()


@pytest.mark.parametrize("case_i,theta", [(0, 0.3), (1, -1.1), (2, math.pi / 2), (3, 2.5)])
def test_rotated_scan_matches_oracle(torch_cuda, case_i, theta):
    case = small_cases()[case_i]
    acq = case.acq
    F = synth.all_frames(acq)
    idx = synth.raster_indices(acq)
    plan, ph_ref = _oracle(acq, case.basis, case.rank_k, F, idx, scan_rotation_rad=theta)
    chi, Wg, ph = _gpu(acq, case.basis, case.rank_k, F, idx, scan_rotation_rad=theta)
    assert rel_l2(chi, plan.chi) < 1e-11
    assert np.abs(Wg - plan.W).max() <= 2e-7 * np.abs(plan.W).max()
    assert phase_err(ph, ph_ref) < PHASE_TOL
    if case_i < 3:                       # the rotation matters: the unrotated tables differ
        plan0 = W.build_plan(oracle_params(acq, case.basis, case.rank_k))
        assert rel_l2(plan0.chi, plan.chi) > 1e-3


def test_rotated_scan_split_path(torch_cuda):
    c2, _ = synth.config("c1")
    acq = dataclasses.replace(c2, scan_y=24, scan_x=20, obj_y=48 + 32, obj_x=40 + 32, det=64,
                              defocus_m=3e-9, dtype="u16", dose=1e4, seed_noise=31)
    F = synth.all_frames(acq)
    idx = synth.raster_indices(acq)
    _, ph_ref = _oracle(acq, "hg_tensor", 64, F, idx, scan_rotation_rad=0.8)
    _, _, ph = _gpu(acq, "hg_tensor", 64, F, idx, precision="split", accum_depth=256,
                    scan_rotation_rad=0.8)
    assert phase_err(ph, ph_ref) < PHASE_TOL


@pytest.mark.parametrize("turns", [1, 3])
def test_quarter_turn_of_the_detector_on_gpu(torch_cuda, turns):
    c1, _ = synth.config("c1")
    acq = dataclasses.replace(c1, scan_y=9, scan_x=11, obj_y=18, obj_x=22, det=15,
                              defocus_m=3e-9, dtype="f64", dose=None)
    F = synth.all_frames(acq)
    idx = synth.raster_indices(acq)
    _, _, ph0 = _gpu(acq, "hg_tensor", 16, F, idx)
    Fr = np.ascontiguousarray(np.rot90(F, k=turns, axes=(1, 2)))
    _, _, ph1 = _gpu(acq, "hg_tensor", 16, Fr, idx, scan_rotation_rad=turns * math.pi / 2)
    assert phase_err(ph1, ph0.astype(np.float64)) < PHASE_TOL
    _, _, ph2 = _gpu(acq, "hg_tensor", 16, Fr, idx)
    assert phase_err(ph2, ph0.astype(np.float64)) > 1e-2


def _frames(shape, dtype, seed):
    rng = np.random.default_rng(seed)
    n, ny, nx = shape
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    cy, cx = 0.37 * ny, 0.61 * nx
    disc = np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (0.1 * ny * nx))
    f = rng.poisson(200.0 * disc[None] * rng.uniform(0.5, 1.5, size=(n, 1, 1)))
    return f.astype(dtype)


@pytest.mark.parametrize("dtype", [np.uint16, np.float32, np.float64])
@pytest.mark.parametrize("source", ["device", "pinned"])
@pytest.mark.parametrize("shape", [(37, 33, 47), (3000, 16, 16), (2, 128, 128)])
def test_detector_center_matches_oracle(torch_cuda, dtype, source, shape):
    from paper_2212_01309_gb300 import wdd
    F = _frames(shape, dtype, seed=shape[0])
    ref = W.detector_center_of_mass(F)
    t = to_source(F, source)
    got = wdd.detector_center(t)
    assert abs(got[0] - ref[0]) < 1e-12 * shape[1] and abs(got[1] - ref[1]) < 1e-12 * shape[2]
    assert wdd.detector_center(t) == got                      # fixed reduction order


def test_detector_center_rejects_bad_input(torch_cuda):
    from paper_2212_01309_gb300 import wdd
    L = wdd.lib()
    cy, cx = ctypes.c_double(), ctypes.c_double()
    host = np.ones((2, 8, 8), np.float32)                     # pageable memory
    assert L.wdd_detector_center(ctypes.c_void_p(host.ctypes.data), 2, 8, 8, 1, ctypes.byref(cy),
                                 ctypes.byref(cx), None) == wdd.ERR_INVALID_ARG
    z = torch_cuda.zeros((2, 8, 8), dtype=torch_cuda.float32, device="cuda")
    with pytest.raises(wdd.WddError) as ei:
        wdd.detector_center(z)
    assert ei.value.status == wdd.ERR_INVALID_ARG
    assert L.wdd_detector_center(ctypes.c_void_p(z.data_ptr()), 0, 8, 8, 1, ctypes.byref(cy),
                                 ctypes.byref(cx), None) == wdd.ERR_INVALID_ARG


def test_plan_on_the_estimated_centre(torch_cuda):
    """A detector whose bright field is off centre: the centre of mass of the frames, given to
    the plan, reproduces the oracle's reconstruction built on the oracle's centre of mass."""
    from paper_2212_01309_gb300 import wdd
    case = small_cases()[0]
    acq = case.acq
    F = np.roll(synth.all_frames(acq), shift=(3, -2), axis=(1, 2))
    idx = synth.raster_indices(acq)
    ref_c = W.detector_center_of_mass(F)
    got_c = wdd.detector_center(to_source(F, "device"))
    assert abs(got_c[0] - ref_c[0]) < 1e-10 and abs(got_c[1] - ref_c[1]) < 1e-10
    assert abs(ref_c[0] - (acq.det // 2 + 3)) < 0.5 and abs(ref_c[1] - (acq.det // 2 - 2)) < 0.5
    _, ph_ref = _oracle(acq, case.basis, case.rank_k, F, idx, det_center_y=ref_c[0],
                        det_center_x=ref_c[1])
    _, _, ph = _gpu(acq, case.basis, case.rank_k, F, idx, det_center_y=got_c[0],
                    det_center_x=got_c[1])
    assert phase_err(ph, ph_ref) < PHASE_TOL
