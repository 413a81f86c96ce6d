"""Row-factorised accumulation (accum_mode="separable") against the FP64 oracle.

The separable mode computes the same accumulator H as Eq. 14, factorising the scan DFT by rows,
in FP32 on the SIMT cores, so it is held to the FP32 path's bounds: phase relative L2 <= 1e-5
and accumulator relative L2 <= 2e-6.  Cases cover ragged scans and detectors, every basis and
frame type, random order with duplicates (frames of many rows in one flush), partial scans,
snapshots during the scan, both projection paths, and a scan taller than 1024 rows (several rows
per thread in the slot scan).
"""
import dataclasses

import numpy as np
import pytest

import oracle.wdd_oracle as W
import synth
from wdd_harness import gpu_plan, oracle_params, phase_err, push_all, rel_l2, small_cases

pytestmark = pytest.mark.gpu

PHASE_TOL = 1e-5
ACCUM_TOL = 2e-6


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def _oracle(acq, basis, k, frames, idx):
    p = oracle_params(acq, basis, k)
    plan = W.build_plan(p)
    H = W.accumulate(W.coefficients(frames, plan), idx, p)
    _, ph = W.finalize(W.deconvolve(H, plan), p)
    return H, ph


@pytest.mark.parametrize("case", small_cases(), ids=lambda c: c.name)
@pytest.mark.parametrize("precision,depth", [("fp32", 0), ("fp32", 100), ("split", 128)])
def test_separable_parity(torch_cuda, case, precision, depth):
    acq = case.acq
    F = synth.all_frames(acq)
    idx = synth.raster_indices(acq)
    H_ref, ph_ref = _oracle(acq, case.basis, case.rank_k, F, idx)
    with gpu_plan(acq, case.basis, case.rank_k, precision=precision, max_batch=37,
                  accum_depth=depth, accum_mode="separable") as g:
        assert g.info()["accum_mode"] == 1
        push_all(g, F, idx, 37)
        _, ph, _, _ = g.finalize()
        g.check_device()
        H = g.copy_array("accum")
    assert rel_l2(H, H_ref) < ACCUM_TOL
    assert phase_err(ph.cpu().numpy(), ph_ref) < PHASE_TOL


def test_separable_random_order_duplicates_partial(torch_cuda):
    case = small_cases()[1]
    acq = case.acq
    F = synth.all_frames(acq)
    rng = np.random.default_rng(5)
    idx = rng.integers(0, acq.n_frames, size=500).astype(np.int32)   # duplicates, gaps
    fr = F[idx]
    H_ref, ph_ref = _oracle(acq, case.basis, case.rank_k, fr, idx)
    with gpu_plan(acq, case.basis, case.rank_k, max_batch=64, accum_depth=200,
                  accum_mode="separable") as g:
        for a in range(0, len(idx), 64):
            g.push(fr[a:a + 64], idx[a:a + 64])
            if a == 256:                                    # a snapshot half way
                g.snapshot()
        _, ph, seen, covered = g.finalize()
        H = g.copy_array("accum")
    assert seen == len(idx) and covered == len(np.unique(idx))
    assert rel_l2(H, H_ref) < ACCUM_TOL
    assert phase_err(ph.cpu().numpy(), ph_ref) < PHASE_TOL


def test_separable_matches_direct_fp32(torch_cuda):
    case = small_cases()[3]
    acq = case.acq
    F = synth.all_frames(acq)
    idx = synth.raster_indices(acq)
    with gpu_plan(acq, case.basis, case.rank_k, max_batch=64) as a, \
            gpu_plan(acq, case.basis, case.rank_k, max_batch=64, accum_depth=1024,
                     accum_mode="separable") as b:
        push_all(a, F, idx, 64)
        push_all(b, F, idx, 64)
        _, pa, _, _ = a.finalize()
        _, pb, _, _ = b.finalize()
        assert rel_l2(b.copy_array("accum"), a.copy_array("accum")) < ACCUM_TOL
        assert phase_err(pb.cpu().numpy(), pa.cpu().numpy().astype(np.float64)) < PHASE_TOL


def test_separable_tall_scan(torch_cuda):
    """1100 scan rows: the slot scan gives each of its 1024 threads two rows."""
    c1, _ = synth.config("c1")
    acq = dataclasses.replace(c1, scan_y=1100, scan_x=3, obj_y=2200, obj_x=22, det=16,
                              dtype="f32", dose=1e3, seed_noise=12)
    F = synth.all_frames(acq)
    idx = synth.raster_indices(acq)
    H_ref, ph_ref = _oracle(acq, "hg_tensor", 9, F, idx)
    with gpu_plan(acq, "hg_tensor", 9, max_batch=256, accum_depth=2048,
                  accum_mode="separable") as g:
        push_all(g, F, idx, 256)
        _, ph, _, _ = g.finalize()
        H = g.copy_array("accum")
    assert rel_l2(H, H_ref) < ACCUM_TOL
    assert phase_err(ph.cpu().numpy(), ph_ref) < PHASE_TOL
