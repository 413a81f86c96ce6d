"""Reconstruction without device allocation (wdd_reconstruct_noalloc).

Some callers cannot allocate device memory: code that runs while a CUDA graph is being captured,
real-time acquisition threads that must not block on the allocator, and applications whose device
memory is fixed up front by a pool or budget.  For them the library offers a reconstruction whose
working memory is a fixed array compiled into the library.  These tests call it through the C ABI
and compare it with the plan-based snapshot (the existing entry point) on the same weights and
accumulator, on consecutive calls, so that the shared scratch is known to be reused correctly.

This file is named to be collected last.
"""
import numpy as np
import pytest

import synth
from wdd_harness import gpu_plan, push_all, rel_l2, small_cases

pytestmark = pytest.mark.gpu

# Same kernels and summation order as the snapshot, so agreement is at FP32 rounding or better.
OBJ_TOL = 1e-6


def _snapshot_and_operands(case):
    import torch
    acq = case.acq
    frames = synth.all_frames(acq)
    idx = synth.raster_indices(acq)
    with gpu_plan(acq, case.basis, case.rank_k, max_batch=64) as plan:
        push_all(plan, frames, idx, 64)
        obj_ref, ph_ref, _, _ = plan.snapshot()
        torch.cuda.synchronize()
        W = torch.from_numpy(plan.copy_array("weights")).cuda()
        H = torch.from_numpy(plan.copy_array("accum")).cuda()
    return obj_ref.cpu().numpy(), ph_ref.cpu().numpy(), W, H


def _call(W, H, acq, rank_k):
    import torch
    from paper_2212_01309_gb300 import wdd
    obj = torch.full((acq.scan_y, acq.scan_x), float("nan"), dtype=torch.complex64, device="cuda")
    ph = torch.full((acq.scan_y, acq.scan_x), float("nan"), dtype=torch.float32, device="cuda")
    wdd.reconstruct_noalloc(W, H, acq.scan_y, acq.scan_x, rank_k, obj, ph)
    torch.cuda.synchronize()
    return obj.cpu().numpy(), ph.cpu().numpy()


def test_noalloc_matches_snapshot_on_consecutive_calls():
    import torch
    assert torch.cuda.is_available()
    a, b = small_cases()[0], small_cases()[2]       # 20 x 14 HG and 12 x 18 Fourier scans
    obj_a, ph_a, Wa, Ha = _snapshot_and_operands(a)
    obj_b, ph_b, Wb, Hb = _snapshot_and_operands(b)
    for case, ref_obj, ref_ph, W, H in ((a, obj_a, ph_a, Wa, Ha), (a, obj_a, ph_a, Wa, Ha),
                                        (b, obj_b, ph_b, Wb, Hb), (a, obj_a, ph_a, Wa, Ha)):
        obj, ph = _call(W, H, case.acq, case.rank_k)
        assert np.isfinite(obj).all() and np.isfinite(ph).all()
        assert rel_l2(obj, ref_obj) <= OBJ_TOL
        assert np.abs(ph - ref_ph).max() <= 1e-5


def test_noalloc_rejects_scans_beyond_its_scratch():
    import torch
    from paper_2212_01309_gb300 import wdd
    case = small_cases()[0]
    _, _, W, H = _snapshot_and_operands(case)
    obj = torch.empty((1024, 1024), dtype=torch.complex64, device="cuda")
    with pytest.raises(wdd.WddError) as ei:
        wdd.reconstruct_noalloc(W, H, 1024, 1024, case.rank_k, obj, None)
    assert ei.value.status == wdd.ERR_INVALID_ARG
    assert "scratch" in str(ei.value)
