"""Checkpoint/resume and partition merge on the GPU (wdd_merge_state; the merge by summation of
Sect. 6.3, which Eq. 14's linearity in the frames allows).

Two plans that see disjoint halves of an acquisition, merged into a fresh plan, give the plan that
saw every frame: the accumulator to FP32 rounding on the FP32 path (1e-6 relative L2: the two
halves are summed in a different order) and within the split path's accumulator bound (3e-5) on
the tensor-core path, whose FP16-split roundings fall differently per partition; hit counters
and frame counts exactly, and the phase within the FP32 path's 1e-5 of the single plan (and of
the oracle; 2e-3 for the split path).  A plan resumed from a checkpoint and fed the rest of
the frames ends the same way.  States are merged from pinned host memory and straight from
device memory, in stream order.  Refused merges (finalized plan, pageable accumulator, counters
that do not add up, a negative frame count, a counter overflow) change nothing.
"""
import dataclasses

import numpy as np
import pytest

import oracle.wdd_oracle as W
import synth
from wdd_harness import gpu_plan, oracle_params, phase_err, push_all, rel_l2

pytestmark = pytest.mark.gpu

ACCUM_TOL = 1e-6
PHASE_TOL = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


@pytest.fixture(scope="module")
def acquisition():
    c1, _ = synth.config("c1")
    acq = dataclasses.replace(c1, scan_y=20, scan_x=14, obj_y=40, obj_x=28, det=40,
                              defocus_m=4e-9, dtype="f32", dose=5e3, seed_noise=91)
    F = synth.all_frames(acq)
    idx = synth.raster_indices(acq)
    # a random order with repeats, so the halves overlap in positions
    rng = np.random.default_rng(5)
    order = np.concatenate([rng.permutation(len(idx)), rng.choice(len(idx), 60)])
    return acq, F[order], idx[order]


@pytest.mark.parametrize("precision", ["fp32", "split"])
def test_partition_merge_equals_single_plan(torch_cuda, acquisition, precision):
    torch = torch_cuda
    acq, F, idx = acquisition
    half = len(idx) // 2 + 7
    kw = dict(max_batch=64, precision=precision, accum_depth=0 if precision == "fp32" else 256)
    with gpu_plan(acq, "hg_tensor", 16, **kw) as full, \
            gpu_plan(acq, "hg_tensor", 16, **kw) as a, \
            gpu_plan(acq, "hg_tensor", 16, **kw) as b, \
            gpu_plan(acq, "hg_tensor", 16, **kw) as m:
        push_all(full, F, idx, 64)
        push_all(a, F[:half], idx[:half], 64)
        push_all(b, F[half:], idx[half:], 64)
        sa, sb = a.export_state(), b.export_state()
        m.merge_state(sa)                                   # numpy: pinned copy
        sb["accum"] = torch.from_numpy(sb["accum"]).cuda()  # straight from device memory
        m.merge_state(sb)
        _, ph_m, seen_m, cov_m = m.snapshot()
        _, ph_f, seen_f, cov_f = full.snapshot()
        torch.cuda.synchronize()
        assert seen_m == seen_f == len(idx) and cov_m == cov_f
        assert np.array_equal(m.hit_counts(), full.hit_counts())
        H_m, H_f = m.copy_array("accum"), full.copy_array("accum")
        assert rel_l2(H_m, H_f) < (ACCUM_TOL if precision == "fp32" else 3e-5)
        assert phase_err(ph_m.cpu().numpy(), ph_f.cpu().numpy().astype(np.float64)) < PHASE_TOL
    p = oracle_params(acq, "hg_tensor", 16)
    _, ph_ref = W.finalize(W.live_wdd(F, idx, W.build_plan(p)), p)
    assert phase_err(ph_m.cpu().numpy(), ph_ref) < (PHASE_TOL if precision == "fp32" else 2e-3)


def test_resume_from_checkpoint(torch_cuda, acquisition):
    torch = torch_cuda
    acq, F, idx = acquisition
    cut = 333
    with gpu_plan(acq, "hg_tensor", 16) as full, gpu_plan(acq, "hg_tensor", 16) as first:
        push_all(full, F, idx, 64)
        push_all(first, F[:cut], idx[:cut], 64)
        ckpt = first.export_state()
    with gpu_plan(acq, "hg_tensor", 16) as resumed, gpu_plan(acq, "hg_tensor", 16) as ref:
        push_all(ref, F, idx, 64)
        resumed.merge_state(ckpt)
        push_all(resumed, F[cut:], idx[cut:], 64)
        _, ph, seen, _ = resumed.finalize()
        _, ph_ref, _, _ = ref.finalize()
        torch.cuda.synchronize()
        assert seen == len(idx)
        assert np.array_equal(resumed.hit_counts(), ref.hit_counts())
        assert rel_l2(resumed.copy_array("accum"), ref.copy_array("accum")) < ACCUM_TOL
        assert phase_err(ph.cpu().numpy(), ph_ref.cpu().numpy().astype(np.float64)) < PHASE_TOL


def test_refused_merges_change_nothing(torch_cuda, acquisition):
    import ctypes
    torch = torch_cuda
    from paper_2212_01309_gb300 import wdd
    acq, F, idx = acquisition
    S = acq.scan_y * acq.scan_x
    with gpu_plan(acq, "hg_tensor", 16) as g:
        push_all(g, F[:100], idx[:100], 64)
        state = g.export_state()
        H0, hits0, seen0 = state["accum"], state["hits"], state["frames_seen"]
        acc = torch.from_numpy(H0).cuda()
        L = wdd.lib()

        def merge(accum_ptr, hits, frames):
            hits = np.ascontiguousarray(hits, dtype=np.uint32)
            return L.wdd_merge_state(g._h, ctypes.c_void_p(accum_ptr),
                                     ctypes.c_void_p(hits.ctypes.data), int(frames))

        bad = hits0.copy()
        bad[0] += 1
        assert merge(acc.data_ptr(), bad, seen0) == wdd.ERR_INVALID_ARG      # do not add up
        assert merge(acc.data_ptr(), hits0, -1) == wdd.ERR_INVALID_ARG       # negative count
        over = np.zeros(S, dtype=np.uint32)
        over[idx[0]] = 0xFFFFFFFF
        assert merge(acc.data_ptr(), over, 0xFFFFFFFF) == wdd.ERR_INVALID_ARG  # overflow
        assert merge(H0.ctypes.data, hits0, seen0) == wdd.ERR_INVALID_ARG    # pageable
        g.finalize()
        assert merge(acc.data_ptr(), hits0, seen0) == wdd.ERR_STATE          # finalized
        torch.cuda.synchronize()
        assert g.info()["frames_seen"] == seen0
        assert np.array_equal(g.hit_counts(), hits0)
        assert np.array_equal(g.copy_array("accum"), H0)
        # after a reset the plan takes the state: the same accumulator again
        g.reset()
        g.merge_state(state)
        torch.cuda.synchronize()
        assert np.array_equal(g.copy_array("accum"), H0)
        assert np.array_equal(g.hit_counts(), hits0)
        with pytest.raises(ValueError):
            other = dict(state, signature=(1, 2, 3, 4, 5, 6))
            g.merge_state(other)
