"""Split-precision tensor-core accumulation (tcgen05) against the FP64 oracle and the FP32 path.

Tolerances: the stated bound for the split path is a phase relative L2 <= 2e-3; the three-product
FP16 split carries about 22 significant bits, so the accumulator itself is also held to 3e-5
relative L2 to catch layout or scaling mistakes that a loose phase bound could hide.
"""
import dataclasses

import numpy as np
import pytest

import oracle.wdd_oracle as W
import synth
from wdd_harness import gpu_plan, oracle_params, phase_err, push_all, rel_l2, small_cases

pytestmark = pytest.mark.gpu

PHASE_TOL_SPLIT = 2e-3
ACCUM_TOL_SPLIT = 3e-5


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def _oracle(acq, basis, k, frames, idx):
    p = oracle_params(acq, basis, k)
    plan = W.build_plan(p)
    H = W.accumulate(W.coefficients(frames, plan), idx, p)
    obj, ph = W.finalize(W.deconvolve(H, plan), p)
    return H, ph


@pytest.mark.parametrize("case", small_cases(), ids=lambda c: c.name)
@pytest.mark.parametrize("depth", [0, 100])
def test_split_parity(torch_cuda, case, depth):
    acq = case.acq
    F = synth.all_frames(acq)
    idx = synth.raster_indices(acq)
    H_ref, ph_ref = _oracle(acq, case.basis, case.rank_k, F, idx)
    with gpu_plan(acq, case.basis, case.rank_k, precision="split", max_batch=45,
                  accum_depth=depth) as g:
        push_all(g, F, idx, 45)
        _, ph, _, _ = g.finalize()
        g.check_device()
        H = g.copy_array("accum")
        assert rel_l2(H, H_ref) < ACCUM_TOL_SPLIT
        assert phase_err(ph.cpu().numpy(), ph_ref) < PHASE_TOL_SPLIT


def test_split_equals_fp32_path_closely(torch_cuda):
    """Same frames through both paths: the split accumulator tracks the FP32 one."""
    case = small_cases()[3]
    acq = case.acq
    F = synth.all_frames(acq)
    idx = synth.raster_indices(acq)
    with gpu_plan(acq, case.basis, case.rank_k, max_batch=64) as a, \
            gpu_plan(acq, case.basis, case.rank_k, precision="split", max_batch=64,
                     accum_depth=512) as b:
        push_all(a, F, idx, 64)
        push_all(b, F, idx, 64)
        _, pa, _, _ = a.finalize()
        _, pb, _, _ = b.finalize()
        assert rel_l2(b.copy_array("accum"), a.copy_array("accum")) < ACCUM_TOL_SPLIT
        assert phase_err(pb.cpu().numpy(), pa.cpu().numpy().astype(np.float64)) < 1e-4


def test_split_random_order_duplicates(torch_cuda):
    case = small_cases()[0]
    acq = case.acq
    F = synth.all_frames(acq)
    rng = np.random.default_rng(21)
    idx = rng.integers(0, acq.n_frames, size=333).astype(np.int32)
    fr = F[idx]
    H_ref, ph_ref = _oracle(acq, case.basis, case.rank_k, fr, idx)
    with gpu_plan(acq, case.basis, case.rank_k, precision="split", max_batch=50,
                  accum_depth=160) as g:
        push_all(g, fr, idx, 50)
        _, ph, seen, _ = g.snapshot()
        g.check_device()
        assert seen == 333
        assert rel_l2(g.copy_array("accum"), H_ref) < ACCUM_TOL_SPLIT
        assert phase_err(ph.cpu().numpy(), ph_ref) < PHASE_TOL_SPLIT


def test_bounded_device_wait_gives_up(torch_cuda):
    """A device wait on a barrier nothing completes returns WDD_ERR_TIMEOUT; the context stays
    usable afterwards."""
    from paper_2212_01309_gb300 import wdd
    assert wdd.selftest_bounded_wait(50_000_000) == wdd.ERR_TIMEOUT
    case = small_cases()[0]
    F = synth.all_frames(case.acq)
    with gpu_plan(case.acq, case.basis, case.rank_k, precision="split", max_batch=64) as g:
        push_all(g, F, synth.raster_indices(case.acq), 64)
        g.finalize()
        g.check_device()
