"""Accuracy of the larger workloads against the FP64 oracle on a 64 x 64 scan crop.

The 256 x 256 scan / 128 x 128 uint16 detector workload (Hermite-Gauss energy basis, K = 128) and
the 512 x 512 scan / 256 x 256 uint16 detector workload (Hermite-Gauss tensor basis, K = 256) are
too large for a full FP64 reconstruction on the host, so each is reconstructed on a 64 x 64 scan
window at the scan origin: the same specimen, optics and frames (the crop's frames are the first
64 rows and columns of the full scan), with its own 64 x 64 scan DFT.  The oracle runs Algorithm 1
and Algorithm 2 in FP64 on the crop; the GPU runs the same crop in the launch configuration of the
streaming benchmark (split tensor-core path: 1024-frame projection launches gathered from the
workload's pushes, 4096 staged frames per flush, overlapped pushes) and through the plain FP32
path.  Bounds: phase relative L2 <= 2e-3 on the split path and <= 1e-5 on the FP32 path; the
accumulator and the deconvolved spectrum <= 3e-5 on both.

The serving mix (six sessions of different scan and detector sizes) is checked the same way on
the split path, one 64 x 64 crop per session (the whole scan for the 64 x 64 session), with the
sessions' pushes interleaved on separate streams as the serving loop issues them.
"""
import numpy as np
import pytest

import oracle.wdd_oracle as W
import synth
from wdd_harness import phase_err, rel_l2

pytestmark = pytest.mark.gpu

SPLIT_PHASE_TOL = 2e-3
FP32_PHASE_TOL = 1e-5
ACCUM_TOL = 3e-5


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def _oracle(acq, F, idx, basis, k):
    p = W.Params.from_acquisition(acq, basis=basis, rank_k=k, epsilon=1e-3)
    plan = W.build_plan(p)
    C = np.concatenate([W.coefficients(F[a:a + 1024], plan) for a in range(0, len(idx), 1024)])
    H = W.accumulate(C, idx, p)
    o = W.deconvolve(H, plan)
    _, ph = W.finalize(o, p)
    return H, o, ph


def _gpu(torch, acq, F, idx, basis, k, batch, precision):
    from paper_2212_01309_gb300 import wdd
    kw = dict(basis=basis, rank_k=k, epsilon=1e-3, max_batch=min(batch, 1024),
              precision=precision)
    if precision == "split":
        kw.update(accum_depth=4096, coalesce_frames=1024, overlap_pushes=True)
    d = torch.from_numpy(F).cuda()
    stream = torch.cuda.Stream()
    with wdd.Plan(wdd.params_from_acquisition(acq, **kw)) as g, torch.cuda.stream(stream):
        for a in range(0, len(idx), batch):
            g.push(d[a:a + batch], idx[a:a + batch], stream=stream)
        _, ph, seen, covered = g.finalize(stream=stream)
        torch.cuda.synchronize()
        g.check_device()
        assert seen == covered == len(idx)
        return g.copy_array("accum"), g.copy_array("spectrum"), ph.cpu().numpy()


@pytest.fixture(scope="module", params=["c3", "c5"])
def crop_case(request):
    acq, rc = synth.config(request.param)
    crop = acq.crop(64, 64)
    F = synth.all_frames(crop)
    idx = synth.raster_indices(crop)
    ref = _oracle(crop, F, idx, rc["basis"], rc["rank_k"])
    return request.param, crop, rc, F, idx, ref


@pytest.mark.parametrize("precision", ["split", "fp32"])
def test_crop_matches_oracle(torch_cuda, crop_case, precision):
    name, crop, rc, F, idx, (H_ref, o_ref, ph_ref) = crop_case
    H, o, ph = _gpu(torch_cuda, crop, F, idx, rc["basis"], rc["rank_k"], rc["batch"], precision)
    assert rel_l2(H, H_ref) < ACCUM_TOL, name
    assert rel_l2(o, o_ref) < ACCUM_TOL, name
    tol = SPLIT_PHASE_TOL if precision == "split" else FP32_PHASE_TOL
    assert phase_err(ph, ph_ref) < tol, name


def test_serving_sessions_crops_interleaved(torch_cuda):
    """Each session of the serving mix on a 64 x 64 crop, all six plans live at once on their own
    streams with their pushes interleaved in arrival order (batches of 16-512 frames), split
    path, against the oracle on each crop."""
    torch = torch_cuda
    from paper_2212_01309_gb300 import wdd
    mix = synth.serving_mix()
    crops, plans, streams, dev, refs = [], [], [], [], []
    for acq, rc in mix:
        crop = acq.crop(min(64, acq.scan_y), min(64, acq.scan_x))
        F = synth.all_frames(crop)
        idx = synth.raster_indices(crop)
        refs.append(_oracle(crop, F, idx, rc["basis"], rc["rank_k"]))
        crops.append((crop, idx))
        dev.append(torch.from_numpy(F).cuda())
        plans.append(wdd.Plan(wdd.params_from_acquisition(
            crop, basis=rc["basis"], rank_k=rc["rank_k"], epsilon=1e-3, precision="split",
            max_batch=512, accum_depth=2048, coalesce_frames=1024)))
        streams.append(torch.cuda.Stream())
    arrivals = synth.serving_arrivals([len(i) for _, i in crops], seed=404)
    try:
        for _, sid, start, count in arrivals:
            _, idx = crops[sid]
            plans[sid].push(dev[sid][start:start + count], idx[start:start + count],
                            stream=streams[sid])
        outs = [g.finalize(stream=s) for g, s in zip(plans, streams)]
        torch.cuda.synchronize()
        for sid, (g, (_, ph, seen, _)) in enumerate(zip(plans, outs)):
            g.check_device()
            H_ref, o_ref, ph_ref = refs[sid]
            assert seen == len(crops[sid][1])
            assert rel_l2(g.copy_array("accum"), H_ref) < ACCUM_TOL, sid
            assert phase_err(ph.cpu().numpy(), ph_ref) < SPLIT_PHASE_TOL, sid
    finally:
        for g in plans:
            g.close()
