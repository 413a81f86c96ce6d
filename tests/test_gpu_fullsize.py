"""Full-size parity in the launch configuration the benchmark times.

128x128 scan / 128x128 float32 detector, Hermite-Gauss K = 64, 64-frame pushes gathered into
4096-frame projection launches, 4096 staged frames per tensor-core flush, pushes overlapped,
the whole acquisition captured once as a CUDA graph and replayed: the accumulator, the spectrum
and the phase against the oracle's full FP64 reconstruction of the same frames (the split path is
held to the FP32 path's phase bound, 1e-5, and 3e-5 on the accumulator).  The same step through
the row-factorised variant and the plain FP32 path.  At 256x256 scan / 128x128 uint16 detector,
K = 128 (65,536 frames) the oracle checks 64 sampled accumulator rows, each computed over every
frame.  The 512x512-scan / 256x256-detector uint16 acquisition (K = 256) streams its first 8,192
frames from pinned host memory in 512-frame pushes through the full-size plan; the oracle checks
64 sampled accumulator rows over those frames.
"""
import numpy as np
import pytest

import oracle.wdd_oracle as W
import synth
from wdd_harness import phase_err, rel_l2

pytestmark = pytest.mark.gpu

PHASE_TOL = 1e-5
ACCUM_TOL = 3e-5


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def _bases_plan(p, k):
    By, Bx, m_idx, comp, m_neg = W._bases(p)
    return W.OraclePlan(params=p, By=By, Bx=Bx, m_idx=m_idx, comp=comp, m_neg=m_neg,
                        chi=np.zeros((1, 1)), W=np.zeros((1, k)), mask=np.ones(1, bool),
                        eps_eff=0.0)


def _coefficients(frames, plan, n):
    return np.concatenate([W.coefficients(frames[a:a + 2048], plan) for a in range(0, n, 2048)])


@pytest.fixture(scope="module")
def c2_reference():
    acq, rc = synth.config("c2")
    frames = synth.all_frames(acq)
    idx = synth.raster_indices(acq)
    p = W.Params.from_acquisition(acq, basis=rc["basis"], rank_k=rc["rank_k"],
                                  epsilon=rc["epsilon"])
    plan = W.build_plan(p)
    H = W.accumulate(_coefficients(frames, plan, len(idx)), idx, p)
    o = W.deconvolve(H, plan)
    _, ph = W.finalize(o, p)
    return acq, rc, frames, idx, H, o, ph


def _graph_step(torch, plan, d_frames, idx, B, stream, obj, phase):
    S = len(idx)

    def step():
        plan.reset(stream=stream)
        for a in range(0, S, B):
            plan.push(d_frames[a:a + B], idx[a:a + B], stream=stream)
        plan.snapshot(obj, phase, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(2):
            step()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            step()
        g.replay()
        g.replay()
    torch.cuda.synchronize()


@pytest.mark.parametrize("variant", ["split", "separable", "fp32_plain"])
def test_c2_bench_configuration(torch_cuda, c2_reference, variant):
    torch = torch_cuda
    from paper_2212_01309_gb300 import wdd
    acq, rc, frames, idx, H_ref, o_ref, ph_ref = c2_reference
    B = rc["batch"]
    kw = dict(basis=rc["basis"], rank_k=rc["rank_k"], epsilon=rc["epsilon"], max_batch=B)
    if variant == "split":
        kw.update(precision="split", accum_depth=4096, overlap_pushes=True, coalesce_frames=4096)
    elif variant == "separable":
        kw.update(precision="split", accum_depth=4096, overlap_pushes=True, coalesce_frames=4096,
                  accum_mode="separable")
    else:
        kw.update(precision="fp32", accum_depth=0)
    d = torch.from_numpy(frames).cuda()
    stream = torch.cuda.Stream()
    obj = torch.empty((acq.scan_y, acq.scan_x), dtype=torch.complex64, device="cuda")
    phase = torch.empty((acq.scan_y, acq.scan_x), dtype=torch.float32, device="cuda")
    with wdd.Plan(wdd.params_from_acquisition(acq, **kw)) as g:
        if variant == "fp32_plain":
            with torch.cuda.stream(stream):
                g.reset(stream=stream)
                for a in range(0, len(idx), B):
                    g.push(d[a:a + B], idx[a:a + B], stream=stream)
                g.snapshot(obj, phase, stream=stream)
            torch.cuda.synchronize()
        else:
            assert g.info()["proj_engine"] == wdd.PROJ_ENGINE["stream"]
            _graph_step(torch, g, d, idx, B, stream, obj, phase)
        g.check_device()
        info = g.info()
        assert info["frames_seen"] == len(idx) and info["positions_covered"] == len(idx)
        H = g.copy_array("accum")
        o = g.copy_array("spectrum")
    assert rel_l2(H, H_ref) < ACCUM_TOL
    assert rel_l2(o, o_ref) < ACCUM_TOL
    assert phase_err(phase.cpu().numpy(), ph_ref) < PHASE_TOL


def test_c3_sampled_rows(torch_cuda):
    torch = torch_cuda
    from paper_2212_01309_gb300 import wdd
    from synth.torch_gen import TorchFrames
    acq, rc = synth.config("c3")
    d = TorchFrames(acq).all()
    frames = d.cpu().numpy()
    idx = synth.raster_indices(acq)
    B = rc["batch"]
    p = W.Params.from_acquisition(acq, basis=rc["basis"], rank_k=rc["rank_k"], epsilon=1e-3)
    C = _coefficients(frames, _bases_plan(p, rc["rank_k"]), len(idx))
    rows = np.sort(np.random.default_rng(7).choice(acq.n_frames, size=64, replace=False))
    H_ref = W.accumulate(C, idx, p, v_rows=rows)
    prm = wdd.params_from_acquisition(acq, basis=rc["basis"], rank_k=rc["rank_k"],
                                      precision="split", max_batch=B, accum_depth=4096,
                                      coalesce_frames=4096, overlap_pushes=True)
    stream = torch.cuda.Stream()
    with wdd.Plan(prm) as g, torch.cuda.stream(stream):
        for a in range(0, len(idx), B):
            g.push(d[a:a + B], idx[a:a + B], stream=stream)
        g.flush(stream=stream)
        torch.cuda.synchronize()
        g.check_device()
        H = g.copy_array("accum")
    assert rel_l2(H[rows], H_ref) < ACCUM_TOL


def test_c5_geometry_streamed_from_pinned_host(torch_cuda):
    """Full c5 geometry (S = 262,144 scan frequencies, 256x256 detector, K = 256, two coefficient
    tiles per CTA), frames pushed from pinned host memory in 512-frame batches: the first 8,192
    frames of the raster scan (a partial scan, as during an acquisition)."""
    torch = torch_cuda
    from paper_2212_01309_gb300 import wdd
    from synth.torch_gen import TorchFrames
    acq, rc = synth.config("c5")
    n = 8192
    B = rc["batch"]
    gen = TorchFrames(acq)
    h = torch.empty((n, acq.det, acq.det), dtype=torch.uint16).pin_memory()
    for b in range(n // 256):
        h[b * 256:(b + 1) * 256].copy_(gen.block(b).cpu())
    frames = h.numpy()
    idx = synth.raster_indices(acq)[:n]
    p = W.Params.from_acquisition(acq, basis=rc["basis"], rank_k=rc["rank_k"], epsilon=1e-3)
    C = _coefficients(frames, _bases_plan(p, rc["rank_k"]), n)
    rows = np.sort(np.random.default_rng(11).choice(acq.n_frames, size=64, replace=False))
    H_ref = W.accumulate(C, idx, p, v_rows=rows)
    prm = wdd.params_from_acquisition(acq, basis=rc["basis"], rank_k=rc["rank_k"],
                                      precision="split", max_batch=B, accum_depth=4096,
                                      coalesce_frames=4096, overlap_pushes=True)
    stream = torch.cuda.Stream()
    with wdd.Plan(prm) as g, torch.cuda.stream(stream):
        for a in range(0, n, B):
            g.push(h[a:a + B], idx[a:a + B], stream=stream)
        _, ph, seen, covered = g.finalize(stream=stream)
        torch.cuda.synchronize()
        g.check_device()
        H = g.copy_array("accum")
    assert seen == n and covered == n
    assert np.isfinite(ph.cpu().numpy()).all()
    assert rel_l2(H[rows], H_ref) < ACCUM_TOL
