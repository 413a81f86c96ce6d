"""Classical (offline) WDD on the GPU against the FP64 oracle (Eq. 2-3).

The GPU path runs the 4-D transform in FP32 (twiddles and Y_v built in FP64), so it is held to
the FP32 path's bounds: spectrum and phase relative L2 <= 1e-5, the Wiener kernel to 1e-5.
Cases cover power-of-two and other scan and detector sizes (four-step, radix-2 and direct-DFT
transforms), detector planes that fit one CTA and ones that take the two-pass transform, every frame type,
device and pinned sources, a scan rotation, the absolute-epsilon mode, the live = classical
identity of the full Fourier basis on the GPU, and a 128^2 scan / 128^2 detector dataset checked
on sampled frequencies.
"""
import dataclasses

import numpy as np
import pytest

import oracle.wdd_oracle as W
import synth
from wdd_harness import gpu_plan, oracle_params, phase_err, push_all, rel_l2, to_source

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def _acq(scan, det, dtype="f32", dose=5e3, seed=3, defocus=3e-9):
    c1, _ = synth.config("c1")
    return dataclasses.replace(c1, scan_y=scan[0], scan_x=scan[1], obj_y=2 * scan[0] + det,
                               obj_x=2 * scan[1] + det, det=det, defocus_m=defocus, dtype=dtype,
                               dose=dose, seed_noise=seed)


def _offline_gpu(acq, frames, source="device", **kw):
    from paper_2212_01309_gb300 import wdd
    p = wdd.params_from_acquisition(acq, basis="hg_tensor", rank_k=1, epsilon=kw.pop("eps", 1e-3),
                                    **kw)
    with wdd.OfflinePlan(p) as g:
        t = frames if hasattr(frames, "data_ptr") else to_source(frames, source)
        obj, ph = g.reconstruct(t)
        o = g.copy_array("spectrum")
        info = g.info()
        n_elems = frames.numel() if hasattr(frames, "numel") else frames.size
        K = g.copy_array("wiener") if n_elems <= (1 << 22) else None
        return o, obj.cpu().numpy(), ph.cpu().numpy(), info, K


def _oracle(acq, frames, **kw):
    p = oracle_params(acq, "hg_tensor", 1, epsilon=kw.pop("eps", 1e-3), **kw)
    o = W.offline_wdd(frames, p)
    obj, ph = W.finalize(o, p)
    return p, o, obj, ph


CASES = [
    # scan, detector, frame type, fused detector plane
    ((16, 16), 32, "f32", 1),
    ((12, 18), 24, "u16", 1),       # direct DFT on both scan axes and the detector
    ((20, 14), 40, "f64", 1),
    ((8, 8), 256, "u16", 0),        # two-pass detector transform (four-step, 16 x 16)
    ((4, 4), 512, "f32", 0),        # two-pass detector transform (four-step, 32 x 16)
    ((6, 7), 120, "f32", 0),        # two-pass detector transform (direct DFT)
    ((32, 32), 128, "u16", 1),      # the 128-pixel detector of the bench
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0][0]}x{c[0][1]}_n{c[1]}_{c[2]}")
def test_offline_matches_oracle(torch_cuda, case):
    scan, det, dtype, fused = case
    acq = _acq(scan, det, dtype=dtype, dose=None if dtype == "f64" else 5e3, seed=det)
    F = synth.all_frames(acq)
    p, o_ref, obj_ref, ph_ref = _oracle(acq, F)
    o, obj, ph, info, K = _offline_gpu(acq, F)
    assert info["fused"] == fused
    assert info["n_active"] == int(W.active_mask(p).sum())
    assert rel_l2(o, o_ref) < TOL
    assert phase_err(ph, ph_ref) < TOL
    assert rel_l2(obj, obj_ref) < TOL
    if K is not None:
        WP = np.stack([W.offline_probe_wigner(p, vy, vx) for vy in range(p.scan_y)
                       for vx in range(p.scan_x)])
        eps = p.epsilon * float(np.max(np.abs(WP) ** 2))
        assert abs(info["eps_eff"] - eps) <= 1e-6 * eps
        K_ref = np.conj(WP) / (np.abs(WP) ** 2 + eps)
        K_ref[~W.active_mask(p)] = 0
        assert rel_l2(K.reshape(K_ref.shape), K_ref) < TOL


def test_offline_sources_and_rotation(torch_cuda):
    acq = _acq((16, 12), 32, dtype="u16", seed=4)
    F = synth.all_frames(acq)
    a = _offline_gpu(acq, F, source="device")
    b = _offline_gpu(acq, F, source="pinned")
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[2], b[2])
    _, o_ref, _, ph_ref = _oracle(acq, F, scan_rotation_rad=0.7)
    o, _, ph, _, _ = _offline_gpu(acq, F, scan_rotation_rad=0.7)
    assert rel_l2(o, o_ref) < TOL and phase_err(ph, ph_ref) < TOL
    _, o_ref, _, ph_ref = _oracle(acq, F, eps=0.3, eps_absolute=True)
    o, _, ph, info, _ = _offline_gpu(acq, F, eps=0.3, eps_absolute=True)
    assert info["eps_eff"] == 0.3
    assert rel_l2(o, o_ref) < TOL and phase_err(ph, ph_ref) < TOL


def test_live_fourier_equals_offline_on_gpu(torch_cuda):
    """The full Fourier basis makes live WDD reproduce classical WDD (reading R1): both GPU paths
    on the 32x32 scan / 32x32 detector workload agree to FP32 rounding."""
    acq, rc = synth.config("c1")
    F = synth.all_frames(acq)
    idx = synth.raster_indices(acq)
    o_off, _, ph_off, _, _ = _offline_gpu(acq, F)
    with gpu_plan(acq, "fourier_full", acq.det * acq.det, max_batch=64) as g:
        push_all(g, F, idx, 64)
        _, ph, _, _ = g.finalize()
        o_live = g.copy_array("spectrum")
    assert rel_l2(o_live, o_off) < TOL
    assert phase_err(ph.cpu().numpy(), ph_off.astype(np.float64)) < TOL


def test_offline_rejects_bad_input(torch_cuda):
    from paper_2212_01309_gb300 import wdd
    acq = _acq((8, 8), 32)
    p = wdd.params_from_acquisition(acq, basis="hg_tensor", rank_k=1, det_center_y=15.5)
    with pytest.raises(wdd.WddError) as ei:
        wdd.OfflinePlan(p)
    assert ei.value.status == wdd.ERR_UNSUPPORTED
    p = wdd.params_from_acquisition(acq, basis="hg_tensor", rank_k=1)
    with wdd.OfflinePlan(p) as g:
        F = synth.all_frames(acq)
        with pytest.raises(wdd.WddError) as ei:
            g.reconstruct(F)                     # pageable numpy array
        assert ei.value.status == wdd.ERR_INVALID_ARG


def test_offline_bench_size_sampled(torch_cuda):
    """128^2 scan / 128^2 float32 detector (the bench workload): sampled frequencies against
    the oracle's one-frequency route.  eps_eff = epsilon |W_P(0, 0)|^2, the maximum over all
    frequencies for an aperture of amplitude 1 (pinned in the oracle tests)."""
    from synth.torch_gen import TorchFrames
    acq, _ = synth.config("c2")
    frames = TorchFrames(acq).all()
    o, _, _, info, _ = _offline_gpu(acq, frames)
    F = frames.cpu().numpy().astype(np.float64)
    del frames
    idx = synth.raster_indices(acq)
    p = oracle_params(acq, "hg_tensor", 1)
    eps = p.epsilon * float(np.abs(W.offline_probe_wigner(p, 0, 0)[0, 0]) ** 2)
    assert abs(info["eps_eff"] - eps) <= 1e-6 * eps
    rng = np.random.default_rng(11)
    vs = [(0, 0), (1, 0), (0, 1), (5, 120)] + [tuple(rng.integers(0, 128, 2)) for _ in range(4)]
    ref = np.array([W.offline_wdd_frequency(F, idx, p, int(a), int(b), eps) for a, b in vs])
    got = np.array([o[a * 128 + b] for a, b in vs])
    assert np.max(np.abs(got - ref)) <= TOL * np.abs(ref).max()
