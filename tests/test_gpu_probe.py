"""Probe reconstruction on the GPU (Sect. 10): the deconvolution run with the roles of probe and
object swapped, and the live plan's Wiener filter rebuilt from a recovered probe.

The swapped classical plan (wdd_offline_probe_plan_create + wdd_offline_reconstruct) is held
against the oracle's offline_probe_wdd / probe_finalize on the same object estimate and frames.
Its arithmetic is the classical path's (FP32 transforms, the object spectrum's trigonometric sums
in FP64), so it takes that path's bound: 1e-5 relative L2 on the probe spectrum p_v and on the
probe.  Cases: the noiseless periodic model of Eq. 1 (every scan frequency on a detector pixel,
an aberrated probe, a random object; the swap also returns the true probe there), and a seeded
weak-phase acquisition whose object estimate is the classical reconstruction.

wdd_plan_set_probe is held against the oracle's updated_plan: chi_v (FP64 on both sides) to
1e-10, eps_eff to 1e-12 relative, the FP32-rounded Wiener weights to 1e-6, and the snapshot's
phase after the update against the oracle's deconvolution of the same accumulator to the FP32
path's 1e-5.  The accumulator is kept across the update, also on a finalized plan.
"""
import dataclasses

import numpy as np
import pytest

import oracle.wdd_oracle as W
import synth
from wdd_harness import oracle_params, phase_err, push_all, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


# ---- the noiseless periodic model of Eq. 1 (scan step = one object pixel, S_y = S_x = N) ----

N = 24
R_PX = 3.5


def _exact_params(eps=1e-3, eps_absolute=False):
    lam = W.electron_wavelength(300e3)
    theta = 0.02
    dk = theta / (R_PX * lam)
    return W.Params(scan_y=N, scan_x=N, scan_step_m=1.0 / (N * dk), det_y=N, det_x=N,
                    det_px_inv_m=dk, voltage_v=300e3, semiconv_rad=theta, defocus_m=3e-9,
                    epsilon=eps, rank_k=N * N, basis="fourier_full", eps_absolute=eps_absolute)


def _exact_frames(seed=5):
    """Frames |F(P(r - r_s) O(r))|^2 on the periodic grid, zero frequency at N // 2, for a
    probe with random phases inside the aperture and a random complex object."""
    rng = np.random.default_rng(seed)
    q = (np.arange(N) - N // 2).astype(np.float64)
    ky, kx = np.meshgrid(q, q, indexing="ij")
    A = (ky * ky + kx * kx <= R_PX * R_PX) * np.exp(1j * rng.uniform(-np.pi, np.pi, (N, N)))
    A[N // 2, N // 2] = 1.0
    O = np.exp(1j * rng.uniform(-1, 1, (N, N))) * (1 + 0.2 * rng.normal(size=(N, N)))
    P = np.fft.ifft2(np.fft.ifftshift(A))
    F = np.empty((N * N, N, N))
    for sy in range(N):
        for sx in range(N):
            psi = np.roll(P, (sy, sx), axis=(0, 1)) * O
            F[sy * N + sx] = np.fft.fftshift(np.abs(np.fft.fft2(psi)) ** 2)
    return A, O, F


def _gpu_params(p: W.Params, frame_dtype):
    from paper_2212_01309_gb300 import wdd
    return wdd.make_params(scan_y=p.scan_y, scan_x=p.scan_x, scan_step_m=p.scan_step_m,
                           det_y=p.det_y, det_x=p.det_x, det_px_inv_m=p.det_px_inv_m,
                           voltage_v=p.voltage_v, semiconv_rad=p.semiconv_rad,
                           defocus_m=p.defocus_m, epsilon=p.epsilon, rank_k=p.rank_k,
                           basis=p.basis, frame_dtype=frame_dtype, eps_absolute=p.eps_absolute)


def _gpu_probe(torch, prm, obj64, frames, obj_source="device"):
    """Runs the swapped classical plan; returns (p_v, probe, eps_eff) from the GPU."""
    from paper_2212_01309_gb300 import wdd
    o = torch.from_numpy(np.ascontiguousarray(obj64))
    o = o.cuda() if obj_source == "device" else o.pin_memory()
    with wdd.OfflinePlan(prm, obj=o) as g:
        probe, _ = g.reconstruct(torch.from_numpy(np.ascontiguousarray(frames)).cuda())
        torch.cuda.synchronize()
        return g.copy_array("spectrum"), probe.cpu().numpy(), g.info()["eps_eff"]


@pytest.mark.parametrize("eps,absolute", [(1e-3, False), (1e-6, True)])
def test_swap_exact_periodic_model(torch_cuda, eps, absolute):
    torch = torch_cuda
    A, O, F = _exact_frames()
    p = _exact_params(eps, absolute)
    obj64 = O.astype(np.complex64)
    pv_ref = W.offline_probe_wdd(F, obj64.astype(np.complex128), p)
    _, probe_ref = W.probe_finalize(pv_ref, p)
    pv, probe, eps_eff = _gpu_probe(torch, _gpu_params(p, "f64"), obj64, F)
    assert rel_l2(pv, pv_ref) < TOL
    assert rel_l2(probe, probe_ref) < TOL
    if absolute:
        assert eps_eff == pytest.approx(eps, rel=1e-6)
    # the swap recovers the probe itself on this model: conj(p_v / sqrt(p_0)) on the scan lattice
    # is the aperture function A at the matching detector pixels (A(0) = 1); with a negligible
    # absolute epsilon up to the FP32 transforms, with the relative one up to its regularisation
    spec = np.conj(pv.astype(np.complex128) / np.sqrt(complex(pv[0]))).reshape(N, N)
    ref = np.fft.ifftshift(A)
    assert rel_l2(spec, ref) < (1e-3 if absolute else 0.05)


def _weak_acq(scan=(16, 12), det=32, dtype="f32", dose=5e3, seed=31):
    c1, _ = synth.config("c1")
    return dataclasses.replace(c1, scan_y=scan[0], scan_x=scan[1], obj_y=2 * scan[0] + det,
                               obj_x=2 * scan[1] + det, det=det, defocus_m=6e-9, dtype=dtype,
                               dose=dose, seed_noise=seed)


@pytest.fixture(scope="module")
def weak_case():
    acq = _weak_acq()
    F = synth.all_frames(acq)
    p = oracle_params(acq, "hg_tensor", 1)
    obj, _ = W.finalize(W.offline_wdd(F, p), p)
    return acq, F, p, obj.astype(np.complex64)


def test_swap_weak_phase_acquisition(torch_cuda, weak_case):
    from paper_2212_01309_gb300 import wdd
    torch = torch_cuda
    acq, F, p, obj64 = weak_case
    pv_ref = W.offline_probe_wdd(F, obj64.astype(np.complex128), p)
    _, probe_ref = W.probe_finalize(pv_ref, p)
    prm = wdd.params_from_acquisition(acq, basis="hg_tensor", rank_k=1, epsilon=1e-3)
    pv, probe, _ = _gpu_probe(torch, prm, obj64, F)
    assert rel_l2(pv, pv_ref) < TOL
    assert rel_l2(probe, probe_ref) < TOL
    # an object estimate in pinned host memory gives the same bits
    pv2, probe2, _ = _gpu_probe(torch, prm, obj64, F, obj_source="pinned")
    assert np.array_equal(pv, pv2) and np.array_equal(probe, probe2)


def test_swap_rejects_bad_input(torch_cuda, weak_case):
    from paper_2212_01309_gb300 import wdd
    torch = torch_cuda
    acq, F, p, obj64 = weak_case
    prm = wdd.params_from_acquisition(acq, basis="hg_tensor", rank_k=1, scan_rotation_rad=0.2)
    with pytest.raises(wdd.WddError) as ei:
        wdd.OfflinePlan(prm, obj=torch.from_numpy(obj64).cuda())
    assert ei.value.status == wdd.ERR_UNSUPPORTED
    prm = wdd.params_from_acquisition(acq, basis="hg_tensor", rank_k=1)
    with pytest.raises(wdd.WddError) as ei:   # pageable host memory
        wdd.OfflinePlan(prm, obj=torch.from_numpy(obj64))
    assert ei.value.status == wdd.ERR_INVALID_ARG
    with pytest.raises(wdd.WddError) as ei:   # nothing to deconvolve by
        wdd.OfflinePlan(prm, obj=torch.zeros(obj64.shape, dtype=torch.complex64, device="cuda"))
    assert ei.value.status == wdd.ERR_INVALID_ARG


# ---- the Wiener filter rebuilt from a recovered probe ----------------------------------------

def _probe_estimate(p):
    """A probe on the scan grid: the model probe's spectrum on the scan lattice with a smooth
    phase error added, transformed to the scan grid (complex64)."""
    vy = np.fft.fftfreq(p.scan_y) * p.scan_y
    vx = np.fft.fftfreq(p.scan_x) * p.scan_x
    gy, gx = np.meshgrid(vy, vx, indexing="ij")
    spec = np.exp(1j * (0.3 * np.sin(0.4 * gy) + 0.2 * np.cos(0.3 * gx) + 0.05 * gx))
    return np.fft.ifft2(spec).astype(np.complex64)


@pytest.mark.parametrize("basis,k,finalize_first",
                         [("hg_tensor", 16, False), ("hg_energy", 10, True),
                          ("fourier_full", 24 * 24, False)])
def test_set_probe_matches_updated_plan(torch_cuda, basis, k, finalize_first):
    torch = torch_cuda
    det = 24 if basis == "fourier_full" else 32
    acq = _weak_acq(scan=(14, 18), det=det, dtype="u16", dose=2e3, seed=41)
    F = synth.all_frames(acq)
    idx = synth.raster_indices(acq)
    p = oracle_params(acq, basis, k)
    probe = _probe_estimate(p)
    ref = W.updated_plan(probe.astype(np.complex128), p)
    from wdd_harness import gpu_plan
    with gpu_plan(acq, basis, k, max_batch=64) as g:
        push_all(g, F, idx, 64)
        if finalize_first:
            g.finalize()
        H_before = g.copy_array("accum")
        g.set_probe(torch.from_numpy(probe).cuda())
        chi = g.copy_array("chi")
        Wt = g.copy_array("weights")
        info = g.info()
        _, ph, seen, _ = g.snapshot()
        torch.cuda.synchronize()
        H_after = g.copy_array("accum")
    assert np.array_equal(H_before, H_after) and seen == len(idx)
    assert rel_l2(chi, ref.chi) < 1e-10
    assert info["eps_eff"] == pytest.approx(float(ref.eps_eff), rel=1e-12)
    assert rel_l2(Wt, ref.W) < 1e-6
    _, ph_ref = W.finalize(W.deconvolve(H_after.astype(np.complex128), ref), p)
    assert phase_err(ph.cpu().numpy(), ph_ref) < TOL


def test_set_probe_with_model_probe_keeps_filter(torch_cuda):
    """On the periodic model, the model probe itself (its spectrum on the scan lattice is the
    aperture's at detector pixels) rebuilds the plan's own filter: weights unchanged to FP32
    rounding."""
    torch = torch_cuda
    from paper_2212_01309_gb300 import wdd
    p = _exact_params()
    q = (np.arange(N) - N // 2).astype(np.float64)
    ky, kx = np.meshgrid(q, q, indexing="ij")
    lam = p.wavelength_m
    A = (ky * ky + kx * kx <= R_PX * R_PX) * np.exp(
        -1j * np.pi * lam * p.defocus_m * p.det_px_inv_m ** 2 * (ky * ky + kx * kx))
    probe = np.fft.ifft2(np.fft.ifftshift(A)).astype(np.complex64)
    prm = _gpu_params(p, "f64")
    with wdd.Plan(prm) as g:
        W0 = g.copy_array("weights")
        g.set_probe(torch.from_numpy(probe).cuda())
        W1 = g.copy_array("weights")
    assert rel_l2(W1, W0) < 1e-6


def test_set_probe_rejects_bad_input(torch_cuda):
    torch = torch_cuda
    from paper_2212_01309_gb300 import wdd
    from wdd_harness import gpu_plan
    acq = _weak_acq(scan=(8, 8), det=32)
    with gpu_plan(acq, "hg_tensor", 16) as g:
        W0 = g.copy_array("weights")
        chi0 = g.copy_array("chi")
        with pytest.raises(wdd.WddError) as ei:   # pageable host memory
            g.set_probe(torch.zeros((8, 8), dtype=torch.complex64))
        assert ei.value.status == wdd.ERR_INVALID_ARG
        rot = wdd.params_from_acquisition(acq, basis="hg_tensor", rank_k=16,
                                          scan_rotation_rad=0.3)
        with wdd.Plan(rot) as g2, pytest.raises(wdd.WddError) as ei:
            g2.set_probe(torch.zeros((8, 8), dtype=torch.complex64, device="cuda"))
        assert ei.value.status == wdd.ERR_UNSUPPORTED
        # the failed calls left the filter as it was
        assert np.array_equal(g.copy_array("weights"), W0)
        assert np.array_equal(g.copy_array("chi"), chi0)
