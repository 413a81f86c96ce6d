"""Scan rotation and the data-estimated detector centre in the oracle (CPU).

Pins (reading R15): with a circular probe, turning every detector image by a quarter turn
(numpy's rot90 over the detector axes) is the same measurement as a scan rotated by +90 degrees,
so reconstructing the turned frames with scan_rotation_rad = pi/2 must give the reconstruction of
the original frames with rotation 0; likewise half turns and pi.  On an odd detector the turn
keeps the zero frequency (and the basis centre) in place, so the identity is exact up to
rounding for the complete Fourier basis and the full Hermite-Gauss tensor basis.  A planted
rotation of the wrong sign must break it.  The centre of mass is pinned on discs whose centre is
known and on simulated frames.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle.wdd_oracle as W
import synth


def odd_acq(defocus_m=3e-9):
    acq, _ = synth.config("c1")
    return dataclasses.replace(acq, scan_y=9, scan_x=11, obj_y=18, obj_x=22, det=15,
                               defocus_m=defocus_m, dtype="f64", dose=None)


def reconstruct(acq, frames, basis, rank_k, rotation=0.0):
    p = W.Params.from_acquisition(acq, basis=basis, rank_k=rank_k, epsilon=1e-3,
                                  scan_rotation_rad=rotation)
    plan = W.build_plan(p)
    o = W.live_wdd(frames, synth.raster_indices(acq), plan)
    return W.finalize(o, p)


@pytest.mark.parametrize("basis,k", [("fourier_full", 225), ("hg_tensor", 16)])
@pytest.mark.parametrize("turns", [1, 2, 3])
def test_quarter_turns_of_the_detector_match_the_rotated_scan(basis, k, turns):
    acq = odd_acq()
    F = synth.all_frames(acq)
    obj0, ph0 = reconstruct(acq, F, basis, k)
    Fr = np.ascontiguousarray(np.rot90(F, k=turns, axes=(1, 2)))
    obj1, ph1 = reconstruct(acq, Fr, basis, k, rotation=turns * math.pi / 2)
    assert W.complex_rel_l2(obj1, obj0) < 1e-9
    assert W.phase_rel_l2(ph1, ph0) < 1e-9
    # the turned frames are not the original measurement: without the rotation they differ
    _, ph2 = reconstruct(acq, Fr, basis, k)
    assert W.phase_rel_l2(ph2, ph0) > 1e-2


def test_full_turn_is_no_rotation():
    acq = odd_acq()
    F = synth.all_frames(acq)
    _, a = reconstruct(acq, F, "hg_tensor", 16)
    _, b = reconstruct(acq, F, "hg_tensor", 16, rotation=2 * math.pi)
    assert W.phase_rel_l2(b, a) < 1e-10


def test_wrong_rotation_sign_is_caught(monkeypatch):
    """A planted mistake: the shift rotated by -theta instead of +theta."""
    orig = W.scan_shift_det_px

    def flipped(p, vy, vx):
        return orig(dataclasses.replace(p, scan_rotation_rad=-p.scan_rotation_rad), vy, vx)

    acq = odd_acq()
    F = synth.all_frames(acq)
    _, ph0 = reconstruct(acq, F, "fourier_full", 225)
    Fr = np.ascontiguousarray(np.rot90(F, k=1, axes=(1, 2)))
    monkeypatch.setattr(W, "scan_shift_det_px", flipped)
    _, ph1 = reconstruct(acq, Fr, "fourier_full", 225, rotation=math.pi / 2)
    assert W.phase_rel_l2(ph1, ph0) > 1e-2


def test_rotation_keeps_the_overlap_mask():
    acq = odd_acq()
    p0 = W.Params.from_acquisition(acq, basis="hg_tensor", rank_k=16, epsilon=1e-3)
    p1 = dataclasses.replace(p0, scan_rotation_rad=0.7)
    assert np.array_equal(W.active_mask(p0), W.active_mask(p1))
    # the rotated shift has the length of the scan-axis one
    qy, qx = W.scan_shift_px(p0)
    for vy, vx in [(1, 2), (3, 0), (8, 10)]:
        dy, dx = W.scan_shift_det_px(p1, vy, vx)
        assert abs(math.hypot(dy, dx) - math.hypot(qy[vy], qx[vx])) < 1e-12


def test_center_of_mass_of_known_discs():
    n = 32
    yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    for cy, cx in [(15.5, 15.5), (12.0, 19.0), (20.0, 9.0)]:
        disc = ((yy - cy) ** 2 + (xx - cx) ** 2 <= 36.0).astype(np.float64)
        got = W.detector_center_of_mass(disc[None])
        assert abs(got[0] - cy) < 1e-12 and abs(got[1] - cx) < 1e-12
        # weights scale out; several frames average
        got2 = W.detector_center_of_mass(np.stack([3 * disc, 5 * disc]))
        assert abs(got2[0] - cy) < 1e-12 and abs(got2[1] - cx) < 1e-12


def test_center_of_mass_of_simulated_frames():
    """Frames of a weak object keep the bright field centred on pixel N // 2."""
    acq = dataclasses.replace(odd_acq(), det=32, dtype="f32", dose=None)
    cy, cx = W.detector_center_of_mass(synth.all_frames(acq))
    assert abs(cy - 16.0) < 0.25 and abs(cx - 16.0) < 0.25


@pytest.mark.parametrize("turns", [1, 2, 3])
def test_quarter_turns_in_classical_wdd(turns):
    """The same identity through the classical route (Eq. 2-3): Y_v with the rotated shift, the
    detector transforms of the turned frames."""
    acq = odd_acq(defocus_m=5e-9)
    F = synth.all_frames(acq)
    p0 = W.Params.from_acquisition(acq, basis="fourier_full", rank_k=acq.det * acq.det,
                                   epsilon=1e-3)
    o0 = W.offline_wdd(F, p0)
    Fr = np.ascontiguousarray(np.rot90(F, k=turns, axes=(1, 2)))
    o1 = W.offline_wdd(Fr, dataclasses.replace(p0, scan_rotation_rad=turns * math.pi / 2))
    assert W.complex_rel_l2(o1, o0) < 1e-9
    # without the rotation the turned frames give another spectrum (compared without the
    # dominant v = 0 term)
    assert W.complex_rel_l2(W.offline_wdd(Fr, p0)[1:], o0[1:]) > 1e-2


@pytest.mark.parametrize("turns", [1, 3])
def test_quarter_turns_in_the_probe_swap(turns):
    """The identity through the swapped deconvolution (Sect. 10, readings R17-R19): the object
    estimate's spectrum is taken along the rotated scan axes, so the turned frames with the
    rotated scan return the probe spectrum of the original frames."""
    acq = odd_acq(defocus_m=5e-9)
    F = synth.all_frames(acq)
    p0 = W.Params.from_acquisition(acq, basis="fourier_full", rank_k=acq.det * acq.det,
                                   epsilon=1e-3)
    obj, _ = W.finalize(W.offline_wdd(F, p0), p0)
    pv0 = W.offline_probe_wdd(F, obj, p0)
    Fr = np.ascontiguousarray(np.rot90(F, k=turns, axes=(1, 2)))
    pr = dataclasses.replace(p0, scan_rotation_rad=turns * math.pi / 2)
    assert W.complex_rel_l2(W.offline_probe_wdd(Fr, obj, pr), pv0) < 1e-9
    assert W.complex_rel_l2(W.offline_probe_wdd(Fr, obj, p0)[1:], pv0[1:]) > 1e-2


def test_wrong_rotation_of_the_estimate_spectrum_is_caught(monkeypatch):
    """A planted mistake: the object estimate's spectrum taken along axes turned by -theta."""
    acq = odd_acq(defocus_m=5e-9)
    F = synth.all_frames(acq)
    p0 = W.Params.from_acquisition(acq, basis="fourier_full", rank_k=acq.det * acq.det,
                                   epsilon=1e-3)
    obj, _ = W.finalize(W.offline_wdd(F, p0), p0)
    pv0 = W.offline_probe_wdd(F, obj, p0)
    Fr = np.ascontiguousarray(np.rot90(F, k=1, axes=(1, 2)))
    pr = dataclasses.replace(p0, scan_rotation_rad=math.pi / 2)
    orig = W.scan_grid_spectrum_at
    monkeypatch.setattr(W, "scan_grid_spectrum_at", lambda X, p, ky, kx: orig(
        X, dataclasses.replace(p, scan_rotation_rad=-p.scan_rotation_rad), ky, kx))
    assert W.complex_rel_l2(W.offline_probe_wdd(Fr, obj, pr)[1:], pv0[1:]) > 1e-2
