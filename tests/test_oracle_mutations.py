"""Planted mistakes in the oracle must be caught by its pins (CPU only).

Each case swaps one oracle function for a plausible wrong variant (a flipped sign, a conjugate on
the wrong factor, a dropped final conjugation, a transposed operand, an unsigned frequency index, a
mis-centred basis) and checks that at least one of the pin quantities moves far outside its pinned
range.  The mistakes are planted in the oracle on the CPU only.
"""
import dataclasses

import numpy as np
import pytest

import oracle.wdd_oracle as W
import synth


def _acq(defocus):
    acq, _ = synth.config("c1")
    return dataclasses.replace(acq, scan_y=31, scan_x=31, obj_y=62, obj_x=62, defocus_m=defocus)


def _truth(acq):
    phi = synth.object_phase(acq)
    k = np.fft.fftfreq(acq.obj_y)
    KY, KX = np.meshgrid(k, k, indexing="ij")
    bl = np.real(np.fft.ifft2(np.fft.fft2(phi) * (KY ** 2 + KX ** 2 < 0.25 ** 2)))
    return bl[::2, ::2]


def pin_quantities():
    """The pinned quantities: live-vs-offline error, recovery correlation and conjugation error."""
    out = {}
    for defocus in (0.0, 8e-9):
        acq = _acq(defocus)
        phi = synth.object_phase(acq)
        idx = synth.raster_indices(acq)
        F = synth.all_frames(acq)
        Fc = synth.all_frames(acq, obj=np.exp(-1j * phi))
        truth = _truth(acq)
        for basis, k in (("fourier_full", acq.det ** 2), ("hg_tensor", 64)):
            p = W.Params.from_acquisition(acq, basis=basis, rank_k=k, epsilon=1e-3)
            plan = W.build_plan(p)
            o = W.live_wdd(F, idx, plan)
            obj, ph = W.finalize(o, p)
            out[f"r_{basis}_{defocus}"] = np.corrcoef(ph.ravel(), truth.ravel())[0, 1]
            if defocus == 0.0:
                objc, _ = W.finalize(W.live_wdd(Fc, idx, plan), p)
                out[f"conj_{basis}"] = W.complex_rel_l2(objc, np.conj(obj))
                if basis == "fourier_full":
                    out["live_vs_offline"] = W.complex_rel_l2(o, W.offline_wdd(F, p))
    return out


def caught(q):
    if any(not np.isfinite(v) for v in q.values()):
        return True
    bad = [k for k, v in q.items() if k.startswith("r_") and v < 0.85]
    bad += [k for k, v in q.items() if (k.startswith("conj_") or k == "live_vs_offline") and v > 1e-10]
    return bool(bad)


_orig = {n: getattr(W, n) for n in ("phase_factor", "finalize", "probe_autocorrelation",
                                    "scan_shift_px", "signed_freq", "hg_functions_1d",
                                    "project_operator", "probe_spectrum", "build_plan")}


def _y_conj_swapped(p, vy, vx):
    qy_all, qx_all = _orig["scan_shift_px"](p)
    qy = np.arange(p.det_y, dtype=np.float64) - p.cy
    qx = np.arange(p.det_x, dtype=np.float64) - p.cx
    ky, kx = np.meshgrid(qy, qx, indexing="ij")
    return np.conj(W.probe_spectrum(ky, kx, p)) * W.probe_spectrum(ky + qy_all[vy], kx + qx_all[vx], p)


def _no_final_conj(o, p):
    o = np.asarray(o).reshape(p.scan_y, p.scan_x)
    obj = np.fft.ifft2(o / np.sqrt(o[0, 0]))
    return obj, np.angle(obj)


def _fourier_pair_sign(p):
    plan = _orig["build_plan"](p)
    if p.basis == "fourier_full":
        plan.W = np.where(plan.comp[None, :] == 1, -plan.W, plan.W)
    return plan


MUTATIONS = {
    "scan kernel sign": ("phase_factor", lambda p, v, s: np.conj(_orig["phase_factor"](p, v, s))),
    "final conjugation dropped": ("finalize", _no_final_conj),
    "conjugate on the wrong probe factor": ("probe_autocorrelation", _y_conj_swapped),
    "probe shift direction": ("scan_shift_px", lambda p: tuple(-a for a in _orig["scan_shift_px"](p))),
    "unsigned frequency index": ("signed_freq", lambda v, n: np.asarray(v)),
    "basis centred one pixel off": ("hg_functions_1d", lambda n, L, s, c: _orig["hg_functions_1d"](n, L, s, c + 1.0)),
    "data transposed before projection": ("project_operator", lambda A, By, Bx: By.T @ A.T @ Bx),
    "defocus phase sign": ("probe_spectrum", lambda ky, kx, p: np.conj(_orig["probe_spectrum"](ky, kx, p))),
    "sin-row weight sign": ("build_plan", _fourier_pair_sign),
}


def test_unmutated_oracle_passes():
    assert not caught(pin_quantities())


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, monkeypatch):
    attr, fn = MUTATIONS[name]
    monkeypatch.setattr(W, attr, fn)
    with np.errstate(all="ignore"):
        q = pin_quantities()
    assert caught(q), (name, q)
