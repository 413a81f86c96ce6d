"""Pins of the probe reconstruction (Sect. 10: the deconvolution run with the roles swapped) and of
the exact-recovery limit of WDD itself.

The pins use a noiseless periodic forward model written here from Eq. 1 alone: the object is
periodic with the detector's real-space period N dx and sampled at dx, the probe is any spectrum on
the detector grid, and the scan visits every object pixel (scan step dx, S_y = S_x = N).  Then
the scan frequencies fall on detector pixels and the scan transform of the frames is exactly
    G_v(q) = (S / N^4) sum_k f_v(q - k) g_v(k),  f_v(u) = A(u) conj A(u + v),
    g_v(k) = Psi(k) conj Psi(k - v),
with A and Psi the probe's and the object's spectra.  So F_q^-1(G_v) = (S / N^2) W_P W_O
pointwise, and a deconvolution by either factor recovers the other wherever it has no zero:
classical WDD returns Psi(0) conj Psi(-v) (the object, unit amplitude scale) and the swapped
deconvolution returns A(0) conj A(v) (the probe).  Every sign, shift, conjugate and
normalisation of both routes has to be right for these to hold to rounding.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle.wdd_oracle as W
import synth

N = 24
R_PX = 3.5


def exact_params(**kw):
    lam = W.electron_wavelength(300e3)
    theta = 0.02
    dk = theta / (R_PX * lam)
    base = dict(scan_y=N, scan_x=N, scan_step_m=1.0 / (N * dk), det_y=N, det_x=N, det_px_inv_m=dk,
                voltage_v=300e3, semiconv_rad=theta, defocus_m=3e-9, epsilon=1e-30,
                rank_k=N * N, basis="fourier_full", eps_absolute=True)
    base.update(kw)
    return W.Params(**base)


def centred_grid():
    q = (np.arange(N) - N // 2).astype(np.float64)
    return np.meshgrid(q, q, indexing="ij")


def forward_frames(A_centred, O):
    """Eq. 1 on the periodic grid: I_s = |F(P(r - r_s) O(r))|^2, stored with q = 0 at N//2."""
    P = np.fft.ifft2(np.fft.ifftshift(A_centred))
    frames = np.empty((N * N, N, N))
    for sy in range(N):
        for sx in range(N):
            psi = np.roll(P, (sy, sx), axis=(0, 1)) * O
            frames[sy * N + sx] = np.fft.fftshift(np.abs(np.fft.fft2(psi)) ** 2)
    return frames


def aberrated_probe(seed=2):
    """An arbitrary probe: the aperture disc with random phases, A(0) = 1."""
    rng = np.random.default_rng(seed)
    ky, kx = centred_grid()
    A = (ky * ky + kx * kx <= R_PX * R_PX) * np.exp(1j * rng.uniform(-np.pi, np.pi, (N, N)))
    A[N // 2, N // 2] = 1.0
    return A


def random_object(seed=2):
    rng = np.random.default_rng(seed)
    return np.exp(1j * rng.uniform(-1, 1, (N, N))) * (1 + 0.2 * rng.normal(size=(N, N)))


def rel(x, ref):
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


@pytest.fixture(scope="module")
def swap_case():
    A = aberrated_probe()
    O = random_object()
    return A, O, forward_frames(A, O)


def test_exact_object_recovery_with_unit_scale():
    """Classical WDD (Eq. 2-3) and live WDD with the full Fourier basis return the object itself,
    amplitude included, up to the global phase of Psi(0), when the object's spectrum lies where
    the probe's Wigner distribution has no zero (here |k| < 2.4 pixels) and epsilon -> 0."""
    p = exact_params()
    ky, kx = centred_grid()
    rng = np.random.default_rng(1)
    f = np.fft.fftfreq(N) * N
    fy, fx = np.meshgrid(f, f, indexing="ij")
    Psi = (rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))) * (fy ** 2 + fx ** 2 < 2.4 ** 2)
    Psi[0, 0] = 30.0 * np.exp(0.4j)
    O = np.fft.ifft2(Psi)
    frames = forward_frames(W.probe_spectrum(ky, kx, p), O)
    truth = np.exp(-0.4j) * O
    obj, _ = W.finalize(W.offline_wdd(frames, p), p)
    assert rel(obj, truth) < 1e-7
    obj_live, _ = W.finalize(W.live_wdd(frames, np.arange(N * N), W.build_plan(p)), p)
    assert rel(obj_live, truth) < 1e-6


def test_swapped_classical_wdd_recovers_the_probe(swap_case):
    A, O, frames = swap_case
    p = exact_params()
    spec, probe = W.probe_finalize(W.offline_probe_wdd(frames, O, p), p)
    assert rel(spec, np.fft.ifftshift(A)) < 1e-10
    assert rel(probe, np.fft.ifft2(np.fft.ifftshift(A))) < 1e-10


def test_swapped_live_wdd_recovers_the_probe(swap_case):
    """The live form (Algorithm 1 with Omega_v for Y_v, applied to the accumulator of Eq. 14)
    with the full Fourier basis equals the classical swap."""
    A, O, frames = swap_case
    p = exact_params()
    H = W.accumulate(W.coefficients(frames, W.build_plan(p)), np.arange(N * N), p)
    spec, _ = W.live_probe(H, O, p)
    assert rel(spec, np.fft.ifftshift(A)) < 1e-10
    ref = W.offline_probe_wdd(frames, O, p)
    assert rel(W.deconvolve(H, W.build_probe_plan(O, p)), ref) < 1e-10


def test_scan_grid_spectrum_is_fft2_at_scan_frequencies():
    """Reading R17: the trigonometric sum over the scan grid equals numpy's fft2 at the detector
    image of every scan frequency, with and without a scan rotation, and is periodic in the
    scan's reciprocal lattice."""
    rng = np.random.default_rng(4)
    for rot in (0.0, 0.37):
        p = W.Params(scan_y=6, scan_x=5, scan_step_m=2e-11, det_y=16, det_x=16,
                     det_px_inv_m=3e9, voltage_v=300e3, semiconv_rad=0.02, defocus_m=0.0,
                     epsilon=1e-3, rank_k=16, scan_rotation_rad=rot)
        X = rng.normal(size=(6, 5)) + 1j * rng.normal(size=(6, 5))
        ref = np.fft.fft2(X)
        for vy in range(6):
            for vx in range(5):
                ky, kx = W.scan_shift_det_px(p, vy, vx)
                assert abs(W.scan_grid_spectrum_at(X, p, ky, kx) - ref[vy, vx]) < 1e-11
        period = 1.0 / (p.det_px_inv_m * p.scan_step_m)     # one reciprocal period in pixels
        c, s = math.cos(rot), math.sin(rot)
        a = W.scan_grid_spectrum_at(X, p, 0.3, -1.1)
        b = W.scan_grid_spectrum_at(X, p, 0.3 + c * period, -1.1 + s * period)
        assert abs(a - b) < 1e-9 * abs(a)


def test_global_epsilon_swamps_a_weak_object():
    """Reading R20: for a weak phase object the object's autocorrelation at v != 0 is far below
    v = 0; a relative epsilon taken over all frequencies then erases the probe, one taken per
    frequency keeps it."""
    ky, kx = centred_grid()
    p = exact_params(epsilon=1e-3, eps_absolute=False)
    A = W.probe_spectrum(ky, kx, p)
    O = np.exp(0.1j * np.random.default_rng(5).uniform(-1, 1, (N, N)))
    frames = forward_frames(A, O)
    ref = np.fft.ifftshift(A)

    def err(spec):
        c = np.vdot(spec, ref) / np.vdot(spec, spec)
        return rel(c * spec, ref)

    spec, _ = W.probe_finalize(W.offline_probe_wdd(frames, O, p), p)
    assert err(spec) < 0.1
    H = W.accumulate(W.coefficients(frames, W.build_plan(p)), np.arange(N * N), p)
    one_max = W.build_plan(p, lambda vy, vx: W.object_autocorrelation(O, p, vy, vx))
    spec_bad, _ = W.probe_finalize(W.deconvolve(H, one_max), p)
    assert err(spec_bad) > 0.5
    spec_live, _ = W.live_probe(H, O, p)
    assert err(spec_live) < 0.1


def test_wiener_update_round_trip(swap_case):
    """Reading R21: the probe recovered from data made with the aperture model (defocus 3 nm)
    rebuilds the same Wiener filter as the model itself."""
    _, O, _ = swap_case
    ky, kx = centred_grid()
    p0 = exact_params()
    frames = forward_frames(W.probe_spectrum(ky, kx, p0), O)
    _, probe = W.probe_finalize(W.offline_probe_wdd(frames, O, p0), p0)
    p = exact_params(epsilon=1e-3, eps_absolute=False)
    model = W.build_plan(p)
    up = W.updated_plan(probe, p)
    assert rel(up.chi, model.chi) < 1e-9
    assert rel(up.W, model.W) < 1e-9


def test_probe_from_synthetic_workload():
    """32x32 scan at 2 object pixels, 32x32 detector, 20 nm defocus, peak phase 1 rad: the live
    swap with the full Fourier basis on the live object estimate finds the defocused probe at
    the scan frequencies that fall on detector pixels (the generator's probe is only defined
    there), far closer than the aperture without its defocus phase."""
    base, _ = synth.config("c1")
    acq = dataclasses.replace(base, obj_y=64, obj_x=64, defocus_m=20e-9, peak_phase=1.0)
    F = synth.all_frames(acq)
    idx = synth.raster_indices(acq)
    p = W.Params.from_acquisition(acq, basis="fourier_full", rank_k=acq.det ** 2, epsilon=1e-3)
    plan = W.build_plan(p)
    H = W.accumulate(W.coefficients(F, plan), idx, p)
    obj, _ = W.finalize(W.deconvolve(H, plan), p)
    spec, _ = W.live_probe(H, obj, p)
    fy, fx = W.scan_shift_px(p)
    ky, kx = np.meshgrid(fy, fx, indexing="ij")
    on_px = (np.abs(ky - np.rint(ky)) < 1e-9) & (np.abs(kx - np.rint(kx)) < 1e-9)
    sel = on_px & (ky * ky + kx * kx <= (0.8 * W.bright_field_radius_px(p)) ** 2)
    a = spec[sel]

    def err(b):
        c = np.vdot(a, b) / np.vdot(a, a)
        return rel(c * a, b)

    truth = W.probe_spectrum(ky, kx, p)[sel]
    assert err(truth) < 0.35
    assert err(np.abs(truth)) > 0.9


MUTATIONS = {
    # the object's autocorrelation shifted the wrong way
    "omega_shift_sign": ("object_autocorrelation",
                         lambda orig: lambda obj, p, vy, vx: _omega_plus(obj, p, vy, vx)),
    # the conjugate of the probe extraction dropped
    "extraction_conjugate": ("probe_finalize",
                             lambda orig: lambda pv, p: _finalize_no_conj(pv, p)),
    # the scan-grid spectrum taken with the wrong sign of the exponent
    "spectrum_sign": ("scan_grid_spectrum_at",
                      lambda orig: lambda X, p, ky, kx: orig(X, p, -np.asarray(ky), -np.asarray(kx))),
}


def _omega_plus(obj, p, vy, vx):
    dy, dx = W.scan_shift_det_px(p, vy, vx)
    ky, kx = centred_grid()
    return (W.scan_grid_spectrum_at(obj, p, ky, kx)
            * np.conj(W.scan_grid_spectrum_at(obj, p, ky + dy, kx + dx)))


def _finalize_no_conj(pv, p):
    pv = np.asarray(pv).reshape(p.scan_y, p.scan_x)
    spec = pv / np.sqrt(pv[0, 0])
    return spec, np.fft.ifft2(spec)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_probe_mistake_is_caught(name, monkeypatch, swap_case):
    A, O, frames = swap_case
    p = exact_params()
    attr, make = MUTATIONS[name]
    monkeypatch.setattr(W, attr, make(getattr(W, attr)))
    spec, _ = W.probe_finalize(W.offline_probe_wdd(frames, O, p), p)
    assert rel(spec, np.fft.ifftshift(A)) > 1e-2
