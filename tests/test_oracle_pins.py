"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU needed).

Each test names the passage it checks.  Together they are chosen so that a plausible mistake in
the oracle (a flipped sign of the scan kernel or the probe shift, a conjugate on the wrong factor,
a missing final conjugation, a transposed operand, a wrong frequency index, a mis-centred basis)
fails at least one of them; test_oracle_mutations.py plants such mistakes and checks that.
"""
import cmath
import dataclasses
import json
import math
import os

import numpy as np
import pytest

import oracle.wdd_oracle as W
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


def c1_odd(defocus_m=0.0):
    """Workload 1 geometry on a 31 x 31 scan (odd: no Nyquist bin), object 62 x 62."""
    acq, _ = synth.config("c1")
    return dataclasses.replace(acq, scan_y=31, scan_x=31, obj_y=62, obj_x=62,
                               defocus_m=defocus_m)


def params(acq, basis="fourier_full", rank_k=None, eps=1e-3, **kw):
    if rank_k is None:
        rank_k = acq.det * acq.det if basis == "fourier_full" else 64
    return W.Params.from_acquisition(acq, basis=basis, rank_k=rank_k, epsilon=eps, **kw)


def reconstruct(acq, p, obj=None):
    F = synth.all_frames(acq, obj=obj)
    idx = synth.raster_indices(acq)
    plan = W.build_plan(p)
    o = W.live_wdd(F, idx, plan)
    return o, W.finalize(o, p)


def bandlimited_truth(acq, kmax_cyc_per_px=0.25):
    """Object phase low-passed to the scan Nyquist (step 2 px) and sampled at scan positions."""
    phi = synth.object_phase(acq)
    ky = np.fft.fftfreq(acq.obj_y)
    kx = np.fft.fftfreq(acq.obj_x)
    KY, KX = np.meshgrid(ky, kx, indexing="ij")
    bl = np.real(np.fft.ifft2(np.fft.fft2(phi) * (KY ** 2 + KX ** 2 < kmax_cyc_per_px ** 2)))
    return bl[::acq.step_px, ::acq.step_px][:acq.scan_y, :acq.scan_x]


# ---- closed forms and printed values ------------------------------------------------------

def test_wavelength_matches_paper_example():
    g = _golden()["wavelength_200kV"]
    lam = W.electron_wavelength(g["voltage_v"])
    assert abs(lam - g["wavelength_m"]) / g["wavelength_m"] < g["rel_tol"]


def test_overlap_bound_matches_paper_example():
    g = _golden()["overlap_example"]
    r = W.overlap_bound_ratio(g["scan_step_m"], g["semiconv_rad"], g["wavelength_m"])
    assert round(r, g["digits"]) == g["s_hat_ratio"]


def test_hg_matches_hermite_polynomials():
    """Recurrence-built columns equal H_n(x/sigma) exp(-x^2/2sigma^2), normalised (Eq. 7)."""
    from numpy.polynomial import hermite as Hm
    for n_pts, L, sigma, c in [(64, 10, 5.3, 32.0), (97, 7, 9.1, 40.5), (33, 16, 3.0, 16.0)]:
        got = W.hg_functions_1d(n_pts, L, sigma, c)
        x = (np.arange(n_pts) - c) / sigma
        for n in range(L):
            coef = np.zeros(n + 1)
            coef[n] = 1.0
            ref = Hm.hermval(x, coef) * np.exp(-x * x / 2)
            ref /= np.linalg.norm(ref)
            assert np.allclose(got[:, n], ref, rtol=0, atol=1e-12), (n_pts, L, n)


def test_hg_orthonormal_when_well_sampled():
    B = W.hg_functions_1d(256, 12, 8.0, 128.0)
    assert np.allclose(B.T @ B, np.eye(12), atol=1e-12)


def test_hg_eigen_energies():
    """Rayleigh quotient of H = -d2/2 + x^2/(2 sigma^4) on psi_n gives sigma^-2 (n + 1/2) (Eq. 6)."""
    off = _golden()["hg_eigen_energy"]["offset_1d"]
    sigma, npts = 50.0, 1200
    B = W.hg_functions_1d(npts, 8, sigma, npts / 2)
    x = np.arange(npts) - npts / 2
    for n in range(8):
        f = B[:, n]
        d2 = np.zeros_like(f)
        # fourth-order central second difference (unit spacing)
        d2[2:-2] = (-f[4:] + 16 * f[3:-1] - 30 * f[2:-2] + 16 * f[1:-3] - f[:-4]) / 12.0
        Hf = -0.5 * d2 + x * x / (2 * sigma ** 4) * f
        E = float(f @ Hf / (f @ f))
        assert abs(E - (n + off) / sigma ** 2) / ((n + off) / sigma ** 2) < 1e-6, n


def test_hg_2d_energy_ordering():
    """Energy-ordered pairs follow E = sigma^-2 (n_y + n_x + 1) (Eq. 10)."""
    pairs = W.energy_pairs(21)
    energies = [a + b for a, b in pairs]
    assert energies == sorted(energies)
    assert pairs[:6] == [(0, 0), (0, 1), (1, 0), (0, 2), (1, 1), (2, 0)]
    assert W.hg_energy_l(128) == 16 and W.hg_energy_l(136) == 16 and W.hg_energy_l(137) == 17


def test_fourier_eigen_property():
    """Sampled psi_n with sigma^2 = N / (2 pi) is a DFT eigenvector with eigenvalue (-i)^n (Eq. 11)."""
    N = 256
    sigma = math.sqrt(N / (2 * math.pi))
    B = W.hg_functions_1d(N, 9, sigma, N / 2)
    for n in range(9):
        f = B[:, n]
        Ff = np.fft.fftshift(np.fft.fft(np.fft.ifftshift(f))) / math.sqrt(N)
        assert np.allclose(Ff, (-1j) ** n * f, atol=1e-10), n


def test_probe_autocorrelation_integer_shift():
    """Y_v = p(q) conj p(q + q_v) (Algorithm 1); for whole-pixel shifts it is a product of the
    simulator's probe grid with a rolled copy of itself."""
    acq, _ = synth.config("c1")
    acq = dataclasses.replace(acq, scan_y=8, scan_x=8, obj_y=16, obj_x=16, defocus_m=7e-9)
    p = params(acq)
    grid = synth.probe_fourier_grid(acq)
    qy, qx = W.scan_shift_px(p)
    for vy, vx in [(0, 0), (1, 0), (0, 3), (2, 5), (7, 7)]:
        sy, sx = int(round(qy[vy])), int(round(qx[vx]))
        assert abs(qy[vy] - sy) < 1e-12 and abs(qx[vx] - sx) < 1e-12
        shifted = np.roll(grid, (-sy, -sx), axis=(0, 1))
        # keep only points that did not wrap around the grid edge
        ok = np.ones_like(grid, dtype=bool)
        iy = np.arange(acq.det)[:, None] + sy
        ix = np.arange(acq.det)[None, :] + sx
        ok &= (iy >= 0) & (iy < acq.det) & (ix >= 0) & (ix < acq.det)
        ref = np.where(ok, grid * np.conj(shifted), 0)
        got = W.probe_autocorrelation(p, vy, vx)
        assert np.allclose(got, ref, atol=1e-14)


def test_projection_operator_brute_force():
    rng = np.random.default_rng(5)
    A = rng.normal(size=(5, 7))
    By = rng.normal(size=(5, 3)) + 1j * rng.normal(size=(5, 3))
    Bx = rng.normal(size=(7, 4)) + 1j * rng.normal(size=(7, 4))
    Z = W.project_operator(A, By, Bx)
    for a in range(3):
        for b in range(4):
            ref = sum(By[i, a] * A[i, j] * Bx[j, b] for i in range(5) for j in range(7))
            assert abs(Z[a, b] - ref) < 1e-12


def test_incremental_phase_sum_is_scan_dft():
    """sum_s F_2D[v, s] c_s (Eq. 14) equals numpy's 2-D FFT over the scan axes."""
    p = W.Params(scan_y=6, scan_x=10, scan_step_m=1e-10, det_y=4, det_x=4, det_px_inv_m=1e9,
                 voltage_v=3e5, semiconv_rad=0.02, defocus_m=0, epsilon=1e-3, rank_k=4)
    rng = np.random.default_rng(1)
    C = rng.normal(size=(60, 7))
    H = W.accumulate(C, np.arange(60), p)
    ref = np.fft.fft2(C.reshape(6, 10, 7), axes=(0, 1)).reshape(60, 7)
    assert np.allclose(H, ref, atol=1e-12)
    # split into partial sums in any order (Sect. 6.1)
    perm = rng.permutation(60)
    H2 = W.accumulate(C[perm[:17]], perm[:17], p) + W.accumulate(C[perm[17:]], perm[17:], p)
    assert np.allclose(H2, ref, atol=1e-12)


@pytest.mark.parametrize("basis,rank_k", [("fourier_full", 36), ("hg_tensor", 4), ("hg_energy", 5)])
def test_pipeline_equals_explicit_linear_operator(basis, rank_k):
    """o_v = sum_{s,q} E[v,s] I_s(q) sum_k W_v[k] P_k(q) by brute-force loops (Algorithm 2)."""
    acq, _ = synth.config("c1")
    acq = dataclasses.replace(acq, scan_y=3, scan_x=4, obj_y=6, obj_x=8, det=6)
    p = params(acq, basis=basis, rank_k=rank_k)
    plan = W.build_plan(p)
    rng = np.random.default_rng(3)
    I = rng.uniform(0, 2, size=(12, 6, 6))
    idx = np.arange(12)
    o = W.live_wdd(I, idx, plan)
    Lx = plan.Bx.shape[1]
    o_ref = np.zeros(12, dtype=complex)
    for v in range(12):
        vy, vx = divmod(v, 4)
        for s in range(12):
            sy, sx = divmod(s, 4)
            e = cmath.exp(-2j * math.pi * (vy * sy / 3 + vx * sx / 4))
            acc = 0
            for k in range(plan.K):
                ly, lx = divmod(int(plan.m_idx[k]), Lx)
                tot = 0
                for i in range(6):
                    for j in range(6):
                        b = plan.By[i, ly] * plan.Bx[j, lx]
                        tot += I[s, i, j] * (b.real if plan.comp[k] == 0 else b.imag)
                acc += plan.W[v, k] * tot
            o_ref[v] += e * acc
    assert np.allclose(o, o_ref, rtol=0, atol=1e-12 * np.abs(o_ref).max())


# ---- the four checks of the live reformulation ---------------------------------------------

def test_live_equals_offline_full_scan():
    """Fourier-basis live WDD equals classical WDD (Eq. 2, Eq. 3) on the full scan (check 1)."""
    for acq in (synth.config("c1")[0], c1_odd(defocus_m=6e-9)):
        p = params(acq)
        F = synth.all_frames(acq)
        o_live = W.live_wdd(F, synth.raster_indices(acq), W.build_plan(p))
        o_off = W.offline_wdd(F, p)
        assert W.complex_rel_l2(o_live, o_off) < 1e-10


def test_offline_per_frequency_equals_fft_route():
    """Classical WDD one frequency at a time (plain scan sum) equals the FFT route (Eq. 2-3), for
    active and inactive frequencies, with and without a scan rotation."""
    acq = c1_odd(defocus_m=4e-9)
    F = synth.all_frames(acq)
    idx = synth.raster_indices(acq)
    for rot in (0.0, 0.6):
        p = dataclasses.replace(params(acq), scan_rotation_rad=rot, epsilon=1e-2)
        o = W.offline_wdd(F, p)
        WP = np.stack([W.offline_probe_wigner(p, vy, vx) for vy in range(p.scan_y)
                       for vx in range(p.scan_x)])
        eps = p.epsilon * float(np.max(np.abs(WP) ** 2))
        for vy, vx in [(0, 0), (1, 0), (0, 3), (acq.scan_y - 1, 2), (4, acq.scan_x - 1)]:
            got = W.offline_wdd_frequency(F, idx, p, vy, vx, eps)
            ref = o[vy * p.scan_x + vx]
            assert abs(got - ref) <= 1e-11 * np.abs(o).max()


def test_offline_probe_wigner_peak_closed_form():
    """With an aperture of amplitude 1, |W_P(v, r)| <= (1/N^2) sum_q A(q) A(q + q_v) <= n_A / N^2,
    reached at v = 0, r = 0: max |W_P|^2 = (n_A / N^2)^2 with n_A the aperture pixel count."""
    acq = c1_odd(defocus_m=7e-9)
    p = params(acq)
    R = W.bright_field_radius_px(p)
    qy = np.arange(p.det_y) - p.cy
    qx = np.arange(p.det_x) - p.cx
    n_a = int(np.sum(qy[:, None] ** 2 + qx[None, :] ** 2 <= R * R))
    peak = max(float(np.max(np.abs(W.offline_probe_wigner(p, vy, vx)) ** 2))
               for vy in range(p.scan_y) for vx in range(p.scan_x))
    assert abs(peak - (n_a / (p.det_y * p.det_x)) ** 2) < 1e-14
    assert abs(W.offline_probe_wigner(p, 0, 0)[0, 0] - n_a / (p.det_y * p.det_x)) < 1e-14


def test_per_frame_equals_batched():
    """Algorithm 2 frame by frame equals the matrix form F_2D C (check 2)."""
    acq, _ = synth.config("c1")
    acq = dataclasses.replace(acq, scan_y=8, scan_x=6, obj_y=16, obj_x=12, det=16)
    for basis, k in [("fourier_full", 256), ("hg_energy", 10)]:
        p = params(acq, basis=basis, rank_k=k)
        plan = W.build_plan(p)
        F = synth.all_frames(acq)
        idx = synth.raster_indices(acq)
        a = W.live_wdd_per_frame(F, idx, plan)
        b = W.live_wdd(F, idx, plan)
        assert W.complex_rel_l2(a, b) < 1e-12


@pytest.mark.parametrize("shape", [(8, 6), (7, 9)])
def test_spectrum_of_real_coefficients_is_hermitian(shape):
    """H[-v, k] = conj(H[v, k]) for every scan frequency (Eq. 14 with real coefficients, for
    every basis family): the property the split path uses to accumulate only the scan columns
    v_x = 0 .. S_x / 2 and mirror the rest.  Checked on even and odd scan sides, with a random
    visiting order and repeated positions, against the oracle's own full accumulation."""
    acq, _ = synth.config("c1")
    acq = dataclasses.replace(acq, scan_y=shape[0], scan_x=shape[1], obj_y=2 * shape[0],
                              obj_x=2 * shape[1], det=16)
    rng = np.random.default_rng(11)
    for basis, k in [("fourier_full", 256), ("hg_energy", 10), ("hg_tensor", 16)]:
        p = params(acq, basis=basis, rank_k=k)
        plan = W.build_plan(p)
        F = synth.all_frames(acq)
        idx = synth.raster_indices(acq)
        order = np.concatenate([rng.permutation(len(idx)), rng.choice(len(idx), 7)])
        C = W.coefficients(F[order], plan)
        assert np.isrealobj(C)
        H = W.accumulate(C, idx[order], p).reshape(p.scan_y, p.scan_x, -1)
        neg = H[(-np.arange(p.scan_y)) % p.scan_y][:, (-np.arange(p.scan_x)) % p.scan_x]
        assert np.max(np.abs(neg - np.conj(H))) <= 1e-12 * np.max(np.abs(H))


@pytest.mark.parametrize("defocus", [0.0, 8e-9])
def test_weak_phase_object_recovered(defocus):
    """Noise-free weak phase object is recovered (check 3; validation protocol of Sect. 3)."""
    acq = c1_odd(defocus)
    truth = bandlimited_truth(acq)
    for basis, k, floor in [("fourier_full", None, 0.95), ("hg_tensor", 64, 0.90)]:
        p = params(acq, basis=basis, rank_k=k)
        _, (obj, ph) = reconstruct(acq, p)
        r = np.corrcoef(ph.ravel(), truth.ravel())[0, 1]
        assert r > floor, (basis, r)
        # orientation: the mirrored or rolled truth must correlate far worse
        assert np.corrcoef(ph.ravel(), truth[::-1, ::-1].ravel())[0, 1] < 0.5
        assert np.corrcoef(ph.ravel(), np.roll(truth, 3, axis=1).ravel())[0, 1] < 0.5


def test_reduced_rank_converges():
    """Keeping the K lowest-|r| Fourier rows converges to the full result as K grows (check 4)."""
    acq, _ = synth.config("c1")
    acq = dataclasses.replace(acq, scan_y=9, scan_x=9, obj_y=18, obj_x=18, det=16)
    p = params(acq)
    F = synth.all_frames(acq)
    idx = synth.raster_indices(acq)
    full = W.live_wdd(F, idx, W.build_plan(p))
    errs = []
    for k in (16, 48, 96, 160, 220, 256):
        o = W.live_wdd(F, idx, W.fourier_window_plan(p, k))
        errs.append(W.complex_rel_l2(o, full))
    assert all(b <= a * (1 + 1e-9) for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-12 and errs[0] > 1e-3


# ---- invariants ----------------------------------------------------------------------------

def test_invariant_scan_roll():
    """Shifting the object by one scan step rolls the reconstruction by one pixel."""
    acq = c1_odd(5e-9)
    phi = synth.object_phase(acq)
    for basis in ("fourier_full", "hg_tensor"):
        p = params(acq, basis=basis)
        _, (a, _) = reconstruct(acq, p, obj=np.exp(1j * phi))
        _, (b, _) = reconstruct(acq, p, obj=np.exp(1j * np.roll(phi, -acq.step_px, axis=1)))
        assert W.complex_rel_l2(b, np.roll(a, -1, axis=1)) < 1e-12


def test_invariant_conjugate_object():
    """Conjugating the object (real probe, defocus 0) conjugates the reconstruction (Sect. 3)."""
    acq = c1_odd(0.0)
    phi = synth.object_phase(acq)
    for basis, k in (("fourier_full", None), ("hg_tensor", 64), ("hg_energy", 128)):
        p = params(acq, basis=basis, rank_k=k)
        _, (a, _) = reconstruct(acq, p, obj=np.exp(1j * phi))
        _, (b, _) = reconstruct(acq, p, obj=np.exp(-1j * phi))
        assert W.complex_rel_l2(b, np.conj(a)) < 1e-12, basis


def test_invariant_vacuum():
    """A vacuum scan has no signal away from zero frequency."""
    acq = c1_odd(4e-9)
    for basis in ("fourier_full", "hg_tensor"):
        p = params(acq, basis=basis)
        o, _ = reconstruct(acq, p, obj=np.ones((acq.obj_y, acq.obj_x), dtype=complex))
        assert np.abs(o[1:]).max() < 1e-12 * abs(o[0])


def test_invariant_order_and_partition_merge():
    """Frame order does not matter and partial results merge by summation (Sect. 6.3 and the live-update figure of Sect. 9)."""
    acq, _ = synth.config("c1")
    F = synth.all_frames(acq)
    idx = synth.raster_indices(acq)
    plan = W.build_plan(params(acq, basis="hg_energy", rank_k=21))
    full = W.live_wdd(F, idx, plan)
    rng = np.random.default_rng(11)
    perm = rng.permutation(len(idx))
    assert W.complex_rel_l2(W.live_wdd(F[perm], idx[perm], plan), full) < 1e-12
    parts = np.array_split(perm, 3)
    merged = sum(W.live_wdd(F[q], idx[q], plan) for q in parts)
    assert W.complex_rel_l2(merged, full) < 1e-12


# ---- overlap criterion (Sect. 6.2) -----------------------------------------------------------

def test_active_mask_matches_disc_geometry():
    acq, _ = synth.config("c1")
    # a scan step of half a pixel puts the aperture-overlap edge inside the frequency grid
    p = W.Params(scan_y=16, scan_x=12, scan_step_m=0.5 * acq.dx_m, det_y=32, det_x=32,
                 det_px_inv_m=acq.det_px_inv_m, voltage_v=acq.voltage_v,
                 semiconv_rad=acq.semiconv_rad, defocus_m=0, epsilon=1e-3, rank_k=4)
    mask = W.active_mask(p).reshape(16, 12)
    qy, qx = W.scan_shift_px(p)
    R = W.bright_field_radius_px(p)
    assert 0 < mask.sum() < mask.size
    # brute force: do the two discs share interior points?  (sampled on a fine grid)
    g = np.linspace(-R, R, 801)
    GY, GX = np.meshgrid(g, g, indexing="ij")
    inside = GY ** 2 + GX ** 2 < R * R
    for vy in range(16):
        for vx in range(12):
            d2 = (GY + qy[vy]) ** 2 + (GX + qx[vx]) ** 2
            overlap = bool(np.any(inside & (d2 < R * R)))
            near_edge = abs(math.hypot(qy[vy], qx[vx]) - 2 * R) < 0.02 * R
            if not near_edge:
                assert overlap == bool(mask[vy, vx]), (vy, vx)
    # Eq. 17 is sufficient: every frequency within the square bound S_hat is active
    fy = W.signed_freq(np.arange(16), 16)
    fx = W.signed_freq(np.arange(12), 12)
    for vy in range(16):
        for vx in range(12):
            shat_y = W.overlap_bound_ratio(p.scan_step_m, p.semiconv_rad, p.wavelength_m) * 16
            shat_x = W.overlap_bound_ratio(p.scan_step_m, p.semiconv_rad, p.wavelength_m) * 12
            # Eq. 17 as printed uses one S for both axes; it is applied per axis here
            if max(abs(fy[vy]) / shat_y, abs(fx[vx]) / shat_x) <= 1 - 1e-9:
                assert mask[vy, vx]


def test_inactive_frequencies_are_zero():
    acq, _ = synth.config("c1")
    acq = dataclasses.replace(acq, scan_y=8, scan_x=8, obj_y=16, obj_x=16, det=16)
    p = dataclasses.replace(params(acq, basis="hg_tensor", rank_k=16), scan_step_m=0.5 * acq.dx_m)
    plan = W.build_plan(p)
    assert (~plan.mask).any()
    assert np.all(plan.W[~plan.mask] == 0)


def test_relative_epsilon_is_scale_free():
    """With the relative epsilon (reading R5) scaling the frames leaves the phase unchanged."""
    acq = c1_odd(3e-9)
    p = params(acq, basis="hg_tensor")
    F = synth.all_frames(acq)
    idx = synth.raster_indices(acq)
    plan = W.build_plan(p)
    _, a = W.finalize(W.live_wdd(F, idx, plan), p)
    _, b = W.finalize(W.live_wdd(17.0 ** 2 * F, idx, plan), p)
    assert np.allclose(a, b, atol=1e-12)


def test_live_equals_offline_non_square_detector():
    """A 24 x 32 detector: rows 4 .. 27 of 32 x 32 frames keep the zero frequency at
    (det_y // 2, det_x // 2); the full Fourier basis still reproduces classical WDD exactly."""
    acq = c1_odd(defocus_m=5e-9)
    acq = dataclasses.replace(acq, scan_y=9, scan_x=11, obj_y=18, obj_x=22)
    F = synth.all_frames(acq)[:, 4:28, :]
    p = W.Params(scan_y=acq.scan_y, scan_x=acq.scan_x, scan_step_m=acq.scan_step_m, det_y=24,
                 det_x=32, det_px_inv_m=acq.det_px_inv_m, voltage_v=acq.voltage_v,
                 semiconv_rad=acq.semiconv_rad, defocus_m=acq.defocus_m, epsilon=1e-3,
                 rank_k=24 * 32, basis="fourier_full")
    idx = synth.raster_indices(acq)
    o_live = W.live_wdd(F, idx, W.build_plan(p))
    o_off = W.offline_wdd(F, p)
    assert W.complex_rel_l2(o_live, o_off) < 1e-10
    # and it is not the square result: dropping detector rows changes the spectrum
    p_sq = dataclasses.replace(p, det_y=32, rank_k=32 * 32)
    o_sq = W.offline_wdd(synth.all_frames(acq), p_sq)
    assert W.complex_rel_l2(o_off, o_sq) > 1e-3


def test_classical_result_ignores_the_detector_roll(monkeypatch):
    """A common circular shift of the data and of Y_v multiplies both inverse detector transforms
    by the same phase ramp, which the conjugate in the Wiener kernel cancels: o_v does not depend
    on how the zero frequency is moved to index 0 (checked on an odd detector, where moving it by
    fftshift instead of ifftshift is a different roll)."""
    c1, _ = synth.config("c1")
    acq = dataclasses.replace(c1, scan_y=9, scan_x=11, obj_y=18, obj_x=22, det=15,
                              defocus_m=4e-9, dtype="f64", dose=None)
    F = synth.all_frames(acq)
    p = W.Params.from_acquisition(acq, basis="fourier_full", rank_k=15 * 15, epsilon=1e-3)
    ref = W.offline_wdd(F, p)
    assert not np.array_equal(np.fft.fftshift(np.arange(15)), np.fft.ifftshift(np.arange(15)))
    monkeypatch.setattr(W.np.fft, "ifftshift", lambda x, axes=None: np.fft.fftshift(x, axes=axes))
    assert W.complex_rel_l2(W.offline_wdd(F, p), ref) < 1e-12
