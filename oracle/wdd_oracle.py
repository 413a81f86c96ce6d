"""FP64 CPU oracle of live Wigner Distribution Deconvolution (WDD), written from the paper.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this module.  It shares no code with the CUDA library.

Everything is float64 / complex128 numpy.  Library routines (numpy FFT, matmul) serve as single
steps; there is no blocking or reordering beyond what each cited equation or algorithm states.

Notation (Sect. 2): scan S = S_y x S_x positions s = s_y*S_x + s_x at r_s = (s_y, s_x) * step;
scan frequencies v = v_y*S_x + v_x; detector N_y x N_x pixels, frames stored with zero frequency
at pixel (c_y, c_x); K reduced coefficients per frame.

Readings of the paper (each one is also listed in the design notes):
  R1 Bases.  "fourier_full": real cos/sin rows of the detector inverse DFT (K = N_y*N_x), which
     makes the live method reproduce classical WDD exactly.  "hg_tensor": the operator H of
     Sect. 5 with L x L Hermite-Gauss functions.  "hg_energy": the first K tensor pairs ordered
     by the 2-D oscillator energy n_y + n_x (Eq. 10), ties by smaller n_y.
  R2 The reduced-space deconvolution is the element-wise product of Algorithm 1 and 2.
  R3 The 2-D eigenfunction is the tensor product of 1-D functions with sigma applied once.
  R4 Hermite-Gauss columns are built by the normalised three-term recurrence and rescaled to unit
     discrete L2 norm; sigma = R_bf / sqrt(2*(L-1)+1) with R_bf the bright-field radius in
     pixels, sampled at x_j = j - c (c = the detector centre N // 2 unless the caller passes
     another, e.g. detector_center_of_mass of the frames, Sect. 5).
  R5 epsilon is relative: eps_eff = epsilon * max_{v,m} |chi_v[m]|^2 (an absolute mode exists).
  R6 Eq. 3's division by sqrt(o_0) is applied (principal root; skipped when o_0 == 0), then the
     conjugated inverse DFT of Algorithm 2 with numpy's 1/S normalisation.
  R7 The sum over every element of D_v is the zero-frequency extraction, used as written.
  R8 A frequency is active iff the two aperture discs overlap: |q_v| < 2 theta / lambda (strict).
  R9 Sign conventions: P_s = p(r - r_s); scan kernel exp(-2 pi i q_v . r_s); Y_v(q) =
     p(q) conj p(q + q_v); probe p(k) = [|k| <= theta/lambda] exp(-i pi lambda df |k|^2).
  R15 Scan rotation (Tables 2 and 3): the scan-axis frequency (q_y, q_x) shifts the probe by
     (q_y cos t - q_x sin t, q_y sin t + q_x cos t) on the detector; t = +90 degrees equals the
     detector images turned by numpy's rot90 over their two axes.
  R17 An object or probe estimate lives on the scan grid; its spectrum at any detector-pixel
     frequency is the trigonometric sum over the scan positions (periodic in the scan's
     reciprocal lattice), which equals fft2 at the scan frequencies.
  R18 The object's counterpart of Y_v is Omega_v(q) = Psi(q) conj Psi(q - q_v): the scan
     transform of noiseless data is the convolution over q of Y_v and Omega_v.
  R19 Probe reconstruction (Sect. 10) runs Algorithm 1-2 (or Eq. 2) with Y_v replaced by
     Omega_v; the zero-frequency sum p_v then carries p(0) conj p(q_v), so the probe spectrum
     on the scan lattice is conj(p_v / sqrt(p_0)).  The updated Wiener filter takes Y_v from the
     recovered probe's spectrum at detector pixels (R17).
  R20 The swapped Wiener filter takes epsilon relative to each frequency's own maximum of
     |Omega_v| (reduced or per pixel): the object's autocorrelation at v != 0 is smaller than at
     v = 0 by the object's contrast squared, so one maximum over all v would swamp every v != 0.
  R21 The updated Wiener filter keeps the known condenser aperture (amplitude 1 for
     |k| <= theta / lambda) and takes only the phase inside it from the recovered probe.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "electron_wavelength", "overlap_bound_ratio", "Params", "signed_freq", "scan_shift_px",
    "bright_field_radius_px", "probe_spectrum", "probe_autocorrelation", "hg_functions_1d",
    "energy_pairs", "hg_energy_l", "OraclePlan", "build_plan", "project_operator",
    "coefficients", "phase_factor", "accumulate", "deconvolve", "finalize", "live_wdd",
    "live_wdd_per_frame", "offline_wdd", "offline_probe_wigner", "offline_wdd_frequency",
    "phase_rel_l2", "complex_rel_l2", "active_mask", "fourier_window_plan", "scan_shift_det_px",
    "detector_center_of_mass", "scan_grid_spectrum_at", "object_autocorrelation",
    "build_probe_plan", "probe_finalize", "live_probe", "offline_probe_wdd",
    "recovered_probe_spectrum_at", "recovered_probe_autocorrelation", "updated_plan",
]

# CODATA 2018 constants (SI).
PLANCK = 6.62607015e-34
ELECTRON_MASS = 9.1093837015e-31
ELEMENTARY_CHARGE = 1.602176634e-19
SPEED_OF_LIGHT = 299792458.0


# ---------------------------------------------------------------------------------------------
# Acquisition geometry (Sect. 6.2, Eq. 15-17)
# ---------------------------------------------------------------------------------------------

def electron_wavelength(voltage_v: float) -> float:
    """Relativistic de Broglie wavelength lambda(V) in metres.

    lambda = h / sqrt(2 m0 e V (1 + e V / (2 m0 c^2))).  Evaluated as a fixed sequence of
    correctly rounded IEEE operations.  Pinned by the 200 kV value 2.508 pm quoted in Sect. 6.2.
    """
    ev = ELEMENTARY_CHARGE * voltage_v
    rel = 1.0 + ev / (2.0 * ELECTRON_MASS * SPEED_OF_LIGHT * SPEED_OF_LIGHT)
    return PLANCK / math.sqrt(2.0 * ELECTRON_MASS * ev * rel)


def overlap_bound_ratio(step_m: float, semiconv_rad: float, wavelength_m: float) -> float:
    """S_hat / S = sqrt(2) * Delta * sin(theta) / lambda (Eq. 17).  Pinned by the 0.47 example."""
    return math.sqrt(2.0) * step_m * math.sin(semiconv_rad) / wavelength_m


@dataclasses.dataclass
class Params:
    """Acquisition and reconstruction parameters (the problem statement of Sect. 2)."""
    scan_y: int
    scan_x: int
    scan_step_m: float
    det_y: int
    det_x: int
    det_px_inv_m: float
    voltage_v: float
    semiconv_rad: float
    defocus_m: float
    epsilon: float
    rank_k: int
    basis: str = "hg_tensor"          # "fourier_full" | "hg_tensor" | "hg_energy"
    det_center_y: float | None = None  # default det_y // 2
    det_center_x: float | None = None
    eps_absolute: bool = False
    scan_rotation_rad: float = 0.0     # scan axes relative to the detector axes (reading R15)

    @property
    def S(self) -> int:
        return self.scan_y * self.scan_x

    @property
    def cy(self) -> float:
        return float(self.det_y // 2) if self.det_center_y is None else float(self.det_center_y)

    @property
    def cx(self) -> float:
        return float(self.det_x // 2) if self.det_center_x is None else float(self.det_center_x)

    @property
    def wavelength_m(self) -> float:
        return electron_wavelength(self.voltage_v)

    @staticmethod
    def from_acquisition(acq, basis: str, rank_k: int, epsilon: float, **kw) -> "Params":
        return Params(scan_y=acq.scan_y, scan_x=acq.scan_x, scan_step_m=acq.scan_step_m,
                      det_y=acq.det, det_x=acq.det, det_px_inv_m=acq.det_px_inv_m,
                      voltage_v=acq.voltage_v, semiconv_rad=acq.semiconv_rad,
                      defocus_m=acq.defocus_m, epsilon=epsilon, rank_k=rank_k, basis=basis, **kw)


def signed_freq(v: np.ndarray | int, n: int):
    """Signed DFT frequency index of bin v (numpy fftfreq ordering times n)."""
    v = np.asarray(v)
    return np.where(v <= (n - 1) // 2, v, v - n)


def scan_shift_px(p: Params) -> tuple[np.ndarray, np.ndarray]:
    """Detector-pixel shift q_v / dk of every scan frequency, per axis (Eq. 16 geometry).

    q_v = (f_y / (S_y * Delta), f_x / (S_x * Delta)) in reciprocal metres with signed
    frequencies f; dividing by the detector sampling dk gives pixels.
    """
    fy = signed_freq(np.arange(p.scan_y), p.scan_y).astype(np.float64)
    fx = signed_freq(np.arange(p.scan_x), p.scan_x).astype(np.float64)
    qy = fy / (p.scan_y * p.scan_step_m * p.det_px_inv_m)
    qx = fx / (p.scan_x * p.scan_step_m * p.det_px_inv_m)
    return qy, qx


def scan_shift_det_px(p: Params, vy, vx):
    """Shift of scan frequency (vy, vx) in detector pixels, along the detector axes.

    The scan frequency vector (q_y, q_x) of scan_shift_px is given along the scan axes; with the
    scan rotated by theta against the detector (the rotation of Tables 2 and 3) it points along
    (q_y cos theta - q_x sin theta, q_y sin theta + q_x cos theta) on the detector (reading R15:
    theta = +90 degrees is the detector image turned by numpy's rot90 over the last two axes).
    """
    qy, qx = scan_shift_px(p)
    a, b = qy[vy], qx[vx]
    c, s = math.cos(p.scan_rotation_rad), math.sin(p.scan_rotation_rad)
    return c * a - s * b, s * a + c * b


def detector_center_of_mass(frames: np.ndarray) -> tuple[float, float]:
    """Centre of mass (row, column) of the summed frames in detector pixels: the data-estimated
    centre for the basis sampling grid (Sect. 5)."""
    f = np.asarray(frames, dtype=np.float64).reshape(-1, *np.shape(frames)[-2:]).sum(axis=0)
    tot = f.sum()
    rows = np.arange(f.shape[0], dtype=np.float64)
    cols = np.arange(f.shape[1], dtype=np.float64)
    return float(f.sum(axis=1) @ rows / tot), float(f.sum(axis=0) @ cols / tot)


def bright_field_radius_px(p: Params) -> float:
    """Aperture radius theta / (lambda dk) in detector pixels."""
    return p.semiconv_rad / (p.wavelength_m * p.det_px_inv_m)


def active_mask(p: Params) -> np.ndarray:
    """Frequencies whose shifted aperture discs intersect: |q_v| < 2 R (reading R8, Eq. 15)."""
    qy, qx = scan_shift_px(p)
    r = bright_field_radius_px(p)
    d2 = qy[:, None] * qy[:, None] + qx[None, :] * qx[None, :]
    return (d2 < 4.0 * (r * r)).reshape(-1)


# ---------------------------------------------------------------------------------------------
# Probe and its autocorrelation (Eq. 2, Algorithm 1)
# ---------------------------------------------------------------------------------------------

def probe_spectrum(ky_px: np.ndarray, kx_px: np.ndarray, p: Params) -> np.ndarray:
    """Probe in reciprocal space, evaluated analytically at (possibly sub-pixel) points.

    p(k) = [|k|^2 <= R^2] * exp(-i pi lambda df dk^2 |k|^2), k in detector pixels, R the
    bright-field radius (Algorithm 1 initialisation: circular aperture).
    """
    r = bright_field_radius_px(p)
    k2 = ky_px * ky_px + kx_px * kx_px
    amp = (k2 <= r * r).astype(np.float64)
    lam = p.wavelength_m
    dk = p.det_px_inv_m
    coef = math.pi * lam * p.defocus_m * (dk * dk)
    return amp * np.exp(-1j * (coef * k2))


def probe_autocorrelation(p: Params, vy: int, vx: int) -> np.ndarray:
    """Y_v(q) = p(q) * conj p(q + q_v) on the detector grid (Algorithm 1, Eq. 2 W_P), q_v along
    the detector axes (scan_shift_det_px)."""
    dy, dx = scan_shift_det_px(p, vy, vx)
    qy = np.arange(p.det_y, dtype=np.float64) - p.cy
    qx = np.arange(p.det_x, dtype=np.float64) - p.cx
    ky, kx = np.meshgrid(qy, qx, indexing="ij")
    a = probe_spectrum(ky, kx, p)
    b = probe_spectrum(ky + dy, kx + dx, p)
    return a * np.conj(b)


# ---------------------------------------------------------------------------------------------
# Hermite-Gauss basis (Sect. 4, Sect. 5)
# ---------------------------------------------------------------------------------------------

def hg_functions_1d(n_pts: int, L: int, sigma: float, center: float) -> np.ndarray:
    """Sampled 1-D oscillator eigenfunctions psi_0..psi_{L-1} (Eq. 7), shape (n_pts, L).

    psi_n(x) is proportional to H_n(x / sigma) exp(-x^2 / (2 sigma^2)); the normalised three-term
    recurrence avoids overflowing H_n.  Each column is then scaled to unit discrete L2 norm
    (reading R4).  Pinned against numpy's Hermite polynomial evaluation and the oscillator
    eigen-energies of Eq. 6.
    """
    x = (np.arange(n_pts, dtype=np.float64) - center) / sigma
    out = np.zeros((n_pts, L), dtype=np.float64)
    out[:, 0] = math.pi ** -0.25 * np.exp(-0.5 * x * x)
    if L > 1:
        out[:, 1] = math.sqrt(2.0) * x * out[:, 0]
    for n in range(1, L - 1):
        out[:, n + 1] = math.sqrt(2.0 / (n + 1)) * x * out[:, n] - math.sqrt(n / (n + 1.0)) * out[:, n - 1]
    norms = np.sqrt((out * out).sum(axis=0))
    norms[norms == 0] = 1.0
    return out / norms


def energy_pairs(K: int) -> list[tuple[int, int]]:
    """First K index pairs (n_y, n_x) by 2-D oscillator energy n_y + n_x (Eq. 10), ties by n_y."""
    pairs = []
    e = 0
    while len(pairs) < K:
        for ny in range(e + 1):
            pairs.append((ny, e - ny))
            if len(pairs) == K:
                break
        e += 1
    return pairs


def hg_energy_l(K: int) -> int:
    """Number of 1-D functions the first K energy-ordered pairs need."""
    return 1 + max(max(a, b) for a, b in energy_pairs(K))


# ---------------------------------------------------------------------------------------------
# Plan: bases, coefficient table, pre-computed Wiener filter (Algorithm 1)
# ---------------------------------------------------------------------------------------------

@dataclasses.dataclass
class OraclePlan:
    params: Params
    By: np.ndarray          # (N_y, L_y) basis along detector rows (real or complex)
    Bx: np.ndarray          # (N_x, L_x)
    m_idx: np.ndarray       # (K,) flat index ly*L_x + lx of each coefficient
    comp: np.ndarray        # (K,) 0 = real part, 1 = imaginary part
    m_neg: np.ndarray       # (K,) flat index of -r (Fourier rows only; else = m_idx)
    chi: np.ndarray         # (S, M) complex projected probe autocorrelation, M = L_y * L_x
    W: np.ndarray           # (S, K) complex Wiener weights (zero on inactive v)
    mask: np.ndarray        # (S,) bool active frequencies
    eps_eff: float

    @property
    def K(self) -> int:
        return int(self.m_idx.shape[0])


def project_operator(A: np.ndarray, By: np.ndarray, Bx: np.ndarray) -> np.ndarray:
    """The reduction operator H of Sect. 5 (Eq. 12) on one detector image: Z = By^T A Bx.

    Z[ly, lx] = sum_{i,j} By[i, ly] A[i, j] Bx[j, lx].  (Sect. 5 writes psi_x^T A^T psi_y, the
    transpose of the same matrix; data and probe pass through the same map, so the orientation
    only relabels coefficients.)
    """
    return By.T @ A @ Bx


def _fourier_tables(ny: int, nx: int):
    m_idx, comp, m_neg = [], [], []
    for ry in range(ny):
        for rx in range(nx):
            m = ry * nx + rx
            n = ((-ry) % ny) * nx + ((-rx) % nx)
            if m > n:
                continue
            m_idx.append(m); comp.append(0); m_neg.append(n)
            if m != n:
                m_idx.append(m); comp.append(1); m_neg.append(n)
    return np.array(m_idx), np.array(comp), np.array(m_neg)


def _bases(p: Params):
    """Basis matrices and coefficient table for the chosen family (reading R1)."""
    if p.basis == "fourier_full":
        ry = np.arange(p.det_y)
        rx = np.arange(p.det_x)
        qy = np.arange(p.det_y, dtype=np.float64) - p.cy
        qx = np.arange(p.det_x, dtype=np.float64) - p.cx
        By = np.exp(2j * np.pi * np.outer(qy, ry) / p.det_y) / p.det_y
        Bx = np.exp(2j * np.pi * np.outer(qx, rx) / p.det_x) / p.det_x
        m_idx, comp, m_neg = _fourier_tables(p.det_y, p.det_x)
        if p.rank_k != m_idx.shape[0]:
            raise ValueError("fourier_full needs rank_k = det_y * det_x")
        return By, Bx, m_idx, comp, m_neg
    r = bright_field_radius_px(p)
    if p.basis == "hg_tensor":
        L = int(round(math.sqrt(p.rank_k)))
        if L * L != p.rank_k:
            raise ValueError("hg_tensor needs a square rank_k")
        pairs = [(a, b) for a in range(L) for b in range(L)]
    elif p.basis == "hg_energy":
        L = hg_energy_l(p.rank_k)
        pairs = energy_pairs(p.rank_k)
    else:
        raise ValueError(p.basis)
    sigma = r / math.sqrt(2.0 * (L - 1) + 1.0)
    By = hg_functions_1d(p.det_y, L, sigma, p.cy)
    Bx = hg_functions_1d(p.det_x, L, sigma, p.cx)
    m_idx = np.array([a * L + b for a, b in pairs])
    comp = np.zeros_like(m_idx)
    return By, Bx, m_idx, comp, m_idx.copy()


def build_plan(p: Params, autocorrelation=None, eps_per_frequency: bool = False) -> OraclePlan:
    """Algorithm 1: for every scan frequency v build Y_v, reduce it, form the Wiener filter.

    chi_v = H(Y_v) (complex), K_v = conj(chi_v) / (|chi_v|^2 + eps_eff), then the weights W_v[k]
    that multiply the real data coefficients: for the Hermite-Gauss families W_v[k] = K_v[m_k];
    for the Fourier family the cos/sin rows of r and -r are paired,
        W[cos r] = K(r) + K(-r)   (K(r) alone when r = -r),   W[sin r] = i (K(r) - K(-r)),
    which is the same sum over all r written with real coefficients.  Inactive v get W_v = 0.

    ``autocorrelation(vy, vx)`` replaces Y_v when given: the object's autocorrelation for the
    swapped deconvolution that recovers the probe, or the autocorrelation of a recovered probe
    for the updated Wiener filter (Sect. 10, readings R17-R21).  With ``eps_per_frequency`` the
    relative epsilon takes the maximum over each frequency's own coefficients (reading R20).
    """
    By, Bx, m_idx, comp, m_neg = _bases(p)
    M = By.shape[1] * Bx.shape[1]
    chi = np.zeros((p.S, M), dtype=np.complex128)
    for vy in range(p.scan_y):
        for vx in range(p.scan_x):
            if autocorrelation is None:
                Y = probe_autocorrelation(p, vy, vx)
            else:
                Y = autocorrelation(vy, vx)
            chi[vy * p.scan_x + vx] = project_operator(Y, By, Bx).reshape(-1)
    used = np.unique(np.concatenate([m_idx, m_neg]))
    if p.eps_absolute:
        eps_eff = p.epsilon
    elif eps_per_frequency:
        eps_eff = p.epsilon * np.max(np.abs(chi[:, used]) ** 2, axis=1, keepdims=True)
    else:
        eps_eff = p.epsilon * float(np.max(np.abs(chi[:, used]) ** 2))
    if eps_per_frequency:   # a frequency whose autocorrelation vanishes carries nothing: 0
        den = np.abs(chi) ** 2 + eps_eff
        Kv = np.divide(np.conj(chi), den, out=np.zeros_like(chi), where=den > 0)
    else:
        Kv = np.conj(chi) / (np.abs(chi) ** 2 + eps_eff)
    if p.basis == "fourier_full":
        self_conj = m_idx == m_neg
        Kr = Kv[:, m_idx]
        Kn = Kv[:, m_neg]
        W = np.where(comp[None, :] == 0, np.where(self_conj[None, :], Kr, Kr + Kn), 1j * (Kr - Kn))
    else:
        W = Kv[:, m_idx]
    mask = active_mask(p)
    W = np.where(mask[:, None], W, 0.0)
    return OraclePlan(params=p, By=By, Bx=Bx, m_idx=m_idx, comp=comp, m_neg=m_neg, chi=chi,
                      W=W, mask=mask, eps_eff=eps_eff)


def fourier_window_plan(p: Params, keep_k: int) -> OraclePlan:
    """Fourier family reduced to the keep_k coefficients of smallest |r| (reduced-rank check)."""
    full = build_plan(dataclasses.replace(p, basis="fourier_full", rank_k=p.det_y * p.det_x))
    Lx = p.det_x
    ry = full.m_idx // Lx
    rx = full.m_idx % Lx
    fy = signed_freq(ry, p.det_y)
    fx = signed_freq(rx, p.det_x)
    order = np.lexsort((np.arange(full.K), fy * fy + fx * fx))[:keep_k]
    order = np.sort(order)
    return dataclasses.replace(full, m_idx=full.m_idx[order], comp=full.comp[order],
                               m_neg=full.m_neg[order], W=full.W[:, order])


# ---------------------------------------------------------------------------------------------
# Streaming path (Algorithm 2, Eq. 14)
# ---------------------------------------------------------------------------------------------

def coefficients(frames: np.ndarray, plan: OraclePlan) -> np.ndarray:
    """Algorithm 2 step 1: c_s = vec(H(I_s)) as K real coefficients, shape (n, K)."""
    f = np.asarray(frames, dtype=np.float64)
    Z = np.einsum("iy,nij,jx->nyx", plan.By, f, plan.Bx, optimize=True)
    Z = Z.reshape(f.shape[0], -1)[:, plan.m_idx]
    return np.where(plan.comp[None, :] == 0, Z.real, Z.imag)


def phase_factor(p: Params, v: np.ndarray, s: np.ndarray) -> np.ndarray:
    """F_2D entries exp(-2 pi i (v_y s_y / S_y + v_x s_x / S_x)) from the two 1-D DFT matrices.

    Returns the (len(v), len(s)) sub-matrix (Algorithm 2: subset of F_2D for the frames at hand).
    """
    v = np.asarray(v, dtype=np.int64)
    s = np.asarray(s, dtype=np.int64)
    vy, vx = v // p.scan_x, v % p.scan_x
    sy, sx = s // p.scan_x, s % p.scan_x
    Fy = np.exp(-2j * np.pi * np.outer(vy, sy) / p.scan_y)
    Fx = np.exp(-2j * np.pi * np.outer(vx, sx) / p.scan_x)
    return Fy * Fx


def accumulate(C: np.ndarray, scan_idx: np.ndarray, p: Params,
               v_rows: np.ndarray | None = None, chunk: int = 2048) -> np.ndarray:
    """H[v, k] = sum_s F_2D[v, s] c_s[k]: Eq. 14 as one matrix product per row block.

    Returns H for the requested rows (all S by default), complex (len(v_rows), K).
    """
    if v_rows is None:
        v_rows = np.arange(p.S)
    C = np.asarray(C, dtype=np.float64)
    H = np.zeros((len(v_rows), C.shape[1]), dtype=np.complex128)
    for a in range(0, len(v_rows), chunk):
        E = phase_factor(p, v_rows[a:a + chunk], scan_idx)
        H[a:a + chunk] = E @ C
    return H


def deconvolve(H: np.ndarray, plan: OraclePlan, v_rows: np.ndarray | None = None) -> np.ndarray:
    """Algorithm 2: D_v = t_v o K_v, o_v = the sum over every element of D_v (reading R2, R7)."""
    W = plan.W if v_rows is None else plan.W[v_rows]
    return (W * H).sum(axis=1)


def finalize(o: np.ndarray, p: Params) -> tuple[np.ndarray, np.ndarray]:
    """Eq. 3 normalisation by sqrt(o_0), then conj(F^-1(O)) of Algorithm 2 (reading R6).

    Returns (complex object transfer function S_y x S_x, phase in radians).  The phase is pinned
    (weak-phase recovery, roll and conjugation invariants), and the amplitude scale by the exact
    recovery of an object from noiseless periodic data (unit scale, up to the phase of Psi(0)).
    """
    o = np.asarray(o, dtype=np.complex128).reshape(p.scan_y, p.scan_x)
    o0 = o[0, 0]
    scale = 1.0 / np.sqrt(o0) if o0 != 0 else 1.0
    obj = np.conj(np.fft.ifft2(o * scale))
    return obj, np.angle(obj)


def live_wdd(frames: np.ndarray, scan_idx: np.ndarray, plan: OraclePlan,
             chunk: int = 4096) -> np.ndarray:
    """Live WDD in batched matrix form: o = deconvolve(F_2D[:, s] @ C) over all frames."""
    p = plan.params
    C = np.concatenate([coefficients(frames[a:a + chunk], plan)
                        for a in range(0, frames.shape[0], chunk)], axis=0)
    H = accumulate(C, np.asarray(scan_idx), p)
    return deconvolve(H, plan)


def live_wdd_per_frame(frames: np.ndarray, scan_idx: np.ndarray, plan: OraclePlan) -> np.ndarray:
    """Algorithm 2 frame by frame: T = f_s i_s^T, D_v = mat(t_v) o K_v, o_v = sum, O += o."""
    p = plan.params
    O = np.zeros(p.S, dtype=np.complex128)
    allv = np.arange(p.S)
    active = np.nonzero(plan.mask)[0]
    for fr, s in zip(frames, scan_idx):
        i_s = coefficients(fr[None], plan)[0]
        f_s = phase_factor(p, allv, np.array([s]))[:, 0]
        T = np.outer(f_s, i_s)
        o = np.zeros(p.S, dtype=np.complex128)
        o[active] = (T[active] * plan.W[active]).sum(axis=1)
        O += o
    return O


# ---------------------------------------------------------------------------------------------
# Classical (offline) WDD, Eq. 2 and Eq. 3
# ---------------------------------------------------------------------------------------------

def offline_probe_wigner(p: Params, vy: int, vx: int) -> np.ndarray:
    """W_P(v, r) = F_q^-1(Y_v): the inverse detector DFT of the probe autocorrelation after moving
    q = 0 to index 0 (Eq. 2; numpy ifft2 normalisation)."""
    return np.fft.ifft2(np.fft.ifftshift(probe_autocorrelation(p, vy, vx)))


def offline_wdd_frequency(frames: np.ndarray, scan_idx: np.ndarray, p: Params, vy: int, vx: int,
                          eps_eff: float) -> complex:
    """o_v of classical WDD for one scan frequency, with the scan transform written as the plain
    sum G_v(q) = sum_s exp(-2 pi i q_v . r_s) I_s(q) over the given frames (Eq. 2), then
    W_O = F_q^-1(G_v) conj(W_P) / (|W_P|^2 + eps_eff) and o_v = sum_r W_O (Eq. 3).  Lets a large
    dataset be checked one frequency at a time; eps_eff is passed in (it is a maximum over all
    frequencies).  Inactive frequencies give 0."""
    if p.cy != p.det_y // 2 or p.cx != p.det_x // 2:
        raise ValueError("offline WDD assumes the detector centre at N//2")
    v = vy * p.scan_x + vx
    if not active_mask(p)[v]:
        return 0j
    E = phase_factor(p, np.array([v]), np.asarray(scan_idx))[0]
    I = np.asarray(frames, dtype=np.float64).reshape(len(E), -1)
    Gv = (E @ I).reshape(p.det_y, p.det_x)
    GP = np.fft.ifft2(np.fft.ifftshift(Gv))
    WP = offline_probe_wigner(p, vy, vx)
    return complex(np.sum(GP * np.conj(WP) / (np.abs(WP) ** 2 + eps_eff)))


def offline_wdd(frames: np.ndarray, p: Params) -> np.ndarray:
    """Classical WDD on the whole 4-D dataset; returns the spectrum o (S complex).

    G = F_rhat(I) (scan DFT), then per frequency: W_P = F_q^-1(Y_v), the data's F_q^-1(G_v),
    W_O = F_q^-1(G_v) conj(W_P) / (|W_P|^2 + eps_eff), o_v = F_r(W_O)|_{q=0} = sum_r W_O.
    Detector arrays are ifftshifted so their zero frequency sits at index 0 (this requires the
    detector centre to be at N//2).  Inactive frequencies (reading R8) are zeroed.
    """
    if p.cy != p.det_y // 2 or p.cx != p.det_x // 2:
        raise ValueError("offline WDD assumes the detector centre at N//2")
    I4 = np.asarray(frames, dtype=np.float64).reshape(p.scan_y, p.scan_x, p.det_y, p.det_x)
    G = np.fft.fft2(I4, axes=(0, 1))
    WP = np.empty((p.scan_y, p.scan_x, p.det_y, p.det_x), dtype=np.complex128)
    for vy in range(p.scan_y):
        for vx in range(p.scan_x):
            WP[vy, vx] = offline_probe_wigner(p, vy, vx)
    eps_eff = p.epsilon if p.eps_absolute else p.epsilon * float(np.max(np.abs(WP) ** 2))
    GP = np.fft.ifft2(np.fft.ifftshift(G, axes=(2, 3)), axes=(2, 3))
    WO = GP * np.conj(WP) / (np.abs(WP) ** 2 + eps_eff)
    o = WO.sum(axis=(2, 3)).reshape(-1)
    return np.where(active_mask(p), o, 0.0)


# ---------------------------------------------------------------------------------------------
# Probe reconstruction by swapping the deconvolution (Sect. 10), readings R17-R21
# ---------------------------------------------------------------------------------------------

def scan_grid_spectrum_at(X: np.ndarray, p: Params, ky_px, kx_px) -> np.ndarray:
    """Spectrum of an array given on the scan grid (an object or probe estimate), evaluated at
    detector-pixel frequencies (ky, kx) along the detector axes (reading R17).

    X(k) = sum_s X_s exp(-2 pi i dk k . r_s), with r_s = (s_y, s_x) * Delta the scan position
    turned onto the detector axes by the scan rotation (R15), so that dk k . r_s is the scan-axis
    frequency R^T k times the position.  At the detector image of a scan frequency q_v this is
    numpy's fft2 of X at v.
    """
    X = np.asarray(X, dtype=np.complex128).reshape(p.scan_y, p.scan_x)
    ky = np.asarray(ky_px, dtype=np.float64)
    kx = np.asarray(kx_px, dtype=np.float64)
    c, s = math.cos(p.scan_rotation_rad), math.sin(p.scan_rotation_rad)
    a = (c * ky + s * kx) * (p.det_px_inv_m * p.scan_step_m)   # cycles per scan step, scan y
    b = (-s * ky + c * kx) * (p.det_px_inv_m * p.scan_step_m)  # and scan x
    Ey = np.exp(-2j * np.pi * a[..., None] * np.arange(p.scan_y))
    Ex = np.exp(-2j * np.pi * b[..., None] * np.arange(p.scan_x))
    return np.einsum("...y,yx,...x->...", Ey, X, Ex, optimize=True)


def object_autocorrelation(obj: np.ndarray, p: Params, vy: int, vx: int) -> np.ndarray:
    """The object's counterpart of Y_v on the detector grid (reading R18):
    Omega_v(q) = Psi(q) conj Psi(q - q_v), Psi the spectrum of the object estimate
    (scan_grid_spectrum_at), q in pixels from the detector centre.  The data's scan transform is
    the convolution over q of Y_v with Omega_v, which is what lets the two swap roles."""
    dy, dx = scan_shift_det_px(p, vy, vx)
    qy = np.arange(p.det_y, dtype=np.float64) - p.cy
    qx = np.arange(p.det_x, dtype=np.float64) - p.cx
    ky, kx = np.meshgrid(qy, qx, indexing="ij")
    a = scan_grid_spectrum_at(obj, p, ky, kx)
    b = scan_grid_spectrum_at(obj, p, ky - dy, kx - dx)
    return a * np.conj(b)


def build_probe_plan(obj: np.ndarray, p: Params) -> OraclePlan:
    """Algorithm 1 with the roles swapped (Sect. 10): the Wiener filter of every scan frequency
    built from the reduced object autocorrelation instead of the probe's, with epsilon relative
    to each frequency's own maximum (reading R20) and the overlap mask of R8."""
    return build_plan(p, lambda vy, vx: object_autocorrelation(obj, p, vy, vx),
                      eps_per_frequency=True)


def probe_finalize(pv: np.ndarray, p: Params) -> tuple[np.ndarray, np.ndarray]:
    """Probe from the swapped deconvolution (reading R19).

    The zero-frequency sum of the deconvolved probe Wigner distribution at scan frequency v is
    p(0) conj p(q_v) times a constant, so the probe spectrum at the scan-lattice frequencies is
    conj(p_v / sqrt(p_0)) (principal root, skipped when p_0 == 0, as R6); its inverse DFT with
    numpy's 1/S is the probe on the scan grid.  Returns (spectrum, probe), both S_y x S_x, with
    the zero frequency and the probe's origin at index 0.
    """
    pv = np.asarray(pv, dtype=np.complex128).reshape(p.scan_y, p.scan_x)
    p0 = pv[0, 0]
    scale = 1.0 / np.sqrt(p0) if p0 != 0 else 1.0
    spec = np.conj(pv * scale)
    return spec, np.fft.ifft2(spec)


def live_probe(H: np.ndarray, obj: np.ndarray, p: Params) -> tuple[np.ndarray, np.ndarray]:
    """Probe from the live accumulator H (Eq. 14) and an object estimate: the swapped filter
    applied to H, the sum over every coefficient (R7), then probe_finalize."""
    return probe_finalize(deconvolve(H, build_probe_plan(obj, p)), p)


def offline_probe_wdd(frames: np.ndarray, obj: np.ndarray, p: Params) -> np.ndarray:
    """Classical WDD with the roles swapped (Eq. 2 with W_O and W_P exchanged, Sect. 10):
    W_O(v, r) = F_q^-1(Omega_v), W_P = F_q^-1(G_v) conj(W_O) / (|W_O|^2 + eps_eff),
    p_v = F_r(W_P)|_{q=0} = sum_r W_P; eps_eff(v) = epsilon * max_r |W_O(v, r)|^2 (reading R20;
    or absolute), inactive frequencies zeroed, and so is a frequency whose W_O vanishes
    everywhere (nothing to divide by).  Returns p (S complex) for probe_finalize."""
    if p.cy != p.det_y // 2 or p.cx != p.det_x // 2:
        raise ValueError("offline WDD assumes the detector centre at N//2")
    I4 = np.asarray(frames, dtype=np.float64).reshape(p.scan_y, p.scan_x, p.det_y, p.det_x)
    G = np.fft.fft2(I4, axes=(0, 1))
    WO = np.empty((p.scan_y, p.scan_x, p.det_y, p.det_x), dtype=np.complex128)
    for vy in range(p.scan_y):
        for vx in range(p.scan_x):
            WO[vy, vx] = np.fft.ifft2(np.fft.ifftshift(object_autocorrelation(obj, p, vy, vx)))
    if p.eps_absolute:
        eps_eff = p.epsilon
    else:
        eps_eff = p.epsilon * np.max(np.abs(WO) ** 2, axis=(2, 3), keepdims=True)
    GP = np.fft.ifft2(np.fft.ifftshift(G, axes=(2, 3)), axes=(2, 3))
    den = np.abs(WO) ** 2 + eps_eff
    K = np.divide(np.conj(WO), den, out=np.zeros_like(WO), where=den > 0)
    WP = GP * K
    pv = WP.sum(axis=(2, 3)).reshape(-1)
    return np.where(active_mask(p), pv, 0.0)


def recovered_probe_spectrum_at(probe: np.ndarray, p: Params, ky_px, kx_px) -> np.ndarray:
    """A recovered probe as a probe model for Algorithm 1 (reading R21): the condenser aperture
    is kept, |k| <= theta / lambda with amplitude 1, and the recovered probe supplies the phase
    inside it (the phase of its spectrum at detector pixels, scan_grid_spectrum_at)."""
    ky = np.asarray(ky_px, dtype=np.float64)
    kx = np.asarray(kx_px, dtype=np.float64)
    r = bright_field_radius_px(p)
    amp = (ky * ky + kx * kx <= r * r).astype(np.float64)
    return amp * np.exp(1j * np.angle(scan_grid_spectrum_at(probe, p, ky, kx)))


def recovered_probe_autocorrelation(probe: np.ndarray, p: Params, vy: int, vx: int) -> np.ndarray:
    """Y_v from a recovered probe (the Wiener update of Sect. 10): p(q) conj p(q + q_v) with p
    the recovered probe model of recovered_probe_spectrum_at."""
    dy, dx = scan_shift_det_px(p, vy, vx)
    qy = np.arange(p.det_y, dtype=np.float64) - p.cy
    qx = np.arange(p.det_x, dtype=np.float64) - p.cx
    ky, kx = np.meshgrid(qy, qx, indexing="ij")
    a = recovered_probe_spectrum_at(probe, p, ky, kx)
    b = recovered_probe_spectrum_at(probe, p, ky + dy, kx + dx)
    return a * np.conj(b)


def updated_plan(probe: np.ndarray, p: Params) -> OraclePlan:
    """Algorithm 1 rebuilt from a recovered probe: the updated Wiener filter that re-deconvolves
    the retained accumulator H into a refined object (Sect. 10)."""
    return build_plan(p, lambda vy, vx: recovered_probe_autocorrelation(probe, p, vy, vx))


# ---------------------------------------------------------------------------------------------
# Error metrics
# ---------------------------------------------------------------------------------------------

def phase_rel_l2(phi: np.ndarray, phi_ref: np.ndarray) -> float:
    """Relative L2 distance of mean-subtracted phase maps."""
    a = np.asarray(phi, dtype=np.float64)
    b = np.asarray(phi_ref, dtype=np.float64)
    a = a - a.mean()
    b = b - b.mean()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def complex_rel_l2(x: np.ndarray, ref: np.ndarray) -> float:
    x = np.asarray(x, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))
