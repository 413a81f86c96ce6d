"""Seeded simulation of 4D-STEM acquisitions of a weak phase object.

Forward model (Eq. 1): for scan position s the detector records
    I_s = |fftshift(FFT2(p(r - r_s) * O(r)))|^2
on an N x N window of object pixels, with O = exp(i*phi) a periodic weak phase object and p the
probe formed by a hard-edged circular aperture with defocus.  Optional Poisson noise follows the
dose model of Sect. 8 (counts ~ Poisson(dose * I_s / sum(I_s))), with the dose given per frame.

Choices the paper leaves open (they are restated in the design notes):
  * object pixel dx = lambda / (4 * theta), so the bright-field disc radius is N/4 detector pixels
    and the detector sampling is 1 / (N * dx);
  * scan step = step_px object pixels (2 in every workload);
  * Gaussian atoms of sigma 1 px at uniform random positions, summed periodically, truncated at
    6 sigma, then scaled so that max(phi) equals the requested peak phase;
  * the probe window is centred on the scan position, and frames are stored fftshifted
    (zero frequency at pixel (N//2, N//2)).

Only numpy is used.  Random draws use numpy's PCG64 keyed by (seed, block) so that any chunking of
the frame stream yields the same frames.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Iterator

import numpy as np

try:  # multi-threaded FFTs when scipy is present (same transform as numpy's)
    import scipy.fft as _sfft

    def _fft2(a):
        return _sfft.fft2(a, axes=(-2, -1), workers=-1)
except ImportError:  # pragma: no cover
    def _fft2(a):
        return np.fft.fft2(a, axes=(-2, -1))

# CODATA 2018 constants (SI).
_H = 6.62607015e-34
_M0 = 9.1093837015e-31
_QE = 1.602176634e-19
_C = 299792458.0

NOISE_BLOCK = 256  # frames per independently seeded noise block


def _wavelength(voltage_v: float) -> float:
    """Relativistic electron wavelength in metres (used only to derive the pixel size)."""
    ev = _QE * voltage_v
    return _H / math.sqrt(2.0 * _M0 * ev * (1.0 + ev / (2.0 * _M0 * _C * _C)))


@dataclasses.dataclass(frozen=True)
class Acquisition:
    scan_y: int
    scan_x: int
    det: int                 # detector is det x det pixels
    obj_y: int
    obj_x: int
    n_atoms: int
    peak_phase: float
    voltage_v: float
    semiconv_rad: float
    defocus_m: float = 0.0
    dose: float | None = None    # electrons per frame; None = noise-free intensities
    dtype: str = "f64"           # "f64", "f32" or "u16"
    step_px: int = 2
    seed_obj: int = 0
    seed_noise: int = 0

    # ---- derived acquisition geometry -------------------------------------------------------
    @property
    def wavelength_m(self) -> float:
        return _wavelength(self.voltage_v)

    @property
    def dx_m(self) -> float:
        return self.wavelength_m / (4.0 * self.semiconv_rad)

    @property
    def scan_step_m(self) -> float:
        return self.step_px * self.dx_m

    @property
    def det_px_inv_m(self) -> float:
        """Detector sampling in reciprocal metres per pixel."""
        return 1.0 / (self.det * self.dx_m)

    @property
    def n_frames(self) -> int:
        return self.scan_y * self.scan_x

    @property
    def np_dtype(self):
        return {"f64": np.float64, "f32": np.float32, "u16": np.uint16}[self.dtype]

    def crop(self, sy: int, sx: int) -> "Acquisition":
        """The same specimen and optics scanned over an sy x sx window at the origin.

        The object keeps its size and content, so frames of the cropped scan are exactly the
        first sy rows and sx columns of the full scan.
        """
        return dataclasses.replace(self, scan_y=sy, scan_x=sx)


# Workloads.  `recon` holds the reconstruction settings that go with each acquisition.
CONFIGS: dict[str, dict] = {
    # One session, FP64, noise-free: 32x32 scan, 32x32 detector, full rank.
    "c1": dict(
        acq=Acquisition(scan_y=32, scan_x=32, det=32, obj_y=64, obj_x=64, n_atoms=40,
                        peak_phase=0.1, voltage_v=300e3, semiconv_rad=20e-3, defocus_m=0.0,
                        dose=None, dtype="f64", seed_obj=1001, seed_noise=2001),
        recon=dict(basis="fourier_full", rank_k=32 * 32, epsilon=1e-3, batch=64)),
    # Same generator at scale, FP32 frames with Poisson noise.
    "c2": dict(
        acq=Acquisition(scan_y=128, scan_x=128, det=128, obj_y=256, obj_x=256, n_atoms=400,
                        peak_phase=0.2, voltage_v=300e3, semiconv_rad=25e-3, defocus_m=5e-9,
                        dose=1e4, dtype="f32", seed_obj=1002, seed_noise=2002),
        recon=dict(basis="hg_tensor", rank_k=64, epsilon=1e-3, batch=64)),
    # Precision path: 256x256 scan, uint16 counts.
    "c3": dict(
        acq=Acquisition(scan_y=256, scan_x=256, det=128, obj_y=512, obj_x=512, n_atoms=400,
                        peak_phase=0.2, voltage_v=300e3, semiconv_rad=25e-3, defocus_m=5e-9,
                        dose=1e3, dtype="u16", seed_obj=1003, seed_noise=2003),
        recon=dict(basis="hg_energy", rank_k=128, epsilon=1e-3, batch=256)),
    # Large single acquisition streamed from host memory.
    "c5": dict(
        acq=Acquisition(scan_y=512, scan_x=512, det=256, obj_y=1024, obj_x=1024, n_atoms=3000,
                        peak_phase=0.3, voltage_v=300e3, semiconv_rad=30e-3, defocus_m=0.0,
                        dose=1e3, dtype="u16", seed_obj=1005, seed_noise=2005),
        recon=dict(basis="hg_tensor", rank_k=256, epsilon=1e-3, batch=512)),
    # Shaped like the paper's timing workload (128,128,128,128), L = 16.
    "paper": dict(
        acq=Acquisition(scan_y=128, scan_x=128, det=128, obj_y=256, obj_x=256, n_atoms=400,
                        peak_phase=0.2, voltage_v=300e3, semiconv_rad=22e-3, defocus_m=0.0,
                        dose=1e4, dtype="u16", seed_obj=1006, seed_noise=2006),
        recon=dict(basis="hg_tensor", rank_k=256, epsilon=1e-3, batch=256)),
}


def config(name: str) -> tuple[Acquisition, dict]:
    c = CONFIGS[name]
    return c["acq"], dict(c["recon"])


# ---- object --------------------------------------------------------------------------------

def object_phase(acq: Acquisition) -> np.ndarray:
    """Phase map phi (obj_y x obj_x, float64) built from periodic Gaussian atoms."""
    rng = np.random.default_rng(acq.seed_obj)
    pos = rng.uniform(0.0, 1.0, size=(acq.n_atoms, 2)) * np.array([acq.obj_y, acq.obj_x])
    phi = np.zeros((acq.obj_y, acq.obj_x), dtype=np.float64)
    sigma = 1.0
    rad = 6  # truncation radius in pixels (6 sigma)
    offs = np.arange(-rad, rad + 1)
    for (py, px) in pos:
        iy0 = int(math.floor(py))
        ix0 = int(math.floor(px))
        ys = iy0 + offs
        xs = ix0 + offs
        dy = ys - py
        dx = xs - px
        g = np.exp(-(dy[:, None] ** 2 + dx[None, :] ** 2) / (2.0 * sigma * sigma))
        phi[np.ix_(ys % acq.obj_y, xs % acq.obj_x)] += g
    m = phi.max()
    if m > 0:
        phi *= acq.peak_phase / m
    return phi


def object_transfer(acq: Acquisition, phi: np.ndarray | None = None) -> np.ndarray:
    if phi is None:
        phi = object_phase(acq)
    return np.exp(1j * phi)


# ---- probe ---------------------------------------------------------------------------------

def probe_fourier_grid(acq: Acquisition) -> np.ndarray:
    """Probe spectrum on the centred detector grid (zero frequency at N//2)."""
    n = acq.det
    dk = acq.det_px_inv_m
    lam = acq.wavelength_m
    q = (np.arange(n) - n // 2).astype(np.float64)
    qy, qx = np.meshgrid(q, q, indexing="ij")
    r2 = qy * qy + qx * qx
    rad = acq.semiconv_rad / (lam * dk)
    amp = (r2 <= rad * rad).astype(np.float64)
    chi = -math.pi * lam * acq.defocus_m * (dk * dk) * r2
    return amp * np.exp(1j * chi)


def probe_real(acq: Acquisition) -> np.ndarray:
    """Real-space probe on the N x N window, centred at pixel (N//2, N//2)."""
    ph = probe_fourier_grid(acq)
    return np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(ph)))


# ---- frames --------------------------------------------------------------------------------

def raster_indices(acq: Acquisition) -> np.ndarray:
    return np.arange(acq.n_frames, dtype=np.int32)


def _frames_clean(acq: Acquisition, obj: np.ndarray, probe: np.ndarray,
                  idx: np.ndarray) -> np.ndarray:
    n = acq.det
    sy = idx // acq.scan_x
    sx = idx % acq.scan_x
    oy = sy * acq.step_px - n // 2
    ox = sx * acq.step_px - n // 2
    ar = np.arange(n)
    rows = (oy[:, None] + ar[None, :]) % acq.obj_y
    cols = (ox[:, None] + ar[None, :]) % acq.obj_x
    patch = obj[rows[:, :, None], cols[:, None, :]]
    wave = _fft2(patch * probe[None, :, :])
    inten = wave.real * wave.real + wave.imag * wave.imag
    return np.fft.fftshift(inten, axes=(-2, -1))


def frames(acq: Acquisition, start: int, count: int, chunk: int = NOISE_BLOCK,
           obj: np.ndarray | None = None) -> Iterator[tuple[np.ndarray, np.ndarray]]:
    """Yield (scan_indices int32, frames) chunks for raster positions [start, start + count).

    Frames have shape (n, N, N) and the acquisition's dtype.  Noise is drawn per block of
    NOISE_BLOCK consecutive positions from a stream keyed by (seed_noise, block), so the frames
    do not depend on the chunking asked for.
    """
    if obj is None:
        obj = object_transfer(acq)
    probe = probe_real(acq)
    nblk = max(1, chunk // NOISE_BLOCK)
    end = start + count
    blk = start // NOISE_BLOCK
    while blk * NOISE_BLOCK < end:
        b0 = blk * NOISE_BLOCK
        b1 = min((blk + nblk) * NOISE_BLOCK, acq.n_frames)
        lo, hi = max(start, b0), min(end, b1)
        if acq.dose is None:
            idx = np.arange(lo, hi, dtype=np.int64)
            out = _frames_clean(acq, obj, probe, idx).astype(acq.np_dtype)
        else:
            idx_full = np.arange(b0, b1, dtype=np.int64)
            clean = _frames_clean(acq, obj, probe, idx_full)
            tot = clean.sum(axis=(-2, -1), keepdims=True)
            lam = acq.dose * clean / tot
            parts = []
            for k in range(0, b1 - b0, NOISE_BLOCK):
                rng = np.random.default_rng([acq.seed_noise, blk + k // NOISE_BLOCK])
                parts.append(rng.poisson(lam[k:k + NOISE_BLOCK]))
            counts = np.concatenate(parts, axis=0)
            if acq.dtype == "u16" and counts.max(initial=0) > 65535:
                raise ValueError("count exceeds uint16 range")
            out = counts[lo - b0:hi - b0].astype(acq.np_dtype)
            idx = np.arange(lo, hi, dtype=np.int64)
        yield idx.astype(np.int32), out
        blk += nblk


def all_frames(acq: Acquisition, obj: np.ndarray | None = None) -> np.ndarray:
    """All frames of the raster scan, shape (S, N, N)."""
    out = np.empty((acq.n_frames, acq.det, acq.det), dtype=acq.np_dtype)
    for idx, fr in frames(acq, 0, acq.n_frames, chunk=1024, obj=obj):
        out[idx] = fr
    return out


# ---- serving mix: several concurrent acquisitions and their frame arrivals -----------------

SERVING_SIZES = [((64, 64), 64), ((128, 128), 64), ((128, 128), 128), ((256, 256), 128),
                 ((192, 256), 96), ((256, 256), 256)]


def serving_mix(seed_obj: int = 1004, seed_noise: int = 2004, sizes=None, scale: int = 1):
    """Sessions of the serving workload: (scan, detector) sizes as listed, uint16 Poisson frames,
    dose log-uniform in [1e2, 1e4] per frame, semiconvergence U[15, 30] mrad, defocus
    U[-10, 10] nm, 300 kV, object twice the scan (scan step 2 px).  K = 64 for detectors up to 96
    pixels, 128 for 128, 256 for 256 (Hermite-Gauss energy basis for 128, tensor otherwise).
    `scale` divides every scan side (smaller copies of the mix for tests).
    Returns a list of (Acquisition, recon dict)."""
    rng = np.random.default_rng(seed_obj)
    out = []
    for i, ((sy, sx), n) in enumerate(sizes or SERVING_SIZES):
        sy, sx = max(4, sy // scale), max(4, sx // scale)
        dose = float(10 ** rng.uniform(2.0, 4.0))
        theta = float(rng.uniform(15e-3, 30e-3))
        df = float(rng.uniform(-10e-9, 10e-9))
        acq = Acquisition(scan_y=sy, scan_x=sx, det=n, obj_y=2 * sy, obj_x=2 * sx,
                          n_atoms=max(8, (sy * sx) // 40), peak_phase=0.2, voltage_v=300e3,
                          semiconv_rad=theta, defocus_m=df, dose=dose, dtype="u16",
                          seed_obj=seed_obj * 10 + i, seed_noise=seed_noise * 10 + i)
        k = 64 if n <= 96 else (128 if n == 128 else 256)
        basis = "hg_energy" if k == 128 else "hg_tensor"
        out.append((acq, dict(basis=basis, rank_k=k, epsilon=1e-3)))
    return out


def serving_arrivals(n_frames, rate_fps: float = 20000.0, seed: int = 3004,
                     bmin: int = 16, bmax: int = 512):
    """Seeded Poisson-process arrivals: batches of b ~ U{bmin..bmax} frames at exponential gaps
    with mean b / rate; each batch goes to a session drawn in proportion to its remaining frames
    and continues that session's raster order.  Returns a list of (t_seconds, session, start,
    count)."""
    rng = np.random.default_rng(seed)
    left = np.array(n_frames, dtype=np.int64)
    nxt = np.zeros(len(n_frames), dtype=np.int64)
    t = 0.0
    out = []
    while left.sum() > 0:
        b = int(rng.integers(bmin, bmax + 1))
        t += float(rng.exponential(b / rate_fps))
        sid = int(rng.choice(len(left), p=left / left.sum()))
        c = int(min(b, left[sid]))
        out.append((t, sid, int(nxt[sid]), c))
        nxt[sid] += c
        left[sid] -= c
    return out
