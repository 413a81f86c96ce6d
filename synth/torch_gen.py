"""GPU simulation of the same acquisitions as synth.generator, for workloads too large for numpy.

The forward model is identical (Eq. 1: window of the periodic object around the scan position,
times the centred probe, FFT, |.|^2, fftshift; Poisson counts at the given dose per frame, Sect. 8)
and the object and probe are the numpy generator's own arrays.  Differences: the FFT runs in
complex64 on the GPU, and Poisson noise is drawn with torch's generator (seeded per 256-frame
block), so noisy frames are a different draw from the numpy generator's.  Noise-free frames agree
with the numpy generator to FP32 rounding (checked by a GPU test).

This module holds none of the reconstruction arithmetic; it is input generation only.
"""
from __future__ import annotations

import numpy as np

from .generator import NOISE_BLOCK, Acquisition, object_transfer, probe_real


class TorchFrames:
    """Frame source on a CUDA device for one acquisition."""

    def __init__(self, acq: Acquisition, device="cuda", obj: np.ndarray | None = None):
        import torch
        self.acq = acq
        self.device = torch.device(device)
        o = object_transfer(acq) if obj is None else obj
        self.obj = torch.from_numpy(o.astype(np.complex64)).to(self.device)
        self.probe = torch.from_numpy(probe_real(acq).astype(np.complex64)).to(self.device)
        self.ar = torch.arange(acq.det, device=self.device)

    def clean(self, idx):
        """Noise-free intensities (float32) for scan positions idx (1-D int tensor)."""
        import torch
        a = self.acq
        n = a.det
        sy = torch.div(idx, a.scan_x, rounding_mode="floor")
        sx = idx - sy * a.scan_x
        oy = sy * a.step_px - n // 2
        ox = sx * a.step_px - n // 2
        rows = torch.remainder(oy[:, None] + self.ar[None, :], a.obj_y)
        cols = torch.remainder(ox[:, None] + self.ar[None, :], a.obj_x)
        patch = self.obj[rows[:, :, None], cols[:, None, :]]
        wave = torch.fft.fft2(patch * self.probe[None])
        inten = wave.real * wave.real + wave.imag * wave.imag
        return torch.fft.fftshift(inten, dim=(-2, -1))

    def block(self, blk: int):
        """Frames of noise block blk (NOISE_BLOCK consecutive positions) in the acquisition dtype."""
        import torch
        a = self.acq
        s0 = blk * NOISE_BLOCK
        s1 = min(s0 + NOISE_BLOCK, a.n_frames)
        idx = torch.arange(s0, s1, device=self.device)
        inten = self.clean(idx)
        if a.dose is None:
            return inten.to(torch.float64 if a.dtype == "f64" else torch.float32)
        lam = a.dose * inten / inten.sum(dim=(-2, -1), keepdim=True)
        g = torch.Generator(device=self.device)
        g.manual_seed(int(a.seed_noise) * 1_000_003 + blk)
        counts = torch.poisson(lam, generator=g)
        if a.dtype == "u16":
            return counts.clamp_(max=65535).to(torch.int32).to(torch.uint16)
        return counts.to(torch.float64 if a.dtype == "f64" else torch.float32)

    def all(self):
        """All frames of the raster scan as one device tensor (S, N, N)."""
        import torch
        a = self.acq
        nblk = (a.n_frames + NOISE_BLOCK - 1) // NOISE_BLOCK
        dt = {"u16": torch.uint16, "f32": torch.float32, "f64": torch.float64}[a.dtype]
        out = torch.empty((a.n_frames, a.det, a.det), dtype=dt, device=self.device)
        for b in range(nblk):
            out[b * NOISE_BLOCK:(b + 1) * NOISE_BLOCK] = self.block(b)
        return out
