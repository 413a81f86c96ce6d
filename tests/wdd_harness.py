"""Shared helpers for the GPU tests: run the CUDA path through the C ABI and the oracle on the
same seeded inputs.  Nothing here computes any part of the method."""
from __future__ import annotations

import dataclasses

import numpy as np

import oracle.wdd_oracle as W
import synth


def oracle_params(acq, basis, rank_k, epsilon=1e-3, **kw):
    return W.Params.from_acquisition(acq, basis=basis, rank_k=rank_k, epsilon=epsilon, **kw)


def gpu_plan(acq, basis, rank_k, epsilon=1e-3, precision="fp32", max_batch=64, accum_depth=0,
             **kw):
    from paper_2212_01309_gb300 import wdd
    p = wdd.params_from_acquisition(acq, basis=basis, rank_k=rank_k, epsilon=epsilon,
                                    precision=precision, max_batch=max_batch,
                                    accum_depth=accum_depth, **kw)
    return wdd.Plan(p)


def to_source(frames: np.ndarray, source: str):
    """Frames as a device tensor, a pinned host tensor or a pageable numpy array."""
    import torch
    if source == "device":
        return torch.from_numpy(np.ascontiguousarray(frames)).cuda()
    if source == "pinned":
        return torch.from_numpy(np.ascontiguousarray(frames)).pin_memory()
    if source == "pageable":
        return np.ascontiguousarray(frames)
    raise ValueError(source)


def push_all(plan, frames: np.ndarray, idx: np.ndarray, batch: int, source="device"):
    for a in range(0, len(idx), batch):
        plan.push(to_source(frames[a:a + batch], source), idx[a:a + batch])


def phase_err(ph_gpu, ph_ref) -> float:
    return W.phase_rel_l2(np.asarray(ph_gpu, dtype=np.float64), ph_ref)


def rel_l2(x, ref) -> float:
    x = np.asarray(x)
    ref = np.asarray(ref)
    return float(np.linalg.norm((x - ref).ravel()) / np.linalg.norm(ref.ravel()))


@dataclasses.dataclass
class Case:
    name: str
    acq: object
    basis: str
    rank_k: int


def small_cases():
    """Ragged shapes that span several tiles: non-square scans, odd and non-multiple-of-16
    detectors, each basis family and frame type."""
    c1, _ = synth.config("c1")
    out = []
    a = dataclasses.replace(c1, scan_y=20, scan_x=14, obj_y=40, obj_x=28, det=40,
                            defocus_m=4e-9, dtype="f32", dose=5e3, seed_noise=77)
    out.append(Case("hg_tensor_f32_20x14_n40", a, "hg_tensor", 16))
    b = dataclasses.replace(c1, scan_y=17, scan_x=23, obj_y=34, obj_x=46, det=36,
                            defocus_m=-3e-9, dtype="u16", dose=2e3, seed_noise=78)
    out.append(Case("hg_energy_u16_17x23_n36", b, "hg_energy", 10))
    c = dataclasses.replace(c1, scan_y=12, scan_x=18, obj_y=24, obj_x=36, det=24,
                            defocus_m=2e-9, dtype="f64", dose=None)
    out.append(Case("fourier_f64_12x18_n24", c, "fourier_full", 24 * 24))
    d = dataclasses.replace(c1, scan_y=65, scan_x=66, obj_y=130, obj_x=132, det=48,
                            defocus_m=1e-9, dtype="u16", dose=1e3, seed_noise=79)
    out.append(Case("hg_energy_u16_65x66_n48_k130", d, "hg_energy", 130))
    return out
