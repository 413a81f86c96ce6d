"""The GPU frame generator simulates the same acquisitions as the numpy generator."""
import dataclasses

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_torch_generator_matches_numpy_noise_free():
    import torch
    from synth.torch_gen import TorchFrames
    acq, _ = synth.config("c2")
    acq = dataclasses.replace(acq, scan_y=24, scan_x=20, obj_y=48, obj_x=40, dose=None, dtype="f32")
    ref = synth.all_frames(acq).astype(np.float64)
    got = TorchFrames(acq).all().cpu().numpy().astype(np.float64)
    assert got.shape == ref.shape
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5


def test_torch_generator_poisson_dose():
    from synth.torch_gen import TorchFrames
    acq, _ = synth.config("c3")
    acq = acq.crop(8, 8)
    f = TorchFrames(acq).all().cpu().numpy().astype(np.float64)
    tot = f.reshape(len(f), -1).sum(axis=1)
    assert abs(tot.mean() - acq.dose) < 5 * np.sqrt(acq.dose / len(f)) + 1
