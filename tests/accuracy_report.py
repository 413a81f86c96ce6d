"""Phase accuracy of the CUDA paths against the FP64 oracle, per workload and arithmetic path.

    python tests/accuracy_report.py [--only c1,c2,...] [--out report.json]

Needs a GPU.  For each workload the same seeded frames go through the oracle (FP64, CPU) and the
library (plain FP32 path and split tensor-core path); printed per line: phase relative L2 (mean
removed), complex relative L2 of the spectrum o, and of the accumulator H.  Workloads whose full
oracle run would take too long on the host are reconstructed on a 64 x 64 scan crop (the same
specimen and optics, its own 64 x 64 scan DFT); for the 256 x 256 scan the accumulator is also
checked at full size on 64 sampled scan frequencies, each computed by the oracle from all frames.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)

import oracle.wdd_oracle as W  # noqa: E402
import synth  # noqa: E402


def gpu_run(acq, frames, idx, basis, k, precision, batch, depth):
    import torch
    from paper_2212_01309_gb300 import wdd
    p = wdd.params_from_acquisition(acq, basis=basis, rank_k=k, precision=precision,
                                    max_batch=batch, accum_depth=depth)
    with wdd.Plan(p) as g:
        d = torch.from_numpy(frames).cuda()
        for a in range(0, len(idx), batch):
            g.push(d[a:a + batch], idx[a:a + batch])
        obj, ph, _, _ = g.finalize()
        torch.cuda.synchronize()
        g.check_device()
        return dict(ph=ph.cpu().numpy().astype(np.float64), o=g.copy_array("spectrum"),
                    H=g.copy_array("accum"))


def compare(name, acq, basis, k, batch, frames=None, idx=None):
    t0 = time.time()
    if frames is None:
        frames = synth.all_frames(acq)
        idx = synth.raster_indices(acq)
    p = W.Params.from_acquisition(acq, basis=basis, rank_k=k, epsilon=1e-3)
    plan = W.build_plan(p)
    C = np.concatenate([W.coefficients(frames[a:a + 2048], plan) for a in range(0, len(idx), 2048)])
    H = W.accumulate(C, idx, p)
    o = W.deconvolve(H, plan)
    _, ph = W.finalize(o, p)
    t_oracle = time.time() - t0
    rows = []
    for precision, depth in (("fp32", 0), ("split", 4096)):
        g = gpu_run(acq, frames, idx, basis, k, precision, batch, depth)
        rows.append({"workload": name, "path": precision, "scan": [acq.scan_y, acq.scan_x],
                     "det": acq.det, "basis": basis, "K": k,
                     "phase_rel_l2": W.phase_rel_l2(g["ph"], ph),
                     "spectrum_rel_l2": W.complex_rel_l2(g["o"], o),
                     "accum_rel_l2": W.complex_rel_l2(g["H"], H),
                     "oracle_s": round(t_oracle, 1)})
    return rows


def sampled_rows(name, acq, basis, k, batch, n_rows=64, seed=7):
    """Full-size check of H on sampled scan frequencies (each row: O(S K) in FP64)."""
    frames = synth.all_frames(acq)
    idx = synth.raster_indices(acq)
    p = W.Params.from_acquisition(acq, basis=basis, rank_k=k, epsilon=1e-3)
    # coefficients only need the bases, not the Wiener filter: build them from a 1-row plan
    By, Bx, m_idx, comp, m_neg = W._bases(p)
    plan = W.OraclePlan(params=p, By=By, Bx=Bx, m_idx=m_idx, comp=comp, m_neg=m_neg,
                        chi=np.zeros((1, 1)), W=np.zeros((1, k)), mask=np.ones(1, bool), eps_eff=0.0)
    C = np.concatenate([W.coefficients(frames[a:a + 2048], plan) for a in range(0, len(idx), 2048)])
    rng = np.random.default_rng(seed)
    rows_v = np.sort(rng.choice(acq.n_frames, size=n_rows, replace=False))
    H_ref = W.accumulate(C, idx, p, v_rows=rows_v)
    out = []
    for precision, depth in (("fp32", 0), ("split", 4096)):
        g = gpu_run(acq, frames, idx, basis, k, precision, batch, depth)
        out.append({"workload": name + " (full size, 64 sampled rows of H)", "path": precision,
                    "scan": [acq.scan_y, acq.scan_x], "det": acq.det, "basis": basis, "K": k,
                    "accum_rel_l2": W.complex_rel_l2(g["H"][rows_v], H_ref)})
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", default="c1,c2,c3crop,c3rows,c5crop,paper,c4crops")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    want = set(a.only.split(","))
    rows = []
    if "c1" in want:
        acq, rc = synth.config("c1")
        rows += compare("c1", acq, rc["basis"], rc["rank_k"], rc["batch"])
    if "c2" in want:
        acq, rc = synth.config("c2")
        rows += compare("c2", acq, rc["basis"], rc["rank_k"], rc["batch"])
    if "c3crop" in want:
        acq, rc = synth.config("c3")
        rows += compare("c3 (64x64 scan crop)", acq.crop(64, 64), rc["basis"], rc["rank_k"],
                        rc["batch"])
    if "c3rows" in want:
        acq, rc = synth.config("c3")
        rows += sampled_rows("c3", acq, rc["basis"], rc["rank_k"], rc["batch"])
    if "c5crop" in want:
        acq, rc = synth.config("c5")
        rows += compare("c5 (64x64 scan crop)", acq.crop(64, 64), rc["basis"], rc["rank_k"],
                        rc["batch"])
    if "paper" in want:
        acq, rc = synth.config("paper")
        rows += compare("paper-shaped", acq, rc["basis"], rc["rank_k"], rc["batch"])
    if "c4crops" in want:
        for i, (acq, rc) in enumerate(synth.serving_mix()):
            crop = acq.crop(min(64, acq.scan_y), min(64, acq.scan_x))
            rows += compare(f"c4 session {i} ({acq.scan_y}x{acq.scan_x} / {acq.det}^2, "
                            f"{crop.scan_y}x{crop.scan_x} crop)", crop, rc["basis"], rc["rank_k"],
                            256)
    for r in rows:
        print(json.dumps(r), flush=True)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(rows, f, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
