"""Grouped flush across plans (wdd_flush_group): the gathered pushes of several live plans are
projected (Eq. 12) by shared launches and their staged frames accumulated (Eq. 14) by one split
launch and one tensor-core launch, as a server holding many sessions issues them.

Every member runs exactly the arithmetic of its own wdd_flush (the same projection body on its
own frames, the same split and accumulation bodies on its own tiles and segments), so the
accumulators of the grouped plans are bit-identical to those of the same plans flushed one by
one; one member is also checked against the FP64 oracle within the split path's bound.  The
members mix frame types, detector sizes and both accumulation kernels (K <= 64 and K > 64).
Refused groups enqueue nothing and leave every plan's staged and gathered frames in place.
"""
import dataclasses

import numpy as np
import pytest

import oracle.wdd_oracle as W
import synth
from wdd_harness import oracle_params, phase_err

pytestmark = pytest.mark.gpu

SPLIT_PHASE_TOL = 2e-3


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def _members():
    """(acquisition, basis, K): u16 and f32 frames, detectors of 36, 40 and 48 pixels, K from 10
    to 130 (both accumulation kernels), two members of one projection class."""
    c1, _ = synth.config("c1")
    a = dataclasses.replace(c1, scan_y=17, scan_x=23, obj_y=34, obj_x=46, det=36,
                            defocus_m=-3e-9, dtype="u16", dose=2e3, seed_noise=78)
    b = dataclasses.replace(c1, scan_y=33, scan_x=40, obj_y=66, obj_x=80, det=48,
                            defocus_m=1e-9, dtype="u16", dose=1e3, seed_noise=79)
    c = dataclasses.replace(c1, scan_y=20, scan_x=14, obj_y=40, obj_x=28, det=40,
                            defocus_m=4e-9, dtype="f32", dose=5e3, seed_noise=77)
    d = dataclasses.replace(a, scan_y=21, scan_x=19, obj_y=42, obj_x=38, seed_noise=80)
    return [(a, "hg_energy", 10), (b, "hg_energy", 130), (c, "hg_tensor", 16),
            (d, "hg_energy", 10)]


@pytest.fixture(scope="module")
def members(torch_cuda):
    torch = torch_cuda
    out = []
    for acq, basis, k in _members():
        F = synth.all_frames(acq)
        idx = synth.raster_indices(acq)
        out.append((acq, basis, k, F, idx, torch.from_numpy(F).cuda()))
    return out


def _plans(members, **kw):
    from paper_2212_01309_gb300 import wdd
    plans = []
    for acq, basis, k, _, _, _ in members:
        p = wdd.params_from_acquisition(acq, basis=basis, rank_k=k, epsilon=1e-3,
                                        precision="split", max_batch=512, accum_depth=4096,
                                        coalesce_frames=kw.get("coalesce", 1024))
        plans.append(wdd.Plan(p))
    return plans


def _push_interleaved(members, plans, stream, seed):
    """Pushes every member's frames in ragged batches (16-300 frames), interleaved across the
    plans in a seeded order, all on one stream."""
    rng = np.random.default_rng(seed)
    pos = [0] * len(plans)
    while any(p < len(m[4]) for p, m in zip(pos, members)):
        j = int(rng.integers(len(plans)))
        n_all = len(members[j][4])
        if pos[j] >= n_all:
            continue
        n = min(int(rng.integers(16, 301)), n_all - pos[j])
        d, idx = members[j][5], members[j][4]
        plans[j].push(d[pos[j]:pos[j] + n], idx[pos[j]:pos[j] + n], stream=stream)
        pos[j] += n


def test_grouped_flush_equals_per_plan_flush(torch_cuda, members):
    torch = torch_cuda
    from paper_2212_01309_gb300 import wdd
    stream = torch.cuda.Stream()
    single, grouped = _plans(members), _plans(members)
    try:
        with torch.cuda.stream(stream):
            _push_interleaved(members, single, stream, seed=11)
            _push_interleaved(members, grouped, stream, seed=11)
            for g in single:
                g.flush(stream)
            infos = [g.info() for g in grouped]
            assert sum(i["pending"] > 0 for i in infos) >= 3   # something left to group
            before = [i["kernel_launches"] for i in infos]
            wdd.flush_group(grouped, stream)
            after = [g.info() for g in grouped]
            assert all(i["staged"] == 0 and i["pending"] == 0 for i in after)
            # one projection launch per class of streaming-projection plans with gathered
            # frames (one per plan for the other engines), then split + accumulation
            rows = [i["proj_engine"] == wdd.PROJ_ENGINE["stream"] for i in infos]
            classes = {(m[0].dtype, (i["basis_ly"] + 3) // 4, 8 if i["basis_lx"] <= 8 else 16,
                        (m[0].det // 4 + 31) // 32)
                       for m, i, r in zip(members, infos, rows) if i["pending"] > 0 and r}
            others = sum(1 for i, r in zip(infos, rows) if i["pending"] > 0 and not r)
            assert sum(rows) >= 3
            assert (sum(a["kernel_launches"] - b for a, b in zip(after, before))
                    == len(classes) + others + 2)
            outs = [g.snapshot(stream=stream) for g in grouped]
        torch.cuda.synchronize()
        for j, (gs, gg) in enumerate(zip(single, grouped)):
            gs.check_device()
            gg.check_device()
            assert np.array_equal(gg.copy_array("accum"), gs.copy_array("accum")), j
            assert np.array_equal(gg.hit_counts(), gs.hit_counts()), j
        acq, basis, k, F, idx, _ = members[0]
        p = oracle_params(acq, basis, k)
        _, ph_ref = W.finalize(W.live_wdd(F, idx, W.build_plan(p)), p)
        assert phase_err(outs[0][1].cpu().numpy(), ph_ref) < SPLIT_PHASE_TOL
    finally:
        for g in single + grouped:
            g.close()


def test_grouped_flush_packs_large_pending_sets(torch_cuda, members):
    """Three plans of one class, each with 1320 frames gathered from 28 pushes: a launch takes
    at most 64 pushes, so the group needs two projection launches; the results stay
    bit-identical."""
    torch = torch_cuda
    from paper_2212_01309_gb300 import wdd
    stream = torch.cuda.Stream()
    sub = [members[1], members[1], members[1]]      # 33 x 40 scans, 1320 frames each
    single, grouped = _plans(sub, coalesce=2048), _plans(sub, coalesce=2048)
    try:
        with torch.cuda.stream(stream):
            for plans in (single, grouped):
                for g, m in zip(plans, sub):
                    for a in range(0, len(m[4]), 48):
                        g.push(m[5][a:a + 48], m[4][a:a + 48], stream=stream)
            for g in single:
                g.flush(stream)
            before = sum(g.info()["kernel_launches"] for g in grouped)
            wdd.flush_group(grouped, stream)
            assert sum(g.info()["kernel_launches"] for g in grouped) - before == 2 + 2
        torch.cuda.synchronize()
        for gs, gg in zip(single, grouped):
            gg.check_device()
            assert np.array_equal(gg.copy_array("accum"), gs.copy_array("accum"))
    finally:
        for g in single + grouped:
            g.close()


def test_refused_groups_enqueue_nothing(torch_cuda, members):
    torch = torch_cuda
    import ctypes
    from paper_2212_01309_gb300 import wdd
    stream = torch.cuda.Stream()
    plans = _plans(members[:2])
    acq, basis, k = members[2][0], members[2][1], members[2][2]
    fp32 = wdd.Plan(wdd.params_from_acquisition(acq, basis=basis, rank_k=k, precision="fp32",
                                                max_batch=64))
    sep = wdd.Plan(wdd.params_from_acquisition(acq, basis=basis, rank_k=k, precision="split",
                                               max_batch=64, accum_depth=256,
                                               accum_mode="separable"))
    try:
        with torch.cuda.stream(stream):
            for g, m in zip(plans, members[:2]):
                g.push(m[5][:100], m[4][:100], stream=stream)
            state = [(g.info()["staged"], g.info()["pending"]) for g in plans]
            L = wdd.lib()

            def call(group, count=None):
                arr = (ctypes.c_void_p * max(1, len(group)))(*[g._h.value for g in group])
                return L.wdd_flush_group(arr, len(group) if count is None else count,
                                         ctypes.c_void_p(int(stream.cuda_stream)))

            assert call(plans + [fp32]) == wdd.ERR_INVALID_ARG       # not SPLIT
            assert call(plans + [sep]) == wdd.ERR_INVALID_ARG        # separable accumulation
            assert call([plans[0], plans[1], plans[0]]) == wdd.ERR_INVALID_ARG   # repeated
            assert call(plans, count=0) == wdd.ERR_INVALID_ARG
            many = [plans[0]] * (wdd.flush_group_max() + 1)
            assert call(many) == wdd.ERR_INVALID_ARG
            assert [(g.info()["staged"], g.info()["pending"]) for g in plans] == state
            done = _plans(members[3:4])[0]
            done.finalize(stream=stream)
            assert call(plans + [done]) == wdd.ERR_STATE
            assert [(g.info()["staged"], g.info()["pending"]) for g in plans] == state
            done.close()
            wdd.flush_group(plans, stream)                           # the valid group runs
        torch.cuda.synchronize()
        for g in plans:
            g.check_device()
            assert g.info()["staged"] == 0
    finally:
        for g in plans + [fp32, sep]:
            g.close()
