"""Multi-process host logic on CPU (torch.distributed, gloo, two ranks on 127.0.0.1).

bench.py under torchrun runs one independent acquisition per rank (replicas, weak scaling) and
reports the slowest rank's step time; these tests run its rank helpers across real processes.
They also pin the exchange step a sharded acquisition would need: the method is linear in the
frames, so frames split across ranks (any partition, here by arrival batch) give partial
accumulators whose sum -- one all-reduce -- equals the single-rank accumulator, and likewise
for the deconvolved spectra (the partition-sum merge of Sect. 6.3).
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

WORLD = 2


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank: int, port: int) -> None:
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)


def _bench_helpers(rank: int, port: int) -> None:
    import bench
    _init(rank, port)
    try:
        ms = [3.5, 5.25][rank]                       # rank 1 is the slow one
        slowest = bench.max_over_ranks(ms, WORLD)
        assert slowest == 5.25
        value = bench.job_throughput(1000, WORLD, slowest)
        assert abs(value - 2000 / 5.25e-3) < 1e-6
        assert bench.max_over_ranks(ms, 1) == ms      # one rank: no collective
    finally:
        dist.destroy_process_group()


def _sharded_accumulator(rank: int, port: int) -> None:
    import oracle.wdd_oracle as W
    import synth
    from wdd_harness import oracle_params
    _init(rank, port)
    try:
        c1, _ = synth.config("c1")
        import dataclasses
        acq = dataclasses.replace(c1, scan_y=9, scan_x=11, obj_y=18, obj_x=22, det=16,
                                  dtype="f32", dose=3e3, seed_noise=31)
        F = synth.all_frames(acq)
        idx = synth.raster_indices(acq)
        p = oracle_params(acq, "hg_tensor", 16)
        plan = W.build_plan(p)
        # arrival batches of 7 frames dealt to the ranks in turn
        batches = [np.arange(a, min(a + 7, len(idx))) for a in range(0, len(idx), 7)]
        mine = np.concatenate(batches[rank::WORLD])
        H_part = W.accumulate(W.coefficients(F[mine], plan), idx[mine], p)
        o_part = W.deconvolve(H_part, plan)
        # one sum all-reduce of each (complex values as float64 pairs)
        H_sum = torch.from_numpy(np.ascontiguousarray(H_part).view(np.float64).copy())
        o_sum = torch.from_numpy(np.ascontiguousarray(o_part).view(np.float64).copy())
        dist.all_reduce(H_sum, op=dist.ReduceOp.SUM)
        dist.all_reduce(o_sum, op=dist.ReduceOp.SUM)
        H_all = H_sum.numpy().view(np.complex128)
        o_all = o_sum.numpy().view(np.complex128)
        H_ref = W.accumulate(W.coefficients(F, plan), idx, p)
        o_ref = W.deconvolve(H_ref, plan)
        assert np.linalg.norm(H_all - H_ref) <= 1e-12 * np.linalg.norm(H_ref)
        assert np.linalg.norm(o_all - o_ref) <= 1e-12 * np.linalg.norm(o_ref)
        _, ph = W.finalize(o_all, p)
        _, ph_ref = W.finalize(o_ref, p)
        assert W.phase_rel_l2(ph, ph_ref) <= 1e-12
        # each rank saw only part of the data: its own result is not the full one
        assert np.linalg.norm(H_part - H_ref) > 1e-3 * np.linalg.norm(H_ref)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("fn", [_bench_helpers, _sharded_accumulator], ids=["bench", "merge"])
def test_two_ranks_gloo(fn):
    mp.spawn(fn, args=(_free_port(),), nprocs=WORLD, join=True)
