"""Multi-session live-WDD serving on one GPU.

Several live acquisitions ("sessions") of different scan and detector sizes stay resident on
the device, each with its own plan (Wiener filter and accumulator in HBM) and CUDA stream.  Frame
batches arrive over time.  The loop:

  * admits waiting sessions first-fit whenever the HBM budget has room for their plan
    (wdd_plan_footprint); a finished session's memory is returned and the next ones start; a
    session whose plan alone exceeds the budget is refused (its frames are dropped) and counted;
  * coalesces each admitted session's contiguous pending batches into pushes on that session's
    stream, cut at its snapshot points, so the work of different sessions overlaps on the
    device;
  * every `snapshot_every` frames of a session, and also whenever its oldest frame not yet in a
    snapshot has waited `snapshot_max_delay_s` (a display refresh deadline, optional),
    accumulates the staged frames (wdd_flush) and replays the session's captured CUDA graph of
    the reconstruction (deconvolution and inverse DFT), recording an event;
  * grouped mode (`grouped=True`): the pushes of every split-precision session only gather
    frames on one shared stream, and at the end of each pass over the sessions those that reached
    a snapshot point are flushed together (wdd_flush_group, up to wdd_flush_group_max() plans per
    call): their gathered frames are projected by shared launches and accumulated by one split
    launch and one tensor-core launch, after which each session's reconstruction graph replays on
    its own stream.  Sessions of other precisions keep the per-session flush;
  * measures each frame's latency from its arrival to the completion of the first snapshot that
    contains it.

All GPU work goes through the C ABI of libwdd.so; this module is scheduling only.  Without a
deadline, results do not depend on the mix: a session's frames are projected one by one and
accumulated in the order they were pushed, with flushes only at its own snapshot points.  With a
deadline the flush points depend on timing, which changes only the FP32 rounding of the sums.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

from . import wdd


@dataclasses.dataclass
class Session:
    """A live acquisition to serve: plan parameters and the device tensor its frames arrive in."""
    sid: int
    params: wdd.Params
    frames: object            # device tensor [S, N, N] holding the detector stream
    n_frames: int


def _groupable(params: wdd.Params) -> bool:
    return (params.precision == wdd.PRECISION["split"]
            and params.accum_mode == wdd.ACCUM_MODE["direct"])


class _Live:
    def __init__(self, spec: Session, use_graph: bool, group_stream=None):
        import torch
        self.spec = spec
        self.plan = wdd.Plan(spec.params)
        self.stream = torch.cuda.Stream()
        # grouped sessions push on the shared stream; their snapshots replay on their own
        self.push_stream = group_stream if group_stream is not None else self.stream
        self.due = False                         # grouped: a snapshot point has been reached
        self.due_final = False
        self.recon_done = None                   # event after the last reconstruction
        sy, sx = spec.params.scan_y, spec.params.scan_x
        self.obj = torch.empty((sy, sx), dtype=torch.complex64, device="cuda")
        self.phase = torch.empty((sy, sx), dtype=torch.float32, device="cuda")
        self.pending = collections.deque()      # (t_arrival, start, count), in arrival order
        self.pushed = 0                          # frames pushed so far (raster order)
        self.unsnapped = []                      # (t_arrival, count) since the last snapshot
        self.inflight = []                       # (event, [(t_arrival, count)], final)
        self.since_snap = 0
        self.closing = False
        self.graph = None
        self.plan.set_stream(self.stream)
        if use_graph:
            # reconstruction with nothing staged: deconvolution + inverse DFT, fixed pointers
            g = torch.cuda.CUDAGraph()
            with torch.cuda.stream(self.stream):
                self.plan.flush()
                g.capture_begin()
                self.plan.snapshot(self.obj, self.phase)
                g.capture_end()
            self.graph = g
        if self.push_stream is not self.stream:
            self.plan.set_stream(self.push_stream)

    def snapshot(self, final: bool):
        import torch
        with torch.cuda.stream(self.stream):
            self.plan.flush(self.stream)
            if self.graph is not None:
                self.graph.replay()
            else:
                self.plan.snapshot(self.obj, self.phase, stream=self.stream)
            ev = torch.cuda.Event()
            ev.record(self.stream)
        self.inflight.append((ev, self.unsnapped, final))
        self.unsnapped = []
        self.since_snap = 0

    def reconstruct_after(self, flushed):
        """Grouped mode: the reconstruction of a session flushed by a group flush, on the
        session's own stream after the event `flushed` of the shared stream."""
        import torch
        self.stream.wait_event(flushed)
        with torch.cuda.stream(self.stream):
            if self.graph is not None:
                self.graph.replay()
            else:
                self.plan.snapshot(self.obj, self.phase, stream=self.stream)
                self.plan.set_stream(self.push_stream)
            ev = torch.cuda.Event()
            ev.record(self.stream)
        self.recon_done = ev
        self.inflight.append((ev, self.unsnapped, self.due_final))
        self.unsnapped = []
        self.since_snap = 0
        self.due = False


class Server:
    """Serving loop.  `hbm_budget_bytes` bounds the summed plan footprints of admitted sessions."""

    def __init__(self, hbm_budget_bytes: int | None = None, snapshot_every: int = 1024,
                 use_graphs: bool = True, clock=time.perf_counter,
                 snapshot_max_delay_s: float | None = None, grouped: bool = False):
        self.budget = hbm_budget_bytes
        self.grouped = grouped
        self.group_stream = None
        self.snapshot_every = snapshot_every
        self.max_delay = snapshot_max_delay_s
        self.use_graphs = use_graphs
        self.clock = clock
        self.waiting: list[Session] = []
        self.live: dict[int, _Live] = {}
        self.backlog: dict[int, collections.deque] = collections.defaultdict(collections.deque)
        self.used = 0
        self.footprint: dict[int, int] = {}
        self.results: dict[int, np.ndarray] = {}
        self.latencies: list[tuple[float, int]] = []   # (seconds, frames)
        self.done_frames = 0
        self.admission_log: list[tuple[float, int, str]] = []
        self.rejected: list[int] = []                   # sessions larger than the whole budget

    # ---- requests -----------------------------------------------------------------------
    def add_session(self, spec: Session) -> None:
        self.footprint[spec.sid] = wdd.plan_footprint(spec.params)
        self.waiting.append(spec)

    def admit_now(self) -> float:
        """Admits every waiting session that fits (building its plan) and returns the seconds
        spent; used to set sessions up before frames start to flow."""
        t0 = self.clock()
        self._admit()
        return self.clock() - t0

    def offer(self, sid: int, start: int, count: int, t_arrival: float | None = None) -> None:
        """Frames [start, start + count) of session sid have arrived."""
        t = self.clock() if t_arrival is None else t_arrival
        if sid in self.rejected:
            return
        if sid in self.live:
            self.live[sid].pending.append((t, start, count))
        else:
            self.backlog[sid].append((t, start, count))

    # ---- loop body ----------------------------------------------------------------------
    def _admit(self) -> None:
        still = []
        for spec in self.waiting:
            need = self.footprint[spec.sid]
            if self.budget is not None and need > self.budget:
                # can never fit: refused outright rather than admitted over the budget
                self.rejected.append(spec.sid)
                self.backlog.pop(spec.sid, None)
                self.admission_log.append((self.clock(), spec.sid, "reject"))
            elif self.budget is None or self.used + need <= self.budget:
                gs = None
                if self.grouped and _groupable(spec.params):
                    if self.group_stream is None:
                        import torch
                        self.group_stream = torch.cuda.Stream()
                    gs = self.group_stream
                lv = _Live(spec, self.use_graphs, gs)
                self.live[spec.sid] = lv
                self.used += need
                lv.pending.extend(self.backlog.pop(spec.sid, ()))
                self.admission_log.append((self.clock(), spec.sid, "admit"))
            else:
                still.append(spec)
        self.waiting = still

    def _service(self, lv: _Live) -> int:
        """Pushes the session's contiguous pending batches, cut at its snapshot points, and
        snapshots every `snapshot_every` frames.  A grouped session instead stops at its
        snapshot point and waits for the group flush at the end of the pass."""
        grouped = lv.push_stream is not lv.stream
        if lv.due:
            return 0
        actions = 0
        while lv.pending and lv.pending[0][1] == lv.pushed:
            run = []                       # contiguous requests: [t_arrival, frames left]
            end = lv.pushed
            while lv.pending and lv.pending[0][1] == end:
                t, _, c = lv.pending.popleft()
                run.append([t, c])
                end += c
            pos, i = lv.pushed, 0
            while pos < end:
                piece_end = min(end, pos + self.snapshot_every - lv.since_snap)
                need = piece_end - pos
                while need > 0:            # attribute the piece's frames to their requests
                    take = min(run[i][1], need)
                    lv.unsnapped.append((run[i][0], take))
                    run[i][1] -= take
                    need -= take
                    if run[i][1] == 0:
                        i += 1
                idx = np.arange(pos, piece_end, dtype=np.int32)
                lv.plan.push(lv.spec.frames[pos:piece_end], idx, stream=lv.push_stream)
                lv.since_snap += piece_end - pos
                pos = piece_end
                actions += 1
                if lv.since_snap >= self.snapshot_every:
                    if not grouped:
                        lv.snapshot(final=False)
                        continue
                    # the rest of the run waits until the group flush has taken this snapshot
                    lv.due = True
                    back, p0 = [], pos
                    for t, c in run[i:]:
                        if c > 0:
                            back.append((t, p0, c))
                            p0 += c
                    lv.pending.extendleft(reversed(back))
                    lv.pushed = pos
                    return actions
            lv.pushed = end
        if lv.pushed == lv.spec.n_frames and not lv.closing:
            if grouped:
                lv.due = lv.due_final = True
            else:
                lv.snapshot(final=True)
            lv.closing = True
            actions += 1
        elif (self.max_delay is not None and lv.unsnapped and not lv.closing and
              self.clock() - lv.unsnapped[0][0] >= self.max_delay):
            if grouped:
                lv.due = True
            else:
                lv.snapshot(final=False)
            actions += 1
        return actions

    def _flush_due(self) -> int:
        """Grouped mode: one wdd_flush_group per wdd_flush_group_max() sessions that reached a
        snapshot point in this pass, then their reconstructions on their own streams."""
        import torch
        due = [lv for lv in self.live.values() if lv.due]
        if not due:
            return 0
        gs = self.group_stream
        m = wdd.flush_group_max()
        for a in range(0, len(due), m):
            chunk = due[a:a + m]
            for lv in chunk:
                if lv.recon_done is not None:
                    gs.wait_event(lv.recon_done)     # the last reconstruction still reads H
            wdd.flush_group([lv.plan for lv in chunk], gs)
            flushed = torch.cuda.Event()
            flushed.record(gs)
            for lv in chunk:
                lv.reconstruct_after(flushed)
        return len(due)

    def _harvest(self, lv: _Live) -> bool:
        """Records latencies of completed snapshots; returns True when the session is finished."""
        now = None
        keep = []
        finished = False
        for ev, frames, final in lv.inflight:
            if ev.query():
                now = self.clock() if now is None else now
                for t, c in frames:
                    self.latencies.append((now - t, c))
                    self.done_frames += c
                if final:
                    finished = True
            else:
                keep.append((ev, frames, final))
        lv.inflight = keep
        return finished and not keep

    def poll(self) -> int:
        self._admit()
        actions = 0
        for sid in list(self.live):
            actions += self._service(self.live[sid])
        if self.grouped:
            actions += self._flush_due()
        for sid in list(self.live):
            lv = self.live[sid]
            if self._harvest(lv):
                lv.plan.check_device()
                self.results[sid] = lv.phase.cpu().numpy()
                lv.plan.close()
                del self.live[sid]
                self.used -= self.footprint[sid]
                self.admission_log.append((self.clock(), sid, "done"))
                actions += 1
        return actions

    def idle(self) -> bool:
        return not self.live and not self.waiting

    # ---- drivers --------------------------------------------------------------------------
    def run(self, arrivals, open_loop: bool = True, timeout_s: float = 600.0) -> dict:
        """Replays an arrival schedule [(t, sid, start, count)].  Open loop: batches arrive at their
        scheduled times; closed loop: all are available at once.  Returns the statistics."""
        t_start = self.clock()
        i = 0
        n = len(arrivals)
        while True:
            now = self.clock() - t_start
            while i < n and (not open_loop or arrivals[i][0] <= now):
                t, sid, start, count = arrivals[i]
                self.offer(sid, start, count, t_arrival=t_start + (t if open_loop else 0.0))
                i += 1
            acted = self.poll()
            if i == n and self.idle():
                break
            if self.clock() - t_start > timeout_s:
                raise TimeoutError("serving loop did not finish in time")
            if not acted and open_loop and i < n:
                wait = arrivals[i][0] - (self.clock() - t_start)
                if wait > 2e-4:
                    time.sleep(min(wait, 1e-3))
        wall = self.clock() - t_start
        return self.stats(wall)

    def stats(self, wall_s: float) -> dict:
        lat = np.concatenate([np.full(c, t) for t, c in self.latencies]) if self.latencies else np.zeros(1)
        return {"frames": int(self.done_frames), "wall_s": wall_s,
                "frames_per_s": self.done_frames / wall_s if wall_s > 0 else 0.0,
                "latency_p50_ms": float(np.percentile(lat, 50) * 1e3),
                "latency_p99_ms": float(np.percentile(lat, 99) * 1e3),
                "sessions": len(self.results), "rejected": len(self.rejected)}
