"""The serving workload's sessions and seeded arrival schedule (CPU)."""
import numpy as np

import synth


def test_serving_mix_shapes():
    mix = synth.serving_mix()
    sizes = [((a.scan_y, a.scan_x), a.det) for a, _ in mix]
    assert sizes == list(synth.SERVING_SIZES)
    for a, rc in mix:
        assert 100 <= a.dose <= 1e4 and 15e-3 <= a.semiconv_rad <= 30e-3
        assert abs(a.defocus_m) <= 10e-9 and a.dtype == "u16"
        assert rc["rank_k"] == (64 if a.det <= 96 else 128 if a.det == 128 else 256)
    assert sum(a.n_frames for a, _ in mix) == 217088


def test_arrivals_cover_every_frame_in_raster_order():
    mix = synth.serving_mix()
    n = [a.n_frames for a, _ in mix]
    arr = synth.serving_arrivals(n)
    nxt = [0] * len(n)
    t_prev = 0.0
    for t, sid, start, count in arr:
        assert t >= t_prev and 1 <= count <= 512
        assert start == nxt[sid]
        nxt[sid] += count
        t_prev = t
    assert nxt == n
    # mean aggregate rate close to 20k frames/s
    rate = sum(n) / arr[-1][0]
    assert 17000 < rate < 23000
    assert synth.serving_arrivals(n) == arr   # seeded


def test_session_above_the_whole_budget_is_refused():
    """Admission never goes over the HBM budget: a session whose plan alone exceeds it is
    refused (and counted), not admitted because nothing else is live.  Host logic only: the
    refused session never builds a plan."""
    import pytest
    wdd = pytest.importorskip("paper_2212_01309_gb300.wdd")
    from paper_2212_01309_gb300 import serving
    acq, rc = synth.serving_mix()[0]
    p = wdd.params_from_acquisition(acq, basis=rc["basis"], rank_k=rc["rank_k"])
    srv = serving.Server(hbm_budget_bytes=wdd.plan_footprint(p) - 1)
    srv.add_session(serving.Session(sid=0, params=p, frames=None, n_frames=acq.n_frames))
    stats = srv.run([(0.0, 0, 0, 64), (0.0, 0, 64, 64)], open_loop=False, timeout_s=5)
    assert stats["rejected"] == 1 and stats["sessions"] == 0 and stats["frames"] == 0
    assert srv.admission_log[0][1:] == (0, "reject") and not srv.live


class _FakePlan:
    """Stands in for wdd.Plan on the CPU: records pushes and flush points."""
    log = {}

    def __init__(self, params):
        self.params = params
        self.sid = None
        self.pushed = 0
        self.events = []

    def set_stream(self, stream):
        pass

    def push(self, frames, idx, stream=None):
        assert idx[0] == self.pushed          # raster order, contiguous
        self.events.append(("push", int(idx[0]), len(idx)))
        self.pushed += len(idx)

    def flush(self, stream=None):
        self.events.append(("flush", self.pushed))

    def snapshot(self, obj=None, phase=None, stream=None):
        self.events.append(("snapshot", self.pushed))

    def check_device(self):
        pass

    def close(self):
        pass


class _FakeTensor:
    def cpu(self):
        return self

    def numpy(self):
        return np.zeros(1)


def _fake_device(monkeypatch, group_max):
    """Fakes the CUDA objects the serving loop touches, and the grouped flush."""
    import contextlib
    import torch
    from paper_2212_01309_gb300 import serving

    class Stream:
        def wait_event(self, ev):
            pass

    class Event:
        def record(self, stream=None):
            pass

        def query(self):
            return True

    class Graph:
        def capture_begin(self):
            pass

        def capture_end(self):
            pass

        def replay(self):
            pass

    groups = []

    def flush_group(plans, stream):
        assert 1 <= len(plans) <= group_max and len(set(map(id, plans))) == len(plans)
        groups.append([p.sid for p in plans])
        for p in plans:
            p.events.append(("flush", p.pushed))

    monkeypatch.setattr(torch.cuda, "Stream", Stream)
    monkeypatch.setattr(torch.cuda, "Event", Event)
    monkeypatch.setattr(torch.cuda, "CUDAGraph", Graph)
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    monkeypatch.setattr(torch, "empty", lambda *a, **k: _FakeTensor())
    monkeypatch.setattr(serving.wdd, "Plan", _FakePlan)
    monkeypatch.setattr(serving.wdd, "plan_footprint", lambda p: 1)
    monkeypatch.setattr(serving.wdd, "flush_group", flush_group)
    monkeypatch.setattr(serving.wdd, "flush_group_max", lambda: group_max)
    return groups


def _serve_fake(grouped, n_frames, arrivals, precision="split"):
    import pytest
    wdd = pytest.importorskip("paper_2212_01309_gb300.wdd")
    from paper_2212_01309_gb300 import serving
    acq, rc = synth.serving_mix()[0]
    srv = serving.Server(snapshot_every=100, grouped=grouped)
    plans = {}
    orig = serving._Live.__init__

    def init(self, spec, use_graph, group_stream=None):
        orig(self, spec, use_graph, group_stream)
        self.plan.sid = spec.sid
        plans[spec.sid] = self.plan

    serving._Live.__init__ = init
    try:
        for sid, n in enumerate(n_frames):
            p = wdd.params_from_acquisition(acq, basis=rc["basis"], rank_k=rc["rank_k"],
                                            precision=precision if sid != 1 else "fp32")
            srv.add_session(serving.Session(sid=sid, params=p, frames=np.zeros(n), n_frames=n))
        stats = srv.run(arrivals, open_loop=False, timeout_s=10)
    finally:
        serving._Live.__init__ = orig
    return stats, {sid: p.events for sid, p in plans.items()}


def test_grouped_serving_schedule_matches_per_session(monkeypatch):
    """Grouped mode on the CPU with faked CUDA objects: every session gets the same pushes and
    flush points as in per-session mode (snapshot points every 100 frames and at the end), the
    groups hold at most wdd_flush_group_max() distinct split sessions, and the FP32 session
    (sid 1) keeps its own flushes."""
    n_frames = [950, 333, 720, 64, 1001]
    arrivals = synth.serving_arrivals(n_frames, seed=5, bmin=16, bmax=150)
    groups = _fake_device(monkeypatch, group_max=3)
    s_ref, ev_ref = _serve_fake(False, n_frames, arrivals)
    assert not groups
    s_grp, ev_grp = _serve_fake(True, n_frames, arrivals)
    assert s_ref["frames"] == s_grp["frames"] == sum(n_frames)
    assert s_grp["sessions"] == len(n_frames)
    for sid in ev_ref:
        pushes = lambda ev: [e for e in ev if e[0] == "push"]
        flushes = lambda ev: [e[1] for e in ev if e[0] == "flush"]
        assert pushes(ev_grp[sid]) == pushes(ev_ref[sid]), sid
        # the graph capture flushes once at admission; then one flush per snapshot
        assert flushes(ev_grp[sid]) == flushes(ev_ref[sid]), sid
        assert all(p[2] <= 100 for p in pushes(ev_grp[sid]))
    members = [sid for g in groups for sid in g]
    assert 1 not in members and set(members) == {0, 2, 3, 4}
    assert max(len(g) for g in groups) == 3
