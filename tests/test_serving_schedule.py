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
