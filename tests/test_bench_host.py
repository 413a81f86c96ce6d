"""Host-side logic of bench.py that needs no GPU: the clock record parsed from nvidia-smi lines,
the stale-capture rule of the traffic record, and the whole-job rate."""
import hashlib
import json
import os

import bench


class _Done:
    """Stands in for a finished nvidia-smi process."""

    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.proc = _Done()
    s.lines = list(lines)
    return s


def test_clock_record_median_max_and_reasons():
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2055, 2070, 1100.4, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
            "garbled line",
            "0, [N/A], 2070, 10, 0x0, Not Active, Not Active, Not Active, Not Active"]
    rec = _sampler(rows).stop()
    assert rec["sm_mhz"] == 2055.0
    assert rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]
    assert rec["samples"] == 3


def test_clock_record_reports_thermal_slowdown():
    rows = ["0, 1500, 2070, 1400, 0x20, Not Active, Active, Active, Not Active"]
    rec = _sampler(rows).stop()
    assert rec["reasons"] == ["hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_record_without_nvidia_smi():
    s = bench.ClockSampler(0)
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_traffic_record_is_dropped_when_the_source_changes(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel v1")
    (tmp_path / "profiles").mkdir()
    rec = {"source": "k.cu", "sha256": hashlib.sha256(b"kernel v1").hexdigest(),
           "bytes_per_launch": 123}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"k@c2": rec}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic("k", "c2")["bytes_per_launch"] == 123
    assert bench._traffic("other", "c2") is None
    assert bench._traffic("k", "c5") is None     # captured on another workload
    src.write_text("kernel v2")
    assert bench._traffic("k", "c2") is None


def test_committed_traffic_records_name_existing_sources():
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        recs = json.load(f)
    for name, rec in recs.items():
        if name.startswith("_"):
            continue
        assert os.path.exists(os.path.join(bench.ROOT, rec["source"])), name
        kernel, _, workload = name.partition("@")
        assert kernel and workload in bench.WORKLOADS, name


def test_whole_job_rate():
    assert bench.job_throughput(1000, 1, 2.0) == 500000.0
    assert bench.job_throughput(1000, 4, 2.0) == 2000000.0
    assert bench.max_over_ranks(3.5, 1) == 3.5


def test_exec_factor_counts_the_computed_scan_columns():
    # three split products (hi*hi, hi*lo, lo*hi) over the S_x / 2 + 1 computed columns
    assert bench.exec_factor({"spectrum_cols": 65, "spectrum_cols_total": 128}) == 3 * 65 / 128
    assert bench.exec_factor({"spectrum_cols": 129, "spectrum_cols_total": 256}) == 3 * 129 / 256
    # every column computed: three products per algorithmic product
    assert bench.exec_factor({"spectrum_cols": 40, "spectrum_cols_total": 40}) == 3.0
