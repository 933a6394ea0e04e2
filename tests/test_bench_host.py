"""Host-side pieces of bench.py on the CPU: the committed DRAM traffic is
used only while the kernel source it was measured on is unchanged, the
clock record flags throttling, and the per-round MIS summary reads the
fl_mis_log rows."""
import json
import os
import shutil

import numpy as np
import pytest

import bench


def test_committed_traffic_matches_the_current_merge_kernel():
    """profiles/traffic.json was taken on the k_sketch.cu that is committed:
    the bench reports it (a change to the kernel must drop it)."""
    t = bench.ncu_traffic("k_merge_hop", "rmat26")
    with open(os.path.join(bench.PROFILE_DIR, "traffic.json")) as fh:
        d = json.load(fh)
    assert t == d["k_merge_hop"]["rmat26"]["dram_bytes_per_launch"]
    assert t > 0


def test_traffic_is_dropped_once_the_kernel_changes(tmp_path, monkeypatch):
    src_dir = tmp_path / "paper_1503_03635_gb300" / "csrc"
    src_dir.mkdir(parents=True)
    prof = tmp_path / "profiles"
    prof.mkdir()
    shutil.copy(os.path.join(bench.PROFILE_DIR, "traffic.json"), prof / "traffic.json")
    orig = os.path.join(bench.ROOT, "paper_1503_03635_gb300", "csrc", "k_sketch.cu")
    shutil.copy(orig, src_dir / "k_sketch.cu")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "PROFILE_DIR", str(prof))
    assert bench.ncu_traffic("k_merge_hop", "rmat26") is not None
    with open(src_dir / "k_sketch.cu", "a") as fh:
        fh.write("\n// edited\n")
    assert bench.ncu_traffic("k_merge_hop", "rmat26") is None
    assert bench.ncu_traffic("k_merge_hop", "rmat20") is None  # no capture for that workload
    assert bench.ncu_traffic("no_such_kernel", "rmat26") is None


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _clock_record(tmp_path, rows):
    c = bench.Clocks(0)
    c.path = str(tmp_path / "clocks.csv")
    with open(c.path, "w") as fh:
        for r in rows:
            fh.write(", ".join(r) + "\n")
    c.fh = open(os.devnull, "w")
    c.proc = _Done()
    return c.stop()


def test_clock_record_median_and_reasons(tmp_path):
    rows = [["0", str(mhz), "2070", "900.0", "0x0", "Not Active", "Not Active", "Not Active", cap]
            for mhz, cap in ((2070, "Not Active"), (1980, "Active"), (2070, "Not Active"))]
    out = _clock_record(tmp_path, rows)
    assert out["sm_mhz"] == 2070 and out["sm_max_mhz"] == 2070 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_record_flags_thermal_slowdown(tmp_path):
    rows = [["0", "1500", "2070", "1300.0", "0x28", "Active", "Active", "Not Active", "Not Active"],
            ["0", "bad", "2070", "1300.0", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]]
    out = _clock_record(tmp_path, rows)
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]
    assert out["sm_mhz"] == 1500 and out["samples"] == 2


def test_clock_record_without_samples():
    c = bench.Clocks(0)
    assert c.stop() is None


def test_mis_summary_reads_the_log_rows():
    # (round, kind, step, frontier, pulled, us)
    rows = np.array([
        [1, 2, 0, 5, 0, 0], [1, 2, 3, 7, 0, 0],
        [1, 0, 0, 12, 0, 150], [1, 0, 1, 900, 1, 2500],
        [1, 1, 1, 800, 1, 1200],
        [1, 4, 1, 40, 0, 90],
        [1, 3, 3, 12, 11, 6000],
        [2, 0, 0, 1, 0, 100], [2, 1, 1, 3, 0, 80], [2, 3, 1, 1, 1, 400],
    ], dtype=np.int64)
    s = bench.mis_summary(rows)
    assert [d["round"] for d in s] == [1, 2]
    assert s[0]["undecided"] == 12 and s[0]["decided"] == 11 and s[0]["T"] == 3 and s[0]["ms"] == 6.0
    assert s[0]["buckets"] == {0: 5, 3: 7}
    assert s[0]["cover"] == [[0, 12, 0, 0.15], [1, 900, 1, 2.5]] and s[0]["gather"] == [[1, 800, 1, 1.2]]
    assert s[1]["decided"] == 1 and s[1]["buckets"] == {}
    assert sum(d["decided"] for d in s) == 12
    assert bench.mis_summary(None) is None and bench.mis_summary(np.zeros((0, 6), np.int64)) is None


def test_measured_peak_is_read_from_the_file():
    peak, kind = bench.measured_peaks()
    p = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            assert peak == pytest.approx(float(json.load(fh)["hbm_gbs"]))
        assert kind == "measured"
    else:
        assert (peak, kind) == (6800.0, "fallback")
