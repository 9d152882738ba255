"""Host-side logic of bench.py that needs no GPU: the DRAM-traffic records the
roofline line reads from profiles/, and the clock sampler's parsing of
nvidia-smi output (throttle reasons decide whether a run is kept)."""
import hashlib
import json
import os
import shutil

import pytest

import bench

RECORDS = sorted(f for f in os.listdir(os.path.join(bench.ROOT, "profiles")) if f.endswith(".json.txt"))


def test_traffic_records_exist():
    assert "sjlt_traffic.json.txt" in RECORDS and "tc_traffic.json.txt" in RECORDS


@pytest.mark.parametrize("name", RECORDS)
def test_traffic_record_matches_its_kernel_source(name):
    """Each record was captured on the kernel source as committed, so the bench
    line's roofline carries its traffic instead of null."""
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", name)))
    src = os.path.join(bench.ROOT, rec["kernel_file"])
    assert hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] == rec["source_sha256_16"], name
    got = bench.traffic_from_profile(os.path.basename(src), name)
    assert got is not None and got["source_sha256_16"] == rec["source_sha256_16"]
    # per-launch bytes are the scaled capture and at least the algorithmic A bytes of n = 32768
    for key in ("rows_bytes_per_launch", "cols_bytes_per_launch"):
        if key in rec:
            assert rec[key] >= 32768 * 32768 * 4


def test_traffic_record_of_a_changed_source_is_ignored(tmp_path, monkeypatch):
    """A kernel edited after its capture gives traffic None (reported as null)."""
    (tmp_path / "profiles").mkdir()
    csrc = tmp_path / "paper_2302_01977_gb300" / "csrc"
    csrc.mkdir(parents=True)
    shutil.copy(os.path.join(bench.ROOT, "profiles", "tc_traffic.json.txt"), tmp_path / "profiles")
    src = open(os.path.join(bench.ROOT, "paper_2302_01977_gb300", "csrc", "gemm_tc.cu"), "rb").read()
    (csrc / "gemm_tc.cu").write_bytes(src)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_from_profile("gemm_tc.cu", "tc_traffic.json.txt") is not None
    (csrc / "gemm_tc.cu").write_bytes(src + b"\n// edited\n")
    assert bench.traffic_from_profile("gemm_tc.cu", "tc_traffic.json.txt") is None
    assert bench.traffic_from_profile("gemm_tc.cu", "absent.json.txt") is None


class _FakeSmi:
    def __init__(self, out):
        self.out = out

    def terminate(self):
        pass

    def communicate(self, timeout=None):
        return self.out, ""


def _clocks_from(monkeypatch, out):
    monkeypatch.setattr(bench.subprocess, "Popen", lambda *a, **k: _FakeSmi(out))
    c = bench.Clocks(0)
    c.start()
    return c.stop()


def test_clocks_median_and_no_reasons(monkeypatch):
    rows = "\n".join(f"0, {mhz}, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active"
                     for mhz in (2070, 2055, 2070, 1980, 2070))
    got = _clocks_from(monkeypatch, rows + "\n")
    assert got["sm_mhz"] == 2070.0 and got["sm_max_mhz"] == 2070.0
    assert got["reasons"] == [] and got["samples"] == 5


def test_clocks_throttle_reasons_are_reported(monkeypatch):
    rows = ["0, 2070, 2070, 1390.0, 0x0, Not Active, Not Active, Not Active, Active",
            "0, 1800, 2070, 1400.0, 0x8, Active, Not Active, Not Active, Active",
            "0, 1700, 2070, 1400.0, 0x40, Not Active, Active, Active, Not Active",
            "garbage line",
            "0, [N/A], 2070, 1400.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    got = _clocks_from(monkeypatch, "\n".join(rows) + "\n")
    assert got["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert got["samples"] == 3 and got["sm_mhz"] == 1800.0


def test_clocks_without_nvidia_smi(monkeypatch):
    def boom(*a, **k):
        raise OSError("no nvidia-smi")

    monkeypatch.setattr(bench.subprocess, "Popen", boom)
    c = bench.Clocks(0)
    c.start()
    got = c.stop()
    assert got["sm_mhz"] is None and got["reasons"] == ["nvidia-smi unavailable"]
