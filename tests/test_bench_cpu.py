"""bench.py's host-side arithmetic on the CPU: the T-table lookup count
behind the roofline, the captured-traffic record and its source-hash guard,
the clock-sample summary, and the workload naming."""
import importlib.util
import json
import os
import sys

import numpy as np
import pytest

from paper_2607_02630_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


def brute_force_lookups(w):
    """16*Nr lookups per block, minus rounds 1-2 for all but the counter-group
    constants: count block by block which counter group each block is in."""
    total = 0
    for n, b, iv in zip(w.lengths, w.bits, w.ivs):
        nb = (int(n) + 15) // 16
        nr = int(b) // 32 + 6
        v0 = int(iv[15])
        groups = set()
        for j in range(nb):
            groups.add((v0 + j) >> 8)
            total += 16 * nr - 32 + 5
        total += 27 * len(groups)
    return total


def test_ttable_lookups_matches_block_by_block_count(bench):
    w = W.batch_varlen(n=24, min_len=1, max_len=20000, seed=11, with_payload=False)
    assert bench.ttable_lookups(w) == brute_force_lookups(w)


def test_ttable_lookups_closed_form_for_one_group(bench):
    class One:
        lengths = np.array([256 * 16])
        bits = np.array([128])
        ivs = np.zeros((1, 16), np.uint8)
    # 256 blocks in one counter group: 256 * (160 - 27) + 27
    assert bench.ttable_lookups(One) == 256 * 133 + 27


def test_captured_traffic_scales_and_guards_the_source_hash(bench, tmp_path, monkeypatch):
    rec = {"kernel": "k", "dram_bytes": 2000, "payload_bytes": 1000, "kernel_src_sha": bench.kernel_source_hash()}
    f = tmp_path / "traffic.txt"
    f.write_text(json.dumps(rec) + "\n")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.captured_traffic(5000) == 10000
    rec["kernel_src_sha"] = "0" * 16
    f.write_text(json.dumps(rec) + "\n")
    assert bench.captured_traffic(5000) is None
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.txt"))
    assert bench.captured_traffic(5000) is None


def test_committed_traffic_record_matches_the_batch_kernel_sources(bench):
    """The committed ncu record is for the batch kernel as it is now."""
    with open(bench.TRAFFIC_FILE) as f:
        rec = json.loads(f.readline())
    assert rec["kernel_src_sha"] == bench.kernel_source_hash()
    assert 1.5 < rec["dram_bytes"] / rec["payload_bytes"] < 2.5  # about 2 bytes moved per payload byte


def test_clock_summary(bench):
    c = bench.ClockSampler(0)
    c.lines = ["0, 2070, 2070, 650.5, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 2055, 2070, 700.0, 0x4, Not Active, Not Active, Not Active, Active",
               "garbage line"]
    s = c.summary()
    assert s["samples"] == 2 and s["sm_max_mhz"] == 2070.0 and s["reasons"] == ["sw_power_cap"]
    assert s["sm_mhz"] == pytest.approx(2062.5) and s["power_w_max"] == 700.0
    empty = bench.ClockSampler(0).summary()
    assert empty["samples"] == 0 and empty["reasons"] == []


def test_workload_name(bench):
    assert bench.workload_name(4096) == bench.WORKLOAD
    assert bench.workload_name(512).startswith("512 requests of: ")


class _FakeProps:
    multi_processor_count = 152


class _FakeCuda:
    @staticmethod
    def get_device_properties(dev):
        return _FakeProps()


class _FakeTorch:
    cuda = _FakeCuda()


def test_bitslice_ops_counts_the_circuit(bench):
    """Per 32 blocks: 16 S-box circuits of 113 gates per round, 416
    MixColumns xors per full round, 128 key xors per round key."""
    class One:
        lengths = np.array([32 * 16, 32 * 16])
        bits = np.array([128, 256])
    want = (16 * 113 * 10 + 416 * 9 + 128 * 11) + (16 * 113 * 14 + 416 * 13 + 128 * 15)
    assert bench.bitslice_ops(One) == pytest.approx(want)


def test_batch_roofline_divides_by_the_measured_rate_of_the_picked_variant(bench):
    w = W.batch_varlen(n=16, min_len=1024, max_len=1 << 20, seed=12, with_payload=False)
    rates = {"lds32_per_clk_sm": 16.0, "lop3_per_clk_sm": 32.0, "zero_copy_each_way_gbs": 100.0}
    step = int(w.lengths.sum())
    tt = bench.batch_roofline(_FakeTorch, 0, w, step, [1e-3], {"variant": 1}, rates)
    bs = bench.batch_roofline(_FakeTorch, 0, w, step, [1e-3], {"variant": 2}, rates)
    f = float(bench.peaks()[0].get("sm_max_mhz", 2070.0)) * 1e6
    assert tt["kernel"] == "batch_ttable_kernel" and bs["kernel"] == "batch_bitslice_kernel"
    assert tt["peak"] == pytest.approx(step / (bench.ttable_lookups(w) / (16.0 * 152 * f)) / 1e9, rel=1e-3)
    assert bs["peak"] == pytest.approx(step / (bench.bitslice_ops(w) / (32.0 * 152 * f)) / 1e9, rel=1e-3)
    assert tt["achieved"] == pytest.approx(step / 1e-3 / 1e9, abs=0.01)  # rounded to 2 decimals
    assert "measured on this GPU" in tt["peak_basis"]
    nominal = bench.batch_roofline(_FakeTorch, 0, w, step, [1e-3], {"variant": 1}, {"error": "no GPU"})
    assert "nominal rate" in nominal["peak_basis"]
    assert nominal["peak"] == pytest.approx(2 * tt["peak"], rel=1e-3)  # 32 per clk instead of the fake 16
