"""The reference arm of bench.py on CPU: one JSON line with the keys the
benchmark contract asks for, on the same metric, unit and direction as the
GPU arm (it times the oracle, so it needs no GPU)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "tiny", "--steps", "1",
                          "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600, check=True)
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    j = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    assert j["impl"] == "reference" and j["metric"] == bench.METRIC and j["unit"] == "Mpts/s"
    assert j["higher_is_better"] is True and j["scaling"] == "weak" and j["vs_baseline"] is None
    assert j["n_gpus"] == 1 and j["steps"] == 1 and j["warmup"] == 0
    assert j["value"] > 0 and j["ms_per_step"] > 0 and j["dtype"] == "int64" and j["data"] == "synthetic"
    assert j["config"]["workload"] == bench.WORKLOADS["tiny"]
    cb = j["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == j["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = j["e2e"]
    assert e2e["value"] == j["value"] and e2e["unit"] == j["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_stage_byte_model():
    """The algorithmic bytes behind stage_bandwidth, per point, for the three
    ways the compaction gets its grid-order rows: rebuilt from a 4-byte
    in-cell offset word (d offsets of bit_length(s - 1) bits fit 32 bits),
    rebuilt from the identifiers alone (s = 1), or gathered from the input
    rows (the offsets exceed 32 bits, or the key is not packed)."""
    sys.path.insert(0, ROOT)
    import bench
    n = 1000
    ms = {"bounds": 1.0, "quantise": 1.0, "sort": 1.0, "compact": 1.0}

    def per_point(d, kc, side, passes=3):
        sb = bench.stage_bandwidth(ms, n, d, {"key_class": kc, "sort_passes": passes, "side": side}, 1.0)
        return {k: v["bytes"] // n for k, v in sb.items()}

    # d = 3, s = 289 (9-bit offsets, 27 bits): key 8, offset word 4, rows padded to 4 ints
    b = per_point(3, 0, 289)
    assert b["bounds"] == 12 and b["quantise"] == 12 + 8 + 4
    assert b["sort"] == 3 * 16 + 2 * 8          # three passes, two upsweeps (the first is quantisation's)
    assert b["compact"] == 2 * 8 + 4 + 4 + 4 + 16
    # d = 3, s = 1: every offset is 0, no word is written or read
    b = per_point(3, 0, 1)
    assert b["quantise"] == 12 + 8 and b["compact"] == 2 * 8 + 4 + 4 + 16
    # d = 5, s = 448 (9-bit offsets, 45 bits): the input rows are gathered
    b = per_point(5, 0, 448)
    assert b["quantise"] == 20 + 8 and b["compact"] == 2 * 8 + 4 + 4 + 20 + 32
    # d = 4, s = 256 (8-bit offsets, exactly 32 bits): rebuilt
    b = per_point(4, 0, 256)
    assert b["compact"] == 2 * 8 + 4 + 4 + 4 + 16
    # 64-bit key with index values: no packed index, rows gathered
    b = per_point(3, 1, 289)
    assert b["quantise"] == 12 + 8 + 4 and b["compact"] == 2 * 8 + 4 + 4 + 4 + 12 + 16
