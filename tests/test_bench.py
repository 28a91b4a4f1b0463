"""bench.py's host logic on the CPU: the DRAM-traffic record written from an ncu CSV and looked up
per launch (keyed by configuration and by the staged kernel's source hash), and the committed
record's plausibility against the algorithmic bytes of a pass."""
import csv
import json
import os
import types

import pytest

import bench

HDR = ["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context", "Stream", "Block Size",
       "Grid Size", "Device", "CC", "Section Name", "Metric Name", "Metric Unit", "Metric Value"]


def _row(launch, name, metric, unit, value):
    return [str(launch), "1", "python", "h", name, "1", "7", "(352, 1, 1)", "(152, 1, 1)", "0", "10.3", "",
            metric, unit, value]


def test_record_then_look_up_traffic(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "traffic.json"))
    even = "void rtpn::stg::<unnamed>::k_stage<0, float, 0>(rtpn::stg::Args)"
    odd = "void rtpn::stg::<unnamed>::k_stage<1, float, 0>(rtpn::stg::Args)"
    rows = [HDR,
            _row(0, even, "dram__bytes_read.sum", "Gbyte", "3.50"),
            _row(0, even, "dram__bytes_write.sum", "Mbyte", "1,750.00"),
            _row(0, even, "gpu__time_duration.sum", "msecond", "1.40"),
            _row(1, odd, "dram__bytes_read.sum", "Gbyte", "3.60"),
            _row(1, odd, "dram__bytes_write.sum", "Gbyte", "1.70"),
            _row(2, even, "dram__bytes_read.sum", "Gbyte", "9.99")]  # a later launch: ignored
    path = tmp_path / "ncu.csv"
    with open(path, "w", newline="") as f:
        csv.writer(f).writerows(rows)
    args = types.SimpleNamespace(record_traffic=str(path), tile="40,2,2", n=80, N=39, precision="fp32", depth=2)
    bench.record_traffic(args)
    rec = json.load(open(bench.TRAFFIC_FILE))
    assert rec["kernel_sha256"] == bench.kernel_source_hash()
    cells = 80 ** 3
    e0 = rec["entries"]["P39 fp32 tile 40x2x2 depth 2 class 0"]
    assert e0["dram_bytes"] == pytest.approx(3.5e9 + 1.75e9) and e0["bytes_per_cell"] == pytest.approx(5.25e9 / cells)
    # scaled to another grid by the cell count; other configurations have no record
    got, why = bench.traffic_per_launch("stage", 39, "fp32", (40, 2, 2), 2, 1, 200 ** 3)
    assert got == pytest.approx(5.3e9 / cells * 200 ** 3) and "80^3" in why
    assert bench.traffic_per_launch("stage", 39, "bf16", (40, 2, 2), 2, 0, 10)[0] is None
    assert bench.traffic_per_launch("window", 39, "fp32", (40, 2, 2), 2, 0, 10)[0] is None
    # a source change since the capture voids the record
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 64)
    got, why = bench.traffic_per_launch("stage", 39, "fp32", (40, 2, 2), 2, 0, 10)
    assert got is None and "changed" in why


def test_committed_traffic_record_is_plausible():
    # DRAM bytes of a pass can only exceed its algorithmic bytes V ((n_c + n_cls) s + 6) (halo
    # re-reads); far above them the tile would re-read its sources
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "stage_traffic.json")))
    assert len(rec["kernel_sha256"]) == 64
    n_c, n_cls = 1600, {0: 820, 1: 780}
    for storage, s in (("fp32", 4), ("bf16", 2)):
        for cls in (0, 1):
            e = rec["entries"][bench._traffic_key(39, storage, (40, 2, 2), 2, cls)]
            alg = (n_c + n_cls[cls]) * s + 6
            assert 1.0 <= e["bytes_per_cell"] / alg <= 1.3, (storage, cls, e["bytes_per_cell"] / alg)
