"""The DRAM-traffic records bench.py reports (paper_1805_06572_gb300.ncu_traffic): reading a
capture's raw page, and the source hash that keeps a record tied to the code it measured."""
import csv
import json

from paper_1805_06572_gb300 import ncu_traffic


def _raw(path, cols, units, row):
    with open(path, "w", newline="") as fh:
        w = csv.writer(fh)
        w.writerow(cols)
        w.writerow(units)
        w.writerow(row)


def test_split_counters(tmp_path):
    p = tmp_path / "raw.csv"
    _raw(p, ["ID", "Kernel Name", "gpu__time_duration.sum", "dram__bytes_read.sum", "dram__bytes_write.sum"],
         ["", "", "us", "Mbyte", "Kbyte"],
         ["0", "void fast_em_kernel<4, 0, 128, 0, 2>(FastEmArgs)", "511.5", "20.5", "12"])
    r = ncu_traffic.read_launch(str(p), "fast_em_kernel<4, 0, 128, 0, 2>")
    assert r["bytes_per_launch"] == 20.5e6 + 12e3
    assert r["duration_us_under_ncu"] == 511.5


def test_rate_times_duration(tmp_path):
    p = tmp_path / "raw.csv"
    _raw(p, ["ID", "Kernel Name", "gpu__time_duration.sum", "dram__bytes.sum.per_second"],
         ["", "", "ms", "Gbyte/s"],
         ["0", "void conv_em_kernel<4, 0, 128, 0, 0>(ConvEmArgs)", "2", "10"])
    r = ncu_traffic.read_launch(str(p), "conv_em_kernel")
    assert abs(r["bytes_per_launch"] - 2e-3 * 10e9) < 1e-3
    assert r["dram_read_bytes"] is None


def test_committed_records_and_the_staleness_rule(monkeypatch):
    """Every committed record carries the hash of the kernels' code lines it was captured at;
    bench.py reports a record's traffic only while that hash matches the sources."""
    import os
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(ncu_traffic.__file__)))
    sys.path.insert(0, root)
    import bench
    table = json.load(open(os.path.join(root, "profiles", "dram_traffic.json")))
    assert table, "no traffic records"
    for key, rec in table.items():
        assert rec["bytes_per_launch"] > 0 and rec["command"].startswith("ncu "), key
        fresh = rec["source_sha"] == ncu_traffic.source_sha()
        assert bench.profiled_traffic(key) == (rec["bytes_per_launch"] if fresh else None), key
    monkeypatch.setattr(ncu_traffic, "source_sha", lambda: "0" * 12)
    assert all(bench.profiled_traffic(k) is None for k in table)


def test_hash_ignores_comments(tmp_path, monkeypatch):
    d = tmp_path / "csrc"
    d.mkdir()
    for f in ncu_traffic.SOURCES:
        (d / f).write_text("int a;  // one\n\n// note\nint b;\n")
    monkeypatch.setattr(ncu_traffic, "HERE", str(tmp_path))
    h0 = ncu_traffic.source_sha()
    (d / ncu_traffic.SOURCES[0]).write_text("int a;  // two\n// other note\nint b;\n")
    assert ncu_traffic.source_sha() == h0
    (d / ncu_traffic.SOURCES[0]).write_text("int a;\nint c;\n")
    assert ncu_traffic.source_sha() != h0
