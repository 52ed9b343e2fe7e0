"""Record the DRAM traffic of a profiled kernel launch in profiles/dram_traffic.json.

The benchmark's roofline records carry, next to the algorithmic bytes, the DRAM bytes one
launch of the kernel actually moved (dram__bytes_read.sum + dram__bytes_write.sum from an
Nsight Compute capture). This module turns the raw page of a capture into that record and
stamps it with a hash of the kernel sources, so that a record taken on older code is not
reported for newer code (bench.py reads it only while the hash matches).

  ncu -i capture.ncu-rep --page raw --csv > raw.csv
  python -m paper_1805_06572_gb300.ncu_traffic raw.csv 'fast_em_kernel<4, 0, 128, 0, 2>' \\
      'fast_em_kernel<4,c64,128,refined>' --command '<the profiled command line>'

The second argument selects the captured launch by a substring of its kernel name; the third
is the key bench.py looks the record up by.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import json
import os

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
PROFILES = os.path.join(ROOT, "profiles", "dram_traffic.json")
SOURCES = ("fca_dev.cuh", "fca_fast.cuh", "fca_conv.cu")


def source_sha() -> str:
    """Hash of the code of the fused EM kernels' sources (both forms): comments and blank lines
    are left out, so that a change to the documentation alone keeps a capture valid."""
    h = hashlib.sha256()
    for f in SOURCES:
        with open(os.path.join(HERE, "csrc", f), encoding="utf-8") as fh:
            for line in fh:
                code = line.split("//", 1)[0].strip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:12]


def _bytes(value: str, unit: str) -> float:
    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9}
    if unit not in scale:
        raise SystemExit(f"unknown byte unit {unit!r}")
    return float(value.replace(",", "")) * scale[unit]


def _usecond(value: str, unit: str) -> float:
    scale = {"nsecond": 1e-3, "usecond": 1.0, "msecond": 1e3, "second": 1e6,
             "ns": 1e-3, "us": 1.0, "ms": 1e3, "s": 1e6}
    if unit not in scale:
        raise SystemExit(f"unknown time unit {unit!r}")
    return float(value.replace(",", "")) * scale[unit]


def read_launch(raw_csv: str, name_part: str) -> dict:
    """The first launch in a raw-page CSV whose kernel name contains name_part."""
    with open(raw_csv, newline="") as fh:
        rows = list(csv.reader(fh))
    head, units = rows[0], rows[1]
    col = {k: i for i, k in enumerate(head)}
    for row in rows[2:]:
        if len(row) < len(head) or name_part not in row[col["Kernel Name"]]:
            continue
        dur = _usecond(row[col["gpu__time_duration.sum"]], units[col["gpu__time_duration.sum"]])
        if "dram__bytes_read.sum" in col:
            rd = _bytes(row[col["dram__bytes_read.sum"]], units[col["dram__bytes_read.sum"]])
            wr = _bytes(row[col["dram__bytes_write.sum"]], units[col["dram__bytes_write.sum"]])
            total = rd + wr
        else:  # sections without the split counters: the summed DRAM rate times the duration
            k = "dram__bytes.sum.per_second"
            rate = float(row[col[k]].replace(",", "")) * {"byte/s": 1, "Kbyte/s": 1e3, "Mbyte/s": 1e6,
                                                          "Gbyte/s": 1e9, "Tbyte/s": 1e12}[units[col[k]]]
            rd = wr = None
            total = rate * dur * 1e-6
        return {"kernel_name": row[col["Kernel Name"]], "dram_read_bytes": rd, "dram_write_bytes": wr,
                "bytes_per_launch": total, "duration_us_under_ncu": dur}
    raise SystemExit(f"no launch of a kernel named like {name_part!r} in {raw_csv}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("raw_csv")
    ap.add_argument("name_part")
    ap.add_argument("key")
    ap.add_argument("--command", required=True, help="the profiled command line, for the record")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="launch units of the benchmarked launch / units of the captured one")
    args = ap.parse_args()
    rec = read_launch(args.raw_csv, args.name_part)
    rec["bytes_per_launch"] *= args.scale
    rec.update({"scale": args.scale, "source_sha": source_sha(), "command": args.command})
    try:
        with open(PROFILES) as fh:
            table = json.load(fh)
    except (OSError, ValueError):
        table = {}
    table[args.key] = rec
    with open(PROFILES, "w") as fh:
        json.dump(table, fh, indent=1, sort_keys=True)
        fh.write("\n")
    print(json.dumps({args.key: rec}))


if __name__ == "__main__":
    main()
