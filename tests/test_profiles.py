"""The committed ncu summaries carry what the benchmark reads from them (CPU):
the kernel, the build digest they were taken on, DRAM bytes per launch and the
metric table; the launch-list summary carries the per-step shares."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))


def _meta(path):
    meta, rows = {}, {}
    with open(path) as fh:
        for line in fh:
            m = re.match(r"^(kernel|build_digest|dram_bytes_per_launch): (.*)$", line)
            if m:
                meta[m.group(1)] = m.group(2).strip()
            elif line.startswith("| ") and line.count("|") == 3:
                k, v = [c.strip() for c in line.strip().strip("|").split("|")]
                rows[k] = v
    return meta, rows


def test_kernel_summaries_have_what_the_bench_reads():
    kern = [p for p in PROFILES if "kernel" in _meta(p)[0]]
    assert len(kern) >= 4
    for p in kern:
        meta, rows = _meta(p)
        assert re.fullmatch(r"[0-9a-f]{64}", meta["build_digest"]), p
        assert int(meta["dram_bytes_per_launch"]) > 0, p
        for label in ("duration under ncu", "L1 throughput, %", "issue active, %",
                      "FMA pipe active, %", "registers / thread"):
            assert float(rows[label].split()[0]) > 0, (p, label)
        with open(p) as fh:
            text = fh.read()
        assert "--clock-control none" in text, p


def test_dominant_kernel_has_a_summary():
    assert any("PassA2<float>" in _meta(p)[0].get("kernel", "") for p in PROFILES)


def test_launch_list_has_per_step_shares():
    path = os.path.join(ROOT, "profiles", "launches_lognormal64_step.md")
    with open(path) as fh:
        text = fh.read()
    assert "--clock-control none" in text
    shares = re.findall(r"^k_sweep<PassA2<float>, \d+, \d+>\s+[\d.]+\s+([\d.]+)%$", text, re.M)
    assert shares and 10.0 < float(shares[0]) < 50.0
