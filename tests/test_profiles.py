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
            m = re.match(r"^(kernel|build_digest|workload|dram_bytes_per_launch): (.*)$", line)
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
        assert re.fullmatch(r"[a-z]+\d+[a-z]*", meta["workload"]), p
        assert int(meta["dram_bytes_per_launch"]) > 0, p
        # a full capture carries the on-chip metrics; a one-pass DRAM capture
        # of a full-size workload carries its duration and DRAM bytes only
        labels = ["duration under ncu", "DRAM read", "DRAM write"]
        if "L1 throughput, %" in rows:
            labels += ["L1 throughput, %", "issue active, %", "FMA pipe active, %",
                       "registers / thread"]
        for label in labels:
            assert float(rows[label].split()[0]) > 0, (p, label)
        with open(p) as fh:
            text = fh.read()
        assert "--clock-control none" in text, p


def test_dominant_kernel_has_a_summary():
    """The adjoint rate sweep: a full capture on the 64^3 box and its DRAM
    traffic on the headline 256^3 box."""
    have = {_meta(p)[0].get("workload") for p in PROFILES
            if "PassA2<float" in _meta(p)[0].get("kernel", "")}
    assert {"lognormal64", "lognormal256"} <= have


@pytest.mark.parametrize("workload", ["lognormal64", "lognormal256"])
def test_launch_list_has_per_step_shares(workload):
    path = os.path.join(ROOT, "profiles", f"launches_{workload}_step.md")
    with open(path) as fh:
        text = fh.read()
    assert "--clock-control none" in text
    shares = re.findall(r"^k_sweep<PassA2<float, 0>, \d+, \d+>\s+1\s+[\d.]+\s+([\d.]+)%$", text,
                        re.M)
    assert shares and 10.0 < float(shares[0]) < 50.0
