"""Write workload_pairs.json: the whole-box pair counts of the benchmark
workloads from the oracle (``oracle.count_pairs``), self excluded -- ordered
gather pairs (r < h_i) and ordered union pairs (r < max(h_i, h_j)) -- for the
inputs each form receives: positions in double, smoothing lengths in double
(fp64) or rounded to float (mixed).  Boxes of a multi-box workload are counted
one by one and summed.  The benchmark's reference arm reports these counts for
the workload whose sample it times.

    python tests/golden/make_workload_pairs.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2511_21921_gb300 import synth  # noqa: E402

WORKLOADS = ["lattice16", "lognormal64", "lognormal128", "clumpy128", "multibox64",
             "lognormal256"]


def counts(d, h):
    if "box_off" not in d:
        return oracle.count_pairs(d["x"], h, d["L"])
    off, L = d["box_off"], d["box_L"]
    g = u = 0
    for b in range(len(off) - 1):
        s = slice(int(off[b]), int(off[b + 1]))
        if s.stop > s.start:
            gb, ub = oracle.count_pairs(np.ascontiguousarray(d["x"][:, s]), h[s], float(L[b]))
            g, u = g + gb, u + ub
    return g, u


def main():
    oracle.build()
    out = {}
    for name in WORKLOADS:
        d = synth.load(name)
        h64 = np.asarray(d["h"], dtype=np.float64)
        h32 = h64.astype(np.float32).astype(np.float64)
        g64, u64 = counts(d, h64)
        g32, u32 = counts(d, h32)
        out[name] = {"n": int(h64.shape[0]), "boxes": int(len(d["box_off"]) - 1) if "box_off" in d else 1,
                     "fp64": {"gather_pairs": g64, "union_pairs": u64},
                     "mixed": {"gather_pairs": g32, "union_pairs": u32}}
        print(name, out[name], flush=True)
    with open(os.path.join(HERE, "workload_pairs.json"), "w") as fh:
        json.dump(out, fh, indent=1, sort_keys=True)
        fh.write("\n")


if __name__ == "__main__":
    main()
