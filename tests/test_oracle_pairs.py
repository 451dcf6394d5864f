"""The oracle's whole-box pair counts (count_pairs), which the full-size GPU
tests and the benchmark's reference arm use: equal to the sizes of the oracle's
neighbor sets (themselves pinned against brute force), and the stored counts
of the small benchmark workloads reproduce."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2511_21921_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "workload_pairs.json")


@pytest.mark.parametrize("case", ["lattice16", "lognormal32", "lognormal32m"])
def test_counts_are_the_set_sizes(case):
    d = synth.load(case)
    n = d["h"].shape[0]
    g, u = oracle.count_pairs(d["x"], d["h"], d["L"])
    _, cg = oracle.neighbors(d["x"], d["h"], d["L"], mode="gather")
    _, cu = oracle.neighbors(d["x"], d["h"], d["L"], mode="union")
    assert g == len(cg) - n  # the gather sets hold the particle itself
    assert u == len(cu)
    assert g <= u <= 2 * g  # a union pair is a gather pair of one side at least


def test_brute_force_counts_on_a_tiny_box():
    rng = np.random.default_rng(3)
    n = 300
    x = rng.random((3, n))
    h = rng.uniform(0.05, 0.2, n)
    d = x[:, :, None] - x[:, None, :]
    d -= np.round(d)  # minimum image in the unit box
    r2 = (d ** 2).sum(0)
    off = ~np.eye(n, dtype=bool)
    g = int(((r2 < h[:, None] ** 2) & off).sum())
    u = int(((r2 < np.maximum(h[:, None], h[None, :]) ** 2) & off).sum())
    assert oracle.count_pairs(x, h, 1.0) == (g, u)


@pytest.mark.parametrize("name", ["lattice16", "lognormal64"])
def test_stored_counts_reproduce(name):
    with open(GOLDEN) as fh:
        want = json.load(fh)[name]
    d = synth.load(name)
    h64 = np.asarray(d["h"], dtype=np.float64)
    h32 = h64.astype(np.float32).astype(np.float64)
    for form, h in (("fp64", h64), ("mixed", h32)):
        g, u = oracle.count_pairs(d["x"], h, d["L"])
        assert (g, u) == (want[form]["gather_pairs"], want[form]["union_pairs"]), form
    assert want["n"] == h64.shape[0]
