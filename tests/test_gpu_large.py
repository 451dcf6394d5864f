"""Full-size parity of the other benchmark configurations, on sampled outputs
the oracle computes one by one (its lazy target mode):

* clumpy128: 2,097,152 particles, 200 Plummer clumps on a variance-3 lognormal
  background, smoothing lengths spanning about two decades;
* multibox64: 64 independent boxes of 8^3 .. 96^3 particles in one call;
* lognormal256: the largest configuration, 16.8 M particles in one box.

All in the mixed form the benchmark runs (float pairs, double-float
separations).  These generate a few million particles and take minutes.  The
whole box's pair counts (ordered gather and union pairs of the lists) must
equal the oracle's exactly (tests/golden/workload_pairs.json, written by
make_workload_pairs.py beside it from the oracle's count_pairs).
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2511_21921_gb300 import synth

from gpu_util import TOL, compare, run_forward, to_dev

pytestmark = pytest.mark.gpu


def _golden_counts(s, name):
    """The list build's whole-box pair counts against the oracle's."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "workload_pairs.json")
    with open(path) as fh:
        want = json.load(fh)[name]["mixed"]
    st = s.stats()
    assert (st["gather_pairs"], st["union_pairs"]) == (want["gather_pairs"], want["union_pairs"])


def _stratified(h, k, rng):
    """k indices spread over the range of h (small-h clump members included)."""
    order = np.argsort(h)
    picks = np.linspace(0, h.size - 1, k).astype(np.int64)
    jitter = rng.integers(-50, 51, size=k)
    return np.unique(order[np.clip(picks + jitter, 0, h.size - 1)])


def test_clumpy128_sampled_parity_mixed():
    d = synth.load("clumpy128")
    assert d["h"].max() / d["h"].min() > 50
    gpu, s = run_forward(d, "mixed")
    assert gpu["status"] == 0
    _golden_counts(s, "clumpy128")
    tg = _stratified(d["h"], 96, np.random.default_rng(5))
    ora = oracle.forward(d["x"], d["h"], d["m"], d["v"], d["u"], 1.0, targets=tg)
    err = compare(gpu, ora, idx=tg)
    for k in ("dvdt", "dudt"):
        assert err[k] < TOL["mixed"], (k, err)
    for k, e in err.items():
        assert e < 5e-5, (k, err)


def test_clumpy128_adjoint_dot_mixed():
    d = synth.load("clumpy128")
    n = d["h"].shape[0]
    from paper_2511_21921_gb300.solver import Solver
    s = Solver(n, 1, "mixed")
    t = to_dev(d, "mixed")
    s.cell_build(t["x"], t["h"])
    s.moments(t["m"])
    s.rates(t["v"], t["u"])
    ga, gu = synth.cotangents(n, seed=14)
    g = s.adjoint(t["v"], t["u"], torch.tensor(ga, dtype=torch.float32, device="cuda"),
                  torch.tensor(gu, dtype=torch.float32, device="cuda"), recompute=False)
    grads = [a.double().cpu().numpy() for a in g]
    assert s.poll() == 0
    rng = np.random.default_rng(15)
    dirs = (rng.normal(size=(3, n)), rng.normal(size=(3, n)), rng.normal(size=n) * d["u"],
            rng.normal(size=n) * d["h"])
    _, tan = oracle.jvp(d["x"], d["h"], d["m"], d["v"], d["u"], 1.0, tx=dirs[0], tv=dirs[1],
                        tu=dirs[2], th=dirs[3])
    lhs = (ga * tan["dvdt"]).sum() + (gu * tan["dudt"]).sum()
    terms = [a * b for a, b in zip(grads, dirs)]
    rhs = sum(x.sum() for x in terms)
    scale = sum(np.abs(x).sum() for x in terms)
    assert abs(lhs - rhs) <= 2e-4 * scale, (lhs, rhs, scale)


def test_multibox64_sampled_parity_mixed():
    d = synth.load("multibox64")
    gpu, s = run_forward(d, "mixed")
    assert gpu["status"] == 0
    _golden_counts(s, "multibox64")
    off = d["box_off"]
    nb = len(off) - 1
    sizes = np.diff(off)
    rng = np.random.default_rng(6)
    boxes = sorted(set([int(np.argmin(sizes)), int(np.argmax(sizes))] +
                       rng.choice(nb, 6, replace=False).tolist()))
    for b in boxes:
        sl = slice(off[b], off[b + 1])
        db = {k: d[k][..., sl] for k in ("x", "v", "u", "h", "m")}
        nbp = db["h"].shape[0]
        tg = np.sort(rng.choice(nbp, min(24, nbp), replace=False))
        ora = oracle.forward(db["x"], db["h"], db["m"], db["v"], db["u"], 1.0, targets=tg)
        gb = {k: (v[..., sl] if isinstance(v, np.ndarray) else v) for k, v in gpu.items()}
        err = compare(gb, ora, idx=tg)
        for k in ("dvdt", "dudt"):
            assert err[k] < TOL["mixed"], (b, sizes[b], k, err)


def test_lognormal256_sampled_parity_mixed():
    """The largest configuration: 256^3 = 16,777,216 particles in one box."""
    d = synth.load("lognormal256")
    n = d["h"].shape[0]
    assert n == 256 ** 3
    gpu, s = run_forward(d, "mixed")
    assert gpu["status"] == 0
    _golden_counts(s, "lognormal256")
    tg = _stratified(d["h"], 48, np.random.default_rng(9))
    ora = oracle.forward(d["x"], d["h"], d["m"], d["v"], d["u"], 1.0, targets=tg)
    err = compare(gpu, ora, idx=tg)
    for k in ("dvdt", "dudt"):
        assert err[k] < TOL["mixed"], (k, err)
    for k, e in err.items():
        assert e < 5e-5, (k, err)
