"""The batched single components of the adjoint (components.py) equal one
oracle JVP per component: the three-hop closures really bound the dependency
of the rates, so summing over disjoint closures loses nothing."""
import numpy as np

import oracle
from paper_2511_21921_gb300 import synth

import components as C


def test_batched_components_equal_single_jvps():
    d = synth.load("lognormal32")
    n = d["h"].shape[0]
    ga, gu = synth.cotangents(n, seed=4)
    batches = C.pick(d, per_kind=2, seed=2)
    assert max(len(b) for b in batches) >= 4  # several components share a JVP
    ex = C.exact(d, ga, gu, batches)
    for kind in C.KINDS:
        p, axis, val = ex[kind][0]
        t = {"x": np.zeros((3, n)), "v": np.zeros((3, n)), "u": np.zeros(n), "h": np.zeros(n)}
        if kind in ("x", "v"):
            t[kind][axis, p] = 1.0
        else:
            t[kind][p] = 1.0
        _, tan = oracle.jvp(d["x"], d["h"], d["m"], d["v"], d["u"], d["L"], tx=t["x"],
                            tv=t["v"], tu=t["u"], th=t["h"], want=("dvdt", "dudt"))
        full = (ga * tan["dvdt"]).sum() + (gu * tan["dudt"]).sum()
        assert abs(val - full) <= 1e-12 * abs(full), (kind, val, full)
