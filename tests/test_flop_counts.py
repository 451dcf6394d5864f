"""The benchmark's algorithmic flops per pair are the oracle's own operation
counts of the formulas (every add, subtract, multiply, divide, sqrt and exp
the oracle performs, one each), stage by stage on the 32^3 clustered box: a
forward sweep counts its stage per pair of its neighbor sets; the adjoint
sweep of a stage counts the stage's forward operations (recomputed) plus the
tangent operations of the oracle's forward-mode derivative of the stage."""
import numpy as np

import bench
import oracle
from paper_2511_21921_gb300 import synth

STAGE = {"b1_volume": 1, "b2_moments": 2, "c1_density": 3, "c2_rates": 4,
         "adj_b1": 1, "adj_b2": 2, "adj_c1": 3, "adj_c2": 4}


def test_bench_flops_equal_the_oracle_count():
    d = synth.load("lognormal32")
    n = d["h"].shape[0]
    o = oracle.forward(d["x"], d["h"], d["m"], L=d["L"], want=("kgather", "kunion"))
    units = {"gather": int(o["kgather"].sum()), "union": int(o["kunion"].sum())}
    rng = np.random.default_rng(0)
    dirs = dict(tx=rng.normal(size=(3, n)), tv=rng.normal(size=(3, n)), tu=rng.normal(size=n),
                th=rng.normal(size=n))
    cum = [(0, 0)] + [oracle.count_ops(d["x"], d["h"], d["m"], d["v"], d["u"], d["L"], st,
                                       derivative=True, **dirs) for st in (1, 2, 3, 4)]
    for name, st in STAGE.items():
        u = units[bench.UNIT_OF[name]]
        val = (cum[st][0] - cum[st - 1][0]) / u
        tan = (cum[st][1] - cum[st - 1][1]) / u
        assert bench.FLOPS_RECOMPUTE[name] == round(val), (name, val)
        want_tan = round(tan) if name.startswith("adj_") else 0
        assert bench.FLOPS_DERIVATIVE[name] == want_tan, (name, tan)
        assert bench.FLOPS_PER_PAIR[name] == bench.FLOPS_RECOMPUTE[name] + want_tan
    # the plain count (no tangent) is the value count of the derivative run
    plain = oracle.count_ops(d["x"], d["h"], d["m"], d["v"], d["u"], d["L"], 4)
    assert plain == (cum[4][0], 0)
