"""The region sample the CPU baseline times: a cube of owned particles with a
ghost margin of three hops of the largest smoothing length.  The oracle
evaluated on the sample alone gives the owned particles exactly the results
of the whole box (bit for bit: the sample keeps the particle order, so every
sum runs in the same order)."""
import numpy as np

import oracle
from paper_2511_21921_gb300 import synth


def test_region_sample_owned_results_equal_whole_box():
    d = synth.load("lognormal64")
    sub, own, idx = synth.region_sample(d, side=0.3)
    assert 0 < own.sum() < sub["h"].shape[0] < d["h"].shape[0]
    o = oracle.forward(sub["x"], sub["h"], sub["m"], sub["v"], sub["u"], sub["L"],
                       want=("rho", "dvdt", "dudt", "kgather"))
    k = np.nonzero(own)[0][::997]
    full = oracle.forward(d["x"], d["h"], d["m"], d["v"], d["u"], d["L"], targets=idx[k],
                          want=("rho", "dvdt", "dudt", "kgather"))
    for key in ("rho", "dvdt", "dudt", "kgather"):
        assert np.array_equal(o[key][..., k], full[key]), key
