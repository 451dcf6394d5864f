"""Overloading (Sec. 2.1): a slab of the box evaluated alone with the ghosts
its particles depend on gives its owned particles the rates of the whole box,
through the C ABI."""
import numpy as np
import pytest
import torch

from paper_2511_21921_gb300 import dist as D
from paper_2511_21921_gb300 import synth
from paper_2511_21921_gb300.solver import Solver

from gpu_util import rel_l2, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_slabs_with_ghosts_reproduce_the_whole_box(precision):
    d = synth.load("lognormal64")
    n = d["h"].shape[0]
    t = to_dev(d, precision)
    sf = Solver(n, 1, precision)
    full = sf.forward(t["x"], t["h"], t["m"], t["v"], t["u"])
    fdv = full["dvdt"].double().cpu().numpy()
    fdu = full["dudt"].double().cpu().numpy()
    row, col = sf.neighbors_csr("union")
    parts = D.overload_slabs(d["x"], d["h"], 2,
                             union_csr=(row.cpu().numpy(), col.cpu().numpy()))
    for owned, ghosts in parts:
        assert owned.size + ghosts.size < n          # the decomposition saves work
        sub = np.concatenate([owned, ghosts])
        ds = {k: (d[k][..., sub] if k in ("x", "v", "u", "h", "m") else d[k]) for k in d}
        ts = to_dev(ds, precision)
        out = Solver(sub.size, 1, precision).forward(ts["x"], ts["h"], ts["m"], ts["v"], ts["u"])
        no = owned.size
        dv = out["dvdt"].double().cpu().numpy()[:, :no]
        du = out["dudt"].double().cpu().numpy()[:no]
        bar = 1e-13 if precision == "fp64" else 1e-5
        assert rel_l2(dv, fdv[:, owned]) <= bar
        assert rel_l2(du, fdu[owned]) <= bar
