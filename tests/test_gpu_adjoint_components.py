"""Per-output errors of the adjoint against exact single components.

For 64 random components of each of g_x, g_v, g_u and g_h, on the 32^3 box
and on the 64^3 clustered box, the exact value <g, J e_k> comes from the
oracle's FP64 forward-mode JVP along the unit direction e_k (batched over
particles with disjoint dependency closures, see components.py).  The library's
adjoint must match them per output within a relative L2 error over the sample
of 1e-13 in the FP64 form and 5e-6 in the mixed form (FP32 pair arithmetic and
accumulation, double-float minimum images; measured on GB300: FP64 at most
2.3e-15, mixed at most 1.5e-6; the sampled errors are printed).
"""
import numpy as np
import pytest
import torch

from paper_2511_21921_gb300 import synth
from paper_2511_21921_gb300.solver import Solver

import components as C
from gpu_util import to_dev

pytestmark = pytest.mark.gpu

BAR = {"fp64": 1e-13, "mixed": 5e-6}
_EXACT = {}


def _exact(case):
    if case not in _EXACT:
        d = synth.load(case)
        n = d["h"].shape[0]
        ga, gu = synth.cotangents(n, seed=4)
        batches = C.pick(d, per_kind=64, seed=1)
        _EXACT[case] = (d, ga, gu, C.exact(d, ga, gu, batches))
    return _EXACT[case]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["lognormal32", "lognormal64"])
def test_adjoint_components_per_output(case, precision):
    d, ga, gu, ex = _exact(case)
    n = d["h"].shape[0]
    s = Solver(n, 1, precision)
    t = to_dev(d, precision)
    s.cell_build(t["x"], t["h"])
    s.moments(t["m"])
    s.rates(t["v"], t["u"])
    dt = t["h"].dtype
    g = s.adjoint(t["v"], t["u"], torch.tensor(ga, dtype=dt, device="cuda"),
                  torch.tensor(gu, dtype=dt, device="cuda"), recompute=False)
    torch.cuda.synchronize()
    assert s.poll() == 0
    gx, gv, gu_, gh = (a.double().cpu().numpy() for a in g)
    got = {"x": lambda p, a: gx[a, p], "v": lambda p, a: gv[a, p], "u": lambda p, a: gu_[p],
           "h": lambda p, a: gh[p]}
    report = {}
    for kind in C.KINDS:
        ref = np.array([v for (_, _, v) in ex[kind]])
        val = np.array([got[kind](p, a) for (p, a, _) in ex[kind]])
        assert ref.size == 64
        rel = np.linalg.norm(val - ref) / np.linalg.norm(ref)
        worst = np.max(np.abs(val - ref) / np.abs(ref).max())
        report[kind] = (rel, worst)
    print(f"\nadjoint components {case} {precision}: " +
          ", ".join(f"g_{k} rel-L2 {r:.2e} (max |err|/max|g| {w:.2e})"
                    for k, (r, w) in report.items()))
    for kind, (rel, _) in report.items():
        assert rel < BAR[precision], (kind, report)
