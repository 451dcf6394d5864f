"""Parity in the launch configuration the benchmark times: the 64^3 lognormal
workload in the mixed form, launch variants chosen by the autotuner, the
union sweeps on the length-balanced work list, and the whole step (build,
moments, rates, adjoint) replayed from a captured CUDA graph.  Rates are
compared with the oracle on sampled particles the oracle computes one by one;
the adjoint through a dot test against the oracle's forward-mode derivative
over the whole box."""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_21921_gb300 import synth
from paper_2511_21921_gb300.solver import Solver

from gpu_util import TOL, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def test_bench_configuration_lognormal64_mixed():
    d = synth.load("lognormal64")
    n = d["h"].shape[0]
    ga, gu = synth.cotangents(n, seed=4)
    t = to_dev(d, "mixed")
    gat = torch.tensor(ga, dtype=torch.float32, device="cuda")
    gut = torch.tensor(gu, dtype=torch.float32, device="cuda")
    s = Solver(n, 1, "mixed")
    s.cell_build(t["x"], t["h"], check=True)
    s.autotune(t["m"], t["v"], t["u"], gat, gut, repeats=1)
    outs = (torch.empty((3, n), device="cuda"), torch.empty(n, device="cuda"))
    grads = (torch.empty((3, n), device="cuda"), torch.empty((3, n), device="cuda"),
             torch.empty(n, device="cuda"), torch.empty(n, device="cuda"))

    def step():
        s.cell_build(t["x"], t["h"], check=False)
        s.moments(t["m"])
        s.rates(t["v"], t["u"], out=outs)
        s.adjoint(t["v"], t["u"], gat, gut, recompute=False, out=grads)

    g = s.capture(step)
    for o in outs + grads:
        o.fill_(float("nan"))
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert s.poll() == 0
    # rates on 160 sampled particles
    rng = np.random.default_rng(77)
    tg = np.sort(rng.choice(n, 160, replace=False))
    ora = oracle.forward(d["x"], d["h"], d["m"], d["v"], d["u"], 1.0, targets=tg)
    dv = outs[0].double().cpu().numpy()[:, tg]
    du = outs[1].double().cpu().numpy()[tg]
    assert rel_l2(dv, ora["dvdt"]) <= TOL["mixed"]
    assert rel_l2(du, ora["dudt"]) <= TOL["mixed"]
    # adjoint: <g, J delta> from the oracle against <J^T g, delta> from the graph
    dirs = (rng.normal(size=(3, n)), rng.normal(size=(3, n)), rng.normal(size=n) * d["u"],
            rng.normal(size=n) * d["h"])
    _, tan = oracle.jvp(d["x"], d["h"], d["m"], d["v"], d["u"], 1.0, tx=dirs[0], tv=dirs[1],
                        tu=dirs[2], th=dirs[3], want=("dvdt", "dudt"))
    lhs = (ga * tan["dvdt"]).sum() + (gu * tan["dudt"]).sum()
    terms = [gg.double().cpu().numpy() * dd for gg, dd in zip(grads, dirs)]
    rhs = sum(x.sum() for x in terms)
    scale = sum(np.abs(x).sum() for x in terms)
    assert abs(lhs - rhs) <= 2e-4 * scale, (lhs, rhs, scale)
