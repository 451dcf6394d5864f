"""Every compiled launch variant of the eight neighbor sweeps -- three register
caps times six ways of bringing the neighbor records to the pair arithmetic
(plain loads, a shared-memory ring filled per lane or by the whole warp in two
layouts, a register double buffer, rotating register buffers with several
records in flight) -- gives the oracle's
results: the forward fields and rates element by element, the adjoint through
a dot test against the oracle's forward-mode derivative, and the active-set
path, whose sweeps walk a compacted work list instead of consecutive warps."""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_21921_gb300 import _lib as L
from paper_2511_21921_gb300 import synth
from paper_2511_21921_gb300.solver import Solver

from gpu_util import DT, TOL, rel_l2, to_dev

pytestmark = pytest.mark.gpu

ADJ_TOL = {"fp64": 1e-10, "mixed": 2e-4}


def _np(t):
    return t.double().cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_every_variant_matches_oracle(precision):
    # 15^3 = 3375 particles: 105 full warps and a ragged tail of 15
    d = synth.lognormal(15, 1.5, seed=31)
    n = d["h"].shape[0]
    assert n % 32 != 0
    ga, gu = synth.cotangents(n, seed=8)
    ref = oracle.forward(d["x"], d["h"], d["m"], d["v"], d["u"], 1.0,
                         want=("V", "rho", "gradv", "dvdt", "dudt"))
    rng = np.random.default_rng(5)
    dirs = (rng.normal(size=(3, n)), rng.normal(size=(3, n)), rng.normal(size=n) * d["u"],
            rng.normal(size=n) * d["h"])
    _, tan = oracle.jvp(d["x"], d["h"], d["m"], d["v"], d["u"], 1.0, tx=dirs[0], tv=dirs[1],
                        tu=dirs[2], th=dirs[3], want=("dvdt", "dudt"))
    lhs = (ga * tan["dvdt"]).sum() + (gu * tan["dudt"]).sum()
    t = to_dev(d, precision)
    dt = DT[precision]
    gat = torch.tensor(ga, dtype=dt, device="cuda")
    gut = torch.tensor(gu, dtype=dt, device="cuda")
    s = Solver(n, 1, precision)
    s.cell_build(t["x"], t["h"])
    for v in range(L.CRK_TUNE_VARIANTS):
        L.crk_tune_set(s.plan, [v] * 8)
        V, _ = s.moments(t["m"], want_V=True)
        dv, du, rho, gv = s.rates(t["v"], t["u"], want_rho=True, want_gradv=True)
        g = s.adjoint(t["v"], t["u"], gat, gut, recompute=False)
        torch.cuda.synchronize()
        assert s.poll() == 0, v
        for name, got in (("V", V), ("rho", rho), ("gradv", gv), ("dvdt", dv), ("dudt", du)):
            assert rel_l2(_np(got), ref[name]) <= TOL[precision], (v, name)
        terms = [_np(a) * b for a, b in zip(g, dirs)]
        rhs = sum(x.sum() for x in terms)
        scale = sum(np.abs(x).sum() for x in terms)
        assert abs(lhs - rhs) <= ADJ_TOL[precision] * scale, (v, lhs, rhs)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_every_variant_active_set(precision):
    """The active-set sweeps of every variant reproduce the plain evaluation
    for the active particles when the stored state is exact."""
    d = synth.lognormal(15, 1.5, seed=33)
    n = d["h"].shape[0]
    t = to_dev(d, precision)
    s = Solver(n, 1, precision)
    s.cell_build(t["x"], t["h"])
    L.crk_tune_set(s.plan, [0] * 8)
    V, coef = s.moments(t["m"], want_V=True, want_coef=True)
    dv0, du0, rho, gv = s.rates(t["v"], t["u"], want_rho=True, want_gradv=True)
    fl = np.random.default_rng(2).choice(np.array([0, 1, 2, 3], np.uint8), size=n,
                                         p=[0.5, 0.3, 0.1, 0.1])
    act = (fl & 1) != 0
    flags = torch.tensor(fl, device="cuda")
    for v in range(L.CRK_TUNE_VARIANTS):
        L.crk_tune_set(s.plan, [v] * 8)
        st = [a.clone() for a in (V, coef, rho, gv)]
        s.moments_active(t["m"], flags, st[0], st[1])
        dv, du = s.rates_active(t["v"], t["u"], st[2], st[3])
        torch.cuda.synchronize()
        assert s.poll() == 0, v
        bar = 1e-13 if precision == "fp64" else 1e-6
        assert rel_l2(_np(dv)[:, act], _np(dv0)[:, act]) <= bar, v
        assert rel_l2(_np(du)[act], _np(du0)[act]) <= bar, v


def test_tune_set_rejects_out_of_range():
    s = Solver(64, 1, "mixed")
    for bad in ([L.CRK_TUNE_VARIANTS] + [0] * 7, [0] * 7 + [-1]):
        with pytest.raises(L.CRKError):
            L.crk_tune_set(s.plan, bad)


def test_tune_set_replays_an_autotuner_choice():
    """A stored autotuner choice, set on a fresh plan, gives the tuned plan's
    results bit for bit (same kernels, same inputs)."""
    d = synth.lognormal(12, 1.5, seed=35)
    n = d["h"].shape[0]
    t = to_dev(d, "mixed")
    s1 = Solver(n, 1, "mixed")
    s1.cell_build(t["x"], t["h"])
    tuned = s1.autotune(t["m"], t["v"], t["u"], repeats=1)
    s1.moments(t["m"])
    r1 = s1.rates(t["v"], t["u"])
    s2 = Solver(n, 1, "mixed")
    s2.tune_set(tuned)
    s2.cell_build(t["x"], t["h"])
    s2.moments(t["m"])
    r2 = s2.rates(t["v"], t["u"])
    torch.cuda.synchronize()
    assert torch.equal(r1[0], r2[0]) and torch.equal(r1[1], r2[1])
