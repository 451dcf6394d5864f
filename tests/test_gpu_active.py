"""GPU active-set evaluation (App. A.1: passive particles reuse their stored
coefficients) against the oracle's active-set evaluation, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_21921_gb300 import _lib as L
from paper_2511_21921_gb300 import synth
from paper_2511_21921_gb300.solver import Solver

from gpu_util import DT, TOL, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def _np(t):
    return t.double().cpu().numpy()


def _as(a, precision):
    return a.astype(np.float32).astype(np.float64) if precision == "mixed" else a


def _plain(s, t):
    V, coef = s.moments(t["m"], want_V=True, want_coef=True)
    dv, du, rho, gv = s.rates(t["v"], t["u"], want_rho=True, want_gradv=True)
    return V, coef, rho, gv, dv, du


def _active(s, t, flags, V, coef, rho, gv):
    st = [a.clone() for a in (V, coef, rho, gv)]
    s.moments_active(t["m"], flags, st[0], st[1])
    dv, du = s.rates_active(t["v"], t["u"], st[2], st[3])
    return st + [dv, du]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_exact_state_reproduces_plain_evaluation(precision):
    d = synth.load("lognormal32")
    n = d["h"].shape[0]
    t = to_dev(d, precision)
    s = Solver(n, 1, precision)
    s.cell_build(t["x"], t["h"])
    plain = _plain(s, t)
    rng = np.random.default_rng(0)
    for probs in ([0, 1, 0, 0], [0.5, 0.3, 0.1, 0.1]):
        fl = rng.choice(np.array([0, 1, 2, 3], np.uint8), size=n, p=probs)
        flags = torch.tensor(fl, device="cuda")
        got = _active(s, t, flags, *plain[:4])
        torch.cuda.synchronize()
        assert s.poll() == 0
        act = (fl & 1) != 0
        for k in (4, 5):   # rates of active particles, bit for bit
            assert np.array_equal(_np(got[k])[..., act], _np(plain[k])[..., act])
        for k in range(4):  # every stored field equals the fresh one
            assert np.array_equal(_np(got[k]), _np(plain[k])), k


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_parity_with_oracle_active_set(precision):
    """Stored fields from the oracle at displaced positions, so passive
    particles really feed stale values to their active neighbors."""
    d = synth.load("lognormal32")
    n = d["h"].shape[0]
    rng = np.random.default_rng(1)
    sp = n ** (-1 / 3)
    xs = np.mod(d["x"] + 0.05 * sp * rng.normal(size=(3, n)), 1.0)
    o = oracle.forward(xs, d["h"], d["m"], d["v"], d["u"], 1.0,
                       want=("V", "coef", "rho", "gradv"))
    state = [_as(o[k], precision) for k in ("V", "coef", "rho", "gradv")]
    fl = rng.choice(np.array([0, 1, 2, 3], np.uint8), size=n, p=[0.55, 0.25, 0.1, 0.1])
    dd = {k: (_as(d[k], precision) if k in ("h", "m", "u", "v") else d[k]) for k in d}
    ref = oracle.forward_state(dd["x"], dd["h"], dd["m"], dd["v"], dd["u"], 1.0, fl, *state)
    t = to_dev(d, precision)
    s = Solver(n, 1, precision)
    s.cell_build(t["x"], t["h"])
    st = [torch.tensor(np.ascontiguousarray(a), dtype=DT[precision], device="cuda")
          for a in state]
    got = _active(s, t, torch.tensor(fl, device="cuda"), *st)
    torch.cuda.synchronize()
    assert s.poll() == 0
    act = (fl & 1) != 0
    rec = (fl & 3) != 0
    bar = TOL[precision]
    errs = {"V": rel_l2(_np(got[0])[rec], ref["V"][rec]),
            "coef": rel_l2(_np(got[1])[:, rec], ref["coef"][:, rec]),
            "rho": rel_l2(_np(got[2])[act], ref["rho"][act]),
            "gradv": rel_l2(_np(got[3])[:, act], ref["gradv"][:, act]),
            "dvdt": rel_l2(_np(got[4])[:, act], ref["dvdt"][:, act]),
            "dudt": rel_l2(_np(got[5])[act], ref["dudt"][act])}
    assert all(e <= bar for e in errs.values()), errs
    # passive stored fields pass through untouched
    assert np.array_equal(_np(got[0])[~rec], state[0][~rec])
    assert np.array_equal(_np(got[2])[~act], state[2][~act])


def test_leaf_mark_and_call_order():
    d = synth.load("lognormal32")
    n = d["h"].shape[0]
    t = to_dev(d, "fp64")
    s = Solver(n, 1, "fp64")
    s.cell_build(t["x"], t["h"])
    rng = np.random.default_rng(2)
    fl = rng.choice(np.array([0, 1], np.uint8), size=n, p=[0.8, 0.2])
    tr = rng.uniform(size=n) < 0.01
    fl[tr] |= 4
    flags = torch.tensor(fl, device="cuda")
    _, leaf = s.leaf_mark(flags, want_leaf=True)
    out = flags.cpu().numpy()
    leaf = leaf.cpu().numpy()
    assert np.array_equal(out & ~np.uint8(2), fl & ~np.uint8(2))   # only bit 1 changes
    counts = np.bincount(leaf, minlength=leaf.max() + 1)
    assert counts.max() <= 8 and counts.sum() == n
    dirty = np.zeros(leaf.max() + 1, bool)
    dirty[leaf[tr]] = True
    assert np.array_equal((out & 2) != 0, dirty[leaf] | ((fl & 2) != 0))
    # call order: rates_active needs moments_active; adjoint reuse is refused after it
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    rc = L.crk_rates_active(s.plan, 0, s._wsp, t["v"].data_ptr(), t["u"].data_ptr(),
                            z.data_ptr(), torch.zeros((9, n), dtype=torch.float64,
                                                      device="cuda").data_ptr(),
                            torch.zeros((3, n), dtype=torch.float64, device="cuda").data_ptr(),
                            z.data_ptr())
    assert rc == L.CRK_ESTATE
    V, coef = s.moments(t["m"], want_V=True, want_coef=True)
    _, _, rho, gv = s.rates(t["v"], t["u"], want_rho=True, want_gradv=True)
    s.moments_active(t["m"], flags, V, coef)
    s.rates_active(t["v"], t["u"], rho, gv)
    g = torch.zeros((3, n), dtype=torch.float64, device="cuda")
    rc = L.crk_adjoint(s.plan, 0, s._wsp, t["v"].data_ptr(), t["u"].data_ptr(), g.data_ptr(),
                       z.data_ptr(), g.data_ptr(), g.data_ptr(), z.data_ptr(), z.data_ptr(), 0)
    assert rc == L.CRK_ESTATE


def test_power_of_two_time_bins_per_leaf():
    """Leaf levels (Sec. 2 power-of-two bins, App. A.4 leaves): one level per
    leaf, the coarsest bin dt_max/2^k not above the leaf's smallest time step,
    and activity on sub-step t iff t is a multiple of 2^(max_level - k)."""
    d = synth.load("lognormal32")
    n = d["h"].shape[0]
    t = to_dev(d, "mixed")
    s = Solver(n, 1, "mixed")
    s.cell_build(t["x"], t["h"])
    rng = np.random.default_rng(3)
    dt = (10 ** rng.uniform(-3.5, 0.2, n)).astype(np.float32)
    max_level, dt_max = 10, 1.0
    flags0 = rng.choice(np.array([0, 2, 4, 6], np.uint8), size=n)
    _, leaf = s.leaf_mark(torch.zeros(n, dtype=torch.uint8, device="cuda"), want_leaf=True)
    leaf = leaf.cpu().numpy()
    for sub in (0, 1, 2, 3, 8, 512, 1023):
        flags = torch.tensor(flags0, device="cuda")
        level, flags = s.time_bins(torch.tensor(dt, device="cuda"), dt_max, max_level, sub, flags)
        lv = level.cpu().numpy().astype(int)
        fl = flags.cpu().numpy()
        nl = leaf.max() + 1
        lmin = np.full(nl, np.inf)
        np.minimum.at(lmin, leaf, dt.astype(np.float64))
        lo = np.full(nl, 99)
        hi = np.full(nl, -1)
        np.minimum.at(lo, leaf, lv)
        np.maximum.at(hi, leaf, lv)
        assert np.array_equal(lo, hi)  # one level per leaf
        k = lv
        ok = (dt_max / 2.0 ** k <= lmin[leaf]) | (k == max_level)
        tight = (k == 0) | (dt_max / 2.0 ** (k - 1) > lmin[leaf])
        assert np.all(ok) and np.all(tight)
        act = (sub % (2 ** (max_level - k))) == 0
        assert np.array_equal((fl & 1) != 0, act)
        assert np.array_equal(fl & ~np.uint8(1), flags0 & ~np.uint8(1))


def test_time_bins_across_boxes_and_ragged_tail():
    """Levels on a multi-box batch whose size is not a multiple of the leaf
    size: every particle gets a level, leaves may span a box boundary."""
    d = synth.multibox(3, seed0=60, nmin=9, nmax=11)
    n = d["h"].shape[0]
    t = to_dev(d, "fp64")
    s = Solver(n, len(d["box_off"]) - 1, "fp64")
    s.cell_build(t["x"], t["h"], t["box_off"], t["box_L"])
    dt = torch.full((n,), 0.3, dtype=torch.float64, device="cuda")
    dt[::7] = 0.01
    level, flags = s.time_bins(dt, 1.0, 8, 0)
    lv = level.cpu().numpy().astype(int)
    assert lv.size == n and lv.min() >= 0 and lv.max() <= 8
    assert np.all((flags.cpu().numpy() & 1) == 1)   # sub-step 0: every leaf is active
    dmin = dt.cpu().numpy()
    assert np.all(1.0 / 2.0 ** lv <= 0.3 + 1e-15)
