"""Pins of the oracle's active-set evaluation (App. A.1: passive particles
reuse the coefficients of their last active step).

With every particle active the stored state is ignored and the result is the
plain evaluation; with the stored state equal to the fresh fields, any choice
of active particles reproduces the plain evaluation for them; a passive
particle's stored fields reach exactly the active particles whose union set
holds it.
"""
import numpy as np

import oracle
from paper_2511_21921_gb300 import synth

KEYS = ("V", "coef", "rho", "gradv", "dvdt", "dudt")


def _plain(d):
    return oracle.forward(d["x"], d["h"], d["m"], d["v"], d["u"], 1.0,
                          want=("V", "coef", "rho", "gradv", "dvdt", "dudt"))


def _state(o):
    return o["V"], o["coef"], o["rho"], o["gradv"]


def test_all_active_ignores_state():
    d = synth.lattice(10, seed=3)
    n = d["h"].shape[0]
    o = _plain(d)
    junk = (np.full(n, 7.0), np.full((16, n), -3.0), np.full(n, 9.0), np.full((9, n), 4.0))
    a = oracle.forward_state(d["x"], d["h"], d["m"], d["v"], d["u"], 1.0, np.ones(n, np.uint8),
                             *junk)
    for k in KEYS:
        assert np.array_equal(a[k], o[k]), k


def test_exact_state_reproduces_plain_evaluation_for_any_active_set():
    d = synth.lognormal(14, 1.5, seed=8)
    n = d["h"].shape[0]
    o = _plain(d)
    rng = np.random.default_rng(0)
    flags = rng.choice(np.array([0, 1, 2, 3], np.uint8), size=n, p=[0.5, 0.3, 0.1, 0.1])
    a = oracle.forward_state(d["x"], d["h"], d["m"], d["v"], d["u"], 1.0, flags, *_state(o))
    act = (flags & 1) != 0
    for k in ("dvdt", "dudt", "rho", "gradv"):
        assert np.allclose(a[k][..., act], o[k][..., act], rtol=1e-13, atol=1e-13 *
                           np.abs(o[k]).max()), k
    assert np.all(a["dvdt"][:, ~act] == 0) and np.all(a["dudt"][~act] == 0)
    for k in ("V", "coef"):
        assert np.allclose(a[k], o[k], rtol=1e-13, atol=1e-13 * np.abs(o[k]).max()), k


def test_passive_state_reaches_exactly_its_union_neighbors():
    d = synth.lognormal(12, 1.5, seed=9)
    n = d["h"].shape[0]
    o = _plain(d)
    flags = np.zeros(n, np.uint8)
    flags[::3] = 1
    V, coef, rho, gv = (np.array(a, copy=True) for a in _state(o))
    base = oracle.forward_state(d["x"], d["h"], d["m"], d["v"], d["u"], 1.0, flags, V, coef, rho,
                                gv)
    k = 1                      # passive
    rho2 = rho.copy()
    rho2[k] *= 1.5             # its stored density -> its pressure in the pair rates
    pert = oracle.forward_state(d["x"], d["h"], d["m"], d["v"], d["u"], 1.0, flags, V, coef, rho2,
                                gv)
    changed = np.any(pert["dvdt"] != base["dvdt"], axis=0)
    row, col = oracle.neighbors(d["x"], d["h"], 1.0, mode="union")
    reach = np.zeros(n, bool)
    for i in np.nonzero(flags & 1)[0]:
        if k in col[row[i]:row[i + 1]]:
            reach[i] = True
    assert np.array_equal(changed, reach)
    assert reach.any()
