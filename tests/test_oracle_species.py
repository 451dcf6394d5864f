"""Pins of the oracle's wind-inclusive density (Sec. 2.5.1 Eq. rhow; App. A.2).

Without winds the evaluation is the gas-only one.  Winds change the gas
particles' density only (through the volume over gas and wind): the gas
volume, coefficients and velocity gradient of the gas are those of the gas
alone, a wind's velocity reaches no gas rate, winds get no rates; the volume
over gas and wind depends on positions and masses only, not on the labels.
"""
import numpy as np

import oracle
from paper_2511_21921_gb300 import synth

WANT = ("V", "coef", "rho", "gradv", "dvdt", "dudt")


def _setup(seed=1, n_wind=200):
    d = synth.lognormal(12, 1.5, seed=seed)
    ng = d["h"].shape[0]
    rng = np.random.default_rng(seed)
    pick = rng.choice(ng, n_wind, replace=False)
    xw = np.mod(d["x"][:, pick] + 0.3 * d["h"][pick] * rng.normal(size=(3, n_wind)), 1.0)
    x = np.concatenate([d["x"], xw], axis=1)
    h = np.concatenate([d["h"], d["h"][pick]])
    m = np.concatenate([d["m"], d["m"][pick]])
    v = np.concatenate([d["v"], rng.normal(0, 0.3, (3, n_wind))], axis=1)
    u = np.concatenate([d["u"], d["u"][pick]])
    sp = np.concatenate([np.zeros(ng, np.uint8), np.ones(n_wind, np.uint8)])
    return d, ng, x, h, m, v, u, sp


def test_all_gas_is_the_plain_evaluation():
    d = synth.lattice(10, seed=2)
    n = d["h"].shape[0]
    o = oracle.forward(d["x"], d["h"], d["m"], d["v"], d["u"], 1.0, want=WANT)
    s = oracle.forward_species(d["x"], d["h"], d["m"], d["v"], d["u"], 1.0, np.zeros(n, np.uint8),
                               want=WANT)
    for k in WANT:
        assert np.array_equal(o[k], s[k]), k
    assert np.array_equal(s["Vgw"], o["V"])


def test_winds_reach_only_the_density():
    d, ng, x, h, m, v, u, sp = _setup(n_wind=3)
    g = oracle.forward(d["x"], d["h"], d["m"], d["v"], d["u"], 1.0, want=WANT)
    w = oracle.forward_species(x, h, m, v, u, 1.0, sp, want=WANT)
    for k in ("V", "coef", "gradv"):
        assert np.allclose(w[k][..., :ng], g[k], rtol=1e-12, atol=1e-12 * np.abs(g[k]).max()), k
    near = np.abs(w["rho"][:ng] / g["rho"] - 1) > 1e-12
    assert near.any() and not near.all()        # winds change the density near them only
    assert np.all(w["dvdt"][:, ng:] == 0) and np.all(w["dudt"][ng:] == 0)
    # a wind's velocity reaches no gas rate
    v2 = v.copy()
    v2[:, ng:] += 5.0
    w2 = oracle.forward_species(x, h, m, v2, u, 1.0, sp, want=WANT)
    assert np.array_equal(w2["dvdt"], w["dvdt"]) and np.array_equal(w2["dudt"], w["dudt"])


def test_gas_plus_wind_volume_ignores_labels():
    d, ng, x, h, m, v, u, sp = _setup(seed=3)
    a = oracle.forward_species(x, h, m, v, u, 1.0, sp, want=("V",))
    sp2 = sp.copy()
    sp2[::7] ^= 1
    b = oracle.forward_species(x, h, m, v, u, 1.0, sp2, want=("V",))
    assert np.allclose(a["Vgw"], b["Vgw"], rtol=1e-14, atol=0)
    # and with no winds it is the gas volume
    c = oracle.forward_species(x, h, m, v, u, 1.0, np.zeros_like(sp), want=("V",))
    assert np.allclose(c["Vgw"], c["V"], rtol=1e-15, atol=0)
    assert np.allclose(a["Vgw"], c["V"], rtol=1e-14, atol=0)
