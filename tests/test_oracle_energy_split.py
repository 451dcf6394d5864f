"""Pins of the two formulation variants of the pair rates (Sec. 2.1: the
compatible energy form and its viscosity, whose details the paper leaves to the
CRKSPH formulation it cites):

* energy split weighted by the specific energies, f_ij + f_ji = 1 (the pair's
  work E_ij goes mostly to the colder particle when it heats, and is drawn
  mostly from the hotter one when it cools);
* per-side viscosity, each Q with its own side's kernel gradient.

Each variant must conserve momentum and energy to roundoff with unequal masses
and energies, reduce to the default form where the mathematics says so, and
the split must favour the colder particle.
"""
import numpy as np
import pytest

import oracle
from paper_2511_21921_gb300 import synth


def _conservation(d, o):
    m, v, a, du = d["m"], d["v"], o["dvdt"], o["dudt"]
    p = (m * a).sum(1)
    e = (m * (v * a).sum(0)).sum() + (m * du).sum()
    ps = np.abs(m * a).sum()
    es = np.abs(m * (v * a).sum(0)).sum() + np.abs(m * du).sum()
    return np.abs(p).max() / ps, abs(e) / es


@pytest.mark.parametrize("mode", [dict(energy_split=1), dict(q_side=1),
                                  dict(energy_split=1, q_side=1)])
def test_variants_conserve_momentum_and_energy(mode):
    d = synth.load("lognormal32m")
    o = oracle.forward(d["x"], d["h"], d["m"], d["v"], d["u"], d["L"],
                       params=oracle.default_params(**mode))
    pm, en = _conservation(d, o)
    assert pm < 1e-13 and en < 1e-13, (mode, pm, en)
    base = oracle.forward(d["x"], d["h"], d["m"], d["v"], d["u"], d["L"])
    if "q_side" not in mode:  # the split leaves the momentum rates alone
        assert np.array_equal(o["dvdt"], base["dvdt"])
    # the variant changes the energy rates (the inputs exercise it)
    assert np.linalg.norm(o["dudt"] - base["dudt"]) > 1e-3 * np.linalg.norm(base["dudt"])


def test_energy_split_is_one_half_for_equal_energies():
    """u_i = u_j on every pair: f_ij = 1/2 exactly, the default rates bit for bit."""
    d = synth.load("lognormal32m")
    u = np.full_like(d["u"], 0.7)
    a = oracle.forward(d["x"], d["h"], d["m"], d["v"], u, d["L"],
                       params=oracle.default_params(energy_split=1))
    b = oracle.forward(d["x"], d["h"], d["m"], d["v"], u, d["L"])
    assert np.array_equal(a["dudt"], b["dudt"]) and np.array_equal(a["dvdt"], b["dvdt"])


def test_per_side_viscosity_equals_default_when_both_sides_agree():
    """Perfect periodic lattice, equal h, uniform u, random velocities: every
    particle has the same density and sound speed and every pair the same mu
    on both sides, so Q_ij = Q_ji and the per-side form is the default form
    (to the rounding of its different operation order)."""
    n = 12
    g = np.stack(np.meshgrid(*(np.arange(n),) * 3, indexing="ij")).reshape(3, -1)
    x = (g + 0.5) / n
    N = n ** 3
    h = np.full(N, (3 * 64 / (4 * np.pi * N)) ** (1 / 3))
    rng = np.random.default_rng(3)
    v = rng.normal(0, 0.3, (3, N))
    m, u = np.full(N, 1.0 / N), np.full(N, 1.3)
    a = oracle.forward(x, h, m, v, u, 1.0, params=oracle.default_params(q_side=1))
    b = oracle.forward(x, h, m, v, u, 1.0)
    assert np.allclose(a["dvdt"], b["dvdt"], rtol=0, atol=1e-13 * np.abs(b["dvdt"]).max())
    assert np.allclose(a["dudt"], b["dudt"], rtol=0, atol=1e-13 * np.abs(b["dudt"]).max())
    # and it differs on a disordered box
    d = synth.load("lognormal32")
    a = oracle.forward(d["x"], d["h"], d["m"], d["v"], d["u"], d["L"],
                       params=oracle.default_params(q_side=1), want=("dvdt",))
    b = oracle.forward(d["x"], d["h"], d["m"], d["v"], d["u"], d["L"], want=("dvdt",))
    assert np.linalg.norm(a["dvdt"] - b["dvdt"]) > 1e-4 * np.linalg.norm(b["dvdt"])


def _pair(u1, u2, approach):
    """Two particles on the x axis inside each other's support, moving toward
    (approach > 0: viscous heating) or apart from each other."""
    x = np.array([[0.45, 0.55], [0.5, 0.5], [0.5, 0.5]])
    h = np.array([0.2, 0.2])
    m = np.array([1.0, 2.0])
    v = np.array([[approach, -approach], [0.0, 0.0], [0.0, 0.0]])
    u = np.array([u1, u2])
    return x, h, m, v, u


@pytest.mark.parametrize("approach", [0.5, -0.5])
def test_energy_split_favours_the_colder_particle(approach):
    """Two particles approaching (the viscosity heats: E > 0) or receding (the
    pressure cools them): with the specific-energy weights the colder one takes
    the larger share of heating and the hotter one the larger share of
    cooling; the total is the pair's kinetic energy loss either way."""
    x, h, m, v, u = _pair(0.2, 1.8, approach)
    out = {}
    for split in (0, 1):
        o = oracle.forward(x, h, m, v, u, 1.0, params=oracle.default_params(energy_split=split),
                           want=("dvdt", "dudt"))
        out[split] = o
    e0 = m * out[0]["dudt"]
    e1 = m * out[1]["dudt"]
    # same kinetic energy loss, shared differently
    assert np.isclose(e0.sum(), e1.sum(), rtol=1e-13)
    assert np.isclose(e1.sum(), -(m * (v * out[1]["dvdt"]).sum(0)).sum(), rtol=1e-13)
    assert np.isclose(e0[0], e0[1], rtol=1e-13)  # f = 1/2
    E = e1.sum()
    assert (E > 0) == (approach > 0)
    # particle 0 is the colder: its share of heating (or of cooling) is larger
    # (smaller) than the hotter one's
    if E > 0:
        assert e1[0] > e1[1] > 0
    else:
        assert e1[1] < e1[0] < 0
    # f_01 = 1/2 (1 + sgn(E) (u_1 - u_0)/(u_0 + u_1)) = 0.9 or 0.1
    assert np.isclose(e1[0] / E, 0.9 if E > 0 else 0.1, rtol=1e-12)


def test_variant_jvp_matches_central_differences():
    """The dual-number tangents of the variant rates agree with central
    differences (the sign of E_ij is held at the primal point, as every branch
    is; the FD step stays inside that branch on this machine)."""
    d = synth.load("lognormal32m")
    x, h, m, v, u, L = d["x"], d["h"], d["m"], d["v"], d["u"], d["L"]
    p = oracle.default_params(energy_split=1, q_side=1)
    rng = np.random.default_rng(9)
    tx = rng.normal(size=x.shape) * 1e-3
    tu = rng.normal(size=u.shape) * u * 0.1
    th = rng.normal(size=h.shape) * h * 0.01
    tg = np.arange(0, h.shape[0], 509)
    _, tan = oracle.jvp(x, h, m, v, u, L, tx=tx, tu=tu, th=th, params=p, targets=tg)
    eps = 1e-6

    def f(s):
        return oracle.forward(np.mod(x + s * tx, L), h + s * th, m, v, u + s * tu, L, params=p,
                              targets=tg, want=("dvdt", "dudt"))
    fp, fm = f(eps), f(-eps)
    for k in ("dvdt", "dudt"):
        fd = (fp[k] - fm[k]) / (2 * eps)
        rel = np.linalg.norm(fd - tan[k]) / np.linalg.norm(fd)
        assert rel < 1e-6, (k, rel)
