"""Pins of the oracle's mass weighting and of its viscosity limiter.

Equal masses hide where m_i and m_j enter the volume (App. A.2, Eq. Vg), the
density (Sec. 2.5.1, Eq. rhow) and the rates (Sec. 2.1), and a viscosity that
is switched off or has mu >= 0 hides the limiter.  Each test here checks a
property the mathematics fixes for any correct implementation:

* conservation of momentum and energy with masses spread over 33x (Sec. 2.1:
  pairwise antisymmetric forces, compatible energy split);
* the textbook SPH reduction of fully relaxed pairs (App. A.1) with unequal
  masses;
* Eq. Vg is linear in the neighbor masses: on a lattice of two interleaved mass
  species, V of one run predicts V of another run with other masses;
* Eq. rhow on that lattice reduces to a two-term closed form in the same
  lattice sums;
* a linear velocity field v = C x + d has grad v_i = C at every interior
  particle (App. A.1, Eq. gradv), so the limiter ratio is 1, phi(1) = 1 and the
  limited relative velocity vanishes: the limited viscosity adds nothing, while
  the unlimited one does; with near-field damping only particles with a pair
  closer than eta_crit * max(h_i, h_j) are affected.
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


def test_unequal_mass_inputs_spread():
    d = synth.load("lognormal32m")
    m = d["m"]
    assert m.max() / m.min() > 10.0
    e = synth.load("lognormal32")
    for k in ("x", "v", "u", "h"):
        assert np.array_equal(d[k], e[k])


@pytest.mark.parametrize("relax", [False, True])
def test_conservation_with_unequal_masses(relax):
    """Sum m_i a_i = 0 and sum m_i (v_i . a_i + du_i/dt) = 0 to roundoff.  With
    unequal masses these fix the 1/m_i of both rates: a 1/m_j (or a missing
    mass) leaves the pair terms m_i a_ij and m_j a_ji unbalanced."""
    d = synth.load("lognormal32m")
    p = oracle.default_params()
    if relax:
        o0 = oracle.forward(d["x"], d["h"], d["m"], d["v"], d["u"], d["L"], want=("gradv",))
        div = np.abs(o0["gradv"][0] + o0["gradv"][4] + o0["gradv"][8])
        p = oracle.default_params(relax_dt=np.log(8.0) / np.quantile(div, 0.85))
    o = oracle.forward(d["x"], d["h"], d["m"], d["v"], d["u"], d["L"], params=p)
    if relax:
        assert 0.05 < o["flag"].mean() < 0.3
    pm, en = _conservation(d, o)
    assert pm < 1e-13 and en < 1e-13, (pm, en)
    # the same pin is blind with equal masses to a swapped mass: check that the
    # spread really enters the pair terms (a_i differs from the equal-mass case)
    e = synth.load("lognormal32")
    oe = oracle.forward(e["x"], e["h"], e["m"], e["v"], e["u"], e["L"], params=p,
                        want=("dvdt",))
    assert np.linalg.norm(o["dvdt"] - oe["dvdt"]) > 0.1 * np.linalg.norm(oe["dvdt"])


def test_fully_relaxed_unequal_masses_reduces_to_standard_sph():
    """All pairs relaxed (A = 1, B = 0), no viscosity, equal h, masses spread
    33x: the rates are textbook SPH, -sum_j V_i V_j (P_i + P_j) grad W_ij / m_i
    and the compatible pdV heating, written here by brute force."""
    d = synth.load("lattice16m")
    x, h, m, v, u, L = d["x"], d["h"], d["m"], d["v"], d["u"], d["L"]
    assert m.max() / m.min() > 10.0
    p = oracle.default_params(Cl=0.0, Cq=0.0, relax_dt=1e9)
    o = oracle.forward(x, h, m, v, u, L, params=p, want=("V", "P", "flag", "dvdt", "dudt"))
    assert o["flag"].all()
    dx = x[:, :, None] - x[:, None, :]
    dx = np.where(dx > L / 2, dx - L, np.where(dx < -L / 2, dx + L, dx))
    r = np.sqrt((dx ** 2).sum(0))
    hh = h[0]
    q = r / hh
    gr = np.where(q < 1, 495 / (32 * np.pi * hh ** 5) * (-56 / 3) * (1 - q) ** 5 * (1 + 5 * q), 0.0)
    np.fill_diagonal(gr, 0.0)
    V, P = o["V"], o["P"]
    coef = V[:, None] * V[None, :] * (P[:, None] + P[None, :]) * gr
    a = -(coef[None] * dx).sum(2) / m
    vij = v[:, :, None] - v[:, None, :]
    du = 0.5 * (coef * (dx * vij).sum(0)).sum(1) / m
    assert np.allclose(o["dvdt"], a, rtol=1e-10, atol=1e-12 * np.abs(a).max())
    assert np.allclose(o["dudt"], du, rtol=1e-10, atol=1e-12 * np.abs(du).max())


# ---------------------------------------------------------------- two-species lattice
def _rocksalt(n=12, ma=1.0, mb=1.0, kn=64):
    """Periodic cubic lattice whose sites carry mass ma or mb by the parity of
    i + j + k (every site keeps the full cubic point symmetry)."""
    g = np.stack(np.meshgrid(*(np.arange(n),) * 3, indexing="ij")).reshape(3, -1)
    x = (g + 0.5) / n
    N = n ** 3
    h = np.full(N, (3 * kn / (4 * np.pi * N)) ** (1 / 3))
    odd = (g.sum(0) % 2) == 1
    m = np.where(odd, mb, ma) / N
    return x, h, m, odd


def test_volume_is_linear_in_the_neighbor_masses():
    """Eq. Vg: m_i / V_i = m_i S_same + m_other S_cross, where S_same and
    S_cross are the kernel sums over sites of the same and of the other parity.
    Two runs with other mass pairs fix S_same and S_cross; a third run must
    then follow from them (a number density 1/sum W, a mass in the wrong place
    or a missing self term fails)."""
    runs = {}
    for ma, mb in ((1.0, 2.0), (1.0, 5.0), (3.0, 0.5), (1.0, 1.0)):
        x, h, m, odd = _rocksalt(ma=ma, mb=mb)
        o = oracle.forward(x, h, m, L=1.0, want=("V",))
        V = o["V"]
        # every site of one parity has the same volume
        for sel in (odd, ~odd):
            assert np.abs(V[sel] / V[sel].mean() - 1).max() < 1e-13
        runs[(ma, mb)] = (V[~odd].mean(), V[odd].mean(), m[~odd][0], m[odd][0])
    (Va, Vb, mA, mB) = runs[(1.0, 2.0)]
    # mA/Va = mA S + mB X ; mB/Vb = mB S + mA X
    M = np.array([[mA, mB], [mB, mA]])
    S, X = np.linalg.solve(M, np.array([mA / Va, mB / Vb]))
    assert S > 0 and X > 0
    for key in ((1.0, 5.0), (3.0, 0.5), (1.0, 1.0)):
        Va2, Vb2, mA2, mB2 = runs[key]
        assert abs(Va2 / (mA2 / (mA2 * S + mB2 * X)) - 1) < 1e-12, key
        assert abs(Vb2 / (mB2 / (mB2 * S + mA2 * X)) - 1) < 1e-12, key


def test_density_on_two_species_lattice():
    """Eq. rhow on the two-species lattice: B = 0 and W^R = A W by symmetry, so
    rho_a = (m_a V_a S + m_b V_b X) / (V_a^2 S + V_b^2 X) with the lattice sums
    S, X of the previous pin (here from the volumes of the same run)."""
    x, h, m, odd = _rocksalt(ma=1.0, mb=4.0)
    o = oracle.forward(x, h, m, L=1.0, want=("V", "coef", "rho"))
    V, rho = o["V"], o["rho"]
    assert np.abs(o["coef"][1:4]).max() * h[0] < 1e-12
    Va, Vb = V[~odd].mean(), V[odd].mean()
    ma, mb = m[~odd][0], m[odd][0]
    S, X = np.linalg.solve(np.array([[ma, mb], [mb, ma]]), np.array([ma / Va, mb / Vb]))
    ra = (ma * Va * S + mb * Vb * X) / (Va * Va * S + Vb * Vb * X)
    rb = (mb * Vb * S + ma * Va * X) / (Vb * Vb * S + Va * Va * X)
    assert np.abs(rho[~odd] / ra - 1).max() < 1e-12
    assert np.abs(rho[odd] / rb - 1).max() < 1e-12
    # and not the single-species value m/V: the masses of the neighbors matter
    assert abs(ra / (ma / Va) - 1) > 1e-3


# ---------------------------------------------------------------- limiter
def _linear_field_box(seed=21):
    d = synth.lattice(24, seed=seed, k_target=64)
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(3, 3)) * 0.3
    B = rng.normal(size=(3, 3)) * 0.3
    C = -(A @ A.T + 0.1 * np.eye(3)) + (B - B.T)  # negative definite symmetric part
    v = C @ d["x"] + rng.normal(size=(3, 1))
    x, h, L = d["x"], d["h"], d["L"]
    n = h.shape[0]
    # particles whose gather set does not wrap: there grad v = C exactly
    flat = np.all((x > h) & (x < L - h), axis=0)
    row, col = oracle.neighbors(x, h, L, mode="union")
    ok = np.array([flat[i] and flat[col[row[i]:row[i + 1]]].all() for i in range(n)])
    return d, v, C, ok, row, col


def test_linear_velocity_field_gives_no_limited_viscosity():
    """v = C x + d (compressive): grad v_i = grad v_j = C, so the limiter ratio
    is 1, phi = 1 and the limited relative velocity v_ij - C x_ij vanishes.
    With the near-field damping off (eta_crit = 0) the limited viscosity then
    adds nothing to the rates, on every particle whose union neighbors all see
    the linear field; the unlimited viscosity heats every one of them."""
    d, v, C, ok, _, _ = _linear_field_box()
    tg = np.nonzero(ok)[0][:400]
    assert tg.size >= 200
    x, h, m, u, L = d["x"], d["h"], d["m"], d["u"], d["L"]
    base = dict(eta_crit=0.0)
    lim = oracle.forward(x, h, m, v, u, L, targets=tg, params=oracle.default_params(**base),
                         want=("gradv", "dvdt", "dudt"))
    assert np.abs(lim["gradv"] - C.reshape(9, 1)).max() < 1e-10
    inv = oracle.forward(x, h, m, v, u, L, targets=tg,
                         params=oracle.default_params(Cl=0.0, Cq=0.0, **base),
                         want=("dvdt", "dudt"))
    unl = oracle.forward(x, h, m, v, u, L, targets=tg,
                         params=oracle.default_params(limiter=0, **base), want=("dvdt", "dudt"))
    sa = np.abs(inv["dvdt"]).max()
    se = np.abs(inv["dudt"]).max()
    assert np.abs(lim["dvdt"] - inv["dvdt"]).max() < 1e-12 * sa
    assert np.abs(lim["dudt"] - inv["dudt"]).max() < 1e-12 * se
    # the unlimited viscosity (compression: mu < 0 on every pair) heats
    assert (unl["dudt"] - inv["dudt"] > 1e-3 * se).all()


def test_near_field_damping_acts_only_on_close_pairs():
    """With eta_crit > 0 the limiter is damped on pairs with
    min(r/h_i, r/h_j) < eta_crit, so in the linear field the limited viscosity
    changes exactly the particles that have such a pair."""
    d, v, C, ok, row, col = _linear_field_box()
    x, h, m, u, L = d["x"], d["h"], d["m"], d["u"], d["L"]
    eta_c = 0.33
    tg = np.nonzero(ok)[0][:600]
    close = np.zeros(tg.size, dtype=bool)
    for k, i in enumerate(tg):
        js = col[row[i]:row[i + 1]]
        dx = x[:, [i]] - x[:, js]
        r = np.sqrt((dx ** 2).sum(0))
        close[k] = (r / np.maximum(h[i], h[js]) < eta_c).any()
    assert close.sum() >= 30 and (~close).sum() >= 30, close.sum()
    lim = oracle.forward(x, h, m, v, u, L, targets=tg,
                         params=oracle.default_params(eta_crit=eta_c), want=("dvdt", "dudt"))
    inv = oracle.forward(x, h, m, v, u, L, targets=tg,
                         params=oracle.default_params(Cl=0.0, Cq=0.0), want=("dvdt", "dudt"))
    se = np.abs(inv["dudt"]).max()
    diff = np.abs(lim["dudt"] - inv["dudt"])
    # roundoff (about 1e-16 of the largest rate) against the smallest damping
    # effect (a pair at 0.9999 eta_crit changes phi by 4e-8)
    assert (diff[~close] < 1e-13 * se).all()
    assert (diff[close] > 1e-12 * se).all()
    # damping reduces phi below 1, so the residual viscosity heats
    assert (lim["dudt"][close] > inv["dudt"][close]).all()
