"""Pins of the oracle's time step (smoothing-length rate, drifts, kicks).

Each test checks a closed form or an invariant the integrator must satisfy,
never the oracle against a retyped copy of itself: the leapfrog recurrence of
a harmonic oscillator, the exact parabola of constant acceleration, quadrature
of the piecewise acceleration behind the refined kick, mass conservation of
the passive drift, the neighbor-count meaning of Delta_N, Galilean invariance
and momentum conservation of whole steps.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import integrate as quad

import oracle
from oracle import integrate as I
from paper_2511_21921_gb300 import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
NH = (3.0 * 100 / (4.0 * np.pi)) ** (1.0 / 3.0)   # the synthetic workloads' ~100 neighbors


def test_kdk_harmonic_oscillator_recurrence():
    """KDK from the oracle's kick and drift on a = -w^2 (x - c): positions obey
    x_{n+1} - 2 x_n + x_{n-1} = -(w dt)^2 (x_n - c) (App. A.4 is leapfrog), and
    the first step is x0 + v0 dt - (w dt)^2 (x0 - c) / 2."""
    w, dt, c, L = 1.3, 0.07, 500.0, 1000.0
    rng = np.random.default_rng(0)
    x = c + rng.normal(size=(3, 5))
    v = rng.normal(size=(3, 5))
    x0, v_init = x.copy(), v.copy()
    acc = lambda y: -w * w * (y - c)
    xs = [x.copy()]
    a = acc(x)
    for _ in range(40):
        vh = I.kick(v, a, 0.5 * dt)
        x = I.drift(x, vh, dt, L)
        a = acc(x)
        v = I.kick(vh, a, 0.5 * dt)
        xs.append(x.copy())
    xs = np.array(xs)
    assert np.allclose(xs[1], x0 + v_init * dt - 0.5 * (w * dt) ** 2 * (x0 - c), rtol=0, atol=1e-12)
    lhs = xs[2:] - 2 * xs[1:-1] + xs[:-2]
    rhs = -(w * dt) ** 2 * (xs[1:-1] - c)
    assert np.max(np.abs(lhs - rhs)) < 1e-11


def test_passive_parabolic_drift_is_exact_parabola():
    """Sub-steps of a passive particle with the local half-step velocity of
    App. A.4 trace x0 + v0 t + a t^2 / 2 exactly under constant acceleration,
    at every sub-step end, for any partition of the active interval."""
    rng = np.random.default_rng(1)
    n, L = 7, 1e6
    x0 = 5e5 + rng.normal(size=(3, n))
    v0 = rng.normal(size=(3, n))
    a = rng.normal(size=(3, n))
    dt_a = 0.25
    cuts = np.sort(rng.uniform(0, dt_a, size=6))
    subs = np.diff(np.concatenate([[0.0], cuts, [dt_a]]))
    vh = I.kick(v0, a, 0.5 * dt_a)
    x = x0.copy()
    te = 0.0
    for dtj in subs:
        x = I.drift(x, vh, dtj, L, a0=a, dt_a=np.full(n, dt_a), t_elapse=np.full(n, te))
        te += dtj
        assert np.allclose(x, x0 + v0 * te + 0.5 * a * te * te, rtol=0, atol=1e-9)
    # with no refinement the end point equals the linear drift with v_half (App. A.4)
    assert np.allclose(x, I.drift(x0, vh, dt_a, L), rtol=0, atol=1e-9)
    # an active particle (dt_a = dt, no elapsed time) drifts linearly
    assert np.array_equal(I.drift(x0, vh, 0.1, L, a0=a), I.drift(x0, vh, 0.1, L))


def test_refined_kick_integrates_piecewise_acceleration():
    """v1 of the refined completion equals v0 plus the exact integral of an
    acceleration held at a0 over dt_b - dt_c and linear from a0 to a1 over the
    last dt_c (App. A.4); dt_c = dt_b is the plain KDK, dt_c = 0 constant a0."""
    rng = np.random.default_rng(2)
    v0, a0, a1 = rng.normal(size=(3, 3, 4))
    dt_b = 0.3
    for dt_c in (0.3, 0.17, 0.05, 0.0):
        got = I.kick_refined(v0, a0, a1, dt_b, dt_c)
        for k in np.ndindex(v0.shape):
            def acc(t, k=k):
                t0 = dt_b - dt_c
                if t < t0 or dt_c == 0:
                    return a0[k]
                return a0[k] + (a1[k] - a0[k]) * (t - t0) / dt_c
            pts = [dt_b - dt_c] if 0 < dt_c < dt_b else None
            val, _ = quad.quad(acc, 0.0, dt_b, points=pts, epsabs=1e-14, epsrel=1e-13)
            assert abs(got[k] - (v0[k] + val)) < 1e-13
    assert np.allclose(I.kick_refined(v0, a0, a1, dt_b, dt_b), v0 + 0.5 * (a0 + a1) * dt_b,
                       rtol=0, atol=1e-15)
    assert np.allclose(I.kick_refined(v0, a0, a1, dt_b, 0.0), v0 + a0 * dt_b, rtol=0, atol=1e-15)
    # the refined first half-kick is the plain half-kick over dt_b
    assert np.array_equal(I.kick(v0, a0, 0.5 * dt_b), v0 + (0.5 * dt_b) * a0)


def test_delta_n_is_neighbor_count_ratio():
    """Delta_N^3 = N_res / N_i (App. A.3): N_res = (4 pi/3) n_h^3 is the target
    count (268 for the paper's gas n_h = 4, App. A.2) and N_i = (4 pi/3) h^3 / V
    the count a particle of volume V sees within h.  With lambda = 1 and no
    divergence, one active step takes h exactly to the target radius."""
    nh = GOLD["gas_nh"]["value"]
    assert round(4 * np.pi / 3 * nh ** 3) == GOLD["gas_neighbors"]["value"]
    rng = np.random.default_rng(3)
    h = rng.uniform(0.02, 0.05, 50)
    V = rng.uniform(0.5, 2.0, 50) * (h / nh) ** 3
    dt_a = 0.01
    hd, hr = I.hdot(h, V, np.zeros(50), dt_a, 1.0, nh)
    n_res = 4 * np.pi / 3 * nh ** 3
    n_i = 4 * np.pi / 3 * h ** 3 / V
    target = h * (n_res / n_i) ** (1.0 / 3.0)
    assert np.allclose(h + hd * dt_a, target, rtol=1e-13, atol=0)
    assert np.allclose(hr, hd / h, rtol=1e-15, atol=0)
    # lambda = 0: continuity only, d ln h / dt = div / 3
    div = rng.normal(size=50)
    _, hr0 = I.hdot(h, V, div, dt_a, 0.0, nh)
    assert np.allclose(hr0, div / 3, rtol=1e-14, atol=1e-16)
    # at the target count the Thacker part vanishes for any lambda
    Vt = (h / nh) ** 3
    _, hr1 = I.hdot(h, Vt, div, dt_a, 0.7, nh)
    assert np.allclose(hr1, div / 3, rtol=1e-12, atol=1e-12)
    with pytest.raises(ValueError):
        I.hdot(h, V, div, 0.0, 0.5, nh)


def test_passive_drift_conserves_mass_and_composes():
    """With h at its target (Delta_N = 1) the passive update V = (h/n_h)^3,
    rho exp(-div dt) keeps V rho (a particle's mass) fixed, and drifts over
    sub-steps compose to one drift over their sum (App. A.3)."""
    rng = np.random.default_rng(4)
    n = 64
    nh = NH
    h = rng.uniform(0.01, 0.03, n)
    V = (h / nh) ** 3
    rho = rng.uniform(0.5, 5.0, n)
    div = rng.normal(scale=3.0, size=n)
    _, hr = I.hdot(h, V, div, 0.02, 0.4, nh)
    dt = 0.02
    h1 = I.drift_h(h, hr, dt)
    V1, rho1 = I.drift_passive(h1, rho, div, dt, nh)
    assert np.allclose(V1 * rho1, V * rho, rtol=1e-13, atol=0)
    hs, rs = h.copy(), rho.copy()
    for dtj in (0.005, 0.0025, 0.0125):
        hs = I.drift_h(hs, hr, dtj)
        _, rs = I.drift_passive(hs, rs, div, dtj, nh)
    assert np.allclose(hs, h1, rtol=1e-14, atol=0)
    assert np.allclose(rs, rho1, rtol=1e-14, atol=0)


def test_wrap_stays_in_box_and_is_congruent():
    L = 1.0
    y = np.array([-1e-18, -0.25, 1.0, 1.0 + 1e-16, 0.999999, 1.5, -0.5, 0.0, 0.3])
    w = I.wrap(y, L)
    assert np.all((w >= 0) & (w < L))
    for a, b in zip(y, w):
        d = (Fraction(a) - Fraction(b)) / Fraction(L)
        # congruent modulo L up to the rounding of the one addition
        assert abs(d - round(d)) <= Fraction(2) ** -52
    assert w[0] == 0.0 and w[7] == 0.0 and w[2] == 0.0


def test_kdk_galilean_invariance_on_lattice():
    """A perfect lattice moving with one velocity feels no force (App. A.4
    KDK around the rates): positions advance by v t modulo the box, velocities
    and energies stay put."""
    n_side = 10
    g = (np.arange(n_side) + 0.5) / n_side
    x = np.stack(np.meshgrid(g, g, g, indexing="ij")).reshape(3, -1).copy()
    n = x.shape[1]
    h = np.full(n, 2.6 / n_side)
    m = np.full(n, 1.0 / n)
    vel = np.array([0.31, -0.12, 0.05])
    v = np.repeat(vel[:, None], n, axis=1)
    u = np.full(n, 0.7)
    dt = 0.011
    d = I.kdk_init(x, v, u, h, m, 1.0, dt, 0.5, NH)
    x1, v1, u1, h1 = x, v, u, h
    for _ in range(3):
        x1, v1, u1, h1, d = I.kdk_step(x1, v1, u1, h1, m, 1.0, d, dt, 0.5, NH)
    expect = np.mod(x + vel[:, None] * 3 * dt, 1.0)
    diff = np.abs(x1 - expect)
    diff = np.minimum(diff, 1.0 - diff)
    assert diff.max() < 1e-13
    assert np.abs(v1 - v).max() < 1e-12
    assert np.abs(u1 - u).max() < 1e-12
    # a uniform lattice keeps a uniform smoothing length
    assert np.ptp(h1) < 1e-12 * h1.mean()


def test_kdk_conserves_momentum_and_converges_in_energy():
    """Pairwise-antisymmetric forces keep sum m v fixed through kicks and drifts;
    the compatible energy update keeps E = sum m (v^2/2 + u) to an error that
    shrinks with the step (Sec. 2.1, App. A.4)."""
    d = synth.lattice(12, seed=5, jitter=0.15, k_target=64)
    x, v, u, h, m = d["x"], d["v"], d["u"], d["h"], d["m"]
    p0 = (m * v).sum(axis=1)
    E0 = (m * (0.5 * (v * v).sum(axis=0) + u)).sum()
    cs = np.sqrt(10.0 / 9.0 * u.max())          # gamma (gamma - 1) u, gamma = 5/3
    dt0 = 0.1 * h.min() / (cs + np.abs(v).max())  # Courant number 0.1, then 0.05
    errs = []
    for k, steps in ((1, 2), (2, 4)):
        dt = dt0 / k
        dd = I.kdk_init(x, v, u, h, m, 1.0, dt, 0.0, NH)
        xs, vs, us, hs = x, v, u, h
        for _ in range(steps):
            xs, vs, us, hs, dd = I.kdk_step(xs, vs, us, hs, m, 1.0, dd, dt, 0.0, NH)
            p = (m * vs).sum(axis=1)
            assert np.abs(p - p0).max() <= 1e-13 * (m * np.abs(vs)).sum()
        E = (m * (0.5 * (vs * vs).sum(axis=0) + us)).sum()
        errs.append(abs(E - E0) / E0)
    assert errs[0] < 1e-3
    assert errs[1] < 0.5 * errs[0], errs
