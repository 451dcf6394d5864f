"""Pins of the subgrid neighbor-sum oracle (App. A.2 Eq. Vsg; Eqs. windmetal,
Anorm, starmetal, AGNE).

Deposits conserve the deposited quantity exactly (the normalisation), skip
ineligible gas, and reach only gas within h_s; the scatter volume reduces to
the gather number density when every h is equal, approaches the lattice
spacing cubed on a uniform lattice, and is invariant under periodic
translation; the kernel is the gas sums' Wendland C4.
"""
import numpy as np

import oracle
from oracle import subgrid as S


def _lattice(ns=12, L=1.0):
    g = (np.arange(ns) + 0.5) / ns * L
    return np.stack(np.meshgrid(g, g, g, indexing="ij")).reshape(3, -1).copy()


def test_kernel_is_the_gas_kernel():
    r = np.linspace(0, 0.25, 101)
    W, _, _ = oracle.kernel(r, 0.2)
    assert np.allclose(S._wendland(r, np.full_like(r, 0.2)), W, rtol=1e-14, atol=1e-14)


def test_deposit_conserves_and_respects_eligibility_and_support():
    rng = np.random.default_rng(0)
    xg = rng.uniform(0, 1, (3, 800))
    Vg = rng.uniform(0.5, 2.0, 800) / 800
    xs = rng.uniform(0, 1, (3, 40))
    hs = rng.uniform(0.08, 0.2, 40)
    q = rng.uniform(0, 1, (2, 40))
    elig = rng.uniform(size=800) > 0.2
    dq, A = S.deposit(xs, hs, q, xg, Vg, eligible=elig)
    has = A > 0
    assert np.allclose(dq.sum(axis=1), q[:, has].sum(axis=1), rtol=1e-13)
    assert np.all(dq[:, ~elig] == 0)
    # a gas particle farther than every h_s from every subgrid particle gets nothing
    d = xs[:, :, None] - xg[:, None, :]
    d -= np.round(d)
    r = np.sqrt((d * d).sum(0))
    far = np.all(r >= hs[:, None], axis=0)
    assert np.all(dq[:, far] == 0)


def test_scatter_volume_equal_h_is_gather_density_and_lattice_spacing():
    ns = 12
    xg = _lattice(ns)
    h = 2.6 / ns
    hg = np.full(xg.shape[1], h)
    rng = np.random.default_rng(1)
    xs = rng.uniform(0, 1, (3, 25))
    V, hv = S.volume(xs, np.full(25, h), xg, hg, n_h=2.0)
    # equal h: the scatter sum is the gather sum of W(r, h)
    d = xs[:, :, None] - xg[:, None, :]
    d -= np.round(d)
    r = np.sqrt((d * d).sum(0))
    W, _, _ = oracle.kernel(r.ravel(), h)
    dens = W.reshape(r.shape).sum(1) + oracle.kernel(np.zeros(1), h)[0][0]
    assert np.allclose(1.0 / V, dens, rtol=1e-13)
    # gas-only part of the sum (self term removed) ~ the lattice number density
    gas_only = 1.0 / V - oracle.kernel(np.zeros(1), h)[0][0]
    # (a kernel sum at h = 2.6 spacings reproduces the density to about a percent
    # at any point and to a few tenths of a percent on average)
    assert np.allclose(gas_only, ns ** 3, rtol=1.5e-2)
    assert abs(gas_only.mean() / ns ** 3 - 1) < 3e-3
    assert np.allclose(hv, 2.0 * np.cbrt(V))


def test_periodic_translation_invariance():
    rng = np.random.default_rng(2)
    xg = rng.uniform(0, 1, (3, 500))
    hg = rng.uniform(0.1, 0.2, 500)
    Vg = rng.uniform(0.5, 2.0, 500) / 500
    xs = rng.uniform(0, 1, (3, 30))
    hs = rng.uniform(0.1, 0.2, 30)
    q = rng.uniform(0, 1, (1, 30))
    V0, _ = S.volume(xs, hs, xg, hg)
    dq0, A0 = S.deposit(xs, hs, q, xg, Vg)
    sh = np.array([[0.37], [0.81], [0.05]])
    V1, _ = S.volume(np.mod(xs + sh, 1), hs, np.mod(xg + sh, 1), hg)
    dq1, A1 = S.deposit(np.mod(xs + sh, 1), hs, q, np.mod(xg + sh, 1), Vg)
    assert np.allclose(V0, V1, rtol=1e-12)
    assert np.allclose(A0, A1, rtol=1e-12)
    assert np.allclose(dq0, dq1, rtol=1e-12, atol=1e-15)
