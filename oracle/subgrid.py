"""FP64 oracle of the subgrid-particle neighbor sums (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
module; the product path never imports it.  Brute force over all gas particles
(small inputs only), float64, periodic minimum image.

What it computes:

* ``volume`` -- App. A.2, Eq. Vsg: the volume of a subgrid particle s (star,
  wind or black hole) from the SPH number density of the gas around it in the
  scatter form, V_s^-1 = sum_{j in gas, r_sj < h_j} W(r_sj, h_j) + W(0, h_s)
  (the self term uses the particle's own smoothing length), and the smoothing
  length n_h V_s^(1/3) it determines.
* ``deposit`` -- Sec. 2.5.3 Eq. windmetal with Eq. Anorm, Sec. 2.6.3 Eq.
  starmetal, Sec. 2.7.4 Eq. AGNE: a quantity q_s carried by a subgrid particle
  is shared among its eligible gas neighbors (gather form, r_sj < h_s) in
  proportion to V_j W(r_sj, h_s), normalised by A_s = 1 / sum_j V_j W(r_sj, h_s);
  every gas particle receives the sum over the subgrid particles that reach it.

Readings: a gas particle at exactly r = h is outside (as for the gas sums); a
subgrid particle with no eligible gas neighbor has A_s = 0 and deposits nothing.
"""
from __future__ import annotations

import numpy as np


def _sep(xs, xg, L):
    d = xs[:, :, None] - xg[:, None, :]          # (3, n_s, n_g)
    return d - L * np.round(d / L)


def _wendland(r, h):
    """Wendland C4 with support h, 3-D (same normalisation as the gas sums)."""
    q = r / h
    om = np.clip(1.0 - q, 0.0, None)
    cw = 495.0 / (32.0 * np.pi)
    return cw / h ** 3 * om ** 6 * (1.0 + 6.0 * q + 35.0 / 3.0 * q * q)


def volume(x_s, h_s, x_g, h_g, L=1.0, n_h=None):
    """(V_s, h_from_V) for subgrid particles x_s (3, n_s) among gas x_g (3, n_g)."""
    x_s = np.asarray(x_s, np.float64)
    x_g = np.asarray(x_g, np.float64)
    h_g = np.asarray(h_g, np.float64)
    d = _sep(x_s, x_g, L)
    r = np.sqrt((d * d).sum(axis=0))               # (n_s, n_g)
    hj = np.broadcast_to(h_g[None, :], r.shape)
    inside = r < hj
    w = np.where(inside, _wendland(r, hj), 0.0)
    s = w.sum(axis=1) + _wendland(np.zeros(x_s.shape[1]), np.asarray(h_s, np.float64))
    V = 1.0 / s
    return V, (None if n_h is None else n_h * np.cbrt(V))


def deposit(x_s, h_s, q_s, x_g, V_g, L=1.0, eligible=None):
    """(dq (n_comp, n_g), A_s (n_s,)) for quantities q_s (n_comp, n_s)."""
    x_s = np.asarray(x_s, np.float64)
    x_g = np.asarray(x_g, np.float64)
    h_s = np.asarray(h_s, np.float64)
    V_g = np.asarray(V_g, np.float64)
    q_s = np.atleast_2d(np.asarray(q_s, np.float64))
    d = _sep(x_s, x_g, L)
    r = np.sqrt((d * d).sum(axis=0))
    hs = np.broadcast_to(h_s[:, None], r.shape)
    ok = r < hs
    if eligible is not None:
        ok &= np.asarray(eligible, bool)[None, :]
    w = np.where(ok, V_g[None, :] * _wendland(r, hs), 0.0)   # V_j W(r_sj, h_s)
    tot = w.sum(axis=1)
    A = np.where(tot > 0, 1.0 / np.where(tot > 0, tot, 1.0), 0.0)
    share = A[:, None] * w                                      # (n_s, n_g)
    dq = q_s @ share                                            # (n_comp, n_g)
    return dq, A
