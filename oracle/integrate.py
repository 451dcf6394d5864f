"""FP64 oracle of the hydro time step around the rates (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
module; the product path never imports it.  Plain numpy, float64, one
operation per line where the GPU path must reproduce the rounding order.

What it computes (paper sections and equations):

* ``hdot``            -- smoothing-length rate of App. A.3 (Smoothing Length
  Integration): the Thacker estimate h^T = h (1 - lambda + lambda Delta_N) with
  Delta_N^3 = V n_h^3 / h^3, its rate (h^T - h)/dt_a, plus the continuity rate
  h (div v)/3.
* ``drift_h``, ``drift_passive`` -- the exponential drift of App. A.3:
  h <- h exp[(hdot/h) dt], V <- (h/n_h)^3, rho <- rho exp[-(div v) dt].
* ``kick``            -- one kick of the KDK update of App. A.4 (K: v + a dt/2).
* ``kick_refined``    -- the piecewise-constant completion of App. A.4 when the
  step is refined from dt_b to dt_c: v0 + a0 (dt_b - dt_c) + (a0 + a1) dt_c / 2.
* ``drift``           -- the drift of App. A.4, with the parabolic passive
  trajectory: the velocity used over sub-step j is
  v_half + a0 [t_elapse + (dt_j - dt_a)/2], and positions accumulate in double.
* ``kdk_step``        -- one global KDK step around ``oracle.forward``.

Readings where the paper leaves a choice (each also listed in the design notes):

* The ratio hdot/h in the drift is the one evaluated with hdot (the logarithmic
  rate is held over the active interval), so drifts over sub-steps compose to
  one drift over their sum, and V rho is conserved when Delta_N = 1.
* The rates at the end of a step use the drifted positions and smoothing
  lengths and the predicted velocity and energy v_half + a0 dt/2,
  u_half + (du/dt)_0 dt/2.
* The internal energy is kicked like the velocity, with du/dt.
* A coordinate that leaves [0, L) is wrapped by one box side; a wrap that
  rounds to exactly L gives 0.
"""
from __future__ import annotations

import numpy as np

from .oracle import forward


def hdot(h, V, div, dt_a, lam, n_h):
    """Smoothing-length rate (App. A.3).  Returns (hdot, hdot / h).

    h, V, div: float64 arrays (n,); dt_a > 0 the active time step; lam the
    Thacker weight; n_h the target number of particles per kernel radius.
    """
    h = np.asarray(h, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    div = np.asarray(div, dtype=np.float64)
    if not dt_a > 0:
        raise ValueError("dt_a must be > 0")
    delta_n = n_h * np.cbrt(V) / h            # Delta_N = (V n_h^3 / h^3)^(1/3)
    one_m = 1.0 - lam
    h_t = h * (one_m + lam * delta_n)         # Thacker estimate
    hd_t = (h_t - h) / dt_a                   # Thacker rate
    hd_c = (h * div) / 3.0                    # continuity rate
    hd = hd_t + hd_c
    return hd, hd / h


def drift_h(h, hrate, dt):
    """h exp[(hdot/h) dt] with the logarithmic rate held fixed (App. A.3)."""
    return np.asarray(h, np.float64) * np.exp(np.asarray(hrate, np.float64) * dt)


def drift_passive(h_new, rho, div, dt, n_h):
    """Passive volume and density after a drift (App. A.3):
    V = (h/n_h)^3 and rho exp(-div dt)."""
    q = np.asarray(h_new, np.float64) / n_h
    V = q * q * q
    r = np.asarray(rho, np.float64) * np.exp(-np.asarray(div, np.float64) * dt)
    return V, r


def kick(v0, a, dt):
    """v0 + dt a (App. A.4, K).  dt is the kick length (dt_a / 2 for a half kick)."""
    v0 = np.asarray(v0, np.float64)
    t = dt * np.asarray(a, np.float64)
    return v0 + t


def kick_refined(v0, a0, a1, dt_b, dt_c):
    """Completion of a refined step (App. A.4):
    v0 + a0 (dt_b - dt_c) + (a0 + a1) dt_c / 2."""
    v0 = np.asarray(v0, np.float64)
    a0 = np.asarray(a0, np.float64)
    a1 = np.asarray(a1, np.float64)
    t1 = a0 * (dt_b - dt_c)
    s = a0 + a1
    t2 = s * (0.5 * dt_c)
    return (v0 + t1) + t2


def wrap(y, L):
    """Map a coordinate that moved by less than one box side back into [0, L)."""
    y = np.array(y, dtype=np.float64)
    L = np.broadcast_to(np.asarray(L, np.float64), y.shape)
    lo = y < 0.0
    y[lo] = y[lo] + L[lo]
    y[lo & (y >= L)] = 0.0
    hi = (~lo) & (y >= L)
    y[hi] = y[hi] - L[hi]
    return y


def drift(x, v_half, dt, L, a0=None, dt_a=None, t_elapse=None):
    """Positions after one drift of length dt (App. A.4), in float64.

    x: (3, n) float64; v_half: (3, n) stored half-step velocity.  Without a0
    the drift is linear in v_half.  With a0, particle i drifts with the local
    half-step velocity v_half + a0 [t_elapse_i + (dt - dt_a_i)/2] (its active
    interval dt_a_i, of which t_elapse_i has passed); dt_a and t_elapse default
    to dt and 0 (an active particle, for which the two drifts agree).
    L: scalar or (n,) box side per particle.
    """
    x = np.asarray(x, np.float64)
    vj = np.asarray(v_half, np.float64)
    if a0 is not None:
        n = x.shape[1]
        dta = np.full(n, dt) if dt_a is None else np.asarray(dt_a, np.float64)
        te = np.zeros(n) if t_elapse is None else np.asarray(t_elapse, np.float64)
        half = 0.5 * (dt - dta)
        w = te + half
        vj = vj + np.asarray(a0, np.float64) * w
    y = x + vj * dt
    return np.stack([wrap(y[k], L) for k in range(3)])


def kdk_init(x, v, u, h, m, L, dt_a, lam, n_h, params=None):
    """Rates and smoothing-length rate at the start of the first step."""
    o = forward(x, h, m, v, u, L, params=params, want=("V", "rho", "gradv", "dvdt", "dudt"))
    div = o["gradv"][0] + o["gradv"][4] + o["gradv"][8]
    _, hr = hdot(h, o["V"], div, dt_a, lam, n_h)
    return {"a": o["dvdt"], "du": o["dudt"], "hrate": hr, "div": div, "V": o["V"],
            "rho": o["rho"]}


def kdk_step(x, v, u, h, m, L, d0, dt, lam, n_h, params=None):
    """One global kick-drift-kick step of length dt (App. A.4) with the
    smoothing-length drift of App. A.3.

    d0: the derivatives at the start ({"a", "du", "hrate"}, from ``kdk_init`` or
    the previous step).  Returns (x1, v1, u1, h1, d1) with d1 the derivatives at
    the end of the step (and "V", "rho", "div" of that evaluation).
    """
    half = 0.5 * dt
    v_h = kick(v, d0["a"], half)
    u_h = kick(u, d0["du"], half)
    x1 = drift(x, v_h, dt, L)
    h1 = drift_h(h, d0["hrate"], dt)
    v_p = kick(v_h, d0["a"], half)
    u_p = kick(u_h, d0["du"], half)
    o = forward(x1, h1, m, v_p, u_p, L, params=params,
                want=("V", "rho", "gradv", "dvdt", "dudt"))
    div = o["gradv"][0] + o["gradv"][4] + o["gradv"][8]
    _, hr = hdot(h1, o["V"], div, dt, lam, n_h)
    v1 = kick(v_h, o["dvdt"], half)
    u1 = kick(u_h, o["dudt"], half)
    d1 = {"a": o["dvdt"], "du": o["dudt"], "hrate": hr, "div": div, "V": o["V"],
          "rho": o["rho"]}
    return x1, v1, u1, h1, d1
