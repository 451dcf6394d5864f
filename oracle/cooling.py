"""FP64 oracle of exact-integration cooling (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
module; the product path never imports it.

What it computes (Sec. 2.3.2, Exact Integration; Eqs. cool, intcool, I, u1, L,
Iu, Iinv): the internal energy u1 at the end of a step dt of du/dt = -Lambda/rho
with rho held fixed, for a source function tabulated at logarithmically spaced
energies and interpolated with piecewise power laws.  The source function is
Lambda(u; rho) = rho^2 lam(u) (the density scaling of the self-similar
power-law test, App. B: Lambda / n_H^2 = A_1 u^beta), so du/dt = -rho lam(u)
and u1 solves

    int_{u1}^{u0} du / lam(u) = rho dt        (cooling, lam > 0),

with the mirror relation for heating (lam < 0).  This module writes that
definition out: per-bin integrals of the power law, summed bin by bin, and the
final energy found by bisection on the integral inside the last bin (not by the
closed-form inverse the kernels use).

Readings where the paper leaves a choice (also in the design notes):

* A bin whose edge values differ in sign (or contain a zero) holds the
  equilibrium: it is crossed at the constant rate max(|lam_k|, |lam_k+1|) in the
  direction the linear interpolant of lam gives at the current energy, and the
  energy stops at the interpolated zero crossing when it lies ahead.
* The table ends are a floor and a ceiling: an energy that reaches u_min
  (u_max) while cooling (heating) stays there; an energy outside the table at
  the start is left unchanged.
"""
from __future__ import annotations

import math

import numpy as np


def nodes(log10_u_min, dlog10_u, n_nodes):
    return 10.0 ** (log10_u_min + dlog10_u * np.arange(n_nodes))


def _G(x, a):
    """int_1^x t^(-a) dt = (x^(1-a) - 1)/(1-a), or ln x for a = 1 (written with
    expm1 so that slopes within rounding of 1 stay accurate)."""
    if a == 1.0:
        return math.log(x)
    return math.expm1((1.0 - a) * math.log(x)) / (1.0 - a)


def _bin(lam, k):
    """Type of bin k: +1 regular cooling, -1 regular heating, 0 equilibrium."""
    a, b = lam[k], lam[k + 1]
    if a > 0 and b > 0:
        return 1
    if a < 0 and b < 0:
        return -1
    return 0


def _alpha(lam, k, dlog10_u):
    return math.log(abs(lam[k + 1]) / abs(lam[k])) / (dlog10_u * math.log(10.0))


def _cost(uk, lk, a, lo, hi):
    """int_lo^hi du / |lam| inside a regular bin with lam = lk (u/uk)^a."""
    return uk / abs(lk) * (_G(hi / uk, a) - _G(lo / uk, a))


def _solve_in_bin(uk, lk, a, u, tau, down, lo, hi):
    """Energy reached from u after tau inside the bin [lo, hi], by bisection
    on the integral (the definition, not the closed-form inverse)."""
    if down:
        f = lambda w: _cost(uk, lk, a, w, u) - tau
        a_, b_ = lo, u
    else:
        f = lambda w: _cost(uk, lk, a, u, w) - tau
        a_, b_ = u, hi
    # f is monotone on [a_, b_]; the root exists because tau < cost to the edge
    for _ in range(200):
        m = 0.5 * (a_ + b_)
        fm = f(m)
        if down:
            if fm > 0:
                a_ = m
            else:
                b_ = m
        else:
            if fm < 0:
                a_ = m
            else:
                b_ = m
        if b_ - a_ <= 1e-17 * max(abs(a_), abs(b_)):
            break
    return 0.5 * (a_ + b_)


def cool_one(u0, rho, dt, lam, log10_u_min, dlog10_u):
    """u1 of one particle (float64)."""
    lam = np.asarray(lam, dtype=np.float64)
    K = lam.size
    un = nodes(log10_u_min, dlog10_u, K)
    u_min, u_max = un[0], un[-1]
    if not (u_min <= u0 <= u_max):
        return float(u0)
    tau = rho * dt
    u = float(u0)
    k = min(int(math.floor((math.log10(u) - log10_u_min) / dlog10_u)), K - 2)
    k = max(k, 0)
    # node k is the largest node <= u (guard the floor of the log)
    while k > 0 and un[k] > u:
        k -= 1
    while k < K - 2 and un[k + 1] <= u:
        k += 1
    direction = 0
    for _ in range(4 * K + 8):
        if tau <= 0:
            return u
        t = _bin(lam, k)
        lo, hi = un[k], un[k + 1]
        if t != 0:
            a = _alpha(lam, k, dlog10_u)
            down = t > 0
            if direction != 0 and (direction < 0) != down:
                return u  # came in from a bin that pushes the other way: equilibrium at the node
            direction = -1 if down else 1
            edge = lo if down else hi
            c = _cost(lo, lam[k], a, edge, u) if down else _cost(lo, lam[k], a, u, edge)
            if tau < c:
                return _solve_in_bin(lo, lam[k], a, u, tau, down, lo, hi)
            tau -= c
            u = edge
            if down:
                if k == 0:
                    return u_min
                k -= 1
            else:
                if k == K - 2:
                    return u_max
                k += 1
            continue
        # equilibrium bin: linear interpolant sets direction and the zero crossing
        la, lb = lam[k], lam[k + 1]
        rate = max(abs(la), abs(lb))
        if rate == 0.0:
            return u
        lin = la + (lb - la) * (u - lo) / (hi - lo)
        if lin == 0.0:
            return u
        down = lin > 0
        if direction != 0 and (direction < 0) != down:
            return u
        direction = -1 if down else 1
        ueq = lo + (hi - lo) * la / (la - lb) if la != lb else None
        if down:
            target = ueq if (ueq is not None and lo <= ueq <= u) else lo
        else:
            target = ueq if (ueq is not None and u <= ueq <= hi) else hi
        need = abs(u - target) / rate
        if tau < need:
            return u - rate * tau if down else u + rate * tau
        tau -= need
        u = target
        if ueq is not None and target == ueq:
            return u
        if down:
            if k == 0:
                return u_min
            k -= 1
        else:
            if k == K - 2:
                return u_max
            k += 1
    return u


def cool(u0, rho, dt, lam, log10_u_min, dlog10_u):
    """u1 for arrays u0, rho (float64 loop; small inputs only)."""
    u0 = np.asarray(u0, dtype=np.float64)
    rho = np.broadcast_to(np.asarray(rho, dtype=np.float64), u0.shape)
    return np.array([cool_one(a, r, dt, lam, log10_u_min, dlog10_u)
                     for a, r in zip(u0.ravel(), rho.ravel())]).reshape(u0.shape)


def power_law_table(A, beta, log10_u_min, dlog10_u, n_nodes):
    """lam_k = A u_k^beta: the self-similar cooling law (App. B) per rho^2."""
    return A * nodes(log10_u_min, dlog10_u, n_nodes) ** beta
