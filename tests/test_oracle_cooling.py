"""Pins of the exact-integration cooling oracle (Sec. 2.3.2, Exact Integration).

Closed forms of single power laws across many table bins (the self-similar
law lam = A u^1.5 of App. B, a linear law and constant heating), an ODE solve of
du/dt = -rho lam(u) through the interpolated table, the semigroup property of
exact integration, and the equilibrium bin: energies approach the interpolated
zero crossing from both sides and never pass it.
"""
import math

import numpy as np
from scipy.integrate import solve_ivp

from oracle import cooling as C

LOGU0, DEX, K = -3.0, 0.05, 161     # table over 8 decades, 0.05 dex bins


def test_self_similar_power_law_closed_form():
    """lam = A u^beta with beta = 1.5 (App. B for n_s = -2): u1 solves
    u1^(1-beta) = u0^(1-beta) - (1-beta) A rho dt, whatever the bins."""
    A, beta = 2.0, 1.5
    lam = C.power_law_table(A, beta, LOGU0, DEX, K)
    rng = np.random.default_rng(0)
    u0 = 10 ** rng.uniform(-1, 3, 40)
    rho = 10 ** rng.uniform(-1, 1, 40)
    for dt in (1e-6, 1e-3, 1e-1):
        got = C.cool(u0, rho, dt, lam, LOGU0, DEX)
        expect = (u0 ** (1 - beta) - (1 - beta) * A * rho * dt) ** (1 / (1 - beta))
        expect = np.maximum(expect, 10 ** LOGU0)  # the floor
        assert np.allclose(got, expect, rtol=1e-11, atol=0), (dt, np.max(np.abs(got / expect - 1)))
    assert abs(1.5 * (3 + -2) / (1 - -2) + 1 - beta) < 1e-15  # beta from n_s = -2 (App. B)


def test_linear_law_and_constant_heating():
    lam = C.power_law_table(3.0, 1.0, LOGU0, DEX, K)          # alpha = 1 in every bin
    u0, rho, dt = np.array([0.5, 7.0, 300.0]), np.array([1.0, 0.3, 2.0]), 0.2
    assert np.allclose(C.cool(u0, rho, dt, lam, LOGU0, DEX), u0 * np.exp(-3.0 * rho * dt),
                       rtol=1e-12, atol=0)
    heat = -np.full(K, 4.0)                                    # lam = -4: du/dt = 4 rho
    assert np.allclose(C.cool(u0, rho, dt, heat, LOGU0, DEX), u0 + 4.0 * rho * dt, rtol=1e-12,
                       atol=0)
    # the ceiling: heating stops at the top of the table
    top = 10 ** (LOGU0 + DEX * (K - 1))
    assert C.cool(np.array([top * 0.9]), 1.0, 1e9, heat, LOGU0, DEX)[0] == top


def _interp(lam, u):
    un = C.nodes(LOGU0, DEX, len(lam))
    k = min(max(int(math.floor((math.log10(u) - LOGU0) / DEX)), 0), len(lam) - 2)
    a = math.log(lam[k + 1] / lam[k]) / (DEX * math.log(10.0))
    return lam[k] * (u / un[k]) ** a


def test_matches_ode_solution_through_the_interpolated_table():
    rng = np.random.default_rng(1)
    lam = np.exp(np.cumsum(rng.normal(0.0, 0.3, K)))          # positive, uneven slopes
    for u0, rho, dt in ((3.0, 0.7, 0.05), (40.0, 2.0, 0.01), (0.2, 1.0, 0.3)):
        got = C.cool_one(u0, rho, dt, lam, LOGU0, DEX)
        sol = solve_ivp(lambda t, y: [-rho * _interp(lam, y[0])], (0.0, dt), [u0],
                        rtol=1e-12, atol=1e-14, method="DOP853")
        assert abs(got / sol.y[0, -1] - 1) < 1e-8, (u0, got, sol.y[0, -1])


def test_exact_integration_is_a_semigroup():
    rng = np.random.default_rng(2)
    u = C.nodes(LOGU0, DEX, K)
    lam = 1.7 * u ** 1.5 - 40.0                               # heating below, cooling above
    u0 = 10 ** rng.uniform(-2, 4, 30)
    rho = 10 ** rng.uniform(-0.5, 0.5, 30)
    one = C.cool(u0, rho, 0.03, lam, LOGU0, DEX)
    two = C.cool(C.cool(u0, rho, 0.01, lam, LOGU0, DEX), rho, 0.02, lam, LOGU0, DEX)
    assert np.allclose(one, two, rtol=1e-10, atol=0)


def test_equilibrium_bin_is_approached_never_crossed():
    u = C.nodes(LOGU0, DEX, K)
    lam = 1.7 * u ** 1.5 - 40.0
    k = int(np.nonzero((lam[:-1] < 0) & (lam[1:] > 0))[0][0])
    ueq = u[k] + (u[k + 1] - u[k]) * lam[k] / (lam[k] - lam[k + 1])
    above = np.array([ueq * 1.001, ueq * 3, ueq * 100])
    below = np.array([ueq * 0.999, ueq / 3, ueq / 100])
    for dt in (1e-4, 1e-2, 10.0):
        ua = C.cool(above, 1.0, dt, lam, LOGU0, DEX)
        ub = C.cool(below, 1.0, dt, lam, LOGU0, DEX)
        assert np.all(ua >= ueq) and np.all(ua <= above)
        assert np.all(ub <= ueq) and np.all(ub >= below)
    assert np.all(C.cool(np.concatenate([above, below]), 1.0, 1e6, lam, LOGU0, DEX) == ueq)
    # outside the table: unchanged
    assert C.cool_one(10 ** (LOGU0 - 1), 1.0, 1.0, lam, LOGU0, DEX) == 10 ** (LOGU0 - 1)
