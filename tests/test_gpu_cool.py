"""GPU exact-integration cooling (Sec. 2.3.2) against the FP64 oracle, through
the C ABI: a table with heating below an equilibrium and the self-similar
power law above it, the closed form of a pure power law at full size,
unchanged energies outside the table, and the semigroup property."""
import numpy as np
import pytest
import torch

from oracle import cooling as C
from paper_2511_21921_gb300 import synth
from paper_2511_21921_gb300.solver import Solver

pytestmark = pytest.mark.gpu

DT = {"fp64": torch.float64, "mixed": torch.float32}
LOGU0, DEX, K = -3.0, 0.004, 1501        # 0.004 dex bins over six decades (the paper's width)
TOL = {"fp64": 1e-12, "mixed": 1e-5}


def _table():
    u = C.nodes(LOGU0, DEX, K)
    return 2.0 * u ** 1.5 - 3.0           # heating below u ~ 1.3, cooling above


def _run(precision, u0, rho, dt, lam, n=None):
    n = u0.size if n is None else n
    s = Solver(max(n, 1), 1, precision)
    t = lambda a: torch.tensor(a, dtype=DT[precision], device="cuda")
    lam_d = torch.tensor(lam, dtype=torch.float64, device="cuda")
    out = s.cool(dt, t(rho), t(u0), lam_d, LOGU0, DEX)
    torch.cuda.synchronize()
    return out.double().cpu().numpy(), s


def _inputs(precision, n, seed=0):
    d = synth.lognormal(16, 1.5, seed=seed)
    rng = np.random.default_rng(seed)
    u0 = np.resize(d["u"], n) * 10 ** rng.uniform(-1, 1, n)
    rho = 10 ** rng.uniform(-1, 1, n)
    if precision == "mixed":
        u0 = u0.astype(np.float32).astype(np.float64)
        rho = rho.astype(np.float32).astype(np.float64)
    return u0, rho


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_parity_with_equilibrium_table(precision):
    lam = _table()
    u0, rho = _inputs(precision, 3000)
    for dt in (1e-4, 1e-2, 1.0):
        got, _ = _run(precision, u0, rho, dt, lam)
        ref = C.cool(u0, rho, dt, lam, LOGU0, DEX)
        rel = np.abs(got - ref) / ref
        assert np.max(rel) <= TOL[precision], (dt, np.max(rel), u0[np.argmax(rel)])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_size_power_law_closed_form(precision):
    """262,144 particles of the 64^3 workload under lam = A u^1.5 (App. B):
    u1 = (u0^-1/2 + A rho dt / 2)^-2, every particle."""
    d = synth.load("lognormal64")
    u0 = d["u"].copy()
    n = u0.size
    rho = 10 ** np.random.default_rng(3).uniform(-1, 1, n)
    if precision == "mixed":
        u0 = u0.astype(np.float32).astype(np.float64)
        rho = rho.astype(np.float32).astype(np.float64)
    A, dt = 4.0, 0.05
    lam = C.power_law_table(A, 1.5, LOGU0, DEX, K)
    got, _ = _run(precision, u0, rho, dt, lam)
    expect = np.maximum((u0 ** -0.5 + 0.5 * A * rho * dt) ** -2.0, 10 ** LOGU0)
    rel = np.abs(got - expect) / expect
    assert np.max(rel) <= (1e-11 if precision == "fp64" else 1e-5), np.max(rel)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_outside_table_and_zero_step_unchanged(precision):
    lam = _table()
    u0 = np.array([10 ** (LOGU0 - 0.5), 10 ** (LOGU0 + DEX * K + 1), 5.0, 0.01])
    rho = np.ones(4)
    got, _ = _run(precision, u0, rho, 0.3, lam)
    assert got[0] == np.float32(u0[0]) or precision == "fp64" and got[0] == u0[0]
    assert got[1] == (np.float32(u0[1]) if precision == "mixed" else u0[1])
    got0, _ = _run(precision, u0, rho, 0.0, lam)
    assert np.array_equal(got0, u0.astype(np.float32).astype(np.float64)
                          if precision == "mixed" else u0)


def test_semigroup_on_gpu_fp64():
    lam = _table()
    u0, rho = _inputs("fp64", 2000, seed=5)
    one, s = _run("fp64", u0, rho, 0.03, lam)
    half, _ = _run("fp64", u0, rho, 0.01, lam)
    two, _ = _run("fp64", half, rho, 0.02, lam)
    assert np.allclose(one, two, rtol=1e-10, atol=0)


def test_two_node_table_and_pure_heating_fp64():
    """The smallest table (one bin) and a heating-only table: closed forms."""
    lam = np.array([-1.5, -1.5])          # constant heating over one bin, 1e-3 .. 1e-3+0.004 dex
    u0 = np.array([1.0e-3, 1.004e-3, 1.009e-3])
    got, _ = _run("fp64", u0, np.ones(3), 1e-7, lam)
    top = 10 ** (LOGU0 + DEX)
    expect = np.minimum(u0 + 1.5e-7, top)
    expect[u0 > top] = u0[u0 > top]
    assert np.allclose(got, expect, rtol=1e-13, atol=0)
