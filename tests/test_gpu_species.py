"""GPU gas + wind evaluation (Sec. 2.5.1 Eq. rhow; App. A.2) against the
oracle's species evaluation, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_21921_gb300 import _lib as L
from paper_2511_21921_gb300 import synth
from paper_2511_21921_gb300.solver import Solver

from gpu_util import DT, TOL, rel_l2, to_dev, compare

pytestmark = pytest.mark.gpu


def _np(t):
    return t.double().cpu().numpy()


def _winds(seed, n_side=32, frac=0.05):
    d = synth.lognormal(n_side, 1.5, seed=seed)
    n = d["h"].shape[0]
    rng = np.random.default_rng(seed)
    sp = (rng.uniform(size=n) < frac).astype(np.uint8)
    d["v"][:, sp == 1] += rng.normal(0, 0.5, (3, int(sp.sum())))   # launched winds
    return d, sp


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_parity_with_oracle_species(precision):
    d, sp = _winds(3)
    n = d["h"].shape[0]
    t = to_dev(d, precision)
    s = Solver(n, 1, precision)
    out = s.forward(t["x"], t["h"], t["m"], t["v"], t["u"],
                    species=torch.tensor(sp, device="cuda"), want_V=True, want_coef=True,
                    want_rho=True, want_gradv=True)
    vgw = s.volume_gw()
    torch.cuda.synchronize()
    assert s.poll() == 0
    dd = {k: (d[k].astype(np.float32).astype(np.float64) if precision == "mixed" and
              k in ("h", "m", "u", "v") else d[k]) for k in d}
    o = oracle.forward_species(dd["x"], dd["h"], dd["m"], dd["v"], dd["u"], 1.0, sp)
    g = {k: _np(v) for k, v in out.items() if v is not None}
    gas = sp == 0
    bar = TOL[precision]
    errs = {"V": rel_l2(g["V"], o["V"]), "Vgw": rel_l2(_np(vgw), o["Vgw"]),
            "rho": rel_l2(g["rho"], o["rho"]),
            "gradv": rel_l2(g["gradv"][:, gas], o["gradv"][:, gas]),
            "coef": rel_l2(g["coef"][:, gas], o["coef"][:, gas]),
            "dvdt": rel_l2(g["dvdt"], o["dvdt"]), "dudt": rel_l2(g["dudt"], o["dudt"])}
    assert all(e <= bar for e in errs.values()), errs
    assert np.all(g["dvdt"][:, ~gas] == 0) and np.all(g["dudt"][~gas] == 0)


def test_no_winds_is_bitwise_the_gas_path_and_guards():
    d = synth.load("lognormal32")
    n = d["h"].shape[0]
    t = to_dev(d, "mixed")
    s = Solver(n, 1, "mixed")
    a = s.forward(t["x"], t["h"], t["m"], t["v"], t["u"], want_rho=True, want_V=True)
    a = {k: v.clone() for k, v in a.items() if v is not None}
    b = s.forward(t["x"], t["h"], t["m"], t["v"], t["u"],
                  species=torch.zeros(n, dtype=torch.uint8, device="cuda"), want_rho=True,
                  want_V=True)
    for k in a:
        assert torch.equal(a[k], b[k]), k
    assert torch.equal(s.volume_gw(), a["V"])
    # with winds the adjoint and the active-set calls are refused
    s.set_species(torch.ones(n, dtype=torch.uint8, device="cuda"))
    s.moments(t["m"])
    z = torch.zeros(n, dtype=torch.float32, device="cuda")
    z3 = torch.zeros((3, n), dtype=torch.float32, device="cuda")
    rc = L.crk_adjoint(s.plan, 0, s._wsp, t["v"].data_ptr(), t["u"].data_ptr(), z3.data_ptr(),
                       z.data_ptr(), z3.data_ptr(), z3.data_ptr(), z.data_ptr(), z.data_ptr(), 1)
    assert rc == L.CRK_ESTATE


def test_subgrid_sums_skip_winds():
    """Winds are subgrid particles: the scatter volume and the deposits of
    other subgrid particles run over the gas only (App. A.2)."""
    from oracle import subgrid as S
    d, sp = _winds(5, n_side=16, frac=0.1)
    n = d["h"].shape[0]
    t = to_dev(d, "fp64")
    s = Solver(n, 1, "fp64")
    s.cell_build(t["x"], t["h"])
    s.set_species(torch.tensor(sp, device="cuda"))
    Vg, _ = s.moments(t["m"], want_V=True)
    rng = np.random.default_rng(6)
    xs = rng.uniform(0, 1, (3, 50))
    hs = rng.uniform(0.08, 0.15, 50)
    xs_d = torch.tensor(xs, device="cuda")
    hs_d = torch.tensor(hs, device="cuda")
    V, _ = s.subgrid_volume(xs_d, hs_d, want_h=False)
    q = np.ones((1, 50))
    dq, A = s.subgrid_deposit(xs_d, hs_d, torch.tensor(q, device="cuda"))
    torch.cuda.synchronize()
    assert s.poll() == 0
    gas = sp == 0
    eV, _ = S.volume(xs, hs, d["x"][:, gas], d["h"][gas])
    assert np.allclose(V.cpu().numpy(), eV, rtol=1e-12)
    edq, eA = S.deposit(xs, hs, q, d["x"][:, gas], Vg.cpu().numpy()[gas])
    got = dq.cpu().numpy()
    assert np.all(got[:, ~gas] == 0)
    assert np.allclose(got[:, gas], edq, rtol=1e-12, atol=1e-15)
    assert np.allclose(A.cpu().numpy(), eA, rtol=1e-12)
