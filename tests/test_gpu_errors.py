"""Argument and call-order errors of the newer entry points are returned
synchronously (no kernel runs on bad arguments)."""
import numpy as np
import pytest
import torch

from paper_2511_21921_gb300 import _lib as L
from paper_2511_21921_gb300 import synth
from paper_2511_21921_gb300.solver import Solver

from gpu_util import to_dev

pytestmark = pytest.mark.gpu


def _built(prec="fp64"):
    d = synth.lattice(8, seed=3)
    n = d["h"].shape[0]
    t = to_dev(d, prec)
    s = Solver(n, 1, prec)
    s.cell_build(t["x"], t["h"])
    return s, t, n


def test_cooling_table_and_step_errors():
    s, t, n = _built()
    lam = torch.ones(4, dtype=torch.float64, device="cuda")
    u = t["u"]
    for K, dex, dt in ((1, 0.1, 0.1), (4, 0.0, 0.1), (4, -1.0, 0.1), (4, 0.1, -1.0),
                       (4, float("nan"), 0.1)):
        tab = L.crk_cool_table(K, 0, -1.0, dex, lam.data_ptr())
        assert L.crk_cool_exact(s.plan, 0, n, tab, dt, u.data_ptr(), u.data_ptr(),
                                u.data_ptr()) == L.CRK_EINVAL
    tab = L.crk_cool_table(4, 0, -1.0, 0.1, None)
    assert L.crk_cool_exact(s.plan, 0, n, tab, 0.1, u.data_ptr(), u.data_ptr(),
                            u.data_ptr()) == L.CRK_EINVAL


def test_subgrid_time_bins_species_and_fused_state_errors():
    s, t, n = _built()
    x_s = torch.rand((3, 4), dtype=torch.float64, device="cuda")
    h_s = torch.full((4,), 0.1, dtype=torch.float64, device="cuda")
    bo = torch.tensor([0, 4], dtype=torch.int64, device="cuda")
    V = torch.empty(4, dtype=torch.float64, device="cuda")
    q = torch.ones(4, dtype=torch.float64, device="cuda")
    dq = torch.zeros(n, dtype=torch.float64, device="cuda")
    # deposits need gas volumes (crk_moments) first
    assert L.crk_subgrid_deposit(s.plan, 0, s._wsp, 4, bo.data_ptr(), x_s.data_ptr(),
                                 h_s.data_ptr(), 1, q.data_ptr(), None, None,
                                 dq.data_ptr()) == L.CRK_ESTATE
    assert L.crk_subgrid_deposit(s.plan, 0, s._wsp, 4, bo.data_ptr(), x_s.data_ptr(),
                                 h_s.data_ptr(), 65, q.data_ptr(), None, None,
                                 dq.data_ptr()) in (L.CRK_ESTATE, L.CRK_EINVAL)
    assert L.crk_subgrid_volume(s.plan, 0, s._wsp, 4, bo.data_ptr(), x_s.data_ptr(),
                                h_s.data_ptr(), -1.0, V.data_ptr(), V.data_ptr()) == L.CRK_EINVAL
    dtp = torch.ones(n, dtype=torch.float64, device="cuda")
    lv = torch.empty(n, dtype=torch.uint8, device="cuda")
    for lvmax, sub in ((-1, 0), (41, 0), (4, 16), (4, -1)):
        assert L.crk_time_bins(s.plan, 0, s._wsp, dtp.data_ptr(), 1.0, lvmax, sub, lv.data_ptr(),
                               None) == L.CRK_EINVAL
    assert L.crk_time_bins(s.plan, 0, s._wsp, dtp.data_ptr(), 0.0, 4, 0, lv.data_ptr(),
                           None) == L.CRK_EINVAL
    # the fused call needs crk_moments; the gas + wind volume needs it too
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    z3 = torch.zeros((3, n), dtype=torch.float64, device="cuda")
    args = [t["v"].data_ptr(), t["u"].data_ptr(), z3.data_ptr(), z.data_ptr(), z3.data_ptr(),
            z.data_ptr(), z3.data_ptr(), z3.data_ptr(), z.data_ptr(), z.data_ptr()]
    assert L.crk_rates_adjoint(s.plan, 0, s._wsp, *args) == L.CRK_ESTATE
    assert L.crk_volume_gw(s.plan, 0, s._wsp, z.data_ptr()) == L.CRK_ESTATE
    s.moments(t["m"])
    assert L.crk_rates_adjoint(s.plan, 0, s._wsp, *args) == L.CRK_OK
    s.set_species(torch.ones(n, dtype=torch.uint8, device="cuda"))
    s.moments(t["m"])
    assert L.crk_rates_adjoint(s.plan, 0, s._wsp, *args) == L.CRK_ESTATE
    torch.cuda.synchronize()
