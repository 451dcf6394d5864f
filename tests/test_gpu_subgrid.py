"""GPU subgrid neighbor sums (App. A.2 Eq. Vsg; Eqs. windmetal/Anorm,
starmetal, AGNE) against the brute-force FP64 oracle, through the C ABI:
scatter volumes and normalised deposits on a clustered box, eligibility,
conservation at full size, and a multi-box batch."""
import numpy as np
import pytest
import torch

import oracle
from oracle import subgrid as S
from paper_2511_21921_gb300 import synth
from paper_2511_21921_gb300.solver import Solver

from gpu_util import DT, to_dev

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-12, "mixed": 1e-5}


def _subgrid(d, n_s, seed, L=1.0):
    """Subgrid particles: half on gas positions (spawned from gas), half at
    random points; h_s from 2.25 times the local spacing."""
    rng = np.random.default_rng(seed)
    n = d["h"].shape[0]
    pick = rng.choice(n, n_s // 2, replace=False)
    xs = np.concatenate([d["x"][:, pick], rng.uniform(0, L, (3, n_s - n_s // 2))], axis=1)
    hs = np.concatenate([d["h"][pick] * 0.6, rng.uniform(0.5, 1.5, n_s - n_s // 2) *
                         np.median(d["h"]) * 0.6])
    return np.ascontiguousarray(xs), hs


def _as(a, precision):
    return a.astype(np.float32).astype(np.float64) if precision == "mixed" else a


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_volume_and_deposit_parity(precision):
    d = synth.lognormal(16, 1.5, seed=4)
    n = d["h"].shape[0]
    xs, hs = _subgrid(d, 300, seed=1)
    hs = _as(hs, precision)
    t = to_dev(d, precision)
    s = Solver(n, 1, precision)
    s.cell_build(t["x"], t["h"])
    Vg, _ = s.moments(t["m"], want_V=True)
    xs_d = torch.tensor(xs, dtype=torch.float64, device="cuda")
    hs_d = torch.tensor(hs, dtype=DT[precision], device="cuda")
    V, hv = s.subgrid_volume(xs_d, hs_d, n_h=2.25)
    rng = np.random.default_rng(2)
    q = _as(rng.uniform(0.1, 1.0, (2, 300)), precision)
    elig = (rng.uniform(size=n) > 0.1).astype(np.uint8)
    dq, A = s.subgrid_deposit(xs_d, hs_d, torch.tensor(q, dtype=DT[precision], device="cuda"),
                              eligible=torch.tensor(elig, device="cuda"))
    torch.cuda.synchronize()
    assert s.poll() == 0
    eV, eh = S.volume(xs, hs, d["x"], _as(d["h"], precision), n_h=2.25)
    Vg_np = Vg.double().cpu().numpy()   # the deposit weights use the GPU's own gas volumes
    edq, eA = S.deposit(xs, hs, q, d["x"], Vg_np, eligible=elig.astype(bool))
    tol = TOL[precision]
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(V.double().cpu().numpy(), eV) <= tol
    assert rel(hv.double().cpu().numpy(), eh) <= tol
    assert rel(A.double().cpu().numpy(), eA) <= tol
    assert rel(dq.double().cpu().numpy(), edq) <= tol
    # the gas volumes themselves are the oracle's
    o = oracle.forward(d["x"], d["h"], d["m"], d["v"], d["u"], 1.0, want=("V",))
    assert rel(Vg_np, o["V"]) <= tol


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_size_deposit_conserves(precision):
    """64^3 workload, 13,107 subgrid particles (5 % of the gas): every
    deposited quantity is conserved to rounding, nothing reaches ineligible gas."""
    d = synth.load("lognormal64")
    n = d["h"].shape[0]
    xs, hs = _subgrid(d, n // 20, seed=3)
    t = to_dev(d, precision)
    s = Solver(n, 1, precision)
    s.cell_build(t["x"], t["h"])
    s.moments(t["m"])
    rng = np.random.default_rng(4)
    q = rng.uniform(0.1, 1.0, (1, xs.shape[1]))
    elig = (rng.uniform(size=n) > 0.05).astype(np.uint8)
    dq, A = s.subgrid_deposit(torch.tensor(xs, device="cuda"),
                              torch.tensor(hs, dtype=DT[precision], device="cuda"),
                              torch.tensor(q, dtype=DT[precision], device="cuda"),
                              eligible=torch.tensor(elig, device="cuda"))
    V, _ = s.subgrid_volume(torch.tensor(xs, device="cuda"),
                            torch.tensor(hs, dtype=DT[precision], device="cuda"), want_h=False)
    torch.cuda.synchronize()
    assert s.poll() == 0
    dq = dq.double().cpu().numpy()
    A = A.double().cpu().numpy()
    qd = q.astype(np.float32).astype(np.float64) if precision == "mixed" else q
    tot = qd[0, A > 0].sum()
    assert abs(dq.sum() / tot - 1) <= (1e-12 if precision == "fp64" else 1e-5)
    assert np.all(dq[:, elig == 0] == 0)
    assert np.all(V.double().cpu().numpy() > 0)
    # sampled scatter volumes against brute force
    k = np.random.default_rng(5).choice(xs.shape[1], 64, replace=False)
    eV, _ = S.volume(xs[:, k], hs[k], d["x"], _as(d["h"], precision))
    assert np.linalg.norm(V.double().cpu().numpy()[k] - eV) / np.linalg.norm(eV) <= \
        (1e-12 if precision == "fp64" else 1e-5)


def test_multibox_subgrid_volume_per_box():
    d = synth.multibox(4, seed0=7, nmin=10, nmax=14)
    off = d["box_off"]
    n = d["h"].shape[0]
    t = to_dev(d, "fp64")
    s = Solver(n, len(off) - 1, "fp64")
    s.cell_build(t["x"], t["h"], t["box_off"], t["box_L"])
    rng = np.random.default_rng(6)
    per = [20, 0, 7, 33]
    xs = np.concatenate([rng.uniform(0, d["box_L"][b], (3, m)) for b, m in enumerate(per)], axis=1)
    hs = rng.uniform(0.05, 0.15, xs.shape[1])
    boff = np.concatenate([[0], np.cumsum(per)]).astype(np.int64)
    V, _ = s.subgrid_volume(torch.tensor(xs, device="cuda"), torch.tensor(hs, device="cuda"),
                            box_off_s=torch.tensor(boff, device="cuda"), want_h=False)
    torch.cuda.synchronize()
    V = V.cpu().numpy()
    for b in range(len(per)):
        sl = slice(boff[b], boff[b + 1])
        if per[b] == 0:
            continue
        g = slice(off[b], off[b + 1])
        eV, _ = S.volume(xs[:, sl], hs[sl], d["x"][:, g], d["h"][g], L=d["box_L"][b])
        assert np.allclose(V[sl], eV, rtol=1e-12)
