"""GPU time step around the rates (kicks, drift, smoothing-length rate, whole
kick-drift-kick steps) against the FP64 oracle, through the C ABI.

Bars: in the FP64 form the kicks and the position drift round exactly like the
oracle (bit-exact); smoothing length, volume and density drifts differ by the
last bits of exp; the rates-derived quantities keep the rates' bar (1e-12
FP64, 1e-5 mixed, relative L2).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import integrate as I
from paper_2511_21921_gb300 import synth
from paper_2511_21921_gb300.solver import Solver

from gpu_util import DT, TOL, rel_l2, to_dev

pytestmark = pytest.mark.gpu

NH = (3.0 * 100 / (4.0 * np.pi)) ** (1.0 / 3.0)


def _dev(a, precision):
    return torch.tensor(np.ascontiguousarray(a), dtype=DT[precision], device="cuda")


def _x(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _np(t):
    return t.double().cpu().numpy()


def _as(a, precision):
    """What the oracle sees of an array the GPU holds in `precision`."""
    return a.astype(np.float32).astype(np.float64) if precision == "mixed" else a


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_kick_and_refined_kick(precision):
    rng = np.random.default_rng(1)
    n = 100_003
    v0, a0, a1 = (_as(rng.normal(size=(3, n)), precision) for _ in range(3))
    u0 = _as(rng.uniform(0.1, 2.0, n), precision)
    du0, du1 = (_as(rng.normal(size=n), precision) for _ in range(2))
    act = (rng.uniform(size=n) < 0.7).astype(np.uint8)
    s = Solver(n, 1, precision)
    tv0, ta0, ta1 = _dev(v0, precision), _dev(a0, precision), _dev(a1, precision)
    tu0, tdu0, tdu1 = _dev(u0, precision), _dev(du0, precision), _dev(du1, precision)
    tact = torch.tensor(act, device="cuda")
    dt = 0.0123
    tol = 0.0 if precision == "fp64" else 2e-7
    # half kick, all active
    vo, uo = s.kick(0.5 * dt, tv0, ta0, tu0, tdu0, v_out=torch.empty_like(tv0),
                    u_out=torch.empty_like(tu0))
    ev, eu = I.kick(v0, a0, 0.5 * dt), I.kick(u0, du0, 0.5 * dt)
    # error relative to the size of the operands (a kick may cancel v0)
    assert np.max(np.abs(_np(vo) - ev) / (np.abs(v0) + np.abs(0.5 * dt * a0))) <= tol
    assert np.max(np.abs(_np(uo) - eu) / (np.abs(u0) + np.abs(0.5 * dt * du0))) <= tol
    # masked, in place
    v_in = tv0.clone()
    s.kick(dt, v_in, ta0, active=tact)
    got = _np(v_in)
    on = act.astype(bool)
    assert np.array_equal(got[:, ~on], _np(tv0)[:, ~on])
    e = I.kick(v0, a0, dt)
    sc = np.abs(v0) + np.abs(dt * a0)
    assert np.max(np.abs(got[:, on] - e[:, on]) / sc[:, on]) <= tol
    # refined completion (App. A.4) for a range of dt_c
    for dt_c in (dt, 0.4 * dt, 0.0):
        vo, uo = s.kick_refined(dt, dt_c, tv0, ta0, ta1, tu0, tdu0, tdu1,
                                v_out=torch.empty_like(tv0), u_out=torch.empty_like(tu0))
        ev = I.kick_refined(v0, a0, a1, dt, dt_c)
        eu = I.kick_refined(u0, du0, du1, dt, dt_c)
        scale_v = np.abs(v0) + np.abs(a0 * dt) + np.abs(a1 * dt)
        scale_u = np.abs(u0) + np.abs(du0 * dt) + np.abs(du1 * dt)
        assert np.max(np.abs(_np(vo) - ev) / scale_v) <= 2 * tol
        assert np.max(np.abs(_np(uo) - eu) / scale_u) <= 2 * tol
        if precision == "fp64":
            assert np.array_equal(_np(vo), ev) and np.array_equal(_np(uo), eu)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_drift_positions_h_volume_density(precision):
    rng = np.random.default_rng(2)
    n = 65_537
    L = 1.0
    x0 = rng.uniform(0, L, size=(3, n))
    # put some particles next to the faces, moving out of the box
    x0[0, :64] = L - 1e-12
    x0[1, 64:128] = 1e-13
    x0[2, 128:130] = 0.0
    vh = _as(rng.normal(size=(3, n)), precision)
    vh[0, :64] = np.abs(vh[0, :64])
    vh[1, 64:128] = -np.abs(vh[1, 64:128])
    vh[2, 128:130] = -1e-30 if precision == "fp64" else -1e-20
    a0 = _as(rng.normal(size=(3, n)), precision)
    dt = 0.003
    dta = rng.choice([dt, 2 * dt, 4 * dt, 8 * dt], size=n)
    te = np.floor(rng.uniform(0, 1, n) * (dta / dt)) * dt
    h = _as(rng.uniform(0.01, 0.05, n), precision)
    hr = _as(rng.normal(scale=2.0, size=n), precision)
    rho = _as(rng.uniform(0.5, 5.0, n), precision)
    div = _as(rng.normal(scale=3.0, size=n), precision)
    s = Solver(n, 1, precision)
    for parabolic in (False, True):
        tx = _x(x0)
        th, trho, tV = _dev(h, precision), _dev(rho, precision), _dev(np.zeros(n), precision)
        kw = dict(a0=_dev(a0, precision), dt_a=_x(dta), t_elapse=_x(te)) if parabolic else {}
        s.drift(dt, tx, _dev(vh, precision), h=th, hrate=_dev(hr, precision), n_h=NH, V=tV,
                rho=trho, div=_dev(div, precision), **kw)
        torch.cuda.synchronize()
        gx = _np(tx)
        if parabolic:
            ex = I.drift(x0, vh, dt, L, a0=a0, dt_a=dta, t_elapse=te)
        else:
            ex = I.drift(x0, vh, dt, L)
        assert np.all((gx >= 0) & (gx < L))
        if precision == "fp64":
            assert np.array_equal(gx, ex), np.argwhere(gx != ex)[:5]
        else:
            dx = np.abs(gx - ex)
            dx = np.minimum(dx, L - dx)
            # the float displacement is good to a few roundings of its operands
            w = te + 0.5 * (dt - dta) if parabolic else 0.0
            scale = (np.abs(vh) + np.abs(a0 * w)) * dt
            assert np.max(dx - 4e-7 * scale) <= 2 ** -52, np.max(dx / (scale + 1e-300))
        eh = I.drift_h(h, hr, dt)
        eV, erho = I.drift_passive(eh, rho, div, dt, NH)
        tolf = 1e-15 if precision == "fp64" else 6e-7
        for got, exp, name in ((th, eh, "h"), (tV, eV, "V"), (trho, erho, "rho")):
            r = np.max(np.abs(_np(got) - exp) / np.abs(exp))
            assert r <= (3 if name == "V" else 1) * tolf, (name, r)


def test_drift_multibox_wraps_each_box():
    rng = np.random.default_rng(3)
    sizes = np.array([5, 0, 1000, 17, 333])
    off = np.concatenate([[0], np.cumsum(sizes)])
    Ls = np.array([1.0, 2.0, 0.5, 3.0, 1.25])
    n = int(off[-1])
    Lp = np.repeat(Ls, sizes)
    x0 = rng.uniform(0, 1, size=(3, n)) * Lp
    vh = rng.normal(size=(3, n)) * Lp
    dt = 0.2
    s = Solver(n, len(sizes), "fp64")
    tx = _x(x0)
    s.drift(dt, tx, _x(vh), box_off=torch.tensor(off, device="cuda"), box_L=_x(Ls))
    gx = _np(tx)
    assert np.array_equal(gx, I.drift(x0, vh, dt, Lp))
    assert np.all((gx >= 0) & (gx < Lp))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_hdot_against_oracle(precision):
    d = synth.load("lognormal32")
    n = d["h"].shape[0]
    t = to_dev(d, precision)
    s = Solver(n, 1, precision)
    s.cell_build(t["x"], t["h"])
    s.moments(t["m"])
    s.rates(t["v"], t["u"])
    dt_a, lam = 2e-3, 0.3
    hd, hr, dv = s.hdot(dt_a, lam, NH)
    torch.cuda.synchronize()
    assert s.poll() == 0
    o = oracle.forward(d["x"], d["h"], d["m"], d["v"], d["u"], 1.0, want=("V", "gradv"))
    div = o["gradv"][0] + o["gradv"][4] + o["gradv"][8]
    ehd, ehr = I.hdot(d["h"], o["V"], div, dt_a, lam, NH)
    for got, exp in ((hd, ehd), (hr, ehr), (dv, div)):
        assert rel_l2(_np(got), exp) <= TOL[precision]


def test_hdot_argument_and_state_errors():
    from paper_2511_21921_gb300 import _lib as L
    d = synth.lattice(8, seed=1)
    n = d["h"].shape[0]
    t = to_dev(d, "fp64")
    s = Solver(n, 1, "fp64")
    s.cell_build(t["x"], t["h"])
    s.moments(t["m"])
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    rc = L.crk_hdot(s.plan, 0, s._wsp, 1e-3, 0.5, NH, out.data_ptr(), None, None)
    assert rc == L.CRK_ESTATE  # no rates yet
    s.rates(t["v"], t["u"])
    for dt_a, nh in ((0.0, NH), (-1.0, NH), (1e-3, 0.0), (float("nan"), NH)):
        assert L.crk_hdot(s.plan, 0, s._wsp, dt_a, 0.5, nh, out.data_ptr(), None, None) == \
            L.CRK_EINVAL
    v = t["v"]
    assert L.crk_kick_refined(s.plan, 0, n, 1e-3, 2e-3, None, v.data_ptr(), v.data_ptr(),
                              v.data_ptr(), v.data_ptr()) == L.CRK_EINVAL  # dt_c > dt_b
    assert L.crk_drift(s.plan, 0, n, 1, None, None, 1e-3, t["x"].data_ptr(),
                       v.data_ptr()) == L.CRK_EINVAL  # no boxes
    assert L.crk_kick(s.plan, 0, n + 1, 1e-3, None, v.data_ptr(), v.data_ptr(),
                      v.data_ptr()) == L.CRK_EINVAL  # n above the plan's n_max


def _min_image(a, L=1.0):
    d = np.abs(a)
    return np.minimum(d, L - d)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_kdk_steps_against_oracle(precision):
    """Three global kick-drift-kick steps (App. A.3 and B.2) on the 32^3
    lognormal box: state and derivatives against the oracle's steps."""
    d = synth.load("lognormal32")
    n = d["h"].shape[0]
    x, v, u, h, m = d["x"], d["v"], d["u"], d["h"], d["m"]
    cs = np.sqrt(10.0 / 9.0 * u.max())
    dt = 0.1 * h.min() / (cs + np.abs(v).max())
    lam = 0.2
    t = to_dev(d, precision)
    s = Solver(n, 1, precision)
    gd = s.kdk_init(t["x"], t["v"], t["u"], t["h"], t["m"], dt, lam, NH)
    od = I.kdk_init(x, _as(v, precision), _as(u, precision), _as(h, precision),
                    _as(m, precision), 1.0, dt, lam, NH)
    ox, ov, ou, oh = x, _as(v, precision), _as(u, precision), _as(h, precision)
    mm = _as(m, precision)
    for _ in range(3):
        s.kdk_step(t["x"], t["v"], t["u"], t["h"], t["m"], gd, dt, lam, NH)
        ox, ov, ou, oh, od = I.kdk_step(ox, ov, ou, oh, mm, 1.0, od, dt, lam, NH)
    torch.cuda.synchronize()
    assert s.poll() == 0
    disp = _min_image(ox - x).max()
    ex = _min_image(_np(t["x"]) - ox).max() / disp
    errs = {"x": ex, "v": rel_l2(_np(t["v"]), ov), "u": rel_l2(_np(t["u"]), ou),
            "h": rel_l2(_np(t["h"]), oh), "a": rel_l2(_np(gd["a"]), od["a"]),
            "du": rel_l2(_np(gd["du"]), od["du"]), "hrate": rel_l2(_np(gd["hrate"]), od["hrate"])}
    bar = TOL[precision]
    assert all(e <= bar for e in errs.values()), errs


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_kdk_conserves_momentum_and_energy_over_steps(precision):
    """Ten steps on the 32^3 lognormal box with a step limited to a tenth of
    the fastest energy change: sum m v is kept to rounding (antisymmetric pair
    forces), and E = sum m (v^2/2 + u) to the integrator's small error
    (compatible energy, Sec. 2.1)."""
    d = synth.load("lognormal32")
    n = d["h"].shape[0]
    t = to_dev(d, precision)
    s = Solver(n, 1, precision)
    gd = s.kdk_init(t["x"], t["v"], t["u"], t["h"], t["m"], 1e-3, 0.2, NH)
    dt = 0.1 * float((t["u"].double() / gd["du"].double().abs()).min())
    gd = s.kdk_init(t["x"], t["v"], t["u"], t["h"], t["m"], dt, 0.2, NH)
    m = t["m"].double()

    def energy():
        vv = t["v"].double()
        return float((m * (0.5 * (vv * vv).sum(dim=0) + t["u"].double())).sum())
    p0 = (m * t["v"].double()).sum(dim=1)
    E0 = energy()
    budget = float((m * t["v"].double().abs()).sum())
    for _ in range(10):
        s.kdk_step(t["x"], t["v"], t["u"], t["h"], t["m"], gd, dt, 0.2, NH)
        budget += float((m * gd["a"].double().abs()).sum()) * dt
    torch.cuda.synchronize()
    assert s.poll() == 0
    dp = float(((m * t["v"].double()).sum(dim=1) - p0).abs().max())
    bar = 1e-13 if precision == "fp64" else 1e-6
    assert dp <= bar * budget, (dp, budget)
    dE = abs(energy() - E0) / E0
    assert dE <= (1e-6 if precision == "fp64" else 1e-5), dE


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_kdk_step_graph_replay_equals_eager(precision):
    """A whole step (kicks, drift, build, moments, rates, hdot) captured into
    one CUDA graph replays bit-identically to the eager step.  The Thacker term
    moves h towards its target by lambda of the gap per step, so the lists get
    room for the growth (no capacity check inside a graph)."""
    d = synth.load("lognormal32")
    n = d["h"].shape[0]
    dt = 1e-4
    outs = []
    for mode in ("eager", "graph"):
        t = to_dev(d, precision)
        s = Solver(n, 1, precision, nbr_cap=384)
        gd = s.kdk_init(t["x"], t["v"], t["u"], t["h"], t["m"], dt, 0.2, NH)
        scratch = (torch.empty_like(t["v"]), torch.empty_like(t["u"]))

        def step():
            s.kdk_step(t["x"], t["v"], t["u"], t["h"], t["m"], gd, dt, 0.2, NH, check=False,
                       scratch=scratch)
        if mode == "eager":
            for _ in range(3):
                step()
        else:
            step()
            g = s.capture(step)  # runs the step once as the capture's warm-up
            g.replay()           # third step
        torch.cuda.synchronize()
        assert s.poll() == 0
        outs.append([_np(a) for a in (t["x"], t["v"], t["u"], t["h"], gd["a"], gd["hrate"])])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_kdk_step_multibox_matches_oracle_per_box():
    """One kick-drift-kick step over a batch of boxes of different sizes (the
    drift wraps each particle into its own box) against the oracle's step of
    every box on its own."""
    d = synth.multibox(5, seed0=40, nmin=10, nmax=14)
    off = d["box_off"]
    n = d["h"].shape[0]
    t = to_dev(d, "fp64")
    s = Solver(n, len(off) - 1, "fp64")
    bo, bl = t["box_off"], t["box_L"]
    dt, lam = 2e-4, 0.2
    gd = s.kdk_init(t["x"], t["v"], t["u"], t["h"], t["m"], dt, lam, NH, box_off=bo, box_L=bl)
    s.kdk_step(t["x"], t["v"], t["u"], t["h"], t["m"], gd, dt, lam, NH, box_off=bo, box_L=bl)
    torch.cuda.synchronize()
    assert s.poll() == 0
    gx, gv = _np(t["x"]), _np(t["v"])
    for b in range(len(off) - 1):
        sl = slice(off[b], off[b + 1])
        if off[b + 1] == off[b]:
            continue
        L = d["box_L"][b]
        od = I.kdk_init(d["x"][:, sl], d["v"][:, sl], d["u"][sl], d["h"][sl], d["m"][sl], L, dt,
                        lam, NH)
        ox, ov, _, _, _ = I.kdk_step(d["x"][:, sl], d["v"][:, sl], d["u"][sl], d["h"][sl],
                                     d["m"][sl], L, od, dt, lam, NH)
        dx = np.abs(gx[:, sl] - ox)
        dx = np.minimum(dx, L - dx)
        assert dx.max() <= 1e-13 * L
        assert rel_l2(gv[:, sl], ov) <= 1e-12
