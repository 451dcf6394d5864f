"""GPU adjoint (vector-Jacobian product) of the rates, through the C ABI.

Checked three independent ways: the dot-product test <g, J d> = <J^T g, d>
with J d from the oracle's dual-number JVP; central finite differences (step
1e-6, FP64) of the GPU forward; and single gradient components from unit
JVPs of the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_21921_gb300 import _lib as L
from paper_2511_21921_gb300 import synth
from paper_2511_21921_gb300.solver import Solver, rates

from gpu_util import to_dev

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 2e-4}


def _box(n_side=16, seed=7):
    return synth.lognormal(n_side, 1.5, seed=seed)


def _gpu_adjoint(d, precision, ga, gu, recompute=False, **params):
    n = d["h"].shape[0]
    s = Solver(n, 1, precision, **params)
    t = to_dev(d, precision)
    s.cell_build(t["x"], t["h"])
    s.moments(t["m"])
    dv, du, _, _ = s.rates(t["v"], t["u"])
    dt = t["h"].dtype
    g = s.adjoint(t["v"], t["u"], torch.tensor(ga, dtype=dt, device="cuda"),
                  torch.tensor(gu, dtype=dt, device="cuda"), recompute=recompute)
    torch.cuda.synchronize()
    assert s.poll() == 0
    return [a.double().cpu().numpy() for a in g], (dv.double().cpu().numpy(),
                                                    du.double().cpu().numpy()), s


def _directions(d, rng, which):
    n = d["h"].shape[0]
    dx = rng.normal(size=(3, n)) if which in ("x", "all") else np.zeros((3, n))
    dv = rng.normal(size=(3, n)) if which in ("v", "all") else np.zeros((3, n))
    du = rng.normal(size=n) * d["u"] if which in ("u", "all") else np.zeros(n)
    dh = rng.normal(size=n) * d["h"] if which in ("h", "all") else np.zeros(n)
    return dx, dv, du, dh


def _pairing(grads, dirs):
    terms = [grads[0] * dirs[0], grads[1] * dirs[1], grads[2] * dirs[2], grads[3] * dirs[3]]
    return sum(t.sum() for t in terms), sum(np.abs(t).sum() for t in terms)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("which", ["x", "v", "u", "h", "all"])
def test_dot_product_against_oracle_jvp(precision, which):
    d = _box()
    n = d["h"].shape[0]
    ga, gu = synth.cotangents(n, seed=4)
    grads, _, _ = _gpu_adjoint(d, precision, ga, gu)
    rng = np.random.default_rng(11)
    dirs = _directions(d, rng, which)
    _, tan = oracle.jvp(d["x"], d["h"], d["m"], d["v"], d["u"], d["L"], tx=dirs[0], tv=dirs[1],
                        tu=dirs[2], th=dirs[3], want=("dvdt", "dudt"))
    lhs = (ga * tan["dvdt"]).sum() + (gu * tan["dudt"]).sum()
    rhs, scale = _pairing(grads, dirs)
    assert abs(lhs - rhs) <= TOL[precision] * scale, (which, lhs, rhs, scale)


def test_dot_product_with_relaxation_and_limiter_off():
    d = _box(seed=9)
    n = d["h"].shape[0]
    o0 = oracle.forward(d["x"], d["h"], d["m"], d["v"], d["u"], 1.0, want=("gradv",))
    div = np.sort(np.abs(o0["gradv"][0] + o0["gradv"][4] + o0["gradv"][8]))
    k0 = int(0.7 * n)
    g = np.argmax(np.diff(div[k0 - 100:k0 + 100]))
    dt = np.log(8.0) / (0.5 * (div[k0 - 100 + g] + div[k0 - 99 + g]))
    ga, gu = synth.cotangents(n, seed=5)
    for kw in ({"relax_dt": dt}, {"limiter": 0}):
        grads, _, _ = _gpu_adjoint(d, "fp64", ga, gu, **kw)
        dirs = _directions(d, np.random.default_rng(2), "all")
        _, tan = oracle.jvp(d["x"], d["h"], d["m"], d["v"], d["u"], 1.0, tx=dirs[0], tv=dirs[1],
                            tu=dirs[2], th=dirs[3], params=oracle.default_params(**kw))
        lhs = (ga * tan["dvdt"]).sum() + (gu * tan["dudt"]).sum()
        rhs, scale = _pairing(grads, dirs)
        assert abs(lhs - rhs) <= 1e-10 * scale, (kw, lhs, rhs)


def test_central_differences_of_gpu_forward_fp64():
    """FD of L = <g, rates> along random directions, step 1e-6, FP64, GPU only,
    on the 32^3 lognormal box."""
    d = synth.load("lognormal32")
    n = d["h"].shape[0]
    ga, gu = synth.cotangents(n, seed=6)
    grads, _, _ = _gpu_adjoint(d, "fp64", ga, gu)
    rng = np.random.default_rng(3)
    sp = n ** (-1.0 / 3.0)
    s = Solver(n, 1, "fp64")

    def L_of(dd):
        t = to_dev(dd, "fp64")
        out = s.forward(t["x"], t["h"], t["m"], t["v"], t["u"])
        return float((torch.tensor(ga, device="cuda") * out["dvdt"]).sum() +
                     (torch.tensor(gu, device="cuda") * out["dudt"]).sum())

    for k in range(6):
        dx, dv, du, dh = _directions(d, rng, "all")
        dx *= 0.01 * sp
        dv *= 0.01
        eps = 1e-6
        vals = []
        for sg in (1, -1):
            dd = dict(d)
            dd["x"] = np.mod(d["x"] + sg * eps * dx, 1.0)
            dd["v"] = d["v"] + sg * eps * dv
            dd["u"] = d["u"] + sg * eps * du
            dd["h"] = d["h"] + sg * eps * dh
            vals.append(L_of(dd))
        fd = (vals[0] - vals[1]) / (2 * eps)
        rhs, scale = _pairing(grads, (dx, dv, du, dh))
        assert abs(fd - rhs) <= 1e-6 * scale, (k, fd, rhs, scale)


def test_gradient_components_from_unit_jvps():
    d = _box(n_side=12, seed=21)
    n = d["h"].shape[0]
    ga, gu = synth.cotangents(n, seed=8)
    grads, _, _ = _gpu_adjoint(d, "fp64", ga, gu)
    rng = np.random.default_rng(4)
    for _ in range(24):
        kind = rng.integers(4)
        i = int(rng.integers(n))
        comp = int(rng.integers(3))
        dirs = [np.zeros((3, n)), np.zeros((3, n)), np.zeros(n), np.zeros(n)]
        if kind < 2:
            dirs[kind][comp, i] = 1.0
            g = grads[kind][comp, i]
        else:
            dirs[kind][i] = 1.0
            g = grads[kind][i]
        _, tan = oracle.jvp(d["x"], d["h"], d["m"], d["v"], d["u"], 1.0, tx=dirs[0], tv=dirs[1],
                            tu=dirs[2], th=dirs[3])
        ref = (ga * tan["dvdt"]).sum() + (gu * tan["dudt"]).sum()
        scale = np.abs(grads[kind]).max()
        assert abs(g - ref) <= 1e-10 * scale, (kind, i, comp, g, ref)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_recompute_equals_reuse(precision):
    d = _box(seed=17)
    n = d["h"].shape[0]
    ga, gu = synth.cotangents(n, seed=9)
    g0, _, _ = _gpu_adjoint(d, precision, ga, gu, recompute=False)
    g1, _, _ = _gpu_adjoint(d, precision, ga, gu, recompute=True)
    for a, b in zip(g0, g1):
        assert np.array_equal(a, b)


def test_autograd_function_matches_direct_adjoint():
    d = _box(seed=19)
    n = d["h"].shape[0]
    t = to_dev(d, "mixed")
    s = Solver(n, 1, "mixed")
    x = t["x"].clone().requires_grad_(True)
    v = t["v"].clone().requires_grad_(True)
    u = t["u"].clone().requires_grad_(True)
    h = t["h"].clone().requires_grad_(True)
    dvdt, dudt = rates(x, v, u, h, t["m"], s)
    ga, gu = synth.cotangents(n, seed=10)
    gat = torch.tensor(ga, dtype=torch.float32, device="cuda")
    gut = torch.tensor(gu, dtype=torch.float32, device="cuda")
    ((gat * dvdt).sum() + (gut * dudt).sum()).backward()
    grads, _, _ = _gpu_adjoint(d, "mixed", ga, gu)
    for a, b in zip((x.grad, v.grad, u.grad, h.grad), grads):
        a = a.double().cpu().numpy()
        assert np.allclose(a, b, rtol=1e-5, atol=1e-5 * np.abs(b).max())


def test_full_size_adjoint_dot_mixed():
    """The benchmark's workload and launch configuration, mixed form."""
    d = synth.load("lognormal64")
    n = d["h"].shape[0]
    ga, gu = synth.cotangents(n, seed=4)
    grads, _, _ = _gpu_adjoint(d, "mixed", ga, gu)
    rng = np.random.default_rng(12)
    dirs = _directions(d, rng, "all")
    _, tan = oracle.jvp(d["x"], d["h"], d["m"], d["v"], d["u"], 1.0, tx=dirs[0], tv=dirs[1],
                        tu=dirs[2], th=dirs[3])
    lhs = (ga * tan["dvdt"]).sum() + (gu * tan["dudt"]).sum()
    rhs, scale = _pairing(grads, dirs)
    assert abs(lhs - rhs) <= TOL["mixed"] * scale, (lhs, rhs, scale)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_autotune_choices_keep_results(precision):
    """The autotuner only changes launch shapes (register caps); the compiler may
    then contract different products into FMAs, so results agree to rounding."""
    d = _box(seed=23)
    n = d["h"].shape[0]
    ga, gu = synth.cotangents(n, seed=11)
    g0, (dv0, du0), s = _gpu_adjoint(d, precision, ga, gu)
    t = to_dev(d, precision)
    dt = t["h"].dtype
    gat = torch.tensor(ga, dtype=dt, device="cuda")
    gut = torch.tensor(gu, dtype=dt, device="cuda")
    tuned = s.autotune(t["m"], t["v"], t["u"], gat, gut, repeats=2)
    assert set(tuned) == {"b1_volume", "b2_moments", "c1_density", "c2_rates", "adj_c2",
                          "adj_c1", "adj_b2", "adj_b1"}
    assert all(v["variant"] in range(L.CRK_TUNE_VARIANTS) and min(v["ms"]) > 0
               for v in tuned.values())
    dv1, du1, _, _ = s.rates(t["v"], t["u"])
    g1 = s.adjoint(t["v"], t["u"], gat, gut, recompute=False)
    torch.cuda.synchronize()
    tol = 1e-13 if precision == "fp64" else 1e-6

    def rel(a, b):
        return np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(dv1.double().cpu().numpy(), dv0) < tol
    assert rel(du1.double().cpu().numpy(), du0) < tol
    for a, b in zip(g1, g0):
        assert rel(a.double().cpu().numpy(), b) < tol


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fused_rates_adjoint_matches_separate_calls(precision):
    """crk_rates_adjoint (the adjoint's pair sweep also forms the rates) gives
    the rates of crk_rates and the gradients of crk_adjoint, to rounding."""
    d = _box(seed=29)
    n = d["h"].shape[0]
    ga, gu = synth.cotangents(n, seed=12)
    grads, (dv0, du0), s = _gpu_adjoint(d, precision, ga, gu)
    t = to_dev(d, precision)
    dt = t["h"].dtype
    s.cell_build(t["x"], t["h"])
    s.moments(t["m"])
    out = s.rates_adjoint(t["v"], t["u"], torch.tensor(ga, dtype=dt, device="cuda"),
                          torch.tensor(gu, dtype=dt, device="cuda"))
    torch.cuda.synchronize()
    assert s.poll() == 0
    tol = 1e-13 if precision == "fp64" else 1e-6

    def rel(a, b):
        return np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(out[0].double().cpu().numpy(), dv0) < tol
    assert rel(out[1].double().cpu().numpy(), du0) < tol
    for a, b in zip(out[2:], grads):
        assert rel(a.double().cpu().numpy(), b) < tol

@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("mode", [dict(energy_split=1), dict(q_side=1),
                                  dict(energy_split=1, q_side=1)])
def test_dot_product_formulation_variants(precision, mode):
    """The adjoint of the variant rates (per-side viscosity, energy split with
    its dependence on u) against the oracle's JVP in the same mode."""
    d = synth.unequal_masses(_box(), seed=8)
    n = d["h"].shape[0]
    ga, gu = synth.cotangents(n, seed=4)
    grads, _, _ = _gpu_adjoint(d, precision, ga, gu, **mode)
    rng = np.random.default_rng(13)
    dirs = _directions(d, rng, "all")
    _, tan = oracle.jvp(d["x"], d["h"], d["m"], d["v"], d["u"], d["L"], tx=dirs[0], tv=dirs[1],
                        tu=dirs[2], th=dirs[3], params=oracle.default_params(**mode),
                        want=("dvdt", "dudt"))
    lhs = (ga * tan["dvdt"]).sum() + (gu * tan["dudt"]).sum()
    rhs, scale = _pairing(grads, dirs)
    assert abs(lhs - rhs) <= TOL[precision] * scale, (mode, lhs, rhs, scale)
    # the u direction alone exercises the split's dependence on u
    dirs = _directions(d, rng, "u")
    _, tan = oracle.jvp(d["x"], d["h"], d["m"], d["v"], d["u"], d["L"], tu=dirs[2],
                        params=oracle.default_params(**mode), want=("dvdt", "dudt"))
    lhs = (ga * tan["dvdt"]).sum() + (gu * tan["dudt"]).sum()
    rhs, scale = _pairing(grads, dirs)
    assert abs(lhs - rhs) <= TOL[precision] * scale, (mode, lhs, rhs, scale)
