"""GPU parity of the forward path (cell build, volume, coefficients, density,
velocity gradient, rates) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_21921_gb300 import synth
from paper_2511_21921_gb300 import _lib as L
from paper_2511_21921_gb300.solver import Solver

from gpu_util import TOL, compare, rel_l2, run_forward, to_dev

pytestmark = pytest.mark.gpu


def _oracle_all(d, **kw):
    return oracle.forward(d["x"], d["h"], d["m"], d["v"], d["u"], d.get("L", 1.0),
                          params=oracle.default_params(**kw))


def _multiscale(n=3000, seed=11):
    rng = np.random.default_rng(seed)
    x = rng.random((3, n))
    h = np.exp(rng.uniform(np.log(0.02), np.log(0.2), n))
    return dict(x=x, h=h, m=np.full(n, 1.0 / n), v=rng.normal(0, 0.1, (3, n)),
                u=np.exp(rng.normal(0, 1, n)), L=1.0)


# ------------------------------------------------------------------ neighbors
@pytest.mark.parametrize("case", ["lattice16", "multiscale", "lognormal32"])
@pytest.mark.parametrize("mode", ["gather", "union"])
def test_neighbor_sets_bit_exact_fp64(case, mode):
    d = _multiscale() if case == "multiscale" else synth.load(case)
    n = d["h"].shape[0]
    s = Solver(n, 1, "fp64")
    t = to_dev(d, "fp64")
    s.cell_build(t["x"], t["h"])
    row, col = s.neighbors_csr(mode)
    row, col = row.cpu().numpy(), col.cpu().numpy()
    orow, ocol = oracle.neighbors(d["x"], d["h"], 1.0, mode=mode, method="tree")
    if mode == "gather":  # the library's gather CSR leaves out the particle itself
        keep = ocol != np.repeat(np.arange(n), np.diff(orow))
        ocol = ocol[keep]
        orow = np.concatenate([[0], np.cumsum(np.diff(orow) - 1)])
    assert np.array_equal(row, orow)
    assert np.array_equal(col, ocol)


def _csr_vs_oracle(d, precision, mode):
    """The library's CSR against the oracle's exact predicate on the smoothing
    lengths the library sees (float32 values in the mixed form)."""
    n = d["h"].shape[0]
    s = Solver(n, 1, precision)
    t = to_dev(d, precision)
    s.cell_build(t["x"], t["h"])
    assert s.poll() == 0
    row, col = (a.cpu().numpy() for a in s.neighbors_csr(mode))
    h = t["h"].double().cpu().numpy()
    orow, ocol = oracle.neighbors(d["x"], h, d.get("L", 1.0), mode=mode, method="tree")
    if mode == "gather":
        keep = ocol != np.repeat(np.arange(n), np.diff(orow))
        ocol = ocol[keep]
        orow = np.concatenate([[0], np.cumsum(np.diff(orow) - 1)])
    return row, col, orow, ocol, s


@pytest.mark.parametrize("case", ["lattice16", "multiscale", "lognormal32", "lognormal64"])
@pytest.mark.parametrize("mode", ["gather", "union"])
def test_neighbor_sets_bit_exact_mixed(case, mode):
    """Mixed form: the float candidate test with the exact re-decision inside
    its rounding band gives the FP64 lists of the same inputs, element for
    element (the 64^3 box is the benchmark's)."""
    d = _multiscale() if case == "multiscale" else synth.load(case)
    row, col, orow, ocol, s = _csr_vs_oracle(d, "mixed", mode)
    assert np.array_equal(row, orow)
    assert np.array_equal(col, ocol)
    if mode == "gather":
        assert s.stats()["gather_pairs"] == len(ocol)


def _dyadic_lattice(n_side, h_pair):
    """Particles at (i + 1/2)/n_side: every separation, r^2 and h^2 below is a
    dyadic rational, exact in float and double, so pairs at r = h tie exactly
    and separations of n_side/2 spacings sit exactly at L/2."""
    g = np.stack(np.meshgrid(*(np.arange(n_side),) * 3, indexing="ij")).reshape(3, -1)
    x = (g + 0.5) / n_side
    N = n_side ** 3
    h = np.where(g.sum(0) % 2 == 0, h_pair[0], h_pair[1]) / n_side
    rng = np.random.default_rng(5)
    return dict(x=x, h=h, m=np.full(N, 1.0 / N), v=rng.normal(0, 0.1, (3, N)),
                u=np.ones(N), L=1.0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", [(16, (2.0, 3.0)), (8, (3.0, 2.0))])
def test_exact_ties_at_the_support_edge(precision, shape):
    """r = h exactly is outside (strict r < h), on both sides of every pair;
    separations of exactly L/2 never enter.  16^3 with h = 2 and 3 spacings
    uses the nearest-image staging of the list build; 8^3 with h up to 3/8 of
    the box takes the general path.  Both forms equal the oracle and the
    count of lattice offsets inside the support."""
    n_side, hp = shape
    d = _dyadic_lattice(n_side, hp)
    for mode in ("gather", "union"):
        row, col, orow, ocol, _ = _csr_vs_oracle(d, precision, mode)
        assert np.array_equal(row, orow) and np.array_equal(col, ocol), mode
    # lattice offsets with |o|^2 < (h n)^2 (strict), excluding the origin
    o = np.arange(-(n_side // 2) + 1, n_side // 2)
    oo = (o[:, None, None] ** 2 + o[None, :, None] ** 2 + o[None, None, :] ** 2).ravel()
    row, _, _, _, _ = _csr_vs_oracle(d, precision, "gather")
    cnt = np.diff(row)
    even = (np.stack(np.meshgrid(*(np.arange(n_side),) * 3, indexing="ij")).reshape(3, -1)
            .sum(0) % 2 == 0)
    assert (cnt[even] == ((oo > 0) & (oo < hp[0] ** 2)).sum()).all()
    assert (cnt[~even] == ((oo > 0) & (oo < hp[1] ** 2)).sum()).all()


# ------------------------------------------------------------------ forward parity
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["lattice16", "lognormal32", "lattice16m", "lognormal32m"])
def test_forward_parity_whole_box(case, precision):
    """Every output of the forward path on whole boxes, equal masses and masses
    spread over 33x (the ``m`` workloads)."""
    d = synth.load(case)
    gpu, s = run_forward(d, precision)
    assert gpu["status"] == 0
    ora = _oracle_all(d)
    err = compare(gpu, ora)
    tol = TOL[precision]
    for k in ("dvdt", "dudt"):
        assert err[k] < tol, (k, err)
    bar = tol if precision == "fp64" else 5e-5
    for k, e in err.items():
        assert e < bar, (k, err)
    st = gpu["stats"]
    h = d["h"].astype(np.float32).astype(np.float64) if precision == "mixed" else d["h"]
    assert st["gather_pairs"] == int(ora_pairs(dict(d, h=h)))


def ora_pairs(d):
    o = oracle.forward(d["x"], d["h"], d["m"], L=d.get("L", 1.0), want=("kgather",))
    return o["kgather"].sum()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_relaxation_partial_flags(precision):
    d = synth.load("lognormal32")
    o0 = oracle.forward(d["x"], d["h"], d["m"], d["v"], d["u"], 1.0, want=("gradv",))
    div = np.sort(np.abs(o0["gradv"][0] + o0["gradv"][4] + o0["gradv"][8]))
    # threshold in the middle of the widest gap near the 80th percentile, so the
    # float and double evaluations of |div| take the same decision
    k0 = int(0.8 * div.size)
    seg = div[k0 - 200:k0 + 200]
    g = np.argmax(np.diff(seg))
    thr = 0.5 * (seg[g] + seg[g + 1])
    dt = np.log(8.0) / thr
    gpu, _ = run_forward(d, precision, relax_dt=dt)
    ora = _oracle_all(d, relax_dt=dt)
    assert 0.1 < ora["flag"].mean() < 0.3
    err = compare(gpu, ora)
    for k in ("dvdt", "dudt"):
        assert err[k] < TOL[precision], (k, err)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["lognormal32", "lognormal32m"])
def test_conservation(precision, case):
    d = synth.load(case)
    gpu, _ = run_forward(d, precision)
    m, v, a, du = d["m"], d["v"], gpu["dvdt"], gpu["dudt"]
    p = np.abs((m * a).sum(1)).max() / np.abs(m * a).sum()
    e = abs((m * (v * a).sum(0)).sum() + (m * du).sum()) / (
        np.abs(m * (v * a).sum(0)).sum() + np.abs(m * du).sum())
    bar = 1e-13 if precision == "fp64" else 1e-6
    assert p < bar and e < bar, (p, e)


# ------------------------------------------------------------------ full size, sampled
@pytest.mark.parametrize("case", ["lognormal64", "lognormal64m"])
def test_full_size_lognormal64_sampled_mixed(case):
    """The 64^3 clustered workload (lognormal, 100 +- 10 neighbors; equal and
    unequal masses) in the mixed form, on outputs the oracle computes one by
    one."""
    d = synth.load(case)
    gpu, s = run_forward(d, "mixed")
    assert gpu["status"] == 0
    rng = np.random.default_rng(123)
    tg = np.sort(rng.choice(d["h"].shape[0], 160, replace=False))
    ora = oracle.forward(d["x"], d["h"], d["m"], d["v"], d["u"], 1.0, targets=tg)
    err = compare(gpu, ora, idx=tg)
    for k in ("dvdt", "dudt"):
        assert err[k] < TOL["mixed"], (k, err)
    for k, e in err.items():
        assert e < 5e-5, (k, err)


@pytest.mark.parametrize("case", ["lognormal64", "lognormal64m"])
def test_full_size_lognormal64_sampled_fp64(case):
    d = synth.load(case)
    gpu, s = run_forward(d, "fp64")
    rng = np.random.default_rng(321)
    tg = np.sort(rng.choice(d["h"].shape[0], 64, replace=False))
    ora = oracle.forward(d["x"], d["h"], d["m"], d["v"], d["u"], 1.0, targets=tg)
    err = compare(gpu, ora, idx=tg)
    for k, e in err.items():
        assert e < TOL["fp64"], (k, err)


# ------------------------------------------------------------------ multi-box
def test_multibox_matches_per_box_oracle():
    d = synth.multibox(n_boxes=6, seed0=300, nmin=8, nmax=18)
    gpu, s = run_forward(d, "fp64")
    assert gpu["status"] == 0
    off = d["box_off"]
    for b in range(len(off) - 1):
        sl = slice(off[b], off[b + 1])
        db = {k: d[k][..., sl] for k in ("x", "v", "u", "h", "m")}
        ora = oracle.forward(db["x"], db["h"], db["m"], db["v"], db["u"], 1.0)
        gb = {k: (v[..., sl] if isinstance(v, np.ndarray) else v) for k, v in gpu.items()}
        err = compare(gb, ora)
        for k, e in err.items():
            assert e < TOL["fp64"], (b, k, err)


# ------------------------------------------------------------------ edge cases
def test_ragged_sizes_and_partial_warps():
    rng = np.random.default_rng(5)
    for n in (37, 200, 1001):
        hval = (3 * 40 / (4 * np.pi * n)) ** (1 / 3)
        hval = min(hval, 0.45)
        d = dict(x=rng.random((3, n)), h=np.full(n, hval) * rng.uniform(0.9, 1.1, n),
                 m=rng.uniform(0.5, 1.5, n) / n, v=rng.normal(0, 0.1, (3, n)),
                 u=np.exp(rng.normal(0, 0.5, n)), L=1.0)
        gpu, _ = run_forward(d, "fp64")
        ora = _oracle_all(d)
        err = compare(gpu, ora)
        for k, e in err.items():
            assert e < 1e-11, (n, k, err)


def test_empty_box_in_batch():
    d = synth.multibox(n_boxes=3, seed0=400, nmin=8, nmax=10)
    off = d["box_off"]
    # insert an empty box between the first and the second
    d["box_off"] = np.array([0, off[1], off[1], off[2], off[3]], dtype=np.int64)
    d["box_L"] = np.ones(4)
    gpu, _ = run_forward(d, "fp64")
    assert gpu["status"] == 0
    sl = slice(off[1], off[2])
    ora = oracle.forward(d["x"][:, sl], d["h"][sl], d["m"][sl], d["v"][:, sl], d["u"][sl], 1.0)
    assert rel_l2(gpu["dvdt"][:, sl], ora["dvdt"]) < 1e-12


def test_isolated_particles_are_singular():
    d = dict(x=np.array([[0.1, 0.6], [0.2, 0.6], [0.3, 0.6]]), h=np.array([0.05, 0.05]),
             m=np.ones(2), v=np.zeros((3, 2)), u=np.ones(2), L=1.0)
    gpu, _ = run_forward(d, "fp64")
    assert gpu["status"] == L.CRK_ESINGULAR
    assert np.all(gpu["coef"][0] == 1) and np.all(gpu["coef"][1:] == 0)
    assert np.all(gpu["dvdt"] == 0)


@pytest.mark.parametrize("bad", ["x_eq_L", "x_neg", "h_half", "nan_x", "nan_h"])
def test_domain_errors_reported_on_device(bad):
    rng = np.random.default_rng(1)
    n = 64
    x = rng.random((3, n))
    h = np.full(n, 0.2)
    code = L.CRK_EDOMAIN
    if bad == "x_eq_L":
        x[0, 5] = 1.0
    elif bad == "x_neg":
        x[2, 7] = -1e-9
    elif bad == "h_half":
        h[3] = 0.5
    elif bad == "nan_x":
        x[1, 2] = np.nan
        code = L.CRK_ENONFINITE
    else:
        h[9] = np.nan
        code = L.CRK_ENONFINITE
    s = Solver(n, 1, "fp64")
    t = to_dev(dict(x=x, h=h, m=np.ones(n), v=np.zeros((3, n)), u=np.ones(n)), "fp64")
    with pytest.raises(L.CRKError) as ei:
        s.cell_build(t["x"], t["h"])
    assert ei.value.code == code


def test_zero_particles():
    s = Solver(0, 1, "mixed")
    x = torch.zeros((3, 0), dtype=torch.float64, device="cuda")
    h = torch.zeros(0, dtype=torch.float32, device="cuda")
    s.cell_build(x, h)
    s.moments(torch.zeros(0, dtype=torch.float32, device="cuda"))
    dv, du, _, _ = s.rates(torch.zeros((3, 0), dtype=torch.float32, device="cuda"),
                           torch.zeros(0, dtype=torch.float32, device="cuda"))
    assert dv.shape == (3, 0) and s.poll() == 0


def test_call_order_enforced():
    s = Solver(100, 1, "mixed")
    rc = L.crk_rates(s.plan, None, 256, 0, 0, 0, 0)
    assert rc == L.CRK_ESTATE


def test_list_capacity_overflow_regrows():
    """A neighbor-list column too small for the longest list is reported on the
    device (CRK_ENOMEM) and the Solver rebuilds with enough slots."""
    d = synth.load("lognormal32")
    n = d["h"].shape[0]
    s = Solver(n, 1, "fp64", nbr_cap=24)
    t = to_dev(d, "fp64")
    s.cell_build(t["x"], t["h"], check=False)
    assert s.poll() == L.CRK_ENOMEM
    gpu, _ = run_forward(d, "fp64", solver=s)
    assert s.params.nbr_cap > 24
    ora = _oracle_all(d)
    err = compare(gpu, ora)
    assert err["dvdt"] < 1e-12 and err["dudt"] < 1e-12, err


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_clumpy_multiscale_parity(precision):
    """Plummer clumps on a lognormal background (smoothing lengths spanning
    about two decades): union sets differ strongly from gather sets."""
    d = synth.clumpy(n_side=32, n_clumps=12, seed=31, nc_min=300, nc_max=1500)
    gpu, s = run_forward(d, precision)
    assert gpu["status"] == 0
    ora = _oracle_all(d)
    err = compare(gpu, ora)
    tol = TOL[precision]
    for k in ("dvdt", "dudt"):
        assert err[k] < tol, (k, err)
    assert d["h"].max() / d["h"].min() > 20


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_replay_equals_eager(precision):
    """The whole step (build, moments, rates, adjoint) captured in one CUDA
    graph gives bit-identical results to eager calls."""
    d = synth.load("lognormal32")
    n = d["h"].shape[0]
    t = to_dev(d, precision)
    ga, gu = synth.cotangents(n, seed=4)
    gat = torch.tensor(ga, dtype=t["h"].dtype, device="cuda")
    gut = torch.tensor(gu, dtype=t["h"].dtype, device="cuda")
    s = Solver(n, 1, precision)
    s.cell_build(t["x"], t["h"])  # sizes the workspace and lists
    outs = (torch.empty((3, n), dtype=t["h"].dtype, device="cuda"),
            torch.empty(n, dtype=t["h"].dtype, device="cuda"))
    grads = tuple(torch.empty(sh, dtype=t["h"].dtype, device="cuda")
                  for sh in ((3, n), (3, n), (n,), (n,)))

    def step():
        s.cell_build(t["x"], t["h"], check=False)
        s.moments(t["m"])
        s.rates(t["v"], t["u"], out=outs)
        s.adjoint(t["v"], t["u"], gat, gut, recompute=False, out=grads)

    step()
    torch.cuda.synchronize()
    eager = [a.clone() for a in outs + grads]
    g = s.capture(step)
    for a in outs + grads:
        a.zero_()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert s.poll() == 0
    for a, b in zip(eager, outs + grads):
        assert torch.equal(a, b)


# ------------------------------------------------------------------ formulation variants
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("mode", [dict(energy_split=1), dict(q_side=1),
                                  dict(energy_split=1, q_side=1)])
def test_formulation_variants_parity_and_conservation(precision, mode):
    """Energy split weighted by the specific energies and per-side viscosity
    (Sec. 2.1, the cited formulation's variants): rates against the oracle in
    the same mode, and momentum and energy conserved, with unequal masses."""
    d = synth.load("lognormal32m")
    gpu, _ = run_forward(d, precision, **mode)
    assert gpu["status"] == 0
    ora = _oracle_all(d, **mode)
    err = compare(gpu, ora, keys=("dvdt", "dudt"), coef=False)
    for k, e in err.items():
        assert e < TOL[precision], (mode, k, err)
    m, v, a, du = d["m"], d["v"], gpu["dvdt"], gpu["dudt"]
    p = np.abs((m * a).sum(1)).max() / np.abs(m * a).sum()
    e = abs((m * (v * a).sum(0)).sum() + (m * du).sum()) / (
        np.abs(m * (v * a).sum(0)).sum() + np.abs(m * du).sum())
    assert p < (1e-13 if precision == "fp64" else 1e-6), p
    assert e < (1e-13 if precision == "fp64" else 1e-6), e
