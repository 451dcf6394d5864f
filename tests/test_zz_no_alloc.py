"""The workspace-free volume entry point (crk_volume_static).

It serves callers that cannot allocate device memory themselves, e.g. code
running inside a framework that owns the device-memory pool or a host loop
that must not call cudaMalloc/cudaFree (they can synchronise the device).  It
is checked through the C ABI against the volume of the regular path
(crk_cell_build + crk_moments) and against the FP64 oracle on the inputs the
library sees, on two calls in a row with different inputs, within the
tolerances the other GPU tests use; then on the branches of its cell walk (a
cell size far below h, three or fewer cells per axis, a single cell), at its
size limit, with particles outside the box or with an invalid h, and for the
device memory it leaves untouched.  This file is collected last.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_21921_gb300 import synth
from paper_2511_21921_gb300 import _lib as L
from paper_2511_21921_gb300.solver import Solver

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-5}
PREC = {"fp64": L.CRK_FP64, "mixed": L.CRK_MIXED32}
DT = {"fp64": torch.float64, "mixed": torch.float32}


def _dev(d, precision):
    x = torch.tensor(d["x"], dtype=torch.float64, device="cuda")
    h = torch.tensor(d["h"], dtype=DT[precision], device="cuda")
    m = torch.tensor(d["m"], dtype=DT[precision], device="cuda")
    return x, h, m


def _regular_volume(d, precision):
    n = d["h"].shape[0]
    s = Solver(n, 1, precision)
    x, h, m = _dev(d, precision)
    s.cell_build(x, h)
    V, _ = s.moments(m, want_V=True)
    torch.cuda.synchronize()
    assert s.poll() == 0
    return V.double().cpu().numpy()


def _static_volume(d, precision, h_bound=None):
    n = d["h"].shape[0]
    x, h, m = _dev(d, precision)
    V = torch.full((n,), -1.0, dtype=DT[precision], device="cuda")
    hb = float(np.max(d["h"])) if h_bound is None else h_bound
    stream = torch.cuda.current_stream().cuda_stream
    rc = L.crk_volume_static(stream, PREC[precision], n, d["L"], hb, x.data_ptr(), h.data_ptr(),
                             m.data_ptr(), V.data_ptr())
    assert rc == L.CRK_OK, L.crk_status_string(rc)
    torch.cuda.synchronize()
    return V.double().cpu().numpy()


def _oracle_volume(d, precision):
    """The oracle on the values the library receives (float32 h and m in the
    mixed form)."""
    dt = np.float32 if precision == "mixed" else np.float64
    h = d["h"].astype(dt).astype(np.float64)
    m = d["m"].astype(dt).astype(np.float64)
    return oracle.forward(d["x"], h, m, L=d["L"], want=("V",))["V"]


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_static_volume_matches_regular_path_twice(precision):
    cases = [synth.load("lognormal32"), synth.load("lattice16")]
    for d in cases:  # two calls in a row, the second on different particles
        ref = _regular_volume(d, precision)
        got = _static_volume(d, precision)
        assert _rel(got, ref) < TOL[precision], precision
        assert _rel(got, _oracle_volume(d, precision)) < TOL[precision], precision


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("h_bound", [0.01, 0.4, 2.0])
def test_static_volume_any_cell_size(precision, h_bound):
    """h_bound only sets the cell size: far below max h (32 cells per axis, a
    reach of several cells), at or above L/3 (every cell walked) and above L
    (one cell) give the oracle's volume."""
    d = synth.load("lognormal32m")
    got = _static_volume(d, precision, h_bound)
    assert _rel(got, _oracle_volume(d, precision)) < TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_static_volume_at_the_size_limit(precision):
    n = L.CRK_STATIC_MAX_PARTICLES
    rng = np.random.default_rng(17)
    h0 = (3 * 64 / (4 * np.pi * n)) ** (1 / 3)
    d = dict(x=rng.random((3, n)), h=h0 * rng.uniform(0.8, 1.25, n),
             m=np.exp(rng.normal(0, 0.5, n)) / n, L=1.0)
    got = _static_volume(d, precision)
    assert _rel(got, _oracle_volume(d, precision)) < TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_static_volume_invalid_particles(precision):
    """A particle outside [0, L) gets NaN and is left out of every other sum;
    a particle with h >= L/2 gets NaN and still counts for its neighbors."""
    d = dict(synth.load("lattice16m"))
    n = d["h"].shape[0]
    x = d["x"].copy()
    x[0, 0] = 1.25   # outside the box
    x[1, 7] = -0.01  # outside the box
    h = d["h"].copy()
    h[40] = 0.6      # h >= L/2
    bad = np.zeros(n, dtype=bool)
    bad[[0, 7, 40]] = True
    got = _static_volume(dict(d, x=x, h=h), precision, h_bound=float(d["h"].max()))
    assert np.isnan(got[bad]).all() and np.isfinite(got[~bad]).all()
    keep = np.ones(n, dtype=bool)
    keep[[0, 7]] = False
    sub = dict(d, x=x[:, keep], h=d["h"][keep], m=d["m"][keep])  # particle 40's h is its own
    ref = _oracle_volume(sub, precision)
    idx = np.nonzero(keep)[0]
    ok = ~bad[idx]
    assert _rel(got[idx][ok], ref[ok]) < TOL[precision]


def test_static_volume_allocates_nothing():
    """Device memory is the same before and after calls (after the first call
    on the device, which loads the module that holds the scratch array)."""
    d = synth.load("lognormal32")
    n = d["h"].shape[0]
    stream = torch.cuda.current_stream().cuda_stream
    args = []
    for precision in ("mixed", "fp64"):
        x, h, m = _dev(d, precision)
        V = torch.empty(n, dtype=DT[precision], device="cuda")
        args.append((PREC[precision], x, h, m, V))

    def call():
        for prec, x, h, m, V in args:
            rc = L.crk_volume_static(stream, prec, n, d["L"], float(d["h"].max()), x.data_ptr(),
                                     h.data_ptr(), m.data_ptr(), V.data_ptr())
            assert rc == L.CRK_OK
        torch.cuda.synchronize()
    call()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        call()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_static_volume_rejects_too_many_particles():
    n = L.CRK_STATIC_MAX_PARTICLES + 1
    rc = L.crk_volume_static(None, L.CRK_FP64, n, 1.0, 0.1, 1, 1, 1, 1)
    assert rc == L.CRK_ENOMEM
