"""The workspace-free volume entry point (crk_volume_static).

It serves callers that cannot allocate device memory themselves, e.g. code
running inside a framework that owns the device-memory pool or a host loop
that must not call cudaMalloc/cudaFree (they can synchronise the device).  It
is checked through the C ABI against the volume of the regular path
(crk_cell_build + crk_moments), on two calls in a row with different inputs,
within the tolerances the other GPU tests use.  This file is collected last.
"""
import numpy as np
import pytest
import torch

from paper_2511_21921_gb300 import synth
from paper_2511_21921_gb300 import _lib as L
from paper_2511_21921_gb300.solver import Solver

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-5}
PREC = {"fp64": L.CRK_FP64, "mixed": L.CRK_MIXED32}
DT = {"fp64": torch.float64, "mixed": torch.float32}


def _regular_volume(d, precision):
    n = d["h"].shape[0]
    s = Solver(n, 1, precision)
    x = torch.tensor(d["x"], dtype=torch.float64, device="cuda")
    h = torch.tensor(d["h"], dtype=DT[precision], device="cuda")
    m = torch.tensor(d["m"], dtype=DT[precision], device="cuda")
    s.cell_build(x, h)
    V, _ = s.moments(m, want_V=True)
    torch.cuda.synchronize()
    assert s.poll() == 0
    return V.double().cpu().numpy()


def _static_volume(d, precision):
    n = d["h"].shape[0]
    x = torch.tensor(d["x"], dtype=torch.float64, device="cuda")
    h = torch.tensor(d["h"], dtype=DT[precision], device="cuda")
    m = torch.tensor(d["m"], dtype=DT[precision], device="cuda")
    V = torch.full((n,), -1.0, dtype=DT[precision], device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = L.crk_volume_static(stream, PREC[precision], n, d["L"], float(d["h"].max()),
                             x.data_ptr(), h.data_ptr(), m.data_ptr(), V.data_ptr())
    assert rc == L.CRK_OK, L.crk_status_string(rc)
    torch.cuda.synchronize()
    return V.double().cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_static_volume_matches_regular_path_twice(precision):
    cases = [synth.load("lognormal32"), synth.load("lattice16")]
    for d in cases:  # two calls in a row, the second on different particles
        ref = _regular_volume(d, precision)
        got = _static_volume(d, precision)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < TOL[precision], (precision, err)


def test_static_volume_rejects_too_many_particles():
    n = L.CRK_STATIC_MAX_PARTICLES + 1
    rc = L.crk_volume_static(None, L.CRK_FP64, n, 1.0, 0.1, 1, 1, 1, 1)
    assert rc == L.CRK_ENOMEM
