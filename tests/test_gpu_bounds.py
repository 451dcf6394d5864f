"""The bounds-checked build (every neighbor index, work-list entry and tree
node checked before it is followed; CRK_EBOUNDS on a bad one) runs the whole
path clean and agrees with the regular build."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from paper_2511_21921_gb300 import synth
from paper_2511_21921_gb300.solver import Solver

from gpu_util import to_dev

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys, json, numpy as np, torch
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[1] + "/tests")
from paper_2511_21921_gb300 import _lib as L, synth
from paper_2511_21921_gb300.solver import Solver
from gpu_util import to_dev
assert L.load()._name.endswith("libcrk_bc.so")
out = {}
for prec in ("fp64", "mixed"):
    d = synth.load("lognormal32"); n = d["h"].shape[0]; t = to_dev(d, prec)
    s = Solver(n, 1, prec)
    r = s.forward(t["x"], t["h"], t["m"], t["v"], t["u"])
    ga, gu = synth.cotangents(n, seed=4)
    g = s.adjoint(t["v"], t["u"], torch.tensor(ga, dtype=t["h"].dtype, device="cuda"),
                  torch.tensor(gu, dtype=t["h"].dtype, device="cuda"), recompute=False)
    torch.cuda.synchronize()
    out[prec] = {"status": s.poll(), "dvdt": r["dvdt"].double().cpu().numpy().tolist(),
                 "gx": g[0].double().cpu().numpy().tolist()}
json.dump(out, open(sys.argv[2], "w"))
"""


def test_bounds_checked_build_runs_clean(tmp_path):
    path = tmp_path / "bc.json"
    env = dict(os.environ, CRK_BOUNDS_CHECK="1")
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT, str(path)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    bc = json.load(open(path))
    for prec, tol in (("fp64", 1e-13), ("mixed", 1e-6)):
        assert bc[prec]["status"] == 0
        d = synth.load("lognormal32")
        n = d["h"].shape[0]
        t = to_dev(d, prec)
        s = Solver(n, 1, prec)
        out = s.forward(t["x"], t["h"], t["m"], t["v"], t["u"])
        ga, gu = synth.cotangents(n, seed=4)
        g = s.adjoint(t["v"], t["u"], torch.tensor(ga, dtype=t["h"].dtype, device="cuda"),
                      torch.tensor(gu, dtype=t["h"].dtype, device="cuda"), recompute=False)
        for a, b in ((out["dvdt"], bc[prec]["dvdt"]), (g[0], bc[prec]["gx"])):
            a = a.double().cpu().numpy()
            b = np.asarray(b)
            assert np.linalg.norm(a - b) <= tol * np.linalg.norm(a)
