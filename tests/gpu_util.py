"""Helpers shared by the GPU tests: run the CUDA path through the C ABI and
compare with the oracle."""
import numpy as np
import torch

from paper_2511_21921_gb300.solver import Solver

DT = {"fp64": torch.float64, "mixed": torch.float32}
# bars: relative L2 per output (the rates' bars are the contract; the
# intermediate fields are reported with the same bar where they are smooth)
TOL = {"fp64": 1e-12, "mixed": 1e-5}


def to_dev(d, precision, device="cuda"):
    dt = DT[precision]
    t = {}
    t["x"] = torch.tensor(np.ascontiguousarray(d["x"]), dtype=torch.float64, device=device)
    for k in ("h", "m", "u"):
        t[k] = torch.tensor(np.ascontiguousarray(d[k]), dtype=dt, device=device)
    t["v"] = torch.tensor(np.ascontiguousarray(d["v"]), dtype=dt, device=device)
    if "box_off" in d:
        t["box_off"] = torch.tensor(d["box_off"], dtype=torch.int64, device=device)
        t["box_L"] = torch.tensor(d["box_L"], dtype=torch.float64, device=device)
    return t


def run_forward(d, precision, solver=None, **params):
    n = d["h"].shape[0]
    nb = len(d["box_off"]) - 1 if "box_off" in d else 1
    s = solver or Solver(max(n, 1), nb, precision, **params)
    t = to_dev(d, precision)
    out = s.forward(t["x"], t["h"], t["m"], t["v"], t["u"], t.get("box_off"), t.get("box_L"),
                    L_box=d.get("L", 1.0), want_V=True, want_coef=True, want_rho=True,
                    want_gradv=True)
    torch.cuda.synchronize()
    res = {k: v.double().cpu().numpy() for k, v in out.items() if v is not None}
    res["stats"] = s.stats()
    res["status"] = s.poll()
    return res, s


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


COEF_GROUPS = {"A": slice(0, 1), "B": slice(1, 4), "gradA": slice(4, 7), "gradB": slice(7, 16)}


def compare(gpu, ora, keys=("V", "rho", "gradv", "dvdt", "dudt"), coef=True, idx=None):
    """Per-output relative L2 errors (optionally on a subset of particles)."""
    err = {}
    for k in keys:
        g = gpu[k] if idx is None else gpu[k][..., idx]
        err[k] = rel_l2(g, ora[k])
    if coef:
        for name, sl in COEF_GROUPS.items():
            g = gpu["coef"][sl] if idx is None else gpu["coef"][sl][:, idx]
            err["coef." + name] = rel_l2(g, ora["coef"][sl])
    return err
