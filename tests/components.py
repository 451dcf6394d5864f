"""Exact single components of the adjoint from the oracle's forward-mode JVP.

The vector-Jacobian product the library computes has components
(J^T g)_k = <g, J e_k> for a unit input direction e_k (one coordinate of x or
v, or one u or h).  One oracle JVP along e_k gives J e_k exactly (dual
numbers, FP64).  To spend one JVP on many components, particles are picked
whose dependency closures are disjoint: the rates of particle i depend on the
inputs of particles at most three union-neighbor hops away (i's union
neighbors j, the gather neighbors k of j whose volumes enter j's coefficients
and density, and the gather neighbors of k that enter V_k), so a unit tangent
on particle p changes only the outputs in p's three-hop closure.  With
disjoint closures the JVP along the sum of the unit tangents splits exactly:
the part of <g, J t> summed over p's closure is <g, J e_p>.
"""
from __future__ import annotations

import numpy as np

import oracle

KINDS = ("x", "v", "u", "h")


def closure(row, col, p, hops=3):
    s = np.array([p])
    for _ in range(hops):
        nb = np.concatenate([col[row[i]:row[i + 1]] for i in s] + [s])
        s = np.unique(nb)
    return s


def pick(d, per_kind=64, seed=0, hops=3, walk=400):
    """Components to check: per kind (x, v, u, h) ``per_kind`` random (particle,
    axis) picks, grouped into batches of particles with disjoint closures.
    Each batch walks up to ``walk`` unused particles in a fixed random order."""
    n = d["h"].shape[0]
    row, col = oracle.neighbors(d["x"], d["h"], d.get("L", 1.0), mode="union")
    rng = np.random.default_rng(seed)
    order = rng.permutation(n)
    pending = [(kind, int(rng.integers(0, 3)) if kind in ("x", "v") else 0)
               for kind in KINDS for _ in range(per_kind)]
    pending = [pending[k] for k in rng.permutation(len(pending))]
    cache, used, batches = {}, set(), []
    while pending:
        taken = np.zeros(n, dtype=bool)
        batch, seen = [], 0
        for p in order:
            if len(batch) == len(pending) or seen >= walk:
                break
            p = int(p)
            if p in used:
                continue
            seen += 1
            if p not in cache:
                cache[p] = closure(row, col, p, hops)
            c = cache[p]
            if taken[c].any():
                continue
            taken[c] = True
            used.add(p)
            kind, axis = pending[len(batch)]
            batch.append((kind, axis, p, c))
        if not batch:
            raise RuntimeError("no particle with a free closure left")
        batches.append(batch)
        pending = pending[len(batch):]
    return batches


def exact(d, ga, gu, batches, params=None):
    """<g, J e_k> for every pick, one oracle JVP per batch.  Returns a dict kind
    -> list of (particle, axis, value)."""
    n = d["h"].shape[0]
    out = {k: [] for k in KINDS}
    for batch in batches:
        t = {"x": np.zeros((3, n)), "v": np.zeros((3, n)), "u": np.zeros(n), "h": np.zeros(n)}
        for kind, axis, p, _ in batch:
            if kind in ("x", "v"):
                t[kind][axis, p] = 1.0
            else:
                t[kind][p] = 1.0
        _, tan = oracle.jvp(d["x"], d["h"], d["m"], d["v"], d["u"], d.get("L", 1.0),
                            tx=t["x"], tv=t["v"], tu=t["u"], th=t["h"], params=params,
                            want=("dvdt", "dudt"))
        contrib = (ga * tan["dvdt"]).sum(0) + gu * tan["dudt"]
        for kind, axis, p, c in batch:
            out[kind].append((p, axis, float(contrib[c].sum())))
    return out
