"""Host-side logic for running independent boxes on several GPUs.

Boxes are independent problems, so N ranks need no data-path collective: each
rank takes a set of whole boxes (balanced by particle count) and runs them in
one batched call; a single-box workload is replicated (weak scaling).  The only
collective is the max over ranks of the step time.

``overload_slabs`` is the paper's "overloading" decomposition of one box (Sec.
2.1: particles near a domain boundary are duplicated in the adjacent domain, so
each domain evaluates its own particles without communication): slabs of the
box along one axis, each with the ghost particles its owned particles' rates
depend on.
"""
from __future__ import annotations

import heapq

import numpy as np


def partition_boxes(sizes, world: int) -> list[list[int]]:
    """Assign box indices to ``world`` ranks, largest first to the least loaded
    rank (deterministic; ties go to the lower rank)."""
    sizes = np.asarray(sizes, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    heap = [(0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for b in sorted(range(sizes.size), key=lambda k: (-int(sizes[k]), k)):
        load, r = heapq.heappop(heap)
        out[r].append(b)
        heapq.heappush(heap, (load + int(sizes[b]), r))
    return [sorted(o) for o in out]


def shard_workload(d: dict, rank: int, world: int) -> dict:
    """The part of workload ``d`` that ``rank`` runs: its boxes for a multi-box
    set (with box offsets rebuilt), the whole box otherwise."""
    if "box_off" not in d or world == 1:
        return d
    off = np.asarray(d["box_off"])
    mine = partition_boxes(np.diff(off), world)[rank]
    cols = np.concatenate([np.arange(off[b], off[b + 1]) for b in mine]) if mine else \
        np.zeros(0, dtype=np.int64)
    out = {k: d[k][..., cols] for k in ("x", "v", "u", "h", "m")}
    sz = np.array([off[b + 1] - off[b] for b in mine], dtype=np.int64)
    out["box_off"] = np.concatenate([[0], np.cumsum(sz)]).astype(np.int64)
    out["box_L"] = np.asarray(d["box_L"])[mine] if mine else np.zeros(0)
    out["L"] = d["L"]
    out["boxes"] = np.asarray(mine, dtype=np.int64)
    return out


def max_over_ranks(value: float, device=None) -> float:
    """Max of ``value`` over the default process group (identity when none)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def _union_neighbors(tree, x, h, hmax, idx, L):
    """Indices j with |x_ij| < max(h_i, h_j) for i in idx (minimum image)."""
    out = set()
    cand = tree.query_ball_point(x[idx], np.maximum(h[idx], hmax))
    for i, cs in zip(idx, cand):
        if not cs:
            continue
        cs = np.asarray(cs)
        d = x[cs] - x[i]
        d -= L * np.round(d / L)
        r = np.sqrt((d * d).sum(axis=1))
        keep = cs[(r < h[i]) | (r < h[cs])]
        out.update(keep.tolist())
    return out


def overload_slabs(x, h, n_slabs, L=1.0, axis=0, union_csr=None):
    """Split a periodic box into ``n_slabs`` slabs along ``axis`` and give each
    the ghosts its owned particles need: the rates of i read the fields of its
    union neighbors j, whose density, gradient and coefficients read their own
    neighbors' volumes, which read theirs -- three levels of union neighbors.
    With those ghosts present the owned particles' rates are those of the whole
    box (up to summation order).  x: (3, n); h: (n,).  Returns a list of
    (owned, ghosts) index arrays, one pair per slab; owned sets partition the box.
    union_csr: optional (row_ptr, col) of the union neighbor sets (as
    crk_neighbors_csr gives them); the closure is then three sparse products
    instead of k-d tree queries.
    """
    x = np.asarray(x, dtype=np.float64).T.copy()
    h = np.asarray(h, dtype=np.float64)
    n = h.shape[0]
    slab = np.minimum((x[:, axis] / L * n_slabs).astype(np.int64), n_slabs - 1)
    if union_csr is not None:
        from scipy.sparse import csr_matrix
        row, col = (np.asarray(a) for a in union_csr)
        A = csr_matrix((np.ones(col.size, dtype=np.int32), col, row), shape=(n, n))
        A = ((A + A.T) > 0).astype(np.int32)   # union sets are symmetric; be safe
        out = []
        for s in range(n_slabs):
            reach = (slab == s)
            owned = np.nonzero(reach)[0]
            for _ in range(3):
                reach = reach | (A @ reach.astype(np.int32) > 0)
            ghosts = np.nonzero(reach & (slab != s))[0]
            out.append((owned, ghosts))
        return out
    from scipy.spatial import cKDTree
    tree = cKDTree(np.mod(x, L), boxsize=L)
    hmax = float(h.max()) if n else 0.0
    out = []
    for s in range(n_slabs):
        owned = np.nonzero(slab == s)[0]
        need = set(owned.tolist())
        frontier = owned
        for _ in range(3):
            nxt = _union_neighbors(tree, x, h, hmax, frontier, L) - need
            need |= nxt
            frontier = np.fromiter(nxt, dtype=np.int64, count=len(nxt))
            if frontier.size == 0:
                break
        ghosts = np.array(sorted(need - set(owned.tolist())), dtype=np.int64)
        out.append((owned, ghosts))
    return out
