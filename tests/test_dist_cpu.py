"""Multi-rank host logic on CPU (gloo, world size 2): box sharding without a
data-path collective, and the max/sum reductions bench.py uses for timing."""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2511_21921_gb300 import dist as D
from paper_2511_21921_gb300 import synth


def test_partition_covers_every_box_once_and_balances():
    rng = np.random.default_rng(0)
    sizes = np.round(np.exp(rng.uniform(np.log(8), np.log(96), 64))).astype(int) ** 3
    for world in (1, 2, 3, 8):
        parts = D.partition_boxes(sizes, world)
        flat = sorted(b for p in parts for b in p)
        assert flat == list(range(64))
        loads = [sizes[p].sum() for p in parts]
        assert max(loads) - min(loads) <= sizes.max()  # greedy LPT bound


def _worker(rank, world, port, d, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sd = D.shard_workload(d, rank, world)
        t = D.max_over_ranks(float(rank + 1))
        n = D.sum_over_ranks(float(sd["h"].shape[0]))
        q.put((rank, sd["boxes"].tolist(), sd["box_off"].tolist(), float(sd["m"].sum()), t, n))
    finally:
        dist.destroy_process_group()


def test_two_rank_sharding_with_gloo():
    d = synth.multibox(n_boxes=6, seed0=500, nmin=8, nmax=14)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, d, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    boxes = sorted(res[0][1] + res[1][1])
    assert boxes == list(range(6))
    n_total = d["h"].shape[0]
    for rank, mine, off, msum, tmax, nsum in res:
        assert tmax == 2.0 and nsum == n_total
        sizes = np.diff(d["box_off"])[mine]
        assert off == [0] + np.cumsum(sizes).tolist()
    assert abs(res[0][3] + res[1][3] - d["m"].sum()) < 1e-12


def test_single_box_is_replicated():
    d = synth.lattice(8, seed=1)
    for r in range(3):
        assert D.shard_workload(d, r, 3) is d


def test_overload_slabs_partition_and_closure():
    """Owned sets partition the box; each slab's ghosts hold every particle
    within three levels of union neighbors of its owned particles (brute force)."""
    import numpy as np
    from paper_2511_21921_gb300 import dist as D
    rng = np.random.default_rng(0)
    n = 600
    x = rng.uniform(0, 1, (3, n))
    h = rng.uniform(0.05, 0.12, n)
    parts = D.overload_slabs(x, h, 3)
    owned = np.concatenate([o for o, _ in parts])
    assert np.array_equal(np.sort(owned), np.arange(n))
    d = x[:, :, None] - x[:, None, :]
    d -= np.round(d)
    r = np.sqrt((d * d).sum(0))
    adj = (r < np.maximum(h[:, None], h[None, :]))
    for o, g in parts:
        reach = np.zeros(n, bool)
        reach[o] = True
        for _ in range(3):
            reach = reach | adj[reach].any(axis=0)
        have = np.zeros(n, bool)
        have[o] = True
        have[g] = True
        assert np.array_equal(reach, have)
        assert not np.intersect1d(o, g).size
    # the same closure from union neighbor sets given as CSR
    rows = [np.nonzero(adj[i] & (np.arange(n) != i))[0] for i in range(n)]
    rp = np.concatenate([[0], np.cumsum([len(c) for c in rows])])
    parts2 = D.overload_slabs(x, h, 3, union_csr=(rp, np.concatenate(rows)))
    for (o1, g1), (o2, g2) in zip(parts, parts2):
        assert np.array_equal(o1, o2) and np.array_equal(g1, g2)
