"""Seeded synthetic particle sets shaped like cosmological gas.

This module holds input generation only (random fields, particle placement,
k-nearest-neighbor smoothing lengths); none of the CRKSPH arithmetic lives here.
Both the CUDA path's tests and the CPU oracle's tests draw their inputs from it.

Every generator draws in a fixed order from ``numpy.random.default_rng(seed)``
and returns a dict with float64 arrays ``x`` (3, n) in ``[0, L)``, ``v`` (3, n),
``u`` (n,), ``h`` (n,), ``m`` (n,) and the box side ``L``; multi-box sets also
carry ``box_off`` (B+1,) and ``box_L`` (B,).

Workload shapes (periodic unit boxes, equal masses m = 1/N; the workloads
named with a trailing ``m`` are the same boxes with lognormal masses, see
``unequal_masses``):

* ``lattice``  -- 16^3 cubic lattice jittered by U(-0.2, 0.2) spacing, constant
  h for about 64 neighbors, v ~ N(0, 0.1), u ~ lognormal(0, 0.5).
* ``lognormal`` -- particles placed multinomially in the cells of a lognormal
  density field exp(delta - s2/2), delta a Gaussian random field with power
  spectrum P(k) ~ k^-2 (the spectral index of the paper's scale-free tests,
  App. B) normalised to variance s2; uniform within a cell; h from the distances
  to the k-th and (k+1)-th nearest neighbors with k ~ U{90..110}; ln u ~ N(0,
  1.151) truncated at 3 sigma (three decades); v ~ N(0, 0.1).
* ``clumpy`` -- 200 Plummer spheres of 1e3..1e4 particles (log-uniform) with
  central contrast 10^U(2,4), truncated at 5 scale radii, plus a lognormal field
  of variance 3.0 for the rest.
* ``multibox`` -- 64 independent boxes with n_b = round(exp(U(ln 8, ln 96))),
  N_b = n_b^3 particles each, variance U(0.5, 3.0), seeds 100 + b.
"""
from __future__ import annotations

import hashlib
import os

import numpy as np

try:  # scipy is present on both the build host and the GPU host
    from scipy.spatial import cKDTree
except Exception:  # pragma: no cover
    cKDTree = None

_CACHE = os.environ.get(
    "CRK_SYNTH_CACHE",
    os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), ".synth_cache"))


def _below(x, L):
    """Fold into [0, L) (guards against rounding up to L)."""
    x = np.mod(x, L)
    return np.where(x >= L, np.nextafter(L, 0.0), x)


def _truncated_normal(rng, n, sigma, cut=3.0):
    z = rng.standard_normal(n)
    bad = np.abs(z) > cut
    while bad.any():
        z[bad] = rng.standard_normal(int(bad.sum()))
        bad = np.abs(z) > cut
    return sigma * z


def gaussian_field(rng, ng, sigma2, slope=-2.0):
    """Periodic Gaussian random field on an ng^3 grid with P(k) ~ k^slope."""
    noise = rng.standard_normal((ng, ng, ng))
    fk = np.fft.rfftn(noise)
    kx = np.fft.fftfreq(ng) * ng
    kz = np.fft.rfftfreq(ng) * ng
    k2 = kx[:, None, None] ** 2 + kx[None, :, None] ** 2 + kz[None, None, :] ** 2
    amp = np.zeros_like(k2)
    nz = k2 > 0
    amp[nz] = k2[nz] ** (slope / 4.0)  # sqrt(P(k)) = k^(slope/2)
    delta = np.fft.irfftn(fk * amp, s=(ng, ng, ng), axes=(0, 1, 2))
    delta *= np.sqrt(sigma2) / delta.std()
    return delta


def place_in_cells(rng, density, n, L=1.0):
    """Multinomial placement of n particles in cells with weights ``density``."""
    ng = density.shape[0]
    p = density.ravel() / density.sum()
    counts = rng.multinomial(n, p)
    cell = np.repeat(np.arange(p.size), counts)
    ci = np.stack(np.unravel_index(cell, density.shape))  # (3, n)
    off = rng.random((3, n))
    return _below((ci + off) * (L / ng), L)


def knn_h(x, L, kmin, kmax, rng, cap=None, chunk=1 << 19):
    """h_i = midpoint of the k_i-th and (k_i+1)-th neighbor distances, k_i ~ U{kmin..kmax}.

    Exactly k_i other particles then lie strictly inside h_i (distinct distances).
    """
    n = x.shape[1]
    k = rng.integers(kmin, kmax + 1, size=n)
    kq = min(kmax + 2, n)
    if cKDTree is None:
        raise RuntimeError("scipy is required for the k-nearest-neighbor smoothing lengths")
    tree = cKDTree(x.T, boxsize=L)
    h = np.empty(n)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        d, _ = tree.query(x[:, s:e].T, k=kq, workers=-1)
        kk = np.minimum(k[s:e], kq - 2)
        rows = np.arange(e - s)
        h[s:e] = 0.5 * (d[rows, kk] + d[rows, kk + 1])  # column 0 is the particle itself
    if cap is not None:
        h = np.minimum(h, cap * L)
    return h, k


def _finish(rng, x, h, L, sigma_v=0.1, sigma_lnu=1.151, lognormal_u_sigma=None):
    n = x.shape[1]
    v = rng.normal(0.0, sigma_v, size=(3, n))
    if lognormal_u_sigma is not None:
        u = np.exp(rng.normal(0.0, lognormal_u_sigma, size=n))
    else:
        u = np.exp(_truncated_normal(rng, n, sigma_lnu))
    m = np.full(n, 1.0 / n)
    return dict(x=np.ascontiguousarray(x), v=v, u=u, h=np.ascontiguousarray(h), m=m, L=float(L))


def lattice(n_side=16, seed=0, jitter=0.2, k_target=64, L=1.0):
    """Jittered cubic lattice with constant h for about ``k_target`` neighbors."""
    rng = np.random.default_rng(seed)
    n = n_side ** 3
    g = np.stack(np.meshgrid(*(np.arange(n_side),) * 3, indexing="ij")).reshape(3, -1)
    x = (g + 0.5 + rng.uniform(-jitter, jitter, size=(3, n))) * (L / n_side)
    x = _below(x, L)
    h = np.full(n, L * (3.0 * k_target / (4.0 * np.pi * n)) ** (1.0 / 3.0))
    return _finish(rng, x, h, L, lognormal_u_sigma=0.5)


def lognormal(n_side=64, sigma2=1.5, seed=1, kmin=90, kmax=110, L=1.0, h_cap=0.45):
    """Lognormal-density box of n_side^3 particles (P(k) ~ k^-2 field on n_side^3 cells)."""
    rng = np.random.default_rng(seed)
    n = n_side ** 3
    delta = gaussian_field(rng, n_side, sigma2)
    rho = np.exp(delta - 0.5 * sigma2)
    x = place_in_cells(rng, rho, n, L)
    h, _ = knn_h(x, L, kmin, kmax, rng, cap=h_cap)
    return _finish(rng, x, h, L)


def clumpy(n_side=128, n_clumps=200, sigma2=3.0, seed=2, kmin=90, kmax=110, L=1.0,
           nc_min=1e3, nc_max=1e4):
    """Plummer clumps on a lognormal background (h spanning about two decades)."""
    rng = np.random.default_rng(seed)
    n = n_side ** 3
    nc = np.round(np.exp(rng.uniform(np.log(nc_min), np.log(nc_max), size=n_clumps))).astype(np.int64)
    contrast = 10.0 ** rng.uniform(2.0, 4.0, size=n_clumps)
    centers = rng.random((3, n_clumps)) * L
    parts = []
    for c in range(n_clumps):
        a = (3.0 * nc[c] / (4.0 * np.pi * n * contrast[c])) ** (1.0 / 3.0) * L
        # Plummer radii by inverting the cumulative mass, truncated at 5a
        r = np.empty(0)
        while r.size < nc[c]:
            q = rng.random(int(nc[c]))
            rr = a / np.sqrt(q ** (-2.0 / 3.0) - 1.0)
            r = np.concatenate([r, rr[rr < 5.0 * a]])
        r = r[: nc[c]]
        dirs = rng.standard_normal((3, int(nc[c])))
        dirs /= np.linalg.norm(dirs, axis=0)
        parts.append(centers[:, c:c + 1] + dirs * r)
    xc = np.concatenate(parts, axis=1)
    n_bg = n - xc.shape[1]
    delta = gaussian_field(rng, n_side, sigma2)
    rho = np.exp(delta - 0.5 * sigma2)
    xb = place_in_cells(rng, rho, n_bg, L)
    x = _below(np.concatenate([xc, xb], axis=1), L)
    h, _ = knn_h(x, L, kmin, kmax, rng, cap=0.45)
    return _finish(rng, x, h, L)


def multibox(n_boxes=64, seed0=100, nmin=8, nmax=96, kmin=90, kmax=110):
    """Independent periodic unit boxes of uneven size, concatenated box by box."""
    meta = np.random.default_rng(seed0 - 1)
    sides = np.round(np.exp(meta.uniform(np.log(nmin), np.log(nmax), size=n_boxes))).astype(int)
    s2 = meta.uniform(0.5, 3.0, size=n_boxes)
    boxes = [lognormal(int(sides[b]), float(s2[b]), seed0 + b, kmin, kmax) for b in range(n_boxes)]
    off = np.zeros(n_boxes + 1, dtype=np.int64)
    off[1:] = np.cumsum([bx["h"].shape[0] for bx in boxes])
    out = {k: np.concatenate([bx[k] for bx in boxes], axis=-1) for k in ("x", "v", "u", "h", "m")}
    out["box_off"] = off
    out["box_L"] = np.ones(n_boxes)
    out["L"] = 1.0
    out["sides"] = sides
    out["sigma2"] = s2
    return out


def cotangents(n, seed=4):
    """Upstream cotangents g ~ N(0, 1) for the momentum and energy rates."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((3, n)), rng.standard_normal(n)


def region_sample(d, side, center=0.5, hops=3):
    """A cubic region of box ``d`` with the particles its results depend on.

    Owned particles lie within ``side``/2 of ``center`` on every axis (no
    periodic wrap, so the cube must sit inside the box).  The sample adds every
    particle within a margin of ``hops`` times the largest smoothing length of
    the sample, grown until it stops changing: a particle's rates depend only
    on particles within three neighbor hops, and a hop is shorter than the
    larger smoothing length of the pair.  Particles keep their relative order,
    so neighbor lists sorted by index are sorted the same way in the sample.
    Returns the sample (same keys as ``d``), the boolean mask of its owned
    particles and the indices of the sample's particles in ``d``.
    """
    x, h = d["x"], d["h"]
    off = np.abs(x - center)
    own = np.all(off < 0.5 * side, axis=0)
    margin = hops * float(h[own].max())
    while True:
        reg = np.all(off < 0.5 * side + margin, axis=0)
        m2 = hops * float(h[reg].max())
        if m2 <= margin:
            break
        margin = m2
    if 0.5 * side + margin >= min(center, d["L"] - center):
        raise ValueError("region with its margin does not fit inside the box")
    idx = np.nonzero(reg)[0]
    out = {k: (d[k][..., idx] if k in ("x", "v", "u", "h", "m") else d[k]) for k in d
           if k not in ("box_off", "box_L", "sides", "sigma2")}
    out["x"] = np.ascontiguousarray(out["x"])
    out["v"] = np.ascontiguousarray(out["v"])
    return out, own[idx], idx


def unequal_masses(d, seed=6, sigma=0.7, cut=2.5):
    """A copy of workload ``d`` whose masses are lognormal: ln(m N) ~ N(0, sigma)
    truncated at ``cut`` sigma (a spread of exp(2 cut sigma) = 33x for the
    defaults), everything else unchanged.  Equal masses hide where m_i and m_j
    enter the sums; these inputs exercise them."""
    rng = np.random.default_rng(seed)
    out = dict(d)
    n = d["h"].shape[0]
    out["m"] = np.exp(_truncated_normal(rng, n, sigma, cut)) / n
    return out


# --------------------------------------------------------------------------
# named workloads with an on-disk cache (generation of the large ones takes
# tens of seconds because of the nearest-neighbor queries)
# --------------------------------------------------------------------------
WORKLOADS = {
    "lattice16": lambda: lattice(16, seed=0),
    "lognormal32": lambda: lognormal(32, 1.5, seed=3),
    "lognormal64": lambda: lognormal(64, 1.5, seed=1),
    "lognormal128": lambda: lognormal(128, 1.5, seed=3),
    "clumpy128": lambda: clumpy(128, seed=2),
    "multibox64": lambda: multibox(64),
    "lognormal256": lambda: lognormal(256, 1.5, seed=5),
    # the same boxes with lognormal masses (33x spread)
    "lattice16m": lambda: unequal_masses(lattice(16, seed=0), seed=6),
    "lognormal32m": lambda: unequal_masses(lognormal(32, 1.5, seed=3), seed=6),
    "lognormal64m": lambda: unequal_masses(lognormal(64, 1.5, seed=1), seed=7),
}


def load(name: str, cache: bool = True) -> dict:
    """Generate (or read from the cache) one of the named workloads."""
    fn = WORKLOADS[name]
    path = os.path.join(_CACHE, f"{name}.npz")
    if cache and os.path.exists(path):
        with np.load(path) as z:
            d = {k: z[k] for k in z.files}
        d["L"] = float(d["L"])
        return d
    d = fn()
    if cache:
        os.makedirs(_CACHE, exist_ok=True)
        tmp = path + f".tmp{os.getpid()}.npz"
        np.savez(tmp, **d)
        os.replace(tmp, path)
    return d


def digest(d: dict) -> str:
    """Short content hash of a workload (recorded next to results)."""
    hs = hashlib.sha256()
    for k in ("x", "v", "u", "h", "m"):
        hs.update(np.ascontiguousarray(d[k]).tobytes())
    return hs.hexdigest()[:16]
