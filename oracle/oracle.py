"""ctypes binding of the FP64 CPU oracle (``crk_oracle.cpp``).

Test infrastructure only: the tests, the smoke check and the benchmark's CPU
baseline call it.  Nothing in the product package imports this module.

Array conventions (shared with the tests, not with the CUDA code):
positions ``x`` and velocities ``v`` are float64 arrays of shape ``(3, n)``;
``h``, ``m``, ``u`` have shape ``(n,)``; the box is ``[0, L)^3``, periodic.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "crk_oracle.cpp")
_OUT = os.path.join(_HERE, "_build", "libcrk_oracle.so")
_lock = threading.Lock()
_lib = None

# Every oracle function has a pin in tests/ (invariants, special cases, brute
# force, quadrature, finite differences, the linear-field and two-species
# lattice reductions).  What no pin fixes: the shape of the limiter function
# phi(r) away from r = 1 (4r/(1+r)^2, a reading of the formulation the paper
# defers to; phi(1) = 1, the limited relative velocity and the side of the
# near-field damping threshold are pinned), the viscosity constants, and so
# the absolute rate values beyond the invariants and reductions.
PARITY_UNPINNED = ("limiter shape phi(r) for r != 1 and the viscosity constants; absolute "
                   "rate values beyond conservation (equal and unequal masses), lattice, "
                   "linear-field, inviscid-limit and standard-SPH reductions")

STATUS = {0: "ok", 1: "invalid argument", 4: "domain (x outside [0,L) or h >= L/2)",
          5: "non-finite input", 6: "singular second moment"}


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build`` (plain g++, FP64, no FMA)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if (not force and os.path.exists(_OUT)
            and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC)):
        return _OUT
    tmp = _OUT + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _OUT)
    return _OUT


class OracleParams(C.Structure):
    _fields_ = [("gamma", C.c_double), ("Cl", C.c_double), ("Cq", C.c_double),
                ("eps2", C.c_double), ("eta_crit", C.c_double), ("eta_fold", C.c_double),
                ("relax_dt", C.c_double), ("limiter", C.c_int32), ("energy_split", C.c_int32),
                ("q_side", C.c_int32), ("pad", C.c_int32)]


def default_params(**kw) -> OracleParams:
    """The reading of the viscosity constants used throughout (configurable)."""
    n_h = (3.0 * 100 / (4.0 * np.pi)) ** (1.0 / 3.0)
    d = dict(gamma=5.0 / 3.0, Cl=2.0, Cq=1.0, eps2=0.01, eta_crit=1.0 / n_h,
             eta_fold=0.2, relax_dt=0.0, limiter=1, energy_split=0, q_side=0)
    d.update(kw)
    return OracleParams(**d, pad=0)


class _Out(C.Structure):
    _fields_ = [("V", C.c_void_p), ("coef", C.c_void_p), ("mom", C.c_void_p),
                ("rho", C.c_void_p), ("gradv", C.c_void_p), ("P", C.c_void_p),
                ("cs", C.c_void_p), ("flag", C.c_void_p), ("dvdt", C.c_void_p),
                ("dudt", C.c_void_p), ("kgather", C.c_void_p), ("kunion", C.c_void_p),
                ("diag", C.c_void_p), ("nsingular", C.c_void_p)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            dp = C.c_void_p
            lib.oracle_forward.restype = C.c_int
            lib.oracle_forward.argtypes = [C.c_int64, dp, dp, dp, dp, dp, C.c_double,
                                           C.POINTER(OracleParams), C.c_int64, dp, C.c_int32,
                                           C.c_int32, C.c_int32, C.POINTER(_Out)]
            lib.oracle_jvp.restype = C.c_int
            lib.oracle_jvp.argtypes = [C.c_int64, dp, dp, dp, dp, dp, C.c_double,
                                       C.POINTER(OracleParams), dp, dp, dp, dp, C.c_int64, dp,
                                       C.c_int32, C.c_int32, C.c_int32, C.POINTER(_Out),
                                       C.POINTER(_Out)]
            lib.oracle_forward_species.restype = C.c_int
            lib.oracle_forward_species.argtypes = [C.c_int64, dp, dp, dp, dp, dp, C.c_double,
                                                   C.POINTER(OracleParams), dp, C.c_int64, dp,
                                                   C.c_int32, C.c_int32, C.c_int32,
                                                   C.POINTER(_Out), dp]
            lib.oracle_forward_state.restype = C.c_int
            lib.oracle_forward_state.argtypes = [C.c_int64, dp, dp, dp, dp, dp, C.c_double,
                                                 C.POINTER(OracleParams), dp, dp, dp, dp, dp,
                                                 C.c_int32, C.POINTER(_Out)]
            lib.oracle_neighbors.restype = C.c_int
            lib.oracle_neighbors.argtypes = [C.c_int32, C.c_int32, C.c_int64, dp, dp,
                                             C.c_double, dp, dp, C.c_int64, dp]
            lib.oracle_kernel.restype = None
            lib.oracle_kernel.argtypes = [C.c_int64, dp, C.c_double, dp, dp, dp]
            lib.oracle_count_pairs.restype = C.c_int
            lib.oracle_count_pairs.argtypes = [C.c_int64, dp, dp, C.c_double,
                                               C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
            lib.oracle_count_ops.restype = C.c_int
            lib.oracle_count_ops.argtypes = [C.c_int64, dp, dp, dp, dp, dp, C.c_double,
                                             C.POINTER(OracleParams), dp, dp, dp, dp, C.c_int32,
                                             C.c_int32, dp]
            lib.oracle_num_threads.restype = C.c_int
            _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        assert a.shape == shape, (a.shape, shape)
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data


_FIELDS = {  # name -> (components, dtype)
    "V": (1, np.float64), "coef": (16, np.float64), "mom": (40, np.float64),
    "rho": (1, np.float64), "gradv": (9, np.float64), "P": (1, np.float64),
    "cs": (1, np.float64), "flag": (1, np.int8), "dvdt": (3, np.float64),
    "dudt": (1, np.float64), "kgather": (1, np.int64), "kunion": (1, np.int64),
    "diag": (16, np.float64),
}
_STAGE_OF = {"V": 1, "kgather": 1, "kunion": 1, "coef": 2, "mom": 2, "diag": 2, "rho": 3,
             "gradv": 3, "P": 3, "cs": 3, "flag": 3, "dvdt": 4, "dudt": 4}


def _alloc(want, nt):
    arrs = {}
    for k in want:
        comp, dt = _FIELDS[k]
        arrs[k] = np.zeros((comp, nt) if comp > 1 else (nt,), dtype=dt)
    arrs["nsingular"] = np.zeros(1, dtype=np.int64)
    o = _Out(**{k: _ptr(v) for k, v in arrs.items()})
    return o, arrs


def _inputs(x, h, m, v, u):
    n = int(np.asarray(h).shape[0])
    x = _f64(x, (3, n))
    h = _f64(h, (n,))
    m = _f64(m, (n,))
    v = _f64(v, (3, n)) if v is not None else np.zeros((3, n))
    u = _f64(u, (n,)) if u is not None else np.zeros(n)
    return n, x, h, m, v, u


def forward(x, h, m, v=None, u=None, L=1.0, params=None, targets=None,
            want=("V", "coef", "rho", "gradv", "P", "cs", "flag", "dvdt", "dudt"),
            nthreads=0, use_tree=True):
    """Evaluate the oracle.  Returns a dict of arrays ``(components, nt)``.

    ``targets`` (int64 indices) restricts outputs to those particles and
    evaluates their neighbor closure lazily; ``None`` evaluates all.
    """
    lib = _load()
    n, x, h, m, v, u = _inputs(x, h, m, v, u)
    p = params if params is not None else default_params()
    stages = max(_STAGE_OF[k] for k in want)
    if targets is not None:
        targets = np.ascontiguousarray(targets, dtype=np.int64)
        nt = targets.shape[0]
    else:
        nt = n
    o, arrs = _alloc(want, nt)
    rc = lib.oracle_forward(n, _ptr(x), _ptr(h), _ptr(m), _ptr(v), _ptr(u), float(L),
                            C.byref(p), nt, _ptr(targets), stages, int(nthreads),
                            1 if use_tree else 0, C.byref(o))
    if rc not in (0, 6):
        raise ValueError(f"oracle_forward: {STATUS.get(rc, rc)}")
    arrs["status"] = rc
    return arrs


def forward_species(x, h, m, v, u, L, species, params=None, targets=None,
                    want=("V", "coef", "rho", "gradv", "P", "cs", "flag", "dvdt", "dudt"),
                    nthreads=0):
    """Evaluation with species (uint8, 0 gas, 1 wind; Sec. 2.5.1, App. A.2):
    winds enter the density with the volume over gas and wind (returned as
    "Vgw") and take part in no other sum; their rates are zero."""
    lib = _load()
    n, x, h, m, v, u = _inputs(x, h, m, v, u)
    p = params if params is not None else default_params()
    sp = np.ascontiguousarray(species, dtype=np.uint8)
    assert sp.shape == (n,)
    stages = max(_STAGE_OF[k] for k in want)
    if targets is not None:
        targets = np.ascontiguousarray(targets, dtype=np.int64)
        nt = targets.shape[0]
    else:
        nt = n
    o, arrs = _alloc(want, nt)
    vgw = np.zeros(nt)
    rc = lib.oracle_forward_species(n, _ptr(x), _ptr(h), _ptr(m), _ptr(v), _ptr(u), float(L),
                                    C.byref(p), _ptr(sp), nt, _ptr(targets), stages,
                                    int(nthreads), 1, C.byref(o), _ptr(vgw))
    if rc not in (0, 6):
        raise ValueError(f"oracle_forward_species: {STATUS.get(rc, rc)}")
    arrs["Vgw"] = vgw
    arrs["status"] = rc
    return arrs


def forward_state(x, h, m, v, u, L, flags, V_state, coef_state, rho_state, gradv_state,
                  params=None, nthreads=0):
    """Active-set evaluation (passive particles reuse stored fields).

    flags (uint8, n): bit 0 active, bit 1 recompute volume and coefficients.
    State arrays (caller order): V (n,), coef (16, n), rho (n,), gradv (9, n).
    Returns V, coef, rho, gradv, P, cs, flag for every particle and dvdt,
    dudt (zero for particles that are not active).
    """
    lib = _load()
    n, x, h, m, v, u = _inputs(x, h, m, v, u)
    p = params if params is not None else default_params()
    flags = np.ascontiguousarray(flags, dtype=np.uint8)
    assert flags.shape == (n,)
    Vs = _f64(V_state, (n,))
    cs_ = _f64(coef_state, (16, n))
    rs = _f64(rho_state, (n,))
    gs = _f64(gradv_state, (9, n))
    o, arrs = _alloc(("V", "coef", "rho", "gradv", "P", "cs", "flag", "dvdt", "dudt"), n)
    rc = lib.oracle_forward_state(n, _ptr(x), _ptr(h), _ptr(m), _ptr(v), _ptr(u), float(L),
                                  C.byref(p), _ptr(flags), _ptr(Vs), _ptr(cs_), _ptr(rs),
                                  _ptr(gs), int(nthreads), C.byref(o))
    if rc not in (0, 6):
        raise ValueError(f"oracle_forward_state: {STATUS.get(rc, rc)}")
    arrs["status"] = rc
    return arrs


def jvp(x, h, m, v, u, L, tx=None, tv=None, tu=None, th=None, params=None, targets=None,
        want=("dvdt", "dudt"), nthreads=0, use_tree=True):
    """Forward-mode tangent of the chosen outputs along (tx, tv, tu, th)."""
    lib = _load()
    n, x, h, m, v, u = _inputs(x, h, m, v, u)
    p = params if params is not None else default_params()
    stages = max(_STAGE_OF[k] for k in want)
    tx = _f64(tx, (3, n)) if tx is not None else None
    tv = _f64(tv, (3, n)) if tv is not None else None
    tu = _f64(tu, (n,)) if tu is not None else None
    th = _f64(th, (n,)) if th is not None else None
    if targets is not None:
        targets = np.ascontiguousarray(targets, dtype=np.int64)
        nt = targets.shape[0]
    else:
        nt = n
    o, arrs = _alloc(want, nt)
    to, tarrs = _alloc(want, nt)
    rc = lib.oracle_jvp(n, _ptr(x), _ptr(h), _ptr(m), _ptr(v), _ptr(u), float(L), C.byref(p),
                        _ptr(tx), _ptr(tv), _ptr(tu), _ptr(th), nt, _ptr(targets), stages,
                        int(nthreads), 1 if use_tree else 0, C.byref(o), C.byref(to))
    if rc not in (0, 6):
        raise ValueError(f"oracle_jvp: {STATUS.get(rc, rc)}")
    return arrs, tarrs


def count_ops(x, h, m, v, u, L, stages, derivative=False, tx=None, tv=None, tu=None, th=None,
              params=None):
    """Operations of a whole-box evaluation up to ``stages`` (1..4) counted by
    the oracle itself (add, subtract, multiply, divide, sqrt, exp = 1 each), on
    one thread.  Returns (value operations, tangent operations); the tangent
    count is 0 unless ``derivative`` (the forward-mode derivative along the
    given tangents)."""
    lib = _load()
    n, x, h, m, v, u = _inputs(x, h, m, v, u)
    p = params if params is not None else default_params()
    t = [_f64(a, s) if a is not None else None
         for a, s in ((tx, (3, n)), (tv, (3, n)), (tu, (n,)), (th, (n,)))]
    ops = np.zeros(2, dtype=np.int64)
    rc = lib.oracle_count_ops(n, _ptr(x), _ptr(h), _ptr(m), _ptr(v), _ptr(u), float(L), C.byref(p),
                              _ptr(t[0]), _ptr(t[1]), _ptr(t[2]), _ptr(t[3]), int(stages),
                              1 if derivative else 0, _ptr(ops))
    if rc not in (0, 6):
        raise ValueError(f"oracle_count_ops: {STATUS.get(rc, rc)}")
    return int(ops[0]), int(ops[1])


def neighbors(x, h, L=1.0, mode="gather", method="tree"):
    """CSR neighbor sets: mode 'gather' (r < h_i, self included) or 'union'."""
    lib = _load()
    n = int(np.asarray(h).shape[0])
    x = _f64(x, (3, n))
    h = _f64(h, (n,))
    row = np.zeros(n + 1, dtype=np.int64)
    nnz = np.zeros(1, dtype=np.int64)
    md = 0 if mode == "gather" else 1
    meth = 1 if method == "tree" else 0
    cap = 0
    col = np.zeros(1, dtype=np.int32)
    for _ in range(2):
        rc = lib.oracle_neighbors(md, meth, n, _ptr(x), _ptr(h), float(L), _ptr(row), _ptr(col),
                                  cap, _ptr(nnz))
        if rc == 0:
            return row, col[: int(nnz[0])]
        if rc != 1 or int(nnz[0]) <= cap:
            raise ValueError(f"oracle_neighbors: {STATUS.get(rc, rc)}")
        cap = int(nnz[0])
        col = np.zeros(max(cap, 1), dtype=np.int32)
    raise RuntimeError("oracle_neighbors: capacity retry failed")


def count_pairs(x, h, L=1.0):
    """(ordered gather pairs, ordered union pairs) of the whole box, self
    excluded, without storing the sets (the sizes of ``neighbors``' sets)."""
    lib = _load()
    n = int(np.asarray(h).shape[0])
    x = _f64(x, (3, n))
    h = _f64(h, (n,))
    g, u = C.c_int64(), C.c_int64()
    rc = lib.oracle_count_pairs(n, _ptr(x), _ptr(h), float(L), C.byref(g), C.byref(u))
    if rc != 0:
        raise ValueError(f"oracle_count_pairs: {STATUS.get(rc, rc)}")
    return int(g.value), int(u.value)


def kernel(r, h):
    """Wendland C4: returns (W, dW/dr, (1/r) dW/dr) at radii ``r``."""
    lib = _load()
    r = _f64(r)
    W = np.zeros_like(r)
    dW = np.zeros_like(r)
    g = np.zeros_like(r)
    lib.oracle_kernel(r.size, _ptr(r), float(h), _ptr(W), _ptr(dW), _ptr(g))
    return W, dW, g

