"""ctypes binding of libcrk (include/crk.h), same names as the C ABI.

Argument marshalling only: every step of the computation runs in the CUDA
library.  Importing this module loads ``_build/libcrk.so`` and raises if it is
missing; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re

from . import build as _build

CRK_OK, CRK_EINVAL, CRK_ENOMEM, CRK_ECUDA, CRK_EDOMAIN, CRK_ENONFINITE, CRK_ESINGULAR, \
    CRK_ETIMEOUT, CRK_ESTATE, CRK_EBOUNDS = range(10)
CRK_FP64, CRK_MIXED32 = 0, 1

STATUS_NAMES = {0: "CRK_OK", 1: "CRK_EINVAL", 2: "CRK_ENOMEM", 3: "CRK_ECUDA", 4: "CRK_EDOMAIN",
                5: "CRK_ENONFINITE", 6: "CRK_ESINGULAR", 7: "CRK_ETIMEOUT", 8: "CRK_ESTATE",
                9: "CRK_EBOUNDS"}


class crk_params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("Cl", C.c_double), ("Cq", C.c_double),
                ("eps2", C.c_double), ("eta_crit", C.c_double), ("eta_fold", C.c_double),
                ("relax_dt", C.c_double), ("limiter", C.c_int32), ("precision", C.c_int32),
                ("nbr_cap", C.c_int32), ("block_threads", C.c_int32),
                ("blocks_per_sm", C.c_int32), ("prefetch", C.c_int32),
                ("energy_split", C.c_int32), ("q_side", C.c_int32)]


class crk_stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_boxes", C.c_int64), ("gather_pairs", C.c_int64),
                ("union_pairs", C.c_int64), ("list_slots", C.c_int64),
                ("list_capacity", C.c_int64), ("tree_nodes", C.c_int64),
                ("launches", C.c_int64), ("tree_tests", C.c_int64), ("bucket_tests", C.c_int64),
                ("status", C.c_int32), ("reserved", C.c_int32)]


class crk_kernel_time(C.Structure):
    _fields_ = [("name", C.c_char * 24), ("ms", C.c_float)]


class crk_cool_table(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("reserved", C.c_int32), ("log10_u_min", C.c_double),
                ("dlog10_u", C.c_double), ("lambda_", C.c_void_p)]


class CRKError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = int(code)
        super().__init__(f"{where}: {STATUS_NAMES.get(self.code, self.code)} "
                         f"({crk_status_string(self.code)})")


_VP = C.c_void_p
_SIGS = {
    "crk_params_default": (None, [C.POINTER(crk_params)]),
    "crk_plan_create": (C.c_int, [C.POINTER(crk_params), C.c_int64, C.c_int32, C.POINTER(_VP)]),
    "crk_plan_destroy": (None, [_VP]),
    "crk_workspace_size": (C.c_int, [_VP, C.c_int64, C.c_int32, C.POINTER(C.c_size_t)]),
    "crk_cell_build": (C.c_int, [_VP, _VP, _VP, C.c_size_t, C.c_int64, C.c_int32, _VP, _VP, _VP,
                                 _VP]),
    "crk_moments": (C.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "crk_rates": (C.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "crk_adjoint": (C.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, C.c_int32]),
    "crk_neighbors_csr": (C.c_int, [_VP, _VP, _VP, C.c_int32, _VP, _VP, C.c_int64,
                                    C.POINTER(C.c_int64)]),
    "crk_stats_get": (C.c_int, [_VP, _VP, _VP, C.POINTER(crk_stats)]),
    "crk_copy": (C.c_int, [_VP, _VP, _VP, C.c_size_t]),
    "crk_status_poll": (C.c_int, [_VP, _VP, _VP, C.POINTER(C.c_int)]),
    "crk_status_string": (C.c_char_p, [C.c_int]),
    "crk_timing_enable": (C.c_int, [_VP, C.c_int32]),
    "crk_timing_read": (C.c_int, [_VP, _VP, C.c_int32, C.POINTER(C.c_int32)]),
    "crk_alu_peak": (C.c_int, [_VP, C.c_int32, C.c_int32, C.POINTER(C.c_double),
                               C.POINTER(C.c_double)]),
    "crk_autotune": (C.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, C.c_int32, _VP, _VP]),
    "crk_tune_set": (C.c_int, [_VP, _VP]),
    "crk_volume_static": (C.c_int, [_VP, C.c_int32, C.c_int64, C.c_double, C.c_double, _VP, _VP,
                                    _VP, _VP]),
    "crk_cool_exact": (C.c_int, [_VP, _VP, C.c_int64, C.POINTER(crk_cool_table), C.c_double, _VP,
                                 _VP, _VP]),
    "crk_subgrid_volume": (C.c_int, [_VP, _VP, _VP, C.c_int64, _VP, _VP, _VP, C.c_double, _VP,
                                     _VP]),
    "crk_subgrid_deposit": (C.c_int, [_VP, _VP, _VP, C.c_int64, _VP, _VP, _VP, C.c_int32, _VP,
                                      _VP, _VP, _VP]),
    "crk_set_species": (C.c_int, [_VP, _VP, _VP, _VP]),
    "crk_rates_adjoint": (C.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP,
                                    _VP]),
    "crk_volume_gw": (C.c_int, [_VP, _VP, _VP, _VP]),
    "crk_leaf_mark": (C.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "crk_time_bins": (C.c_int, [_VP, _VP, _VP, _VP, C.c_double, C.c_int32, C.c_int64, _VP, _VP]),
    "crk_moments_active": (C.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "crk_rates_active": (C.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "crk_hdot": (C.c_int, [_VP, _VP, _VP, C.c_double, C.c_double, C.c_double, _VP, _VP, _VP]),
    "crk_kick": (C.c_int, [_VP, _VP, C.c_int64, C.c_double, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "crk_kick_refined": (C.c_int, [_VP, _VP, C.c_int64, C.c_double, C.c_double, _VP, _VP, _VP,
                                   _VP, _VP, _VP, _VP, _VP, _VP]),
    "crk_drift": (C.c_int, [_VP, _VP, C.c_int64, C.c_int32, _VP, _VP, C.c_double, _VP, _VP, _VP,
                            _VP, _VP, _VP, _VP, C.c_double, _VP, _VP, _VP]),
}
CRK_STATIC_MAX_PARTICLES = 65536
CRK_TUNE_VARIANTS = 18  # launch variants per sweep (include/crk.h)

_lib = None


def load(build_if_missing: bool = True) -> C.CDLL:
    """Load libcrk.so (building it first when allowed); raises if unavailable.
    With CRK_BOUNDS_CHECK=1 in the environment the bounds-checked build is
    loaded instead."""
    global _lib
    if _lib is not None:
        return _lib
    bc = os.environ.get("CRK_BOUNDS_CHECK", "0") == "1"
    path = _build.LIB_BC if bc else _build.LIB
    if build_if_missing:
        path = _build.build_library(bounds_check=bc)
    if not os.path.exists(path):
        raise ImportError(f"libcrk.so not built at {path}; run paper_2511_21921_gb300.build")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def header_symbols() -> list[str]:
    """Function names declared in include/crk.h."""
    with open(os.path.join(_build.INCLUDE, "crk.h")) as fh:
        src = fh.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(crk_[a-z_]+)\s*\(", src)))


def crk_status_string(code: int) -> str:
    s = load().crk_status_string(int(code))
    return s.decode() if s else "?"


def check(code: int, where: str) -> None:
    if code != CRK_OK:
        raise CRKError(code, where)


# thin same-name wrappers -----------------------------------------------------
def crk_params_default() -> crk_params:
    p = crk_params()
    load().crk_params_default(C.byref(p))
    return p


def crk_plan_create(params: crk_params, n_max: int, n_boxes_max: int) -> int:
    h = _VP()
    check(load().crk_plan_create(C.byref(params), int(n_max), int(n_boxes_max), C.byref(h)),
          "crk_plan_create")
    return h.value


def crk_plan_destroy(plan: int) -> None:
    if plan:
        load().crk_plan_destroy(_VP(plan))


def crk_workspace_size(plan: int, n: int, n_boxes: int) -> int:
    b = C.c_size_t()
    check(load().crk_workspace_size(_VP(plan), int(n), int(n_boxes), C.byref(b)),
          "crk_workspace_size")
    return int(b.value)


def crk_cell_build(plan, stream, ws, ws_bytes, n, n_boxes, box_off, box_L, x, h) -> int:
    return load().crk_cell_build(_VP(plan), _VP(stream), _VP(ws), int(ws_bytes), int(n),
                                 int(n_boxes), _VP(box_off), _VP(box_L), _VP(x), _VP(h))


def crk_moments(plan, stream, ws, m, V_out=None, coef_out=None) -> int:
    return load().crk_moments(_VP(plan), _VP(stream), _VP(ws), _VP(m), _VP(V_out),
                              _VP(coef_out))


def crk_rates(plan, stream, ws, v, u, dvdt, dudt, rho_out=None, gradv_out=None) -> int:
    return load().crk_rates(_VP(plan), _VP(stream), _VP(ws), _VP(v), _VP(u), _VP(dvdt),
                            _VP(dudt), _VP(rho_out), _VP(gradv_out))


def crk_adjoint(plan, stream, ws, v, u, g_dvdt, g_dudt, g_x, g_v, g_u, g_h, recompute) -> int:
    return load().crk_adjoint(_VP(plan), _VP(stream), _VP(ws), _VP(v), _VP(u), _VP(g_dvdt),
                              _VP(g_dudt), _VP(g_x), _VP(g_v), _VP(g_u), _VP(g_h),
                              int(recompute))


def crk_neighbors_csr(plan, stream, ws, mode, row_ptr, col, cap):
    nnz = C.c_int64()
    rc = load().crk_neighbors_csr(_VP(plan), _VP(stream), _VP(ws), int(mode), _VP(row_ptr),
                                  _VP(col), int(cap), C.byref(nnz))
    return rc, int(nnz.value)


def crk_stats_get(plan, stream, ws) -> crk_stats:
    s = crk_stats()
    check(load().crk_stats_get(_VP(plan), _VP(stream), _VP(ws), C.byref(s)), "crk_stats_get")
    return s


def crk_copy(stream, dst, src, nbytes) -> None:
    check(load().crk_copy(_VP(stream), _VP(dst), _VP(src), int(nbytes)), "crk_copy")


def crk_status_poll(plan, stream, ws) -> int:
    v = C.c_int()
    check(load().crk_status_poll(_VP(plan), _VP(stream), _VP(ws), C.byref(v)), "crk_status_poll")
    return int(v.value)


def crk_timing_enable(plan, enable: bool) -> None:
    check(load().crk_timing_enable(_VP(plan), 1 if enable else 0), "crk_timing_enable")


def crk_timing_read(plan) -> list[tuple[str, float]]:
    buf = (crk_kernel_time * 256)()
    cnt = C.c_int32()
    check(load().crk_timing_read(_VP(plan), buf, 256, C.byref(cnt)), "crk_timing_read")
    return [(buf[k].name.decode(), float(buf[k].ms)) for k in range(cnt.value)]


def crk_alu_peak(stream, fp64: bool, iters: int) -> tuple[float, float]:
    """(flops/s, ms) of the FMA-chain microbenchmark in float or double."""
    f, ms = C.c_double(), C.c_double()
    check(load().crk_alu_peak(_VP(stream), 1 if fp64 else 0, int(iters), C.byref(f), C.byref(ms)),
          "crk_alu_peak")
    return float(f.value), float(ms.value)


def crk_volume_static(stream, precision, n, L, h_bound, x, h, m, V_out) -> int:
    return load().crk_volume_static(_VP(stream), int(precision), int(n), float(L),
                                    float(h_bound), _VP(x), _VP(h), _VP(m), _VP(V_out))


def crk_hdot(plan, stream, ws, dt_a, lam, n_h, hdot_out=None, hrate_out=None,
             div_out=None) -> int:
    return load().crk_hdot(_VP(plan), _VP(stream), _VP(ws), float(dt_a), float(lam),
                           float(n_h), _VP(hdot_out), _VP(hrate_out), _VP(div_out))


def crk_kick(plan, stream, n, dt, active, v0, a, v_out, u0=None, dudt=None, u_out=None) -> int:
    return load().crk_kick(_VP(plan), _VP(stream), int(n), float(dt), _VP(active), _VP(v0),
                           _VP(a), _VP(v_out), _VP(u0), _VP(dudt), _VP(u_out))


def crk_kick_refined(plan, stream, n, dt_b, dt_c, active, v0, a0, a1, v_out, u0=None, du0=None,
                     du1=None, u_out=None) -> int:
    return load().crk_kick_refined(_VP(plan), _VP(stream), int(n), float(dt_b), float(dt_c),
                                   _VP(active), _VP(v0), _VP(a0), _VP(a1), _VP(v_out), _VP(u0),
                                   _VP(du0), _VP(du1), _VP(u_out))


def crk_drift(plan, stream, n, n_boxes, box_off, box_L, dt, x, v_half, a0=None, dt_a=None,
              t_elapse=None, h=None, hrate=None, n_h=0.0, V=None, rho=None, div=None) -> int:
    return load().crk_drift(_VP(plan), _VP(stream), int(n), int(n_boxes), _VP(box_off),
                            _VP(box_L), float(dt), _VP(x), _VP(v_half), _VP(a0), _VP(dt_a),
                            _VP(t_elapse), _VP(h), _VP(hrate), float(n_h), _VP(V), _VP(rho),
                            _VP(div))


def crk_cool_exact(plan, stream, n, table: crk_cool_table, dt, rho, u0, u1) -> int:
    return load().crk_cool_exact(_VP(plan), _VP(stream), int(n), C.byref(table), float(dt),
                                 _VP(rho), _VP(u0), _VP(u1))


def crk_subgrid_volume(plan, stream, ws, n_s, box_off_s, x_s, h_s, n_h, V_out, h_out=None):
    return load().crk_subgrid_volume(_VP(plan), _VP(stream), _VP(ws), int(n_s), _VP(box_off_s),
                                     _VP(x_s), _VP(h_s), float(n_h), _VP(V_out), _VP(h_out))


def crk_subgrid_deposit(plan, stream, ws, n_s, box_off_s, x_s, h_s, n_comp, q_s, eligible, A_out,
                        dq) -> int:
    return load().crk_subgrid_deposit(_VP(plan), _VP(stream), _VP(ws), int(n_s), _VP(box_off_s),
                                      _VP(x_s), _VP(h_s), int(n_comp), _VP(q_s), _VP(eligible),
                                      _VP(A_out), _VP(dq))


def crk_leaf_mark(plan, stream, ws, flags, leaf_out=None) -> int:
    return load().crk_leaf_mark(_VP(plan), _VP(stream), _VP(ws), _VP(flags), _VP(leaf_out))


def crk_rates_adjoint(plan, stream, ws, v, u, g_dvdt, g_dudt, dvdt, dudt, g_x, g_v, g_u,
                      g_h) -> int:
    return load().crk_rates_adjoint(_VP(plan), _VP(stream), _VP(ws), _VP(v), _VP(u),
                                    _VP(g_dvdt), _VP(g_dudt), _VP(dvdt), _VP(dudt), _VP(g_x),
                                    _VP(g_v), _VP(g_u), _VP(g_h))


def crk_set_species(plan, stream, ws, species) -> int:
    return load().crk_set_species(_VP(plan), _VP(stream), _VP(ws), _VP(species))


def crk_volume_gw(plan, stream, ws, Vgw_out) -> int:
    return load().crk_volume_gw(_VP(plan), _VP(stream), _VP(ws), _VP(Vgw_out))


def crk_time_bins(plan, stream, ws, dt, dt_max, max_level, substep, level_out, flags) -> int:
    return load().crk_time_bins(_VP(plan), _VP(stream), _VP(ws), _VP(dt), float(dt_max),
                                int(max_level), int(substep), _VP(level_out), _VP(flags))


def crk_moments_active(plan, stream, ws, m, flags, V_state, coef_state) -> int:
    return load().crk_moments_active(_VP(plan), _VP(stream), _VP(ws), _VP(m), _VP(flags),
                                     _VP(V_state), _VP(coef_state))


def crk_rates_active(plan, stream, ws, v, u, rho_state, gradv_state, dvdt, dudt) -> int:
    return load().crk_rates_active(_VP(plan), _VP(stream), _VP(ws), _VP(v), _VP(u),
                                   _VP(rho_state), _VP(gradv_state), _VP(dvdt), _VP(dudt))


SWEEPS = ("b1_volume", "b2_moments", "c1_density", "c2_rates", "adj_c2", "adj_c1", "adj_b2",
          "adj_b1")


def crk_tune_set(plan, choice) -> None:
    """Set the launch variant of every sweep (8 ints in the order of SWEEPS)."""
    arr = (C.c_int32 * 8)(*[int(c) for c in choice])
    check(load().crk_tune_set(_VP(plan), arr), "crk_tune_set")


def crk_autotune(plan, stream, ws, m, v, u, g_dvdt, g_dudt, repeats=3):
    nv = CRK_TUNE_VARIANTS
    choice = (C.c_int32 * 8)()
    ms = (C.c_float * (8 * nv))()
    check(load().crk_autotune(_VP(plan), _VP(stream), _VP(ws), _VP(m), _VP(v), _VP(u),
                              _VP(g_dvdt), _VP(g_dudt), int(repeats), choice, ms),
          "crk_autotune")
    return {SWEEPS[q]: {"variant": int(choice[q]), "ms": [round(float(ms[nv * q + k]), 4)
                                                          for k in range(nv)]} for q in range(8)}
