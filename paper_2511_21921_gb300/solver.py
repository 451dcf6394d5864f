"""Torch-facing wrapper of libcrk: one plan plus one workspace tensor.

PyTorch supplies device memory and the current stream; every computation is a
libcrk call.  Arrays follow the C ABI: positions ``x`` are float64 (3, n);
other real arrays are float64 for ``precision="fp64"`` and float32 for
``precision="mixed"``; all tensors are contiguous on one CUDA device.
"""
from __future__ import annotations

import math

import torch

from . import _lib as L

_DT = {"fp64": torch.float64, "mixed": torch.float32}
_PREC = {"fp64": L.CRK_FP64, "mixed": L.CRK_MIXED32}


def make_params(precision="mixed", **kw) -> L.crk_params:
    """Library defaults (gamma 5/3, Cl 2, Cq 1, eps2 0.01, eta_crit 1/n_h, eta_fold 0.2,
    no relaxation, limiter on) overridden by keyword."""
    p = L.crk_params_default()
    p.precision = _PREC[precision]
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


def _ptr(t):
    return None if t is None else t.data_ptr()


def _stream():
    return torch.cuda.current_stream().cuda_stream


class Solver:
    """Plan + workspace for up to ``n_max`` particles in ``n_boxes_max`` boxes."""

    def __init__(self, n_max: int, n_boxes_max: int = 1, precision: str = "mixed",
                 device=None, **params):
        if not torch.cuda.is_available():
            raise RuntimeError("libcrk needs a CUDA device; there is no CPU path")
        L.load()
        self.precision = precision
        self.dtype = _DT[precision]
        self.device = torch.device(device if device is not None else "cuda")
        self.params = make_params(precision, **params)
        self.n_max, self.nb_max = int(n_max), int(n_boxes_max)
        self.plan = L.crk_plan_create(self.params, self.n_max, self.nb_max)
        self.ws = None
        self.ws_bytes = 0
        self.n = 0
        self.nb = 1
        self._keep = []

    def __del__(self):
        try:
            L.crk_plan_destroy(self.plan)
        except Exception:
            pass

    # -- workspace ----------------------------------------------------------
    def _ensure_ws(self, n, nb):
        need = L.crk_workspace_size(self.plan, n, nb)
        if self.ws is None or self.ws_bytes < need:
            self.ws = torch.empty(need + 256, dtype=torch.uint8, device=self.device)
            self.ws_bytes = need
        base = self.ws.data_ptr()
        return base + ((-base) % 256)

    def _regrow(self, slots_per_particle):
        self.params.nbr_cap = int(slots_per_particle)
        L.crk_plan_destroy(self.plan)
        self.plan = L.crk_plan_create(self.params, self.n_max, self.nb_max)
        self.ws = None  # the layout changed

    # -- (a) cell build -----------------------------------------------------
    def cell_build(self, x, h, box_off=None, box_L=None, L_box=1.0, check=True):
        """Sort, build the tree and the neighbor lists.  With ``check`` the
        call synchronises once, raises on a device error and grows the
        neighbor-list capacity when it overflowed."""
        n = int(h.shape[0])
        assert x.dtype == torch.float64 and x.shape == (3, n) and x.is_contiguous()
        assert h.dtype == self.dtype and h.is_contiguous()
        if box_off is None:
            # single box: made once and reused (no host copy inside graph capture)
            key = (n, float(L_box))
            if getattr(self, "_box_key", None) != key:
                self._box_default = (
                    torch.tensor([0, n], dtype=torch.int64, device=self.device),
                    torch.tensor([float(L_box)], dtype=torch.float64, device=self.device))
                self._box_key = key
            box_off, box_L = self._box_default
        nb = int(box_off.shape[0]) - 1
        self._keep = [box_off, box_L]
        for _ in range(3):
            ws = self._ensure_ws(n, nb)
            rc = L.crk_cell_build(self.plan, _stream(), ws, self.ws_bytes, n, nb,
                                  box_off.data_ptr(), box_L.data_ptr(), x.data_ptr(),
                                  h.data_ptr())
            L.check(rc, "crk_cell_build")
            self.n, self.nb, self._wsp = n, nb, ws
            if not check:
                return self
            st = L.crk_stats_get(self.plan, _stream(), ws)
            code = L.crk_status_poll(self.plan, _stream(), ws)
            if code == L.CRK_ENOMEM and st.list_slots > st.list_capacity:
                self._regrow(int(math.ceil(st.list_slots * 1.05)) + 8)
                continue
            L.check(code, "crk_cell_build (device)")
            return self
        raise L.CRKError(L.CRK_ENOMEM, "crk_cell_build: neighbor-list capacity")

    # -- (b) moments ----------------------------------------------------------
    def moments(self, m, want_V=False, want_coef=False):
        n = self.n
        V = torch.empty(n, dtype=self.dtype, device=self.device) if want_V else None
        coef = torch.empty((16, n), dtype=self.dtype, device=self.device) if want_coef else None
        L.check(L.crk_moments(self.plan, _stream(), self._wsp, m.data_ptr(), _ptr(V), _ptr(coef)),
                "crk_moments")
        return V, coef

    # -- (c) rates ------------------------------------------------------------
    def rates(self, v, u, want_rho=False, want_gradv=False, out=None):
        n = self.n
        if out is None:
            dvdt = torch.empty((3, n), dtype=self.dtype, device=self.device)
            dudt = torch.empty(n, dtype=self.dtype, device=self.device)
        else:
            dvdt, dudt = out
        rho = torch.empty(n, dtype=self.dtype, device=self.device) if want_rho else None
        gv = torch.empty((9, n), dtype=self.dtype, device=self.device) if want_gradv else None
        L.check(L.crk_rates(self.plan, _stream(), self._wsp, v.data_ptr(), u.data_ptr(),
                            dvdt.data_ptr(), dudt.data_ptr(), _ptr(rho), _ptr(gv)), "crk_rates")
        return dvdt, dudt, rho, gv

    # -- (d) adjoint ----------------------------------------------------------
    def adjoint(self, v, u, g_dvdt, g_dudt, recompute=True, out=None):
        n = self.n
        if out is None:
            gx = torch.empty((3, n), dtype=self.dtype, device=self.device)
            gv = torch.empty((3, n), dtype=self.dtype, device=self.device)
            gu = torch.empty(n, dtype=self.dtype, device=self.device)
            gh = torch.empty(n, dtype=self.dtype, device=self.device)
        else:
            gx, gv, gu, gh = out
        L.check(L.crk_adjoint(self.plan, _stream(), self._wsp, v.data_ptr(), u.data_ptr(),
                              g_dvdt.data_ptr(), g_dudt.data_ptr(), gx.data_ptr(), gv.data_ptr(),
                              gu.data_ptr(), gh.data_ptr(), 1 if recompute else 0),
                "crk_adjoint")
        return gx, gv, gu, gh

    # -- inspection -------------------------------------------------------------
    def neighbors_csr(self, mode="gather"):
        n = self.n
        md = 0 if mode == "gather" else 1
        row = torch.zeros(n + 1, dtype=torch.int64, device=self.device)
        rc, nnz = L.crk_neighbors_csr(self.plan, _stream(), self._wsp, md, row.data_ptr(), None, 0)
        if rc not in (L.CRK_OK, L.CRK_ENOMEM):
            L.check(rc, "crk_neighbors_csr")
        col = torch.zeros(max(nnz, 1), dtype=torch.int32, device=self.device)
        rc, nnz = L.crk_neighbors_csr(self.plan, _stream(), self._wsp, md, row.data_ptr(),
                                      col.data_ptr(), col.numel())
        L.check(rc, "crk_neighbors_csr")
        return row, col[:nnz]

    def stats(self) -> dict:
        s = L.crk_stats_get(self.plan, _stream(), self._wsp)
        return {k: getattr(s, k) for k, _ in s._fields_ if k != "reserved"}

    def poll(self) -> int:
        return L.crk_status_poll(self.plan, _stream(), self._wsp)

    # -- autotuner ---------------------------------------------------------------
    def autotune(self, m, v, u, g_dvdt=None, g_dudt=None, repeats=3) -> dict:
        """Pick the fastest compiled launch variant of every sweep on this data
        (after cell_build); the plan keeps the choice.  Synchronises."""
        return L.crk_autotune(self.plan, _stream(), self._wsp, m.data_ptr(), v.data_ptr(),
                              u.data_ptr(), _ptr(g_dvdt), _ptr(g_dudt), repeats)

    # -- CUDA graph of a whole step ---------------------------------------------
    def capture(self, fn):
        """Capture ``fn`` (a sequence of this solver's calls with ``check=False``
        builds) into a CUDA graph and return it; replay with ``graph.replay()``.
        Every libcrk call is asynchronous and host-synchronisation free, so the
        whole step -- sort, tree, lists, all sweeps -- becomes one graph."""
        side = torch.cuda.Stream(device=self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(side):
            fn()  # warm-up on a side stream, as torch requires before capture
        torch.cuda.current_stream(self.device).wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        return g

    # -- one call for the whole forward path ------------------------------------
    def forward(self, x, h, m, v, u, box_off=None, box_L=None, L_box=1.0, **want):
        self.cell_build(x, h, box_off, box_L, L_box)
        V, coef = self.moments(m, want.get("want_V", False), want.get("want_coef", False))
        dvdt, dudt, rho, gv = self.rates(v, u, want.get("want_rho", False),
                                         want.get("want_gradv", False))
        return dict(V=V, coef=coef, dvdt=dvdt, dudt=dudt, rho=rho, gradv=gv)


class CRKRates(torch.autograd.Function):
    """(dv/dt, du/dt) = CRKSPH rates of (x, v, u, h) with masses m; the backward
    pass is libcrk's adjoint (no per-pair storage; forward state is reused)."""

    @staticmethod
    def forward(ctx, x, v, u, h, m, solver: Solver, box_off=None, box_L=None, L_box=1.0):
        solver.cell_build(x.detach(), h.detach(), box_off, box_L, L_box)
        solver.moments(m.detach())
        dvdt, dudt, _, _ = solver.rates(v.detach(), u.detach())
        ctx.solver = solver
        ctx.save_for_backward(v, u)
        return dvdt, dudt

    @staticmethod
    def backward(ctx, g_dvdt, g_dudt):
        v, u = ctx.saved_tensors
        s = ctx.solver
        if g_dvdt is None:
            g_dvdt = torch.zeros((3, s.n), dtype=s.dtype, device=s.device)
        if g_dudt is None:
            g_dudt = torch.zeros(s.n, dtype=s.dtype, device=s.device)
        gx, gv, gu, gh = s.adjoint(v.detach(), u.detach(), g_dvdt.contiguous(),
                                   g_dudt.contiguous(), recompute=True)
        return gx.to(torch.float64), gv, gu, gh, None, None, None, None, None


def rates(x, v, u, h, m, solver: Solver, box_off=None, box_L=None, L_box=1.0):
    """Differentiable CRKSPH rates; see :class:`CRKRates`."""
    return CRKRates.apply(x, v, u, h, m, solver, box_off, box_L, L_box)
