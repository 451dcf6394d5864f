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


def copy_(dst: torch.Tensor, src: torch.Tensor) -> torch.Tensor:
    """``dst.copy_(src)`` for contiguous tensors of one dtype and shape through
    ``crk_copy`` (the SMs move the bytes) on the current stream: the staging
    copy between page-locked host memory and the device each step."""
    if dst.dtype != src.dtype or dst.shape != src.shape:
        raise ValueError("copy_: dtype and shape must match")
    if not (dst.is_contiguous() and src.is_contiguous()):
        raise ValueError("copy_: tensors must be contiguous")
    L.crk_copy(_stream(), dst.data_ptr(), src.data_ptr(), src.numel() * src.element_size())
    return dst


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

    def _boxes(self, n, box_off, box_L, L_box):
        if box_off is not None:
            return box_off, box_L
        # single box: made once and reused (no host copy inside graph capture)
        key = (n, float(L_box))
        if getattr(self, "_box_key", None) != key:
            self._box_default = (
                torch.tensor([0, n], dtype=torch.int64, device=self.device),
                torch.tensor([float(L_box)], dtype=torch.float64, device=self.device))
            self._box_key = key
        return self._box_default

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
        box_off, box_L = self._boxes(n, box_off, box_L, L_box)
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

    def rates_adjoint(self, v, u, g_dvdt, g_dudt, out=None):
        """Rates and their VJP for cotangents known in advance, in one pass
        structure (the adjoint's pair sweep also accumulates the rates)."""
        n = self.n
        if out is None:
            out = (torch.empty((3, n), dtype=self.dtype, device=self.device),
                   torch.empty(n, dtype=self.dtype, device=self.device),
                   torch.empty((3, n), dtype=self.dtype, device=self.device),
                   torch.empty((3, n), dtype=self.dtype, device=self.device),
                   torch.empty(n, dtype=self.dtype, device=self.device),
                   torch.empty(n, dtype=self.dtype, device=self.device))
        dvdt, dudt, gx, gv, gu, gh = out
        L.check(L.crk_rates_adjoint(self.plan, _stream(), self._wsp, v.data_ptr(), u.data_ptr(),
                                    g_dvdt.data_ptr(), g_dudt.data_ptr(), dvdt.data_ptr(),
                                    dudt.data_ptr(), gx.data_ptr(), gv.data_ptr(), gu.data_ptr(),
                                    gh.data_ptr()), "crk_rates_adjoint")
        return out

    # -- gas and wind ----------------------------------------------------------------
    def set_species(self, species):
        """Species of the last build's particles (uint8, 0 gas, nonzero wind);
        None returns to all gas.  Call after every cell_build."""
        L.check(L.crk_set_species(self.plan, _stream(), self._wsp, _ptr(species)),
                "crk_set_species")

    def volume_gw(self):
        out = torch.empty(self.n, dtype=self.dtype, device=self.device)
        L.check(L.crk_volume_gw(self.plan, _stream(), self._wsp, out.data_ptr()), "crk_volume_gw")
        return out

    # -- active-set evaluation (passive particles reuse their stored fields) -------
    def leaf_mark(self, flags, want_leaf=False):
        """Set bit 1 on the leaf-mates of transformed particles (bit 2), in place."""
        leaf = torch.empty(self.n, dtype=torch.int32, device=self.device) if want_leaf else None
        L.check(L.crk_leaf_mark(self.plan, _stream(), self._wsp, flags.data_ptr(), _ptr(leaf)),
                "crk_leaf_mark")
        return flags, leaf

    def time_bins(self, dt, dt_max, max_level, substep, flags=None):
        """Per-leaf power-of-two levels and the active bit for one sub-step."""
        level = torch.empty(self.n, dtype=torch.uint8, device=self.device)
        if flags is None:
            flags = torch.zeros(self.n, dtype=torch.uint8, device=self.device)
        L.check(L.crk_time_bins(self.plan, _stream(), self._wsp, dt.data_ptr(), dt_max, max_level,
                                substep, level.data_ptr(), flags.data_ptr()), "crk_time_bins")
        return level, flags

    def moments_active(self, m, flags, V_state, coef_state):
        L.check(L.crk_moments_active(self.plan, _stream(), self._wsp, m.data_ptr(),
                                     flags.data_ptr(), V_state.data_ptr(), coef_state.data_ptr()),
                "crk_moments_active")
        return V_state, coef_state

    def rates_active(self, v, u, rho_state, gradv_state, out=None):
        n = self.n
        if out is None:
            out = (torch.zeros((3, n), dtype=self.dtype, device=self.device),
                   torch.zeros(n, dtype=self.dtype, device=self.device))
        dvdt, dudt = out
        L.check(L.crk_rates_active(self.plan, _stream(), self._wsp, v.data_ptr(), u.data_ptr(),
                                   rho_state.data_ptr(), gradv_state.data_ptr(), dvdt.data_ptr(),
                                   dudt.data_ptr()), "crk_rates_active")
        return dvdt, dudt

    # -- (e)-(h) time step around the rates --------------------------------------
    def hdot(self, dt_a, lam, n_h, out=None):
        """(hdot, hdot/h, div v) of the last rates evaluation, caller order."""
        n = self.n
        if out is None:
            out = tuple(torch.empty(n, dtype=self.dtype, device=self.device) for _ in range(3))
        hd, hr, dv = out
        L.check(L.crk_hdot(self.plan, _stream(), self._wsp, dt_a, lam, n_h, _ptr(hd), _ptr(hr),
                           _ptr(dv)), "crk_hdot")
        return hd, hr, dv

    def kick(self, dt, v0, a, u0=None, dudt=None, v_out=None, u_out=None, active=None):
        """v0 + dt a (and u0 + dt dudt); in place when no outputs are given."""
        n = int(v0.shape[1])
        v_out = v0 if v_out is None else v_out
        if u0 is not None and u_out is None:
            u_out = u0
        L.check(L.crk_kick(self.plan, _stream(), n, dt, _ptr(active), v0.data_ptr(), a.data_ptr(),
                           v_out.data_ptr(), _ptr(u0), _ptr(dudt), _ptr(u_out)), "crk_kick")
        return v_out, u_out

    def kick_refined(self, dt_b, dt_c, v0, a0, a1, u0=None, du0=None, du1=None, v_out=None,
                     u_out=None, active=None):
        n = int(v0.shape[1])
        v_out = v0 if v_out is None else v_out
        if u0 is not None and u_out is None:
            u_out = u0
        L.check(L.crk_kick_refined(self.plan, _stream(), n, dt_b, dt_c, _ptr(active),
                                   v0.data_ptr(), a0.data_ptr(), a1.data_ptr(), v_out.data_ptr(),
                                   _ptr(u0), _ptr(du0), _ptr(du1), _ptr(u_out)),
                "crk_kick_refined")
        return v_out, u_out

    def drift(self, dt, x, v_half, a0=None, dt_a=None, t_elapse=None, h=None, hrate=None,
              n_h=0.0, V=None, rho=None, div=None, box_off=None, box_L=None, L_box=1.0):
        """In-place drift of x (and h, V, rho when given)."""
        n = int(x.shape[1])
        box_off, box_L = self._boxes(n, box_off, box_L, L_box)
        L.check(L.crk_drift(self.plan, _stream(), n, int(box_off.shape[0]) - 1, box_off.data_ptr(),
                            box_L.data_ptr(), dt, x.data_ptr(), v_half.data_ptr(), _ptr(a0),
                            _ptr(dt_a), _ptr(t_elapse), _ptr(h), _ptr(hrate), n_h, _ptr(V),
                            _ptr(rho), _ptr(div)), "crk_drift")
        return x

    # -- subgrid particles over the gas of the last build --------------------------
    def _sub_boxes(self, n_s, box_off_s):
        if box_off_s is not None:
            return box_off_s
        assert self.nb == 1, "pass box_off_s for a multi-box build"
        return torch.tensor([0, n_s], dtype=torch.int64, device=self.device)

    def subgrid_volume(self, x_s, h_s, n_h=2.25, box_off_s=None, want_h=True):
        """Scatter volumes of subgrid particles (and n_h V^(1/3))."""
        n_s = int(h_s.shape[0])
        bo = self._sub_boxes(n_s, box_off_s)
        V = torch.empty(n_s, dtype=self.dtype, device=self.device)
        h = torch.empty(n_s, dtype=self.dtype, device=self.device) if want_h else None
        L.check(L.crk_subgrid_volume(self.plan, _stream(), self._wsp, n_s, bo.data_ptr(),
                                     x_s.data_ptr(), h_s.data_ptr(), n_h, V.data_ptr(), _ptr(h)),
                "crk_subgrid_volume")
        return V, h

    def subgrid_deposit(self, x_s, h_s, q_s, eligible=None, box_off_s=None, dq=None):
        """Normalised kernel deposit of q_s (n_comp, n_s) into the gas; returns
        (dq (n_comp, n), A_s)."""
        n_s = int(h_s.shape[0])
        q_s = q_s.reshape(-1, n_s).contiguous()
        nc = int(q_s.shape[0])
        bo = self._sub_boxes(n_s, box_off_s)
        if dq is None:
            dq = torch.zeros((nc, self.n), dtype=self.dtype, device=self.device)
        A = torch.empty(n_s, dtype=self.dtype, device=self.device)
        L.check(L.crk_subgrid_deposit(self.plan, _stream(), self._wsp, n_s, bo.data_ptr(),
                                      x_s.data_ptr(), h_s.data_ptr(), nc, q_s.data_ptr(),
                                      _ptr(eligible), A.data_ptr(), dq.data_ptr()),
                "crk_subgrid_deposit")
        return dq, A

    def cool(self, dt, rho, u, lam, log10_u_min, dlog10_u, out=None):
        """Exact-integration cooling/heating over dt (lam: float64 device tensor
        of Lambda(u_k)/rho^2 at the table nodes)."""
        n = int(u.shape[0])
        assert lam.dtype == torch.float64 and lam.is_cuda and lam.is_contiguous()
        tab = L.crk_cool_table(int(lam.shape[0]), 0, float(log10_u_min), float(dlog10_u),
                               lam.data_ptr())
        out = torch.empty_like(u) if out is None else out
        L.check(L.crk_cool_exact(self.plan, _stream(), n, tab, dt, rho.data_ptr(), u.data_ptr(),
                                 out.data_ptr()), "crk_cool_exact")
        return out

    def kdk_init(self, x, v, u, h, m, dt_a, lam, n_h, box_off=None, box_L=None, L_box=1.0):
        """Rates and smoothing-length rate at the start of the first step."""
        self.cell_build(x, h, box_off, box_L, L_box)
        self.moments(m)
        a, du, _, _ = self.rates(v, u)
        _, hr, dv = self.hdot(dt_a, lam, n_h)
        return {"a": a, "du": du, "hrate": hr, "div": dv}

    def kdk_step(self, x, v, u, h, m, d, dt, lam, n_h, box_off=None, box_L=None, L_box=1.0,
                 check=True, scratch=None):
        """One global kick-drift-kick step of length dt, in place on x, v, u, h
        and on the derivative set d (rates and hrate of the previous
        evaluation in, of the new one out).  Half kick; drift of x and h; rates
        at the new positions with the predicted velocity and energy
        v_half + a dt/2, u_half + du dt/2; smoothing-length rate; half kick.
        With fixed tensors and check=False the step can be graph-captured."""
        half = 0.5 * dt
        if scratch is None:
            scratch = (torch.empty_like(v), torch.empty_like(u))
        v_p, u_p = scratch
        self.kick(half, v, d["a"], u, d["du"])
        self.drift(dt, x, v, h=h, hrate=d["hrate"], box_off=box_off, box_L=box_L, L_box=L_box)
        self.kick(half, v, d["a"], u, d["du"], v_out=v_p, u_out=u_p)
        self.cell_build(x, h, box_off, box_L, L_box, check=check)
        self.moments(m)
        self.rates(v_p, u_p, out=(d["a"], d["du"]))
        self.hdot(dt, lam, n_h, out=(None, d["hrate"], d["div"]))
        self.kick(half, v, d["a"], u, d["du"])
        return d

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

    def tune_set(self, choice) -> None:
        """Set the launch variant of every sweep without timing: ``choice`` is the
        dict ``autotune`` returned (replaying a stored choice) or eight ints in
        the order of ``_lib.SWEEPS``."""
        if isinstance(choice, dict):
            choice = [choice[k]["variant"] if isinstance(choice[k], dict) else choice[k]
                      for k in L.SWEEPS]
        L.crk_tune_set(self.plan, choice)

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
    def forward(self, x, h, m, v, u, box_off=None, box_L=None, L_box=1.0, species=None, **want):
        self.cell_build(x, h, box_off, box_L, L_box)
        if species is not None:
            self.set_species(species)
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
