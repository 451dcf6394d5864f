#!/usr/bin/env python
"""Benchmark: CRKSPH pair interactions per second on GB300.

One step = one pass of the whole hot path on one batch of synthetic gas:
cell build (sort, tree, neighbor lists) -> volume and RK coefficients ->
density, velocity gradient and pair rates -> adjoint of the rates.  The unit is
the ordered gather pair (j != i, |x_ij| < h_i) counted once per step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on the host cores instead (the arm the GPU path is compared against).
"""
from __future__ import annotations

import argparse
import math
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "CRKSPH pair interactions/s (fwd+adjoint step) on 1 GB300"
UNIT = "pair interactions/s"
# the largest single-GPU configuration (one 256^3 box) is the headline; the
# clustered 64^3 box is reported beside it
WORKLOAD = "lognormal256"
SMALL_WORKLOAD = "lognormal64"
WORKLOAD_DESCS = {
    "lognormal256": ("256^3 = 16,777,216 gas particles in one periodic unit box, lognormal "
                     "density (P(k)~k^-2 field, variance 1.5, seed 5), h for 100+-10 neighbors, "
                     "u lognormal over 3 decades"),
    "lognormal64": ("64^3 = 262,144 gas particles, lognormal density (P(k)~k^-2 field, variance "
                    "1.5, seed 1), h for 100+-10 neighbors, u lognormal over 3 decades, periodic "
                    "unit box"),
}
# boxes above this size are timed on the CPU through a region sample
REGION_SAMPLE_ABOVE = 1 << 21

# Algorithmic flops per unit of each sweep: the oracle's own operation count
# (add, subtract, multiply, divide, sqrt, exp = 1; oracle.count_ops), per unit
# of the sweep, averaged over the 32^3 clustered box (the 64^3 box gives the
# same to 0.3 %).  Units: ordered union pairs for the rates and their adjoint,
# ordered gather pairs (j != i) for the others.  A forward sweep counts the
# operations of its stage of the oracle (per-particle work included); the
# adjoint sweep of a stage counts that stage's forward operations, which it
# recomputes, plus the derivative operations of the oracle's forward-mode
# differentiation of the stage (one tangent).  tests/test_flop_counts.py
# recounts them.
FLOPS_RECOMPUTE = {"b1_volume": 30, "b2_moments": 215, "c1_density": 131, "c2_rates": 317,
                   "adj_c2": 317, "adj_c1": 131, "adj_b2": 215, "adj_b1": 30}
FLOPS_DERIVATIVE = {"b1_volume": 0, "b2_moments": 0, "c1_density": 0, "c2_rates": 0,
                    "adj_c2": 720, "adj_c1": 302, "adj_b2": 505, "adj_b1": 64}
FLOPS_PER_PAIR = {k: FLOPS_RECOMPUTE[k] + FLOPS_DERIVATIVE[k] for k in FLOPS_RECOMPUTE}
# The kernels' own tally of the expressions they evaluate (reduced moment
# sums, intermediates shared between the forward recompute and the reverse):
# lower than the oracle's count; reported beside it.
FLOPS_KERNEL_TALLY = {"b1_volume": 31, "b2_moments": 114, "c1_density": 117, "c2_rates": 253,
                      "adj_c2": 654, "adj_c1": 511, "adj_b2": 458, "adj_b1": 93}
UNIT_OF = {"b1_volume": "gather", "b2_moments": "gather", "c1_density": "gather",
           "c2_rates": "union", "adj_c2": "union", "adj_c1": "gather", "adj_b2": "gather",
           "adj_b1": "gather"}
# FP32 lanes x 2 flops x SMs x max SM clock (152 SMs, 128 FP32 lanes/SM, 2070 MHz)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


# kernel names of the sweeps as they appear in ncu captures (profiles/*.md)
PROFILE_KERNEL = {"b1_volume": "PassB1<float", "b2_moments": "PassB2<float",
                  "c1_density": "PassC1<float", "c2_rates": "PassC2<float",
                  "adj_c2": "PassA2<float", "adj_c1": "PassA1<float", "adj_b2": "PassAB2<float",
                  "adj_b1": "PassAB1<float"}


def _profile_of(kernel: str, workload: str, need=None):
    """(path, metadata, table rows) of the committed ncu summary of ``kernel``
    on ``workload``, only if it was taken on the current sources (same build
    digest); ``need`` names a metadata field the summary must carry."""
    import glob
    from paper_2511_21921_gb300 import build as B
    want = PROFILE_KERNEL.get(kernel)
    if not want:
        return None
    digest = B._digest()
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        meta, rows = {}, {}
        with open(path) as fh:
            for line in fh:
                if ":" in line and line.split(":", 1)[0] in ("kernel", "build_digest", "workload",
                                                            "dram_bytes_per_launch"):
                    k, v = line.split(":", 1)
                    meta[k] = v.strip()
                elif line.startswith("| ") and line.count("|") == 3:
                    k, v = [c.strip() for c in line.strip().strip("|").split("|")]
                    rows[k] = v
        if (want in meta.get("kernel", "") and meta.get("build_digest") == digest and
                meta.get("workload") == workload and (need is None or need in meta)):
            return path, meta, rows
    return None


def profiled_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of ``kernel`` on ``workload`` from a committed ncu
    summary, only if that summary was taken on the current sources."""
    p = _profile_of(kernel, workload, need="dram_bytes_per_launch")
    return int(p[1]["dram_bytes_per_launch"]) if p else None


def profiled_limiter(kernel: str, workload: str):
    """The busiest on-chip unit of ``kernel`` in its committed ncu summary (same
    build digest): L1 throughput, issue activity and FMA-pipe activity, in %.
    A full-size workload is captured for DRAM bytes only (one pass), so its
    on-chip figures come from the same kernel's full capture on the small box."""
    p = None
    for wl in (workload, SMALL_WORKLOAD):
        p = _profile_of(kernel, wl)
        if p and "L1 throughput, %" in p[2]:
            break
        p = None
    if not p:
        return None
    path, _, rows = p

    def pct(label):
        v = rows.get(label, "").split()
        try:
            return round(float(v[0]), 1)
        except (IndexError, ValueError):
            return None
    return {"l1_throughput_pct": pct("L1 throughput, %"), "issue_active_pct": pct("issue active, %"),
            "fma_pipe_pct": pct("FMA pipe active, %"), "workload": p[1].get("workload"),
            "source": os.path.relpath(path, ROOT)}


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


# ---------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region.

    The GPU is addressed by its UUID (``nvidia-smi --id`` uses the physical
    numbering, which CUDA_VISIBLE_DEVICES does not change), and only samples
    whose timestamps fall between ``mark_start`` and ``mark_stop`` count."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device=None, out_dir=None):
        self.proc = None
        self.gpu = self.device_id(device)
        self.path = None
        self.out_dir = out_dir
        self.t0 = self.t1 = None

    @staticmethod
    def device_id(device):
        """UUID of a torch device in the form nvidia-smi takes (GPU-...), or
        the index when the UUID is not available."""
        try:
            import torch
            u = str(torch.cuda.get_device_properties(device).uuid)
            return u if u.startswith("GPU-") else "GPU-" + u
        except Exception:
            return str(getattr(device, "index", 0) or 0)

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv", prefix="clocks_")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv",
                 "-lms", "50"], stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def mark_start(self):
        self.t0 = time.time()

    def mark_stop(self):
        self.t1 = time.time()

    @staticmethod
    def _when(ts):
        import datetime
        for fmt in ("%Y/%m/%d %H:%M:%S.%f", "%Y/%m/%d %H:%M:%S"):
            try:
                return datetime.datetime.strptime(ts.strip(), fmt).timestamp()
            except ValueError:
                pass
        return None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh.read().splitlines()[1:]:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 10:
                    continue
                try:
                    sm = float(parts[2].split()[0])
                    smax = float(parts[3].split()[0])
                except ValueError:
                    continue
                rows.append((self._when(parts[0]), sm, smax, parts[6], parts[7], parts[8], parts[9]))
        try:
            if self.out_dir:
                os.makedirs(self.out_dir, exist_ok=True)
                os.replace(self.path, os.path.join(self.out_dir, "clocks.csv"))
            else:
                os.remove(self.path)
        except OSError:
            pass
        if not rows:
            return None
        inside = [r for r in rows if r[0] is not None and self.t0 is not None and
                  self.t1 is not None and self.t0 <= r[0] <= self.t1]
        use = inside if inside else rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in use for k in range(4) if r[3 + k] == "Active"})
        return {"sm_mhz": statistics.median(r[1] for r in use),
                "sm_max_mhz": max(r[2] for r in use), "reasons": reasons,
                "samples": len(rows), "samples_in_timed_region": len(inside),
                "gpu": self.gpu,
                "region": "samples inside the timed region" if inside else
                          "no sample fell inside the timed region: all samples"}


# ---------------------------------------------------------------------------- GPU arm
def run_ours(args, rank, world, workload=None, light=False):
    """The GPU arm on ``workload`` (default: the command line's).  ``light``
    times the graph-replayed step and its kernels only (the 64^3 box reported
    beside the headline)."""
    import torch
    from paper_2511_21921_gb300 import synth
    from paper_2511_21921_gb300 import _lib as L
    from paper_2511_21921_gb300.solver import Solver, copy_

    from paper_2511_21921_gb300 import dist as D
    dev = torch.device("cuda", _env_int("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    name = workload or args.workload
    # independent boxes are sharded whole across ranks; one box is replicated
    d = D.shard_workload(synth.load(name), rank, world)
    n = d["h"].shape[0]
    prec = args.precision
    dt = torch.float32 if prec == "mixed" else torch.float64
    gx_h, gu_h = synth.cotangents(n, seed=4)
    # pinned host copies (end-to-end leg) and resident device copies
    host = {"x": torch.tensor(d["x"], dtype=torch.float64).pin_memory()}
    for k in ("h", "m", "u"):
        host[k] = torch.tensor(d[k], dtype=dt).pin_memory()
    host["v"] = torch.tensor(d["v"], dtype=dt).pin_memory()
    host["ga"] = torch.tensor(gx_h, dtype=dt).pin_memory()
    host["gu"] = torch.tensor(gu_h, dtype=dt).pin_memory()
    dv = {k: t.to(dev) for k, t in host.items()}
    nb = 1
    boxes = (None, None)
    if "box_off" in d:  # many independent boxes in one call
        nb = len(d["box_off"]) - 1
        boxes = (torch.tensor(d["box_off"], dtype=torch.int64, device=dev),
                 torch.tensor(d["box_L"], dtype=torch.float64, device=dev))
    s = Solver(n, nb, prec, device=dev, prefetch=args.prefetch)
    s.cell_build(dv["x"], dv["h"], *boxes, check=True)  # sizes the neighbor lists once
    st0 = s.stats()
    pairs = st0["gather_pairs"]
    upairs = st0["union_pairs"]
    outs = (torch.empty((3, n), dtype=dt, device=dev), torch.empty(n, dtype=dt, device=dev))
    grads = tuple(torch.empty(sh, dtype=dt, device=dev) for sh in ((3, n), (3, n), (n,), (n,)))
    with_adj = not args.fwd_only

    def step(src):
        s.cell_build(src["x"], src["h"], *boxes, check=False)
        s.moments(src["m"])
        s.rates(src["v"], src["u"], out=outs)
        if with_adj:
            s.adjoint(src["v"], src["u"], src["ga"], src["gu"], recompute=False, out=grads)

    tuned = None
    if args.tune:  # a stored autotuner choice (8 variants in the order of _lib.SWEEPS)
        s.tune_set([int(c) for c in args.tune.split(",")])
    elif args.autotune:
        tuned = s.autotune(dv["m"], dv["v"], dv["u"], dv["ga"] if with_adj else None,
                           dv["gu"] if with_adj else None, repeats=3)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        step(dv)
    torch.cuda.synchronize()
    if s.poll() != 0:
        raise RuntimeError("device status set during warm-up")

    def timed(fn, k_steps, flush_l2=True):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(k_steps)]
        for k in range(k_steps):
            if flush_l2:
                flush.fill_(k & 0xff)
            evs[k][0].record(stream)
            fn()
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs]

    # the whole step captured once as a CUDA graph and replayed per timed step
    l0 = s.stats()["launches"]
    step(dv)
    per_step_launches = s.stats()["launches"] - l0
    graph = s.capture(lambda: step(dv)) if args.graph else None
    run = graph.replay if graph is not None else (lambda: step(dv))
    for _ in range(2):
        run()
    torch.cuda.synchronize()
    ms_eager = timed(lambda: step(dv), max(3, args.steps // 4))

    # CRK_CLOCKS_DIR (optional): a folder that receives the raw clock samples
    sampler = ClockSampler(dev, out_dir=os.environ.get("CRK_CLOCKS_DIR") or None)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    sampler.mark_start()
    ms = timed(run, args.steps)
    sampler.mark_stop()
    launches = per_step_launches * args.steps
    clocks = sampler.stop()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    step_ms = D.max_over_ranks(sum(ms) / len(ms), device=dev)
    job_pairs = D.sum_over_ranks(pairs, device=dev)
    status = s.poll()

    def kernel_times(nk):
        """Mean per-launch milliseconds of every library phase over ``nk`` steps
        (library CUDA events on the launching stream)."""
        L.crk_timing_enable(s.plan, True)
        kt = {}
        for k in range(nk):
            flush.fill_(k & 0xff)
            step(dv)
            for nm, t in L.crk_timing_read(s.plan):
                kt.setdefault(nm, []).append(t)
        L.crk_timing_enable(s.plan, False)
        return {k: sum(v) / len(v) for k, v in kt.items()}

    def roofline_of(kmean, alu_fp32=None):
        units = {"gather": pairs, "union": upairs}
        dom = max((k for k in kmean if k in FLOPS_PER_PAIR), key=lambda k: kmean[k])
        achieved = FLOPS_PER_PAIR[dom] * units[UNIT_OF[dom]] / (kmean[dom] * 1e-3) / 1e12
        per_kernel = {k: round(FLOPS_PER_PAIR[k] * units[UNIT_OF[k]] / (kmean[k] * 1e-3) / 1e12, 3)
                      for k in kmean if k in FLOPS_PER_PAIR}
        tally = FLOPS_KERNEL_TALLY[dom] * units[UNIT_OF[dom]] / (kmean[dom] * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": dom, "achieved": round(achieved, 3),
                "peak": round(FP32_PEAK_TFLOPS, 2), "unit": "TFLOP/s",
                "frac": round(achieved / FP32_PEAK_TFLOPS, 4),
                "traffic": profiled_traffic(dom, name),
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz",
                "flops_per_pair": FLOPS_PER_PAIR[dom],
                "flops_per_pair_split": {"recompute": FLOPS_RECOMPUTE[dom],
                                         "derivative": FLOPS_DERIVATIVE[dom]},
                "flops_source": "the oracle's operation count of the formulas (oracle.count_ops)",
                "pairs": units[UNIT_OF[dom]],
                "kernel_ms": round(kmean[dom], 4),
                "frac_of_measured_fp32": round(achieved / alu_fp32, 4) if alu_fp32 else None,
                "kernel_tally": {"flops_per_pair": FLOPS_KERNEL_TALLY[dom],
                                 "achieved": round(tally, 3),
                                 "frac": round(tally / FP32_PEAK_TFLOPS, 4)},
                "on_chip": profiled_limiter(dom, name)}
        return roof, per_kernel

    if light:
        kmean = kernel_times(max(3, min(args.steps, 20)))
        roof, per_kernel = roofline_of(kmean)
        return {"workload": WORKLOAD_DESCS.get(name, name), "name": name, "n": n,
                "gather_pairs": pairs, "union_pairs": upairs,
                "value": job_pairs / (step_ms * 1e-3), "unit": UNIT,
                "ms_per_step": round(step_ms, 4), "steps": args.steps,
                "ms_per_step_median": round(float(np.median(ms)), 4),
                "roofline": roof, "kernel_ms": {k: round(v, 4) for k, v in sorted(kmean.items())},
                "kernel_tflops": per_kernel, "gpu_launches": launches, "clocks": clocks,
                "autotune": {k: v["variant"] for k, v in tuned.items()} if tuned else None,
                "device_status": status}, pairs

    # end to end: pinned host inputs -> device, step, results -> pinned host
    out_h = (torch.empty((3, n), dtype=dt).pin_memory(), torch.empty(n, dtype=dt).pin_memory())
    grad_h = tuple(torch.empty(g.shape, dtype=dt).pin_memory() for g in grads)
    stage = {k: torch.empty_like(t) for k, t in dv.items()}

    # the staging copies go through crk_copy (copy_): the SMs move the bytes,
    # which keeps the host link's rate right after a step, where a copy engine
    # falls to a tenth of it
    def e2e_step():
        for k, t in host.items():
            copy_(stage[k], t)
        step(stage)
        copy_(out_h[0], outs[0])
        copy_(out_h[1], outs[1])
        if with_adj:
            for a, b in zip(grad_h, grads):
                copy_(a, b)

    # The same step with the copies a step does not wait for taken off its
    # path: positions and smoothing lengths go in first (the cell build needs
    # only them) and the other inputs follow on a side stream (copy engine)
    # while the lists are built; the rates go out on the side stream while the
    # adjoint runs.  The step ends when its last copy has landed.
    side = torch.cuda.Stream(device=dev)
    ev_in, ev_rates, ev_out = torch.cuda.Event(), torch.cuda.Event(), torch.cuda.Event()
    late = [k for k in host if k not in ("x", "h")]

    def e2e_step_overlap():
        cur = torch.cuda.current_stream()
        copy_(stage["x"], host["x"])
        copy_(stage["h"], host["h"])
        side.wait_stream(cur)  # the previous step is done with the staged inputs
        with torch.cuda.stream(side):
            for k in late:
                stage[k].copy_(host[k], non_blocking=True)
            ev_in.record(side)
        s.cell_build(stage["x"], stage["h"], *boxes, check=False)
        cur.wait_event(ev_in)
        s.moments(stage["m"])
        s.rates(stage["v"], stage["u"], out=outs)
        ev_rates.record(cur)
        side.wait_event(ev_rates)
        with torch.cuda.stream(side):
            out_h[0].copy_(outs[0], non_blocking=True)
            out_h[1].copy_(outs[1], non_blocking=True)
            ev_out.record(side)
        if with_adj:
            s.adjoint(stage["v"], stage["u"], stage["ga"], stage["gu"], recompute=False, out=grads)
            for a, b in zip(grad_h, grads):
                copy_(a, b)
        cur.wait_event(ev_out)  # the rates have landed before the next step overwrites them

    h2d = sum(t.numel() * t.element_size() for t in host.values())
    d2h = sum(t.numel() * t.element_size() for t in out_h)
    if with_adj:
        d2h += sum(t.numel() * t.element_size() for t in grad_h)
    e2e_step()  # warm-up: first use of the staging buffers and the copy kernels
    torch.cuda.synchronize()
    e2e_ms = timed(e2e_step, max(3, args.steps // 4))
    e2e_mean = sum(e2e_ms) / len(e2e_ms)
    e2e_step_overlap()
    torch.cuda.synchronize()
    e2e_ov_ms = timed(e2e_step_overlap, max(3, args.steps // 4))
    e2e_ov_mean = sum(e2e_ov_ms) / len(e2e_ov_ms)

    # the same loop as a user would pipeline it: the inputs of step k+1 are
    # copied in and the results of step k-1 copied out (two copy streams,
    # double buffers) while step k computes; wall time of all steps
    pipe = None
    if world == 1:
        h2d_s, d2h_s = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
        stg = [{k: torch.empty_like(t) for k, t in dv.items()} for _ in range(2)]
        obuf = [(torch.empty_like(outs[0]), torch.empty_like(outs[1])) +
                tuple(torch.empty_like(g) for g in grads) for _ in range(2)]
        hbuf = [tuple(torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in ob) for ob in obuf]
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_done = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]
        for e in ev_done + ev_out:
            e.record(stream)

        def pstep(b):
            sb, ob = stg[b], obuf[b]
            s.cell_build(sb["x"], sb["h"], *boxes, check=False)
            s.moments(sb["m"])
            s.rates(sb["v"], sb["u"], out=ob[:2])
            if with_adj:
                s.adjoint(sb["v"], sb["u"], sb["ga"], sb["gu"], recompute=False, out=ob[2:])

        def issue_in(b):
            with torch.cuda.stream(h2d_s):
                h2d_s.wait_event(ev_done[b])  # the step that last read buffer b is done
                for k, t in host.items():
                    stg[b][k].copy_(t, non_blocking=True)
                ev_in[b].record(h2d_s)

        def run_pipe(k_steps):
            issue_in(0)
            for k in range(k_steps):
                b = k & 1
                if k + 1 < k_steps:
                    issue_in(b ^ 1)
                stream.wait_event(ev_in[b])
                stream.wait_event(ev_out[b])  # results of step k-2 are out of buffer b
                if pgraphs is not None:
                    pgraphs[b].replay()
                else:
                    pstep(b)
                ev_done[b].record(stream)
                with torch.cuda.stream(d2h_s):
                    d2h_s.wait_event(ev_done[b])
                    nout = 2 + (4 if with_adj else 0)
                    for hh, dd in zip(hbuf[b][:nout], obuf[b][:nout]):
                        hh.copy_(dd, non_blocking=True)
                    ev_out[b].record(d2h_s)
            stream.wait_stream(d2h_s)
            stream.wait_stream(h2d_s)

        # one captured graph per buffer set, as for the device-timed step
        pgraphs = None
        if args.graph:
            for b in range(2):
                for k, t in dv.items():
                    stg[b][k].copy_(t)
            pgraphs = [s.capture(lambda b=b: pstep(b)) for b in range(2)]
        run_pipe(3)
        torch.cuda.synchronize()
        kp = max(3, args.steps // 4)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        run_pipe(kp)
        t1.record(stream)
        torch.cuda.synchronize()
        pms = t0.elapsed_time(t1) / kp
        pipe = {"value": pairs / (pms * 1e-3), "unit": UNIT, "ms_per_step": round(pms, 4),
                "steps": kp, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "how": "inputs of step k+1 copied in and results of step k-1 copied out on two "
                       "copy streams while step k computes (double buffers, one graph per "
                       "buffer set); no L2 flush: each step's lists and records (> 300 MB) "
                       "exceed L2"}

    # the same step with the fused rates + adjoint call (cotangents known in
    # advance): the adjoint's pair sweep also forms the rates
    fused = None
    if with_adj and nb == 1:
        fout = (outs[0], outs[1]) + grads

        def fstep():
            s.cell_build(dv["x"], dv["h"], *boxes, check=False)
            s.moments(dv["m"])
            s.rates_adjoint(dv["v"], dv["u"], dv["ga"], dv["gu"], out=fout)
        fstep()
        fgraph = s.capture(fstep) if args.graph else None
        frun = fgraph.replay if fgraph is not None else fstep
        for _ in range(2):
            frun()
        fms = timed(frun, max(3, min(args.steps, 50)))
        fmean = sum(fms) / len(fms)
        fused = {"ms_per_step": round(fmean, 4), "value": pairs / (fmean * 1e-3),
                 "step": "build+moments+rates_adjoint (fused rates and adjoint sweep)"}

    # the step without the cell build: moments, rates and adjoint over the
    # lists of the last build (what a caller that reuses the lists pays)
    def nbstep():
        s.moments(dv["m"])
        s.rates(dv["v"], dv["u"], out=outs)
        if with_adj:
            s.adjoint(dv["v"], dv["u"], dv["ga"], dv["gu"], recompute=False, out=grads)
    step(dv)
    nbgraph = s.capture(nbstep) if args.graph else None
    nbrun = nbgraph.replay if nbgraph is not None else nbstep
    for _ in range(2):
        nbrun()
    nbms = timed(nbrun, max(3, min(args.steps, 50)))
    nbmean = sum(nbms) / len(nbms)
    no_build = {"ms_per_step": round(nbmean, 4), "value": pairs / (nbmean * 1e-3),
                "step": "moments+rates" + ("+adjoint" if with_adj else "") +
                        " over the lists of the last build"}

    # per-kernel durations (library CUDA events on the launching stream)
    kmean = kernel_times(max(3, min(args.steps, 20)))
    fwd_names = ("build.check", "build.keys_sort", "build.tree", "build.lists", "pack_b1",
                 "b1_volume", "b2_moments", "pack_c1", "c1_density", "c2_rates")
    fwd_ms = sum(kmean.get(k, 0.0) for k in fwd_names)
    # measured FMA-chain rates (same clocks and power state as the sweeps)
    f32, _ = L.crk_alu_peak(stream.cuda_stream, False, 16384)
    f64, _ = L.crk_alu_peak(stream.cuda_stream, True, 512)
    alu_peak = {"fp32_tflops": round(f32 / 1e12, 3), "fp64_tflops": round(f64 / 1e12, 4),
                "fp32_over_fp64": round(f32 / f64, 1) if f64 > 0 else None,
                "method": "FMA chains, 8 per thread, 8 x 256 threads per SM, best of 3"}
    roofline, per_kernel_tflops = roofline_of(kmean, alu_peak["fp32_tflops"])
    res = {
        "metric": METRIC, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(step_ms, 4),
        "ms_per_step_median": round(float(np.median(ms)), 4),
        "value": job_pairs / (step_ms * 1e-3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == "mixed" else "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_DESCS.get(name, name),
                   "name": name, "n": n, "boxes": nb,
                   "gather_pairs": pairs, "union_pairs": upairs,
                   "precision": prec, "step": "build+moments+rates" + ("+adjoint" if with_adj
                                                                       else ""),
                   "l2": "flushed (256 MB write) before every timed step",
                   "parallelism": f"replica x{world}" if world > 1 else "1 GPU"},
        "e2e": {"value": job_pairs / (D.max_over_ranks(e2e_mean, device=dev) * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_steps": [round(x, 3) for x in e2e_ms],
                "copies": "crk_copy (SM-driven) from and to page-locked host memory"},
        "e2e_overlap": {"value": job_pairs / (D.max_over_ranks(e2e_ov_mean, device=dev) * 1e-3),
                        "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                        "ms_steps": [round(x, 3) for x in e2e_ov_ms],
                        "copies": "positions and h by crk_copy first; the other inputs and the rates "
                                  "by copy engine on a side stream under the list build and the "
                                  "adjoint; the gradients by crk_copy"},
        "e2e_pipelined": pipe,
        "gpu_launches": launches,
        "fused_rates_adjoint": fused,
        "autotune": {k: v["variant"] for k, v in tuned.items()} if tuned else None,
        "autotune_ms": {k: v["ms"] for k, v in tuned.items()} if tuned else None,
        "graph": bool(graph is not None),
        "eager_ms_per_step": round(sum(ms_eager) / len(ms_eager), 4),
        "fwd_pairs_per_s": pairs / (fwd_ms * 1e-3) if fwd_ms > 0 else None,
        "fwd_pairs_per_s_no_build": (pairs / ((fwd_ms - sum(kmean.get(k, 0.0) for k in
                                                             fwd_names if k.startswith("build.")))
                                              * 1e-3)) if fwd_ms > 0 else None,
        "no_build": no_build,
        "alu_peak_measured": alu_peak,
        "kernel_ms": {k: round(v, 4) for k, v in sorted(kmean.items())},
        "kernel_tflops": per_kernel_tflops,
        "roofline": roofline,
        "clocks": clocks,
        "device_status": status,
    }
    if args.hydro and world == 1:
        # the other rows of the path, on the clustered 64^3 box
        ds = synth.load(SMALL_WORKLOAD)
        res["other_rows_workload"] = SMALL_WORKLOAD
        res["hydro_step"] = hydro_step(args, ds, dev, flush)
        res["cooling"] = cooling_leg(args, ds, dev, flush)
        res["subgrid"] = subgrid_leg(args, ds, dev, flush)
        res["active_set"] = active_leg(args, ds, dev, flush)
    if args.fp64_compare and world == 1 and prec == "mixed":
        res["fp64_gpu"] = fp64_compare(args, d, dev)
        if res["fp64_gpu"]:
            res["speedup_vs_fp64_gpu"] = round(step_ms and res["fp64_gpu"]["ms_per_step"] /
                                               step_ms, 2)
    return res, pairs


def hydro_step(args, d, dev, flush):
    """One kick-drift-kick step (half kick, drift of x and h, cell build,
    moments, rates at the predicted velocity, smoothing-length rate, half kick)
    of the whole box, graph-replayed, each from the same initial state."""
    import torch
    from paper_2511_21921_gb300.solver import Solver
    n = d["h"].shape[0]
    prec = args.precision
    dt_ = torch.float32 if prec == "mixed" else torch.float64
    t = {"x": torch.tensor(d["x"], dtype=torch.float64, device=dev)}
    for k in ("h", "m", "u"):
        t[k] = torch.tensor(d[k], dtype=dt_, device=dev)
    t["v"] = torch.tensor(d["v"], dtype=dt_, device=dev)
    nh = (3.0 * 100 / (4.0 * math.pi)) ** (1.0 / 3.0)
    lam = 0.2
    s = Solver(n, 1, prec, device=dev, nbr_cap=320)
    gd = s.kdk_init(t["x"], t["v"], t["u"], t["h"], t["m"], 1e-3, lam, nh)
    step_dt = 0.1 * float((t["u"].double() / gd["du"].double().abs()).min())
    gd = s.kdk_init(t["x"], t["v"], t["u"], t["h"], t["m"], step_dt, lam, nh)
    if args.autotune:
        s.autotune(t["m"], t["v"], t["u"], repeats=2)
        gd = s.kdk_init(t["x"], t["v"], t["u"], t["h"], t["m"], step_dt, lam, nh)
    pairs = s.stats()["gather_pairs"]
    scratch = (torch.empty_like(t["v"]), torch.empty_like(t["u"]))
    # every timed step starts from the same state (a device copy inside the
    # graph): the synthetic velocity field is transonic in its cold regions,
    # so a fixed step taken again and again would run into negative energies
    saved = {k: v.clone() for k, v in t.items()}
    saved_d = {k: v.clone() for k, v in gd.items()}

    def step():
        for k in ("x", "v", "u", "h"):
            t[k].copy_(saved[k])
        for k, v in saved_d.items():
            gd[k].copy_(v)
        s.kdk_step(t["x"], t["v"], t["u"], t["h"], t["m"], gd, step_dt, lam, nh, check=False,
                   scratch=scratch)
    l0 = s.stats()["launches"]
    step()
    launches = s.stats()["launches"] - l0
    g = s.capture(step)
    stream = torch.cuda.current_stream()
    k_steps = max(3, min(args.steps, 20))
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(k_steps)]
    for k in range(k_steps):
        flush.fill_(k & 0xff)
        evs[k][0].record(stream)
        g.replay()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in evs]
    st = s.stats()
    status = s.poll()
    mean = sum(ms) / len(ms)
    # the step's rates run on the drifted state: count its pairs
    return {"ms_per_step": round(mean, 4), "pairs_per_s": st["gather_pairs"] / (mean * 1e-3),
            "steps": k_steps, "dt": step_dt, "restart": "state restored before each step", "lambda": lam, "n_h": round(nh, 4),
            "gather_pairs_first": pairs, "gather_pairs_last": st["gather_pairs"],
            "launches_per_step": launches, "device_status": status,
            "step": "kick+drift+build+moments+rates+hdot+kick (graph)"}


def cooling_leg(args, d, dev, flush):
    """Exact-integration cooling (Sec. 2.3.2) of the whole box over one step:
    a 0.004 dex table over six decades holding the self-similar law
    lam = A u^1.5 above an equilibrium and heating below it; rho from the
    density of the box's own rates evaluation."""
    import torch
    from paper_2511_21921_gb300.solver import Solver
    n = d["h"].shape[0]
    prec = args.precision
    dt_ = torch.float32 if prec == "mixed" else torch.float64
    s = Solver(n, 1, prec, device=dev)
    t = {"x": torch.tensor(d["x"], dtype=torch.float64, device=dev)}
    for k in ("h", "m", "u"):
        t[k] = torch.tensor(d[k], dtype=dt_, device=dev)
    t["v"] = torch.tensor(d["v"], dtype=dt_, device=dev)
    rho = s.forward(t["x"], t["h"], t["m"], t["v"], t["u"], want_rho=True)["rho"]
    lu0, dex, K = -3.0, 0.004, 1501
    un = 10.0 ** (lu0 + dex * np.arange(K))
    A, H = 1.0, 0.5
    lam = torch.tensor(A * un ** 1.5 - H, dtype=torch.float64, device=dev)
    dt = 0.1 / float(rho.double().median())   # typical energies move by a few to tens of bins
    out = torch.empty_like(t["u"])
    stream = torch.cuda.current_stream()
    for _ in range(3):
        s.cool(dt, rho, t["u"], lam, lu0, dex, out=out)
    k_steps = max(3, min(args.steps, 20))
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(k_steps)]
    for k in range(k_steps):
        flush.fill_(k & 0xff)
        evs[k][0].record(stream)
        s.cool(dt, rho, t["u"], lam, lu0, dex, out=out)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs) / k_steps
    bins = np.abs(np.log10(out.double().cpu().numpy() / d["u"])) / dex
    nbytes = 3 * n * (4 if prec == "mixed" else 8)
    return {"ms": round(ms, 5), "particles_per_s": n / (ms * 1e-3),
            "bytes_per_particle": nbytes // n, "hbm_gbs": nbytes / (ms * 1e-3) / 1e9,
            "bins_walked_median": float(np.median(bins)), "bins_walked_max": float(bins.max()),
            "table": "lam = u^1.5 - 0.5 over 1e-3..1e3, 0.004 dex", "dt_rho_median": 0.1}


def subgrid_leg(args, d, dev, flush):
    """Subgrid particles over the gas (App. A.2 Eq. Vsg; Eqs. windmetal,
    starmetal, AGNE): 5 % of the gas count as star particles, half spawned on
    gas positions and half at random points, h_s = 0.6 h of the local gas;
    their scatter volumes and a two-component normalised deposit, timed after
    one build + moments of the box."""
    import torch
    from paper_2511_21921_gb300.solver import Solver
    n = d["h"].shape[0]
    prec = args.precision
    dt_ = torch.float32 if prec == "mixed" else torch.float64
    rng = np.random.default_rng(11)
    n_s = n // 20
    pick = rng.choice(n, n_s // 2, replace=False)
    xs = np.concatenate([d["x"][:, pick], rng.uniform(0, 1, (3, n_s - n_s // 2))], axis=1)
    hs = np.concatenate([d["h"][pick], rng.uniform(0.5, 1.5, n_s - n_s // 2) *
                         np.median(d["h"])]) * 0.6
    s = Solver(n, 1, prec, device=dev)
    t = {"x": torch.tensor(d["x"], dtype=torch.float64, device=dev),
         "h": torch.tensor(d["h"], dtype=dt_, device=dev),
         "m": torch.tensor(d["m"], dtype=dt_, device=dev)}
    s.cell_build(t["x"], t["h"])
    s.moments(t["m"])
    xs_d = torch.tensor(xs, dtype=torch.float64, device=dev).contiguous()
    hs_d = torch.tensor(hs, dtype=dt_, device=dev)
    q = torch.ones((2, n_s), dtype=dt_, device=dev)
    dq = torch.zeros((2, n), dtype=dt_, device=dev)
    stream = torch.cuda.current_stream()
    res = {}
    for name, fn in (("volume", lambda: s.subgrid_volume(xs_d, hs_d, 2.25)),
                     ("deposit", lambda: s.subgrid_deposit(xs_d, hs_d, q, dq=dq))):
        for _ in range(3):
            fn()
        k_steps = max(3, min(args.steps, 20))
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(k_steps)]
        for k in range(k_steps):
            flush.fill_(k & 0xff)
            evs[k][0].record(stream)
            fn()
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in evs) / k_steps
        res[name + "_ms"] = round(ms, 5)
        res[name + "_per_s"] = n_s / (ms * 1e-3)
    res["n_subgrid"] = n_s
    res["device_status"] = s.poll()
    return res


def active_leg(args, d, dev, flush):
    """Active-set evaluation (App. A.1): one step of a time-bin hierarchy in
    which a quarter of the particles (whole tree leaves, chosen at random) is
    active; passive particles reuse their stored coefficients and fields.  The
    timed call is moments + rates over the active set after one build."""
    import torch
    from paper_2511_21921_gb300.solver import Solver
    n = d["h"].shape[0]
    prec = args.precision
    dt_ = torch.float32 if prec == "mixed" else torch.float64
    t = {"x": torch.tensor(d["x"], dtype=torch.float64, device=dev)}
    for k in ("h", "m", "u"):
        t[k] = torch.tensor(d[k], dtype=dt_, device=dev)
    t["v"] = torch.tensor(d["v"], dtype=dt_, device=dev)
    s = Solver(n, 1, prec, device=dev)
    s.cell_build(t["x"], t["h"])
    V, coef = s.moments(t["m"], want_V=True, want_coef=True)
    _, _, rho, gv = s.rates(t["v"], t["u"], want_rho=True, want_gradv=True)
    # leaves (8 consecutive sorted particles) drawn at random: mark one particle
    # per chosen leaf as transformed and let the library expand it
    rng = np.random.default_rng(12)
    flags = torch.zeros(n, dtype=torch.uint8, device=dev)
    _, leaf = s.leaf_mark(flags, want_leaf=True)
    lf = leaf.cpu().numpy()
    chosen = rng.uniform(size=lf.max() + 1) < 0.25
    fl = np.where(chosen[lf], 1, 0).astype(np.uint8)
    flags = torch.tensor(fl, device=dev)
    out = (torch.zeros((3, n), dtype=dt_, device=dev), torch.zeros(n, dtype=dt_, device=dev))
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(3):
            fn()
        k_steps = max(3, min(args.steps, 20))
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(k_steps)]
        for k in range(k_steps):
            flush.fill_(k & 0xff)
            evs[k][0].record(stream)
            fn()
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs) / k_steps

    def full():
        s.moments(t["m"])
        s.rates(t["v"], t["u"], out=out)

    def part():
        s.moments_active(t["m"], flags, V, coef)
        s.rates_active(t["v"], t["u"], rho, gv, out=out)
    ms_full = timed(full)
    ms_part = timed(part)
    return {"active_fraction": float(fl.mean()), "ms_active_set": round(ms_part, 4),
            "ms_all_active": round(ms_full, 4), "speedup": round(ms_full / ms_part, 3),
            "device_status": s.poll()}


def fp64_compare(args, d, dev):
    """The plain FP64 GPU form on the same workload (same step, fewer repeats)."""
    import torch
    from paper_2511_21921_gb300.solver import Solver
    from paper_2511_21921_gb300 import synth
    n = d["h"].shape[0]
    t64 = {k: torch.tensor(d[k], dtype=torch.float64, device=dev) for k in ("x", "h", "m", "u",
                                                                           "v")}
    ga, gu = synth.cotangents(n, seed=4)
    t64["ga"] = torch.tensor(ga, dtype=torch.float64, device=dev)
    t64["gu"] = torch.tensor(gu, dtype=torch.float64, device=dev)
    nb, boxes = 1, (None, None)
    if "box_off" in d:
        nb = len(d["box_off"]) - 1
        boxes = (torch.tensor(d["box_off"], dtype=torch.int64, device=dev),
                 torch.tensor(d["box_L"], dtype=torch.float64, device=dev))
    s = Solver(n, nb, "fp64", device=dev)
    s.cell_build(t64["x"], t64["h"], *boxes, check=True)

    def step():
        s.cell_build(t64["x"], t64["h"], *boxes, check=False)
        s.moments(t64["m"])
        s.rates(t64["v"], t64["u"])
        if not args.fwd_only:
            s.adjoint(t64["v"], t64["u"], t64["ga"], t64["gu"], recompute=False)

    big = n > REGION_SAMPLE_ABOVE  # a step of the FP64 form takes seconds there
    for _ in range(1 if big else 2):
        step()
    torch.cuda.synchronize()
    k = 2 if big else max(2, min(5, args.steps))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(k):
        step()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / k
    return {"ms_per_step": round(ms, 4), "value": s.stats()["gather_pairs"] / (ms * 1e-3),
            "steps": k}


# ---------------------------------------------------------------------------- CPU arm
def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_pass(d, with_derivative=True):
    """One oracle evaluation of the step: forward values and, for the adjoint
    part, the oracle's derivative pass (forward-mode JVP; it has no reverse).
    Returns (seconds, gather pairs per particle)."""
    import oracle
    n = d["h"].shape[0]
    t0 = time.perf_counter()
    if with_derivative:
        rng = np.random.default_rng(0)
        o, _ = oracle.jvp(d["x"], d["h"], d["m"], d["v"], d["u"], d["L"],
                          tx=rng.normal(size=(3, n)) * 1e-4, want=("dvdt", "dudt", "kgather"))
    else:
        o = oracle.forward(d["x"], d["h"], d["m"], d["v"], d["u"], d["L"],
                           want=("dvdt", "dudt", "kgather"))
    return time.perf_counter() - t0, o["kgather"]


def cpu_sample(name, side):
    """The oracle's input for a bounded sample of workload ``name``: the whole
    box when it is small, otherwise a cube of ``side`` (box units) at the box
    center with the particles its results depend on (synth.region_sample).
    Returns (input, owned mask, description)."""
    from paper_2511_21921_gb300 import synth
    d = synth.load(name)
    n = d["h"].shape[0]
    if n <= REGION_SAMPLE_ABOVE:
        return d, np.ones(n, dtype=bool), f"whole {name} workload"
    sub, own, _ = synth.region_sample(d, side)
    desc = (f"region of {name}: the {int(own.sum())} particles of a cube of side {side} at the "
            f"box center (owned) plus the {int((~own).sum())} within three times the largest "
            "smoothing length of them (ghosts, which the owned particles' rates depend on); "
            "the owned particles' results equal the whole box's; pairs counted = the owned "
            "particles' gather pairs")
    return sub, own, desc


def cpu_baseline(args, min_seconds=10.0, max_passes=20, side=0.3):
    """The oracle as it stands on the host cores: passes over a bounded sample of
    the benchmark workload (each one forward-mode pass with one JVP), repeated
    until about ten seconds of wall time have been spent."""
    import oracle
    d, own, desc = cpu_sample(args.workload, side)
    t, k, pairs = 0.0, 0, 0
    while k < max_passes and (k == 0 or t < min_seconds):
        dt_, kg = oracle_pass(d, not args.fwd_only)
        t += dt_
        pairs = int(kg[own].sum())
        k += 1
    return {"value": k * pairs / t, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{desc} ({pairs} pairs) x {k} passes, each one oracle forward pass with "
                      "one forward-mode derivative (JVP), FP64, OpenMP over particles",
            "seconds": round(t, 3)}


def reference_config(args):
    """The workload the reference arm samples, described as the GPU arm describes
    it: its whole-box pair counts are the oracle's (tests/golden/workload_pairs.json,
    written by the committed script beside it from oracle.count_pairs)."""
    cfg = {"workload": WORKLOAD_DESCS.get(args.workload, args.workload), "name": args.workload}
    path = os.path.join(ROOT, "tests", "golden", "workload_pairs.json")
    try:
        with open(path) as fh:
            w = json.load(fh)[args.workload]
    except (OSError, KeyError, ValueError):
        return cfg
    c = w["mixed" if args.precision == "mixed" else "fp64"]
    cfg.update({"n": w["n"], "boxes": w["boxes"], "gather_pairs": c["gather_pairs"],
                "union_pairs": c["union_pairs"],
                "step": "build+moments+rates" + ("" if args.fwd_only else "+adjoint")})
    return cfg


def run_reference(args):
    """Reference arm: the FP64 CPU oracle timed step by step on the host cores,
    each step one oracle pass over a bounded sample of the workload."""
    import oracle
    oracle.build()
    side = 0.2
    d, own, sample = cpu_sample(args.workload, side)
    _, kg = oracle_pass(d, not args.fwd_only)  # also warms the oracle
    pairs = int(kg[own].sum())
    for _ in range(max(0, args.warmup - 1)):
        oracle_pass(d, not args.fwd_only)
    ts = [oracle_pass(d, not args.fwd_only)[0] for _ in range(args.steps)]
    mean = sum(ts) / len(ts)
    val = pairs / mean
    cores = oracle.num_threads()
    return {
        "impl": "reference", "metric": METRIC, "unit": UNIT, "value": val,
        "higher_is_better": True, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(mean * 1e3, 3), "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": reference_config(args),
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample + "; forward values plus one JVP per step",
                         "sample_gather_pairs_per_step": pairs},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


# ---------------------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--fwd-only", action="store_true")
    ap.add_argument("--no-graph", dest="graph", action="store_false", default=True)
    ap.add_argument("--no-autotune", dest="autotune", action="store_false", default=True)
    ap.add_argument("--tune", default="",
                    help="set a stored autotuner choice instead of tuning: 8 comma-separated "
                         "variants (volume, moments, density, rates, adjoint rates, adjoint "
                         "density, adjoint moments, adjoint volume)")
    ap.add_argument("--prefetch", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-small", dest="small", action="store_false", default=True,
                    help="skip the 64^3 box reported beside the headline")
    ap.add_argument("--no-hydro", dest="hydro", action="store_false", default=True)
    ap.add_argument("--fp64-compare", action="store_true", default=True)
    ap.add_argument("--no-fp64-compare", dest="fp64_compare", action="store_false")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    res, _ = run_ours(args, rank, world)
    if args.small and world == 1 and args.workload != SMALL_WORKLOAD:
        res[SMALL_WORKLOAD], _ = run_ours(args, rank, world, workload=SMALL_WORKLOAD, light=True)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            res["cpu_baseline"] = cpu_baseline(args)
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
