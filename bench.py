#!/usr/bin/env python3
"""Benchmark: photon-packet cell-crossings/s (and ray-cell steps/s) of the
full Monte Carlo radiative-transfer step on one GB300.

One step = one pass of the hot path over the r^-2 shell model (128^3 cells,
tau(1 um) = 10, 64 frequencies, central 2500 K star): Bjorkman & Wood
transport of 1e7 packets in FP32 with FP64 energy accumulators, Lucy
deposits in thin cells and the scattering-event store; the Eq. 4 dust
temperatures; ray-traced images (5 inclinations x 12 frequencies x 256^2
pixels) and SEDs from the temperatures and the stored events.

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle on the
same workload (bounded packet samples on the host cores) instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "photon-packet cell-crossings/s"
UNIT = "crossings/s"
# DRAM bytes (read + write) of one full-size transport launch of this
# workload, from a single-pass ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum; the command is in the transport kernel's summary
# under profiles/); to be re-measured (or set to None) whenever the transport
# kernel changes
TRANSPORT_DRAM_BYTES = 32.065e6 + 31.657e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--packets", type=float, default=1e7)
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--tau", type=float, default=10.0)
    ap.add_argument("--npix", type=int, default=256)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--forms", default="", help="measure other forms instead of the step: "
                    "all or a comma list of fp64_debug, plain_fp32, mrw_disk, adjoint, batched, "
                    "refined_shell, next_rows")
    return ap.parse_args()


def workload_config(a, extra=None):
    cfg = {"workload": f"r^-2 spherical shell {a.n}^3, tau(1um)={a.tau:g}, 64 freq 0.1-1000um, "
                       f"2500 K star; {a.packets:.0e} packets B&W FP32+FP64 acc, Lucy thin, "
                       f"events; Eq.4 temperatures; images 5 incl x 12 freq x {a.npix}^2",
           "grid": a.n, "n_packets": int(a.packets), "n_freq": 64, "mode": "bjorkman-wood",
           "images": [5, 12, a.npix], "l2": "flushed between steps (512 MiB write)"}
    if extra:
        cfg.update(extra)
    return cfg


def build_model(a):
    import workloads as W
    return W.r2_shell(n=a.n, tau_1um=a.tau, nf=64)


def image_setup(m, a):
    import math as _m
    import workloads as W
    fidx = W.nearest_freq_indices(m.nu, W.image_wavelengths_um())
    D = 140 * W.PC
    cams = [W.Camera(_m.radians(t), 0.0, a.npix, D) for t in W.inclinations_deg()]
    return cams, fidx


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(self.rows)}


def cpu_baseline(m, a, budget_s=12.0):
    """The FP64 oracle, as it stands, on a bounded packet sample of the same
    workload (B&W is sequential by definition: one host core)."""
    from oracle import oracle as O
    om = O.OracleModel(m)
    N = int(a.packets)
    t0 = time.perf_counter()
    r = O.transport(om, N, seed=99, pid_begin=0, pid_end=200, mode=O.MODE_BW)
    dt = time.perf_counter() - t0
    n = max(200, min(int(200 * budget_s / max(dt, 1e-3)), 200000))
    t0 = time.perf_counter()
    r = O.transport(om, N, seed=99, pid_begin=0, pid_end=n, mode=O.MODE_BW)
    dt = time.perf_counter() - t0
    out = {"value": r["stats"]["crossings"] / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{n} packets of the {N:.0e}-packet B&W emission (packet ids 0..{n - 1}), "
                     f"{r['stats']['crossings']} crossings in {dt:.1f} s"}
    # the iterative (frozen-T) scheme is order independent: the oracle splits
    # packet-id ranges over all host cores
    cores = os.cpu_count() or 1
    T0 = O.temperature_guess(m)
    n1 = 2000 * cores
    t0 = time.perf_counter()
    O.transport(om, N, seed=98, pid_begin=0, pid_end=n1, mode=O.MODE_FROZEN_T, T_prev=T0,
                n_threads=cores)
    dt = time.perf_counter() - t0
    n2 = max(n1, min(int(n1 * 0.6 * budget_s / max(dt, 1e-3)), 4000000))
    t0 = time.perf_counter()
    r2 = O.transport(om, N, seed=98, pid_begin=0, pid_end=n2, mode=O.MODE_FROZEN_T, T_prev=T0,
                     n_threads=cores)
    dt = time.perf_counter() - t0
    out["frozen_t_all_cores"] = {
        "value": r2["stats"]["crossings"] / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
        "sample": f"{n2} packets, iterative scheme at the optically thin starting temperatures, "
                  f"{r2['stats']['crossings']} crossings in {dt:.1f} s"}
    return out


# ---------------------------------------------------------------------------
# Other forms of the hot path (opt-in, --forms): each on its own workload,
# timed with CUDA events after warm-up, reported with its roofline fraction.

def _peak_hbm():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def _timed(fn, reps, warm, flush=None):
    import torch
    for _ in range(warm):
        fn(-1)
    torch.cuda.synchronize()
    ts = []
    for r in range(reps):
        if flush is not None:
            flush.fill_(float(r))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn(r)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    return ts


def _transport_bytes(S, ns):
    return (4 * ns * S["crossings"] + 32 * ns * S["lucy_deposits"] + 40 * S["absorptions"]
            + 20 * S["scatters"] + 32 * S["escaped"] + 64 * S["mrw_steps"])


def _roof(bytes_, secs):
    peak, src = _peak_hbm()
    gbs = bytes_ / secs / 1e9
    return {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
            "peak_source": src}


def _stats_delta(out, s0):
    from paper_1203_2941_gb300 import rtgb as R
    st = (out.stats - s0).cpu().numpy()
    return {k: int(st[i]) for i, k in enumerate(R.STAT_NAMES)}


def form_fp64_debug(rt, ctx, flush):
    """Homogeneous sphere 32^3 (tau_V = 1, 30 frequencies, 1e5 packets):
    the FP64 debug build against the FP32 production build, same packets."""
    import torch
    import workloads as W
    from paper_1203_2941_gb300 import rtgb as R
    m = W.homogeneous_sphere(n=32, tau_v=1.0, nf=30)
    grid, opac, srcs = ctx.grid(m), ctx.opacity(m), rt.Sources(m.sources)
    N = 100000
    res = {}
    for name, prec in (("fp64_debug", R.RT_PREC_FP64), ("fp32_fp64acc", R.RT_PREC_FP32)):
        out = rt.TransportOut(grid.ncell, 1, opac.nf)
        s0 = [None]

        def run(r):
            out.zero_()
            rt.transport(ctx, grid, opac, srcs, N, out=out, seed=3 + max(r, 0), precision=prec)
        ts = _timed(run, 5, 2, flush)
        S = _stats_delta(out, torch.zeros_like(out.stats))
        t = statistics.median(ts)
        res[name] = {"value": S["crossings"] / t, "unit": UNIT, "ms": 1e3 * t,
                     "roofline": _roof(_transport_bytes(S, 1), t)}
    res["ratio_fp64_over_fp32"] = res["fp64_debug"]["value"] / res["fp32_fp64acc"]["value"]
    res["workload"] = "homogeneous sphere 32^3, tau_V=1, 30 freq, 1e5 packets, B&W, Lucy thin"
    return res


def form_plain_fp32(rt, ctx, flush, packets=1e7):
    """The benchmark's transport (128^3 r^-2 shell, tau(1 um) = 10, 1e7
    packets, B&W, Lucy thin, events) in the production form (FP32 transport,
    FP64 accumulators) and in the plain-FP32 form (FP32 accumulators), same
    packets."""
    import torch
    import workloads as W
    from paper_1203_2941_gb300 import rtgb as R
    m = W.r2_shell(n=128, tau_1um=10.0, nf=64)
    grid, opac, srcs = ctx.grid(m), ctx.opacity(m), rt.Sources(m.sources)
    N = int(packets)
    res = {}
    for name, prec in (("fp32_fp64acc", R.RT_PREC_FP32), ("fp32_fp32acc", R.RT_PREC_FP32_ACC32)):
        out = rt.TransportOut(grid.ncell, 1, opac.nf, event_cap=6 * N)

        def run(r):
            out.zero_()
            out.stats[13:].zero_()
            rt.transport(ctx, grid, opac, srcs, N, out=out, record_events=True, seed=7 + max(r, 0),
                         precision=prec)
        ts = _timed(run, 5, 2, flush)
        S = _stats_delta(out, torch.zeros_like(out.stats))
        t = statistics.median(ts)
        res[name] = {"value": S["crossings"] / t, "unit": UNIT, "ms": 1e3 * t,
                     "roofline": _roof(_transport_bytes(S, 1), t)}
    res["ratio_fp32acc_over_fp64acc"] = res["fp32_fp32acc"]["value"] / res["fp32_fp64acc"]["value"]
    res["workload"] = f"r^-2 shell 128^3 tau1um=10, 64 freq, {N:.0e} packets, B&W, Lucy thin, events"
    return res


def form_next_rows(rt, ctx, flush, packets=1e7):
    """The later rows on their own workloads: the PAH re-emission pass
    (128^3 clumpy torus with PAH, the records of a 1e7-packet B&W run), Eq. 1
    equal-energy source bins against random bins on the benchmark's
    transport, photon-counting cameras (5 cones) on the same transport, and
    visibilities of the benchmark's images (5 x 12 images of 256^2 at 1024
    (u, v) points)."""
    import math as _m
    import numpy as _np
    import torch
    import workloads as W
    N = int(packets)
    res = {}
    # PAH pass
    mt = W.clumpy_torus(n=128, n_clump=1000, seed=77, nf=100)
    eps, cls = W.pah_emissivity(mt)
    gt, ot, st_ = ctx.grid(mt), ctx.opacity(mt), rt.Sources(mt.sources)
    o1 = rt.transport(ctx, gt, ot, st_, N, pah_cap=N, seed=3)
    torch.cuda.synchronize()
    n_rec = int(min(o1.stats[14].item(), N))
    cls_t = torch.tensor(cls, device="cuda")
    o2 = rt.TransportOut(gt.ncell, gt.ns, ot.nf, pah_cap=n_rec)

    def pah(r):
        o2.zero_()
        o2.stats[13:].zero_()
        rt.pah_reemit(ctx, gt, ot, o1, o1.xi, eps, cls_t, out=o2, pah_cap=n_rec, seed=4 + max(r, 0),
                      model_id=1)
    ts = _timed(pah, 3, 1, flush)
    S = _stats_delta(o2, torch.zeros_like(o2.stats))
    t = statistics.median(ts)
    res["pah_pass"] = {"value": S["crossings"] / t, "unit": UNIT, "ms": 1e3 * t, "packets": n_rec,
                       "roofline": _roof(_transport_bytes(S, 3), t),
                       "workload": "128^3 clumpy torus (1000 clumps, 3 species), records of a "
                                   f"{N:.0e}-packet B&W run, 4 emissivity classes"}
    # Eq. 1 source bins and photon counting on the benchmark's transport
    m = W.r2_shell(n=128, tau_1um=10.0, nf=64)
    grid, opac, srcs = ctx.grid(m), ctx.opacity(m), rt.Sources(m.sources)
    out = rt.TransportOut(grid.ncell, 1, opac.nf, event_cap=6 * N)
    cams = [rt.PcCamera(_m.radians(th), 0.0, 256, _m.cos(_m.radians(5.0))) for th in W.inclinations_deg()]
    for name, kw in (("random_bins", {}), ("source_bins_1000", {"source_bins": 1000}),
                     ("photon_counting_5_cameras", {"pc_cams": cams})):
        def run(r):
            out.zero_()
            out.stats[13:].zero_()
            rt.transport(ctx, grid, opac, srcs, N, out=out, record_events=True, seed=7 + max(r, 0), **kw)
        ts = _timed(run, 3, 1, flush)
        S = _stats_delta(out, torch.zeros_like(out.stats))
        t = statistics.median(ts)
        res[name] = {"value": S["crossings"] / t, "unit": UNIT, "ms": 1e3 * t,
                     "roofline": _roof(_transport_bytes(S, 1), t)}
    # visibilities of the benchmark's images
    T = rt.temperatures(ctx, grid, opac, out.E_abs)
    fidx = W.nearest_freq_indices(m.nu, W.image_wavelengths_um())
    rcams = [W.Camera(_m.radians(th), 0.0, 256, 140 * W.PC) for th in W.inclinations_deg()]
    img, _ = rt.raytrace(ctx, grid, opac, T, out, out.xi, srcs, rcams, fidx)
    uv = _np.random.default_rng(1).normal(size=(1024, 2)) * 1e5
    vis = {}

    def vrun(r):
        vis["v"] = rt.visibilities(ctx, grid, rcams, img, uv)
    ts = _timed(vrun, 3, 1, flush)
    t = statistics.median(ts)
    n_img = len(rcams) * len(fidx)
    nbytes = n_img * len(uv) * 256 * 256 * 4
    res["visibilities"] = {"value": n_img * len(uv) / t, "unit": "visibilities/s", "ms": 1e3 * t,
                           "roofline": _roof(nbytes, t),
                           "workload": f"{n_img} images of 256^2 at {len(uv)} (u, v) points"}
    return res


def form_mrw_disk(rt, ctx, flush, packets=1e7, npix=512):
    """Flared disk 256^3 (midplane tau_V = 1e4, 100 frequencies) with the
    modified random walk in cells of tau > 10; then Eq. 4 temperatures and
    images at 12 frequencies x 5 inclinations."""
    import math as _m
    import torch
    import workloads as W
    m = W.flared_disk(n=256, tau_v=1e4, nf=100)
    grid, opac, srcs = ctx.grid(m), ctx.opacity(m), rt.Sources(m.sources)
    N = int(packets)
    out = rt.TransportOut(grid.ncell, 1, opac.nf, event_cap=4 * N)
    state = {}

    def run(r):
        out.zero_()
        out.stats[13:].zero_()
        rt.transport(ctx, grid, opac, srcs, N, out=out, record_events=True, mrw=True,
                     seed=11 + max(r, 0))
    ts = _timed(run, 3, 1, flush)
    S = _stats_delta(out, torch.zeros_like(out.stats))
    t = statistics.median(ts)
    res = {"transport": {"value": S["crossings"] / t, "unit": UNIT, "ms": 1e3 * t,
                         "mrw_steps": S["mrw_steps"], "crossings": S["crossings"],
                         "interactions": S["interactions"], "absorptions": S["absorptions"],
                         "lucy_deposits": S["lucy_deposits"], "stuck": S["stuck"],
                         "roofline": _roof(_transport_bytes(S, 1), t)}}
    T = rt.temperatures(ctx, grid, opac, out.E_abs)
    fidx = W.nearest_freq_indices(m.nu, W.image_wavelengths_um())
    cams = [W.Camera(_m.radians(th), 0.0, npix, 140 * W.PC) for th in W.inclinations_deg()]
    steps = torch.zeros(1, dtype=torch.int64, device="cuda")

    def ray(r):
        steps.zero_()
        rt.raytrace(ctx, grid, opac, T, out, out.xi, srcs, cams, fidx, steps=steps)
    ts = _timed(ray, 3, 1, flush)
    t = statistics.median(ts)
    n = int(steps.item())
    nfp = (len(fidx) + 3) // 4 * 4
    res["raytrace"] = {"value": n / t, "unit": "ray-cell steps/s", "ms": 1e3 * t, "steps": n,
                       "roofline": _roof(n * (4 + 4 * nfp), t)}
    res["workload"] = (f"flared disk 256^3, midplane tau_V=1e4, 100 freq, {N:.0e} packets, B&W, "
                       f"MRW tau_cell>10, Lucy thin, events; images {len(cams)} incl x {len(fidx)} freq "
                       f"x {npix}^2")
    return res


def form_refined_shell(rt, ctx, flush, packets=1e7, npix=256):
    """r^-2 shell (tau(1 um) = 10, 64 frequencies) on 64^3 cubes, the cubes
    within 6 cube edges of the star divided into 4^3 sub-cubes (one level of
    refinement): B&W transport, Eq. 4 temperatures and images (5
    inclinations x 12 frequencies), against the same shell on the uniform
    64^3 grid."""
    import math as _m
    import torch
    import workloads as W
    mr = W.r2_shell_refined(n=64, tau_1um=10.0, nf=64, r=4, refine_radius=6.0)
    mu = W.r2_shell(n=64, tau_1um=10.0, nf=64)
    N = int(packets)
    res = {}
    for name, m in (("refined", mr), ("uniform", mu)):
        grid, opac, srcs = ctx.grid(m), ctx.opacity(m), rt.Sources(m.sources)
        out = rt.TransportOut(grid.ncell, 1, opac.nf, event_cap=6 * N)

        def run(r):
            out.zero_()
            out.stats[13:].zero_()
            rt.transport(ctx, grid, opac, srcs, N, out=out, record_events=True, seed=5 + max(r, 0))
        ts = _timed(run, 3, 1, flush)
        S = _stats_delta(out, torch.zeros_like(out.stats))
        t = statistics.median(ts)
        res[name] = {"transport": {"value": S["crossings"] / t, "unit": UNIT, "ms": 1e3 * t,
                                   "crossings": S["crossings"], "cells": grid.ncell,
                                   "roofline": _roof(_transport_bytes(S, 1), t)}}
        T = rt.temperatures(ctx, grid, opac, out.E_abs)
        fidx = W.nearest_freq_indices(m.nu, W.image_wavelengths_um())
        cams = [W.Camera(_m.radians(th), 0.0, npix, 140 * W.PC) for th in W.inclinations_deg()]
        steps = torch.zeros(1, dtype=torch.int64, device="cuda")

        def ray(r):
            steps.zero_()
            rt.raytrace(ctx, grid, opac, T, out, out.xi, srcs, cams, fidx, steps=steps)
        ts = _timed(ray, 3, 1, flush)
        t = statistics.median(ts)
        n = int(steps.item())
        nfp = (len(fidx) + 3) // 4 * 4
        res[name]["raytrace"] = {"value": n / t, "unit": "ray-cell steps/s", "ms": 1e3 * t,
                                 "steps": n, "roofline": _roof(n * (4 + 4 * nfp), t)}
    res["workload"] = (f"r^-2 shell tau1um=10, 64 freq, {N:.0e} packets, B&W, Lucy thin, events; "
                       f"64^3 cubes, {int(mr.refined.sum())} cubes within 6 edges of the star divided "
                       f"into 4^3 ({mr.ncell} cells); images 5 incl x 12 freq x {npix}^2")
    return res


def form_batched(rt, ctx, flush, per_model=1e6, n_models=64):
    """64 clumpy tori of uneven size (64^3 .. 192^3, silicate + carbon + PAH,
    100 frequencies) in one persistent launch replayed from a CUDA graph,
    against the same models run one after another through the single-model
    path."""
    import torch
    import workloads as W
    models = W.batched_tori(n_models=n_models)
    opac = ctx.opacity(models[0])
    N = [int(per_model)] * n_models
    b = rt.Batch(ctx, opac, models, N, seed=21, pah_cap=int(per_model))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.run(s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    gr = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gr):
        b.run(torch.cuda.current_stream())
    s0 = [o.stats.clone() for o in b.outs]

    def run(r):
        gr.replay()
    reps = 3
    ts = _timed(run, reps, 1, flush)
    S = {}
    for o, z in zip(b.outs, s0):
        for k, v in _stats_delta(o, z).items():
            S[k] = S.get(k, 0) + v
    S = {k: v // (reps + 1) for k, v in S.items()}
    t = statistics.median(ts)
    res = {"batched_graph": {"value": S["crossings"] / t, "unit": UNIT, "ms": 1e3 * t,
                             "crossings": S["crossings"], "roofline": _roof(_transport_bytes(S, 3), t)}}
    grids, srcs = b.grids, b.sources
    outs = [rt.TransportOut(g.ncell, g.ns, opac.nf, pah_cap=int(per_model)) for g in grids]

    def single(r):
        for i in range(n_models):
            outs[i].zero_()
            rt.transport(ctx, grids[i], opac, srcs[i], N[i], out=outs[i], seed=21, model_id=i)
    ts = _timed(single, 2, 1, flush)
    t1 = statistics.median(ts)
    c1 = sum(int(o.stats[0].item()) for o in outs)
    res["single_model_loop"] = {"value": c1 / t1, "unit": UNIT, "ms": 1e3 * t1, "crossings": c1}
    res["ratio_batched_over_single"] = res["batched_graph"]["value"] / res["single_model_loop"]["value"]
    sizes = [m_.rho.shape[-1] for m_ in models]
    res["workload"] = (f"{n_models} clumpy tori {min(sizes)}^3..{max(sizes)}^3 "
                       f"(3 species incl. PAH, 100 freq), {per_model:.0e} packets each, B&W, Lucy thin")
    return res


def form_adjoint(rt, ctx, flush, npix=256):
    """Ray-tracer adjoint on a 128^3 clumpy torus (1000 clumps, temperatures
    fixed from a prior transport): 8 views at 10 um plus the SED at 16 of
    the model frequencies, d(loss)/d(rho) and d/d(scale)."""
    import math as _m
    import torch
    import workloads as W
    m = W.clumpy_torus(n=128, n_clump=1000, seed=77, nf=40)
    grid, opac, srcs = ctx.grid(m), ctx.opacity(m), rt.Sources(m.sources)
    out = rt.transport(ctx, grid, opac, srcs, 1000000, event_cap=4000000, seed=31)
    T = rt.temperatures(ctx, grid, opac, out.E_abs)
    fidx = W.nearest_freq_indices(m.nu, [10.0])
    cams = [W.Camera(_m.radians(th), _m.radians(45.0 * k), npix, 14e6 * W.PC)
            for k, th in enumerate((10, 30, 50, 70, 90, 110, 130, 150))]
    g = torch.Generator(device="cuda").manual_seed(5)
    dimg = torch.randn((len(cams), len(fidx), npix, npix), device="cuda", generator=g)
    dsed = torch.randn((len(cams), len(fidx)), device="cuda", dtype=torch.float64, generator=g)
    steps = torch.zeros(1, dtype=torch.int64, device="cuda")

    def fwd(r):
        steps.zero_()
        rt.raytrace(ctx, grid, opac, T, out, out.xi, srcs, cams, fidx, steps=steps)
    tf = statistics.median(_timed(fwd, 3, 1, flush))
    nf_ = int(steps.item())

    def bwd(r):
        steps.zero_()
        rt.raytrace_backward(ctx, grid, opac, T, out, out.xi, srcs, cams, fidx, dL_dimg=dimg,
                             dL_dsed=dsed, steps=steps)
    tb = statistics.median(_timed(bwd, 3, 1, flush))
    nb = int(steps.item())
    nfp = (len(fidx) + 3) // 4 * 4
    br = 4 * 4 + 4 * nfp
    res = {"forward": {"value": nf_ / tf, "unit": "ray-cell steps/s", "ms": 1e3 * tf,
                       "roofline": _roof(nf_ * br, tf)},
           "adjoint": {"value": nb / tb, "unit": "ray-cell steps/s", "ms": 1e3 * tb,
                       "roofline": _roof(nb * (2 * br + 4), tb)}}
    res["workload"] = f"clumpy torus 128^3, 1000 clumps, 3 species, 8 views x 10 um x {npix}^2 + SED"
    return res


def run_forms(a):
    import torch
    import paper_1203_2941_gb300 as rt
    rt.build()
    ctx = rt.Context(0)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    forms = {}
    for name, fn in (("fp64_debug", form_fp64_debug), ("plain_fp32", form_plain_fp32),
                     ("mrw_disk", form_mrw_disk), ("adjoint", form_adjoint),
                     ("batched", form_batched), ("refined_shell", form_refined_shell),
                     ("next_rows", form_next_rows)):
        if a.forms != "all" and name not in a.forms.split(","):
            continue
        t0 = time.perf_counter()
        kw = {"packets": a.packets} if name in ("mrw_disk", "refined_shell", "plain_fp32", "next_rows") else {}
        forms[name] = fn(rt, ctx, flush, **kw)
        forms[name]["wall_s"] = time.perf_counter() - t0
        print(json.dumps({"form": name, **forms[name]}), flush=True)
    return forms


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    m = build_model(a)
    from oracle import oracle as O
    om = O.OracleModel(m)
    N = int(a.packets)
    t0 = time.perf_counter()
    O.transport(om, N, seed=7, pid_begin=0, pid_end=100, mode=O.MODE_BW)
    per = (time.perf_counter() - t0) / 100
    n = max(100, int(6.0 / max(per, 1e-6)))
    n = max(1, min(n, N // max(1, a.warmup + a.steps)))     # the samples stay inside [0, N)
    cross, times = 0, []
    for i in range(a.warmup + a.steps):
        t0 = time.perf_counter()
        r = O.transport(om, N, seed=7, pid_begin=i * n, pid_end=(i + 1) * n, mode=O.MODE_BW)
        dt = time.perf_counter() - t0
        if i >= a.warmup:
            cross += r["stats"]["crossings"]
            times.append(dt)
    v = cross / sum(times)
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "impl": "reference",
            "data": "synthetic (seeded generator shaped like the paper's 1D benchmark shell)",
            "config": workload_config(a, {"reference_sample": f"{n} packets per step"}),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{n} packets per step of the {N:.0e}-packet B&W emission"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
        return
    if a.forms:
        run_forms(a)
        return
    import numpy as np
    import torch

    import paper_1203_2941_gb300 as rt
    from paper_1203_2941_gb300 import rtgb as R

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    rt.build()
    m = build_model(a)
    ctx = rt.Context(local)
    grid, opac, srcs = ctx.grid(m), ctx.opacity(m), rt.Sources(m.sources)
    cams, fidx = image_setup(m, a)
    N = int(a.packets)
    ev_cap = 6 * N
    out = rt.TransportOut(grid.ncell, 1, opac.nf, event_cap=ev_cap)
    ray_steps = torch.zeros(1, dtype=torch.int64, device="cuda")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    seed_base = 1000 * rank

    def step(i, ev_pairs=None):
        for t in (out.E_abs, out.count, out.esq, out.sed_esc, out.sed_cnt):
            t.zero_()
        out.stats[13:].zero_()                      # event/PAH/trajectory cursors restart
        if ev_pairs is not None:
            ev_pairs[0].record(stream)
        rt.transport(ctx, grid, opac, srcs, N, out=out, record_events=True, seed=seed_base + i + 1)
        if ev_pairs is not None:
            ev_pairs[1].record(stream)
        T = rt.temperatures(ctx, grid, opac, out.E_abs)
        if ev_pairs is not None:
            ev_pairs[2].record(stream)
        img, sed = rt.raytrace(ctx, grid, opac, T, out, out.xi, srcs, cams, fidx, steps=ray_steps)
        if ev_pairs is not None:
            ev_pairs[3].record(stream)
        return T, img, sed

    for i in range(a.warmup):
        step(i)
    torch.cuda.synchronize()
    stats0 = out.stats.clone()
    rs0 = ray_steps.clone()
    launches0 = R.rt_kernel_launches()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(a.steps)]
    with ClockSampler(local) as clk:
        for k in range(a.steps):
            flush.fill_(float(k))                   # evict the grid and tables from L2
            step(a.warmup + k, evs[k])
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = R.rt_kernel_launches() - launches0
    if dist:
        # replicas of the B&W solve: average the accumulated outputs (untimed)
        from paper_1203_2941_gb300.shard import allreduce_mean
        allreduce_mean([out.E_abs, out.sed_esc])
    t_step = [e[0].elapsed_time(e[3]) for e in evs]
    t_tr = [e[0].elapsed_time(e[1]) for e in evs]
    t_T = [e[1].elapsed_time(e[2]) for e in evs]
    t_ray = [e[2].elapsed_time(e[3]) for e in evs]
    st = (out.stats - stats0).cpu().numpy()
    S = {k: int(st[i]) for i, k in enumerate(R.STAT_NAMES)}
    rsteps = int((ray_steps - rs0).item())
    tot_s = sum(t_step) / 1e3
    if dist:
        tt = torch.tensor([tot_s], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        cc = torch.tensor([S["crossings"]], device="cuda", dtype=torch.float64)
        dist.all_reduce(cc)
        tot_s, crossings_all = float(tt.item()), float(cc.item())
    else:
        crossings_all = S["crossings"]
    value = crossings_all / tot_s

    # roofline of the dominant kernel (transport): algorithmic bytes per launch
    K = a.steps
    ns = 1
    bytes_alg = (4 * ns * S["crossings"] + 32 * ns * S["lucy_deposits"] + 40 * S["absorptions"]
                 + 20 * min(S["scatters"], K * ev_cap) + 32 * S["escaped"]) / K
    t_tr_s = sum(t_tr) / K / 1e3
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    achieved = bytes_alg / t_tr_s / 1e9
    default_work = (a.n == 128 and a.tau == 10.0 and int(a.packets) == 10**7)
    # sector-granular view of the same launch: every gather, deposit pair,
    # absorption tally, event record and escape tally touches a 32-byte sector
    bytes_sec = (32 * S["crossings"] + 32 * S["lucy_deposits"] + 64 * S["absorptions"]
                 + 32 * min(S["scatters"], K * ev_cap) + 32 * S["escaped"]) / K
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": TRANSPORT_DRAM_BYTES if default_work else None,
            "kernel": "transport_kernel<float,1,12>", "peak_source": peak_src,
            "bytes_per_launch": bytes_alg, "launch_ms": t_tr_s * 1e3,
            "sector_bytes_per_launch": bytes_sec, "sector_achieved": bytes_sec / t_tr_s / 1e9}

    # end to end through the public API with host buffers
    e2e = None
    if not a.no_e2e:
        rho_h = torch.from_numpy(m.rho.copy()).pin_memory()
        E_h = torch.empty((1, grid.ncell), dtype=torch.float64).pin_memory()
        T_h = torch.empty((1, grid.ncell), dtype=torch.float64).pin_memory()
        img_h = torch.empty((len(cams), len(fidx), a.npix, a.npix), dtype=torch.float32).pin_memory()
        sed_h = torch.empty((len(cams), len(fidx)), dtype=torch.float64).pin_memory()
        st_h = torch.empty(R.RT_STAT_COUNT, dtype=torch.int64).pin_memory()
        e2e_out = rt.TransportOut(grid.ncell, 1, opac.nf, event_cap=ev_cap)
        cross_e2e = 0
        g2 = rt.Grid(ctx, rho_h, m.box_min, m.cell)               # the caller's grid handle
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(a.steps):
            g2.update(rho_h)                                      # H2D of the step's density
            e2e_out.zero_()
            o = rt.transport(ctx, g2, opac, srcs, N, out=e2e_out, record_events=True, seed=50 + k)
            T = rt.temperatures(ctx, g2, opac, o.E_abs)
            img, sed = rt.raytrace(ctx, g2, opac, T, o, o.xi, srcs, cams, fidx)
            E_h.copy_(o.E_abs, non_blocking=True)
            T_h.copy_(T, non_blocking=True)
            img_h.copy_(img, non_blocking=True)
            sed_h.copy_(sed, non_blocking=True)
            st_h.copy_(o.stats, non_blocking=True)
            torch.cuda.synchronize()
            cross_e2e += int(st_h[0])
        dt = time.perf_counter() - t0
        del g2
        e2e = {"value": cross_e2e / dt, "unit": UNIT,
               "h2d_bytes_per_step": int(rho_h.numel() * 4),
               "d2h_bytes_per_step": int(E_h.numel() * 8 + T_h.numel() * 8 + img_h.numel() * 4
                                         + sed_h.numel() * 8 + st_h.numel() * 8),
               "ms_per_step": 1e3 * dt / a.steps}

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        cpu = cpu_baseline(m, a)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": sum(t_step) / len(t_step),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (seeded generator shaped like the paper's 1D benchmark shell)",
                "config": workload_config(a, {"parallelism": f"replicas x{world}" if world > 1 else "1 GPU"}),
                "phases_ms": {"transport": sum(t_tr) / K, "temperatures": sum(t_T) / K,
                              "raytrace": sum(t_ray) / K},
                "raytrace": {"metric": "ray-cell steps/s", "value": rsteps / (sum(t_ray) / 1e3),
                             "ray_cell_steps_per_step": rsteps // K},
                "stats_per_step": {k: v // K for k, v in S.items() if not k.startswith("n_")},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk.summary(),
                "gpu_launches": launches}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
