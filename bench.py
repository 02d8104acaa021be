#!/usr/bin/env python3
"""Benchmark: photon-packet cell-crossings/s (and ray-cell steps/s) of the
full Monte Carlo radiative-transfer step on one GB300.

One step = one pass of the hot path over one model:

* ``--workload disk`` (default, the largest single-GPU configuration): the
  flared disk on a 256^3 grid (rho ~ r^-1 exp(-z^2 / 2 h^2), h ~ r^1.125,
  midplane tau_V = 1e4, 100 frequencies, central 5800 K star): Bjorkman &
  Wood transport of 1e8 packets in FP32 with FP64 energy accumulators, the
  modified random walk in cells of tau > 10, Lucy deposits in thin cells and
  the scattering events at the image frequencies; the Eq. 4 temperatures;
  ray-traced images (5 inclinations x 12 frequencies x 512^2 pixels) and SEDs.
  The same disk at midplane tau_V = 1e5 (a step takes over a minute) is the
  opt-in form ``--forms disk_tau1e5``.
* ``--workload shell``: the r^-2 shell on 128^3 cells (tau(1 um) = 10, 64
  frequencies, 2500 K star), 1e7 packets, images of 256^2; it also appears
  as the ``shell_128`` sub-object of the default line.

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
L2_BYTES = 126.5 * 2 ** 20          # GB300 L2 (nominal 129 MB)
# DRAM bytes (read + write) of one transport launch of each workload at its
# default packet count, from single-pass ncu captures (profiles/): the disk's
# taken on 1e7 packets and scaled by 10 (its traffic grows with the packets),
# the shell's on the full launch, each at the schedule the autotuner chose
# (march_min_active 6 and 16), on the build of commit 445f240; emptied when
# the transport kernel changes until it is captured again.
TRANSPORT_DRAM = {"disk": (25.136743680e9 + 10.662938112e9) * 10, "shell": 29.148672e6 + 0.595456e6}

WORKLOADS = {
    "disk": dict(n=256, tau=1e4, nf=100, packets=1e8, npix=512, mrw=True,
                 text="flared disk 256^3 (r^-1 exp(-z^2/2h^2), h~r^1.125), midplane tau_V={tau:g}, "
                      "100 freq 0.1-1000um, 5800 K star; {packets:.0e} packets B&W FP32+FP64 acc, "
                      "MRW tau_cell>10, Lucy thin, events at the image freq; Eq.4 temperatures; "
                      "images 5 incl x 12 freq x {npix}^2"),
    "shell": dict(n=128, tau=10.0, nf=64, packets=1e7, npix=256, mrw=False,
                  text="r^-2 spherical shell {n}^3, tau(1um)={tau:g}, 64 freq 0.1-1000um, 2500 K star; "
                       "{packets:.0e} packets B&W FP32+FP64 acc, Lucy thin, events at the image freq; "
                       "Eq.4 temperatures; images 5 incl x 12 freq x {npix}^2"),
}


_T0 = time.perf_counter()


def log(msg):
    """Progress on stderr (the JSON line alone goes to stdout)."""
    sys.stderr.write(f"[bench {time.perf_counter() - _T0:7.1f} s] {msg}\n")
    sys.stderr.flush()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="disk", choices=sorted(WORKLOADS))
    ap.add_argument("--packets", type=float, default=None)
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--tau", type=float, default=None)
    ap.add_argument("--npix", type=int, default=None)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-shell", action="store_true", help="skip the 128^3 shell sub-object")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the schedule autotuner (library default march_min_active)")
    ap.add_argument("--march-min-active", type=int, default=None,
                    help="fixed march_min_active instead of the autotuner's choice")
    ap.add_argument("--schedule", default="persistent", choices=["persistent", "compact"],
                    help="transport schedule: dynamic refill per warp, or with per-warp packet compaction")
    ap.add_argument("--sharded", action="store_true",
                    help="the sharded iterative solve (the mode used under torchrun) at any world size")
    ap.add_argument("--forms", default="", help="measure other forms instead of the step: "
                    "all or a comma list of fp64_debug, plain_fp32, mrw_disk, adjoint, batched, "
                    "refined_shell, next_rows")
    a = ap.parse_args()
    a.packets_given = a.packets
    w = WORKLOADS[a.workload]
    for k in ("packets", "n", "tau", "npix"):
        if getattr(a, k) is None:
            setattr(a, k, w[k])
    a.nf, a.mrw = w["nf"], w["mrw"]
    return a


def workload_config(a, extra=None):
    w = WORKLOADS[a.workload]
    cfg = {"workload": w["text"].format(n=a.n, tau=a.tau, packets=a.packets, npix=a.npix),
           "grid": a.n, "n_packets": int(a.packets), "n_freq": a.nf, "mode": "bjorkman-wood",
           "mrw": a.mrw, "images": [5, 12, a.npix], "schedule": getattr(a, "schedule", "persistent"),
           "l2": "inputs larger than L2 and flushed between steps (512 MiB write)"}
    if extra:
        cfg.update(extra)
    return cfg


def build_model(a):
    import workloads as W
    if a.workload == "disk":
        return W.flared_disk(n=a.n, tau_v=a.tau, nf=a.nf)
    return W.r2_shell(n=a.n, tau_1um=a.tau, nf=a.nf)


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


def _oracle_sample(O, om, N, budget_s, first, **kw):
    """Consecutive packet-id ranges of the emission, four times longer each
    from `first` packets, until the oracle's packet loops have taken
    budget_s (a heavy tail of slow packets overruns it by at most one range).  Returns
    (packets, crossings, loop seconds, grid set-up seconds of one call)."""
    done, cross, loop, n, setup = 0, 0, 0.0, first, None
    while loop < budget_s and done < N:
        n = min(n, N - done)
        t0 = time.perf_counter()
        r = O.transport(om, N, pid_begin=done, pid_end=done + n, **kw)
        if setup is None:
            setup = time.perf_counter() - t0 - r["loop_seconds"]
        done += n
        cross += r["stats"]["crossings"]
        loop += r["loop_seconds"]
        n *= 4
    return done, cross, loop, setup


def cpu_baseline(m, a, budget_s=10.0):
    """The FP64 oracle, as it stands, on bounded packet samples of the same
    workload: B&W on one host core (sequential by definition) and the
    iterative (frozen-T) scheme over packet-id ranges on every host core.
    Rates count the oracle's packet loop; its grid set-up (cell sizes and the
    Lucy flag of every cell) is timed apart and reported."""
    from oracle import oracle as O
    om = O.OracleModel(m)
    N = int(a.packets)
    n, cross, dt, setup = _oracle_sample(O, om, N, budget_s, 50, seed=99, mode=O.MODE_BW, mrw=a.mrw)
    out = {"value": cross / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{n} packets of the {N:.0e}-packet B&W emission (packet ids 0..{n - 1}, in "
                     f"growing ranges, each from empty accumulators), {cross} crossings in {dt:.1f} s of packet "
                     f"loops (grid set-up {setup:.1f} s per call, not counted)",
           "setup_s": setup}
    cores = os.cpu_count() or 1
    T0 = O.temperature_guess(m)
    n2, c2, dt2, _ = _oracle_sample(O, om, N, budget_s, 100 * cores, seed=98, mode=O.MODE_FROZEN_T,
                                    T_prev=T0, n_threads=cores, mrw=a.mrw)
    out["frozen_t_all_cores"] = {
        "value": c2 / dt2, "unit": UNIT, "cores": cores, "kind": "oracle",
        "sample": f"{n2} packets, iterative scheme at the optically thin starting temperatures, "
                  f"{c2} crossings in {dt2:.1f} s of packet loops"}
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


def form_batched(rt, ctx, flush, per_model=1e7, n_models=64):
    """64 clumpy tori of uneven size (64^3 .. 192^3, silicate + carbon + PAH,
    100 frequencies) in one persistent launch replayed from a CUDA graph,
    against the same models run one after another through the single-model
    path.  Every repetition of either starts from zeroed outputs (B&W
    temperatures follow the accumulated energy, so accumulating across
    repetitions would change the work); both take the march_min_active the
    schedule autotuner picks on a mid-size model."""
    import torch
    import workloads as W
    from paper_1203_2941_gb300.autotune import tune_transport
    models = W.batched_tori(n_models=n_models)
    opac = ctx.opacity(models[0])
    N = [int(per_model)] * n_models
    mid = models[n_models // 2]
    g_mid = ctx.grid(mid)
    tr = tune_transport(ctx, g_mid, opac, rt.Sources(mid.sources), N[0], sample=2_000_000,
                        grid_values={"threads_per_block": (256,)}, repeats=2)
    del g_mid
    mma = tr.params["march_min_active"]
    b = rt.Batch(ctx, opac, models, N, seed=21, pah_cap=int(per_model), march_min_active=mma)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.run(s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    gr = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gr):
        for o in b.outs:
            o.zero_()
        b.run(torch.cuda.current_stream())

    def run(r):
        gr.replay()
    ts = _timed(run, 3, 1, flush)
    S = {}
    for o in b.outs:
        for k, v in _stats_delta(o, torch.zeros_like(o.stats)).items():
            S[k] = S.get(k, 0) + v
    t = statistics.median(ts)
    res = {"march_min_active": mma,
           "batched_graph": {"value": S["crossings"] / t, "unit": UNIT, "ms": 1e3 * t,
                             "crossings": S["crossings"], "roofline": _roof(_transport_bytes(S, 3), t)}}
    grids, srcs = b.grids, b.sources
    outs = [rt.TransportOut(g.ncell, g.ns, opac.nf, pah_cap=int(per_model)) for g in grids]

    def single(r):
        for i in range(n_models):
            outs[i].zero_()
            rt.transport(ctx, grids[i], opac, srcs[i], N[i], out=outs[i], seed=21, model_id=i,
                         march_min_active=mma)
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
    """The ray-tracer adjoint of a density fit on a 128^3 clumpy torus (1000
    clumps, 3 species, temperatures and events from a prior 2e6-packet
    transport): loss = chi^2 of the SED at 40 wavelengths (0.3-500 um) seen
    from one view + chi^2 of 256^2 images at 10 um from 8 views, against a
    synthetic observation (perturbed density, 10 % noise).  Times one
    evaluation of the loss (forward) and of its gradient (forward + adjoint)
    and reports ray-cell steps/s of each."""
    import torch
    import workloads as W
    m = W.clumpy_torus(n=128, n_clump=1000, seed=77, nf=100)
    grid, opac, srcs = ctx.grid(m), ctx.opacity(m), rt.Sources(m.sources)
    out = rt.transport(ctx, grid, opac, srcs, 2_000_000, event_cap=8_000_000, seed=31, record_events=True)
    T = rt.temperatures(ctx, grid, opac, out.E_abs)
    sed_f = W.nearest_freq_indices(m.nu, W.adjoint_sed_wavelengths_um())
    chunks = [sed_f[i:i + 16] for i in range(0, len(sed_f), 16)]
    img_f = W.nearest_freq_indices(m.nu, [10.0])
    D = 14e6 * W.PC
    views = [W.Camera(th, ph, npix, D) for th, ph in W.adjoint_view_angles()]
    steps = torch.zeros(1, dtype=torch.int64, device="cuda")

    def forward(g):
        img, _ = rt.raytrace(ctx, g, opac, T, out, out.xi, srcs, views, img_f, steps=steps)
        sed = torch.cat([rt.raytrace(ctx, g, opac, T, out, out.xi, srcs, views[:1], ch, steps=steps)[1]
                         for ch in chunks], dim=1)
        return img, sed

    gt = rt.Grid(ctx, torch.tensor(W.perturbed_density(m), device="cuda"), m.box_min, m.cell)
    I_obs, F_obs = forward(gt)
    gen = torch.Generator(device="cuda").manual_seed(78)
    I_obs = I_obs.double() * (1 + 0.1 * torch.randn(I_obs.shape, device="cuda", dtype=torch.float64, generator=gen))
    F_obs = F_obs * (1 + 0.1 * torch.randn(F_obs.shape, device="cuda", dtype=torch.float64, generator=gen))
    sI = 0.1 * I_obs.abs() + 1e-3 * I_obs.abs().max()
    sF = 0.1 * F_obs.abs()
    res = {}

    def loss(r):
        img, sed = forward(grid)
        return (((sed - F_obs) / sF) ** 2).sum() + (((img.double() - I_obs) / sI) ** 2).sum()

    def grad(r):
        img, sed = forward(grid)
        gi = (2 * (img.double() - I_obs) / sI ** 2).float()
        gs = 2 * (sed - F_obs) / sF ** 2
        rt.raytrace_backward(ctx, grid, opac, T, out, out.xi, srcs, views, img_f, dL_dimg=gi, steps=steps)
        o = 0
        for ch in chunks:
            rt.raytrace_backward(ctx, grid, opac, T, out, out.xi, srcs, views[:1], ch,
                                 dL_dsed=gs[:, o:o + len(ch)].contiguous(), steps=steps)
            o += len(ch)

    for name, fn in (("loss_forward", loss), ("loss_gradient", grad)):
        steps.zero_()
        ts = _timed(fn, 3, 1, flush)
        n = int(steps.item()) // 4
        t = statistics.median(ts)
        res[name] = {"value": n / t, "unit": "ray-cell steps/s", "ms": 1e3 * t, "ray_cell_steps": n}
    res["workload"] = ("clumpy torus 128^3, 1000 clumps, 3 species; loss = chi^2 of a 40-point SED "
                       f"(0.3-500 um, one view) + chi^2 of 8 views x 10 um x {npix}^2 images")
    return res


def form_disk_tau1e5(rt, ctx, flush, packets=1e8):
    """The benchmark step on the 256^3 flared disk at midplane tau_V = 1e5
    (1e8 packets, MRW, 5 x 12 x 512^2 images): one warm-up and one timed
    step (a step takes over a minute)."""
    import torch
    a = argparse.Namespace(workload="disk", n=256, tau=1e5, nf=100, packets=packets, npix=512, mrw=True,
                           schedule="persistent")
    m = build_model(a)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    gp = gather_peaks(rt, ctx, m.rho[0].size * 12)
    r = run_step_bench(a, rt, ctx, m, 1, 1, flush, 0, 0, 1, None, peaks, gp, 0)
    S = r["S"]
    r["roofline"]["kernel"] = "transport_kernel<float,1,13>"
    return {"workload": workload_config(a)["workload"], "metric": METRIC,
            "value": S["crossings"] / r["tot_s"], "unit": UNIT, "steps": 1, "warmup": 1,
            "ms_per_step": r["t_step"][0],
            "phases_ms": {"transport": r["t_tr"][0], "temperatures": r["t_T"][0], "raytrace": r["t_ray"][0]},
            "stats_per_step": {k: v for k, v in S.items() if not k.startswith("n_")},
            "raytrace": {"metric": "ray-cell steps/s", "value": r["rsteps"] / (r["t_ray"][0] / 1e3),
                         "roofline": r["ray_roofline"]},
            "roofline": r["roofline"]}


def form_compaction(rt, ctx, flush, packets=1e7):
    """Per-warp packet compaction (RT_SCHED_COMPACT) against the persistent
    schedule on the same packets: the 128^3 r^-2 shell (1e7 packets, B&W,
    Lucy thin, events at the image frequencies) and the 256^3 flared disk
    (midplane tau_V = 1e4, MRW; 1e7 packets), with a sweep of the lanes left
    marching at which the stopped lanes trade (compact_swap) and at which a
    march phase ends (march_min_active)."""
    import torch
    import workloads as W
    from paper_1203_2941_gb300 import rtgb as R
    res = {}
    for wname, m, kw in (("shell_128", W.r2_shell(n=128, tau_1um=10.0, nf=64), {}),
                         ("disk_256", W.flared_disk(n=256, tau_v=1e4, nf=100), {"mrw": True})):
        grid, opac, srcs = ctx.grid(m), ctx.opacity(m), rt.Sources(m.sources)
        fidx = sorted(set(W.nearest_freq_indices(m.nu, W.image_wavelengths_um())))
        N = int(packets)
        out = rt.TransportOut(grid.ncell, 1, opac.nf, event_cap=6 * N)
        rows = {}
        cases = [("persistent", dict(schedule=R.RT_SCHED_PERSISTENT))]
        for sw in (24, 28):
            for ma in (4, 8):
                cases.append((f"compact_swap{sw}_end{ma}",
                              dict(schedule=R.RT_SCHED_COMPACT, compact_swap=sw, march_min_active=ma)))
        for name, ck in cases:
            def run(r):
                out.zero_()
                out.stats[13:].zero_()
                rt.transport(ctx, grid, opac, srcs, N, out=out, record_events=True, record_nu=fidx,
                             seed=7 + max(r, 0), **kw, **ck)
            ts = _timed(run, 3, 1, flush)
            S = _stats_delta(out, torch.zeros_like(out.stats))
            t = statistics.median(ts)
            rows[name] = {"value": S["crossings"] / t, "unit": UNIT, "ms": 1e3 * t}
        base = rows["persistent"]["value"]
        for v in rows.values():
            v["speedup"] = v["value"] / base
        res[wname] = rows
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
                     ("next_rows", form_next_rows), ("compaction", form_compaction),
                     ("disk_tau1e5", form_disk_tau1e5)):
        if (a.forms != "all" or name == "disk_tau1e5") and name not in a.forms.split(","):
            continue
        t0 = time.perf_counter()
        kw = ({"packets": a.packets_given if a.packets_given is not None else 1e7}
              if name in ("mrw_disk", "refined_shell", "plain_fp32", "next_rows", "compaction") else {})
        forms[name] = fn(rt, ctx, flush, **kw)
        forms[name]["wall_s"] = time.perf_counter() - t0
        print(json.dumps({"form": name, **forms[name]}), flush=True)
    return forms


def run_reference(a):
    """The FP64 oracle as it stands (the paper's code is not available) on
    the same workload: each step is B&W (sequential: one host core) on the
    next bounded packet-id range of the emission; the rate counts the
    oracle's packet loops (its per-call grid set-up is timed apart and
    reported)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    m = build_model(a)
    from oracle import oracle as O
    om = O.OracleModel(m)
    N = int(a.packets)
    t0 = time.perf_counter()
    r = O.transport(om, N, seed=7, pid_begin=0, pid_end=20, mode=O.MODE_BW, mrw=a.mrw)
    setup = time.perf_counter() - t0 - r["loop_seconds"]
    per = max(r["loop_seconds"] / 20, 1e-6)
    n = max(20, int(3.0 / per))
    n = max(1, min(n, N // max(1, a.warmup + a.steps)))     # the samples stay inside [0, N)
    cross, times = 0, []
    for i in range(a.warmup + a.steps):
        r = O.transport(om, N, seed=7, pid_begin=i * n, pid_end=(i + 1) * n, mode=O.MODE_BW, mrw=a.mrw)
        if i >= a.warmup:
            cross += r["stats"]["crossings"]
            times.append(r["loop_seconds"])
    v = cross / sum(times)
    sample = (f"{n} packets per step of the {N:.0e}-packet B&W emission, one host core; packet loops "
              f"only (grid set-up {setup:.1f} s per call, not counted)")
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "impl": "reference",
            "data": "synthetic (seeded generators shaped like the paper's benchmark models)",
            "config": workload_config(a, {"reference_sample": f"{n} packets per step"}),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "setup_s": setup},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def gather_peaks(rt, ctx, working_set):
    """Random 32-byte sector reads (rt_probe_gather, the access pattern of
    the transport's density gathers) from a buffer of the workload's
    working-set size and from a 2 GiB buffer: the sector bandwidths that the
    L2 and HBM serve to such gathers, CUDA events on the launching stream,
    best of 5 after 2 warm-up launches."""
    import torch
    from paper_1203_2941_gb300 import rtgb as R
    big = 2 * 2 ** 30
    buf = torch.zeros(big, dtype=torch.uint8, device="cuda")
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.cuda.current_stream()
    res = {}
    for name, nbytes in (("working_set", int(max(32, working_set) // 32 * 32)), ("hbm_2GiB", big)):
        n_reads = 2 ** 30
        ts = []
        for r in range(7):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            R.rt_probe_gather(ctx.h, buf.data_ptr(), nbytes, n_reads, 17 + r, sink.data_ptr(), st.cuda_stream)
            e1.record(st)
            torch.cuda.synchronize()
            if r >= 2:
                ts.append(e0.elapsed_time(e1) / 1e3)
        res[name] = {"bytes": nbytes, "sector_gbs": n_reads * 32 / min(ts) / 1e9,
                     "reads_per_s": n_reads / min(ts)}
    del buf
    torch.cuda.empty_cache()
    return res


def transport_roofline(S, K, t_launch_s, ns, ncell, gp, peaks):
    """The dominant kernel's roofline with the algorithmic bytes of one
    launch: 4 n_s per crossing (density gather), 16 n_s per Lucy deposit
    (FP64 read-modify-write of E_abs), 44 per absorption, scattering, escape
    and MRW step (16 energy tally + 20 event record + 8 table read).  The
    roof is the L2 when the working set, ncell (4 n_s + 8) bytes, fits in
    half of it (measured by the gather probe at that size), else the
    measured HBM copy bandwidth."""
    events = S["absorptions"] + S["scatters"] + S["escaped"] + S["mrw_steps"]
    per = {"density_gathers": 4 * ns * S["crossings"] / K, "lucy_rmw": 16 * ns * S["lucy_deposits"] / K,
           "events": 44 * events / K}
    bytes_alg = sum(per.values())
    ws = ncell * (4 * ns + 8)
    achieved = bytes_alg / t_launch_s / 1e9
    sector = (32 * S["crossings"] + 32 * ns * S["lucy_deposits"] + 96 * events) / K
    if ws <= 0.5 * L2_BYTES:
        bound, peak = "l2", gp["working_set"]["sector_gbs"]
        src = f"measured: rt_probe_gather, random 32-byte sectors in {ws / 1e6:.0f} MB (L2-resident)"
        sector_peak = peak
    else:
        bound, peak = "hbm", float(peaks.get("hbm_gbs") or 6800.0)
        src = "measured (HBM copy bandwidth)" if peaks.get("hbm_gbs") else "fallback"
        sector_peak = gp["hbm_2GiB"]["sector_gbs"]
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_source": src, "bytes_per_launch": bytes_alg, "bytes_by_kind": per,
            "esq_bytes_per_launch": 16 * ns * S["lucy_deposits"] / K,
            "working_set_bytes": ws, "launch_ms": 1e3 * t_launch_s,
            "sector_bytes_per_launch": sector, "sector_achieved": sector / t_launch_s / 1e9,
            "sector_peak": sector_peak, "sector_frac": sector / t_launch_s / 1e9 / sector_peak}


def raytrace_roofline(steps, K, t_s, ns, nfi, ncell, ncam, gp, peaks):
    """Ray march: 4 n_s + 8 F bytes per ray-cell step (density and the thermal
    and scattering emissivities of F image frequencies); the tables of all
    cameras, ncam ncell F 4 bytes, against the roof as for the transport.
    The kernel reads one fused emissivity table (4 n_s + 4 F bytes per step),
    reported as `fused_bytes_per_step`."""
    b = (4 * ns + 8 * nfi) * steps / K
    ws = ncam * ncell * 4 * nfi
    achieved = b / t_s / 1e9
    if ws <= 0.5 * L2_BYTES:
        bound, peak, src = "l2", gp["working_set"]["sector_gbs"], "measured: rt_probe_gather (L2)"
    else:
        bound, peak = "hbm", float(peaks.get("hbm_gbs") or 6800.0)
        src = "measured (HBM copy bandwidth)" if peaks.get("hbm_gbs") else "fallback"
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_source": src, "bytes_per_step": 4 * ns + 8 * nfi,
            "fused_bytes_per_step": 4 * ns + 4 * ((nfi + 3) // 4 * 4), "working_set_bytes": ws}


def run_step_bench(a, rt, ctx, m, K, Wu, flush, local, rank, world, dist, peaks, gp, e2e_steps):
    """Time K steps of the hot path on model m after Wu warm-up steps; returns
    the measurements (per-rank values: the caller reduces over ranks)."""
    import torch
    from paper_1203_2941_gb300 import rtgb as R
    grid, opac, srcs = ctx.grid(m), ctx.opacity(m), rt.Sources(m.sources)
    cams, fidx = image_setup(m, a)
    N = int(a.packets)
    ev_cap = (30 if a.workload == "disk" else 6) * N       # events at the image frequencies
    out = rt.TransportOut(grid.ncell, grid.ns, opac.nf, event_cap=ev_cap)
    ray_steps = torch.zeros(1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    seed_base = 1000 * rank
    tkw = dict(record_events=True, record_nu=sorted(set(fidx)), mrw=a.mrw,
               schedule=R.RT_SCHED_COMPACT if a.schedule == "compact" else R.RT_SCHED_PERSISTENT)
    tuned = None
    if getattr(a, "march_min_active", None) is not None:
        tkw["march_min_active"] = a.march_min_active
        tuned = {"params": {"march_min_active": a.march_min_active}, "fixed": True}
    elif a.schedule == "persistent" and not getattr(a, "no_tune", False):
        # the schedule autotuner (lanes still marching below which a warp
        # serves its interactions) on a bounded sample of the same emission,
        # before and outside the timed steps; the e2e steps use it too
        from paper_1203_2941_gb300.autotune import tune_transport
        t0 = time.perf_counter()
        n_tune = min(N, 10_000_000)
        tr = tune_transport(ctx, grid, opac, srcs, N, sample=n_tune, event_cap=ev_cap * n_tune // N,
                            grid_values={"threads_per_block": (256,)}, repeats=2, **tkw)
        tkw.update(tr.params)
        tuned = {"params": tr.params, "sample_packets": n_tune, "seconds": time.perf_counter() - t0,
                 "candidates_ms": {str(c["march_min_active"]): round(1e3 * t, 3) for c, t in tr.table}}
        log(f"schedule tuned: {tr.params} ({tuned['seconds']:.1f} s)")

    def step(i, ev=None):
        for t in (out.E_abs, out.count, out.esq, out.sed_esc, out.sed_cnt):
            t.zero_()
        out.stats[13:].zero_()                      # event/PAH/trajectory cursors restart
        if ev is not None:
            ev[0].record(stream)
        rt.transport(ctx, grid, opac, srcs, N, out=out, seed=seed_base + i + 1, **tkw)
        if ev is not None:
            ev[1].record(stream)
        T = rt.temperatures(ctx, grid, opac, out.E_abs)
        if ev is not None:
            ev[2].record(stream)
        img, sed = rt.raytrace(ctx, grid, opac, T, out, out.xi, srcs, cams, fidx, steps=ray_steps)
        if ev is not None:
            ev[3].record(stream)
        return T, img, sed

    for i in range(Wu):
        t0 = time.perf_counter()
        step(i)
        torch.cuda.synchronize()
        log(f"warm-up step {i}: {time.perf_counter() - t0:.2f} s, {int(out.stats[0].item())} crossings so far")
    stats0 = out.stats.clone()
    rs0 = ray_steps.clone()
    launches0 = R.rt_kernel_launches()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    with ClockSampler(local) as clk:
        for k in range(K):
            flush.fill_(float(k))                   # evict the grid and tables from L2
            step(Wu + k, evs[k])
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = R.rt_kernel_launches() - launches0
    t_step = [e[0].elapsed_time(e[3]) for e in evs]
    t_tr = [e[0].elapsed_time(e[1]) for e in evs]
    t_T = [e[1].elapsed_time(e[2]) for e in evs]
    t_ray = [e[2].elapsed_time(e[3]) for e in evs]
    st = (out.stats - stats0).cpu().numpy()
    S = {k: int(st[i]) for i, k in enumerate(R.STAT_NAMES)}
    rsteps = int((ray_steps - rs0).item())
    res = {"K": K, "S": S, "rsteps": rsteps, "tot_s": sum(t_step) / 1e3, "t_step": t_step,
           "t_tr": t_tr, "t_T": t_T, "t_ray": t_ray, "launches": launches, "clocks": clk.summary(),
           "roofline": transport_roofline(S, K, sum(t_tr) / K / 1e3, grid.ns, grid.ncell, gp, peaks),
           "ray_roofline": raytrace_roofline(rsteps, K, sum(t_ray) / K / 1e3, grid.ns, len(fidx),
                                             grid.ncell, len(cams), gp, peaks),
           "tuned": tuned}
    log(f"timed {K} steps: {sum(t_step) / 1e3:.2f} s")
    # end to end through the public API with host buffers
    if e2e_steps:
        rho_h = torch.from_numpy(m.rho.copy()).pin_memory()
        E_h = torch.empty((grid.ns, grid.ncell), dtype=torch.float64).pin_memory()
        T_h = torch.empty((grid.ns, grid.ncell), dtype=torch.float64).pin_memory()
        img_h = torch.empty((len(cams), len(fidx), a.npix, a.npix), dtype=torch.float32).pin_memory()
        sed_h = torch.empty((len(cams), len(fidx)), dtype=torch.float64).pin_memory()
        st_h = torch.empty(R.RT_STAT_COUNT, dtype=torch.int64).pin_memory()
        e2e_out = rt.TransportOut(grid.ncell, grid.ns, opac.nf, event_cap=ev_cap)
        cross_e2e = 0
        g2 = grid                                                 # the caller's grid handle, refilled
                                                                  # from host memory every step
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        clk_e2e = ClockSampler(local).__enter__()
        for k in range(-1, e2e_steps):                            # k = -1: untimed warm-up
            if k == 0:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                cross_e2e = 0
            ts0 = time.perf_counter()
            g2.update(rho_h)                                      # H2D of the step's density
            e2e_out.zero_()
            o = rt.transport(ctx, g2, opac, srcs, N, out=e2e_out, seed=50 + k, **tkw)
            torch.cuda.synchronize()
            ts1 = time.perf_counter()
            T = rt.temperatures(ctx, g2, opac, o.E_abs)
            img, sed = rt.raytrace(ctx, g2, opac, T, o, o.xi, srcs, cams, fidx)
            E_h.copy_(o.E_abs, non_blocking=True)
            T_h.copy_(T, non_blocking=True)
            img_h.copy_(img, non_blocking=True)
            sed_h.copy_(sed, non_blocking=True)
            st_h.copy_(o.stats, non_blocking=True)
            torch.cuda.synchronize()
            cross_e2e += int(st_h[0])
            log(f"e2e step {k}: {time.perf_counter() - t0:.2f} s since the timed start "
                f"(update + transport {ts1 - ts0:.3f} s, the rest {time.perf_counter() - ts1:.3f} s)")
        dt = time.perf_counter() - t0
        clk_e2e.__exit__(None, None, None)
        del g2, e2e_out
        res["e2e"] = {"value": cross_e2e / dt, "unit": UNIT,
                      "h2d_bytes_per_step": int(rho_h.numel() * 4),
                      "d2h_bytes_per_step": int(E_h.numel() * 8 + T_h.numel() * 8 + img_h.numel() * 4
                                                + sed_h.numel() * 8 + st_h.numel() * 8),
                      "ms_per_step": 1e3 * dt / e2e_steps, "steps": e2e_steps, "clocks": clk_e2e.summary()}
    del out
    torch.cuda.empty_cache()
    return res


def run_sharded_bench(a, rt, ctx, m, K, Wu, flush, local, rank, world, dist):
    """The multi-GPU form: the iterative scheme sharded by packet id.  Each
    step, every rank transports its N packets of a world * N emission at the
    previous step's temperatures (frozen-T, Eq. 5), the accumulators are summed
    over the ranks (one all-reduce per array), the Eq. 4 temperatures follow
    on every rank, the scattering events are gathered and the cameras traced
    round robin, the images assembled on every rank.  Weak scaling: N packets
    per GPU.  Returns this rank's timings and the summed counters."""
    import torch
    from paper_1203_2941_gb300 import rtgb as R
    from paper_1203_2941_gb300 import shard
    grid, opac, srcs = ctx.grid(m), ctx.opacity(m), rt.Sources(m.sources)
    cams, fidx = image_setup(m, a)
    N = int(a.packets)
    be = shard.DeviceBackend(ctx, grid, opac, srcs, fidx, a.npix, event_cap=6 * N, record_events=True,
                             record_nu=sorted(set(fidx)), mrw=a.mrw)
    state = {"T": rt.temperature_guess(ctx, grid, srcs)}
    stream = torch.cuda.current_stream()

    def step(i, ev=None):
        if ev is not None:
            ev[0].record(stream)
        T, out, local_ev = shard.frozen_t_iterations(be, state["T"], 1, world * N, seed=i + 1,
                                                     rank=rank, world=world)
        if ev is not None:
            ev[1].record(stream)
        events = shard.gather_events(local_ev, world)
        img, sed = shard.raytrace_views(be, T, events, cams, rank, world)
        if ev is not None:
            ev[2].record(stream)
        state["T"] = T
        return out

    for i in range(Wu):
        step(i)
    torch.cuda.synchronize()
    launches0 = R.rt_kernel_launches()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    cross = 0
    with ClockSampler(local) as clk:
        for k in range(K):
            flush.fill_(float(k))
            out = step(Wu + k, evs[k])
            cross += int(out["stats"][0].item())
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_step = [e[0].elapsed_time(e[2]) for e in evs]
    t_tr = [e[0].elapsed_time(e[1]) for e in evs]
    return {"K": K, "crossings_all": cross, "tot_s": sum(t_step) / 1e3, "t_step": t_step, "t_tr": t_tr,
            "launches": R.rt_kernel_launches() - launches0, "clocks": clk.summary()}


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
        return
    if a.forms:
        run_forms(a)
        return
    import torch

    import paper_1203_2941_gb300 as rt

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    rt.build()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    log(f"building the {a.workload} model")
    m = build_model(a)
    ctx = rt.Context(local)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    log("gather probe")
    ncell = int(m.rho.reshape(m.rho.shape[0], -1).shape[1])
    gp = gather_peaks(rt, ctx, ncell * (4 * m.rho.shape[0] + 8))
    K = a.steps
    if world > 1 or a.sharded:
        rs = run_sharded_bench(a, rt, ctx, m, K, a.warmup, flush, local, rank, world, dist)
        tot = torch.tensor([rs["tot_s"]], device="cuda")
        if dist:
            dist.all_reduce(tot, op=dist.ReduceOp.MAX)
        if rank == 0:
            line = {"metric": METRIC, "value": rs["crossings_all"] / float(tot.item()), "unit": UNIT,
                    "n_gpus": world, "steps": K, "warmup": a.warmup,
                    "ms_per_step": 1e3 * float(tot.item()) / K, "higher_is_better": True, "scaling": "weak",
                    "vs_baseline": None, "dtype": "f32",
                    "data": "synthetic (seeded generators shaped like the paper's benchmark models)",
                    "config": workload_config(a, {"mode": "iterative (frozen-T), sharded by packet id",
                                                  "parallelism": f"packet-id shards x{world}, NCCL sum per "
                                                                 "iteration; cameras round robin"}),
                    "phases_ms": {"transport_and_reduce": sum(rs["t_tr"]) / K,
                                  "temperatures_events_raytrace": (sum(rs["t_step"]) - sum(rs["t_tr"])) / K},
                    "clocks": rs["clocks"], "gpu_launches": rs["launches"]}
            print(json.dumps(line), flush=True)
        if dist:
            dist.destroy_process_group()
        return
    r = run_step_bench(a, rt, ctx, m, K, a.warmup, flush, local, rank, world, dist, peaks, gp,
                       0 if a.no_e2e else min(K, 3))
    S = r["S"]
    tot_s = r["tot_s"]
    if dist:
        tt = torch.tensor([tot_s], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        cc = torch.tensor([S["crossings"]], device="cuda", dtype=torch.float64)
        dist.all_reduce(cc)
        tot_s, crossings_all = float(tt.item()), float(cc.item())
    else:
        crossings_all = S["crossings"]
    value = crossings_all / tot_s
    roof = r["roofline"]
    roof["kernel"] = "transport_kernel<float,1,13>" if a.mrw else "transport_kernel<float,1,12>"
    wd = WORKLOADS[a.workload]
    captured = (a.schedule == "persistent" and int(a.packets) == int(wd["packets"]) and a.n == wd["n"]
                and a.tau == wd["tau"] and a.nf == wd["nf"] and bool(a.mrw) == wd["mrw"])
    roof["traffic"] = TRANSPORT_DRAM.get(a.workload) if captured else None
    # the 128^3 r^-2 shell, the other full-size configuration, as a sub-object
    shell = None
    if a.workload == "disk" and not a.no_shell:
        b = argparse.Namespace(**vars(a))
        b.workload = "shell"
        b.march_min_active = None              # tuned for its own workload
        for k in ("packets", "n", "tau", "npix", "nf", "mrw"):
            setattr(b, k, WORKLOADS["shell"][k])
        log("shell sub-object")
        ms = build_model(b)
        gps = gather_peaks(rt, ctx, ms.rho[0].size * 12)
        rs = run_step_bench(b, rt, ctx, ms, min(K, 10), 2, flush, local, rank, world, dist, peaks, gps, 0)
        rs["roofline"]["kernel"] = "transport_kernel<float,1,12>"
        rs["roofline"]["traffic"] = TRANSPORT_DRAM.get("shell")
        shell = {"workload": workload_config(b)["workload"], "metric": METRIC,
                 "value": rs["S"]["crossings"] / rs["tot_s"], "unit": UNIT,
                 "ms_per_step": sum(rs["t_step"]) / len(rs["t_step"]), "steps": rs["K"],
                 "phases_ms": {"transport": sum(rs["t_tr"]) / rs["K"], "temperatures": sum(rs["t_T"]) / rs["K"],
                               "raytrace": sum(rs["t_ray"]) / rs["K"]},
                 "raytrace": {"metric": "ray-cell steps/s", "value": rs["rsteps"] / (sum(rs["t_ray"]) / 1e3),
                              "roofline": rs["ray_roofline"]},
                 "roofline": rs["roofline"], "gather_probe": gps, "schedule_tuning": rs["tuned"]}
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        log("oracle baseline")
        cpu = cpu_baseline(m, a)
        log("oracle baseline done")
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
                "warmup": a.warmup, "ms_per_step": sum(r["t_step"]) / len(r["t_step"]),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (seeded generators shaped like the paper's benchmark models)",
                "config": workload_config(a, {"parallelism": "1 GPU"}),
                "phases_ms": {"transport": sum(r["t_tr"]) / K, "temperatures": sum(r["t_T"]) / K,
                              "raytrace": sum(r["t_ray"]) / K},
                "raytrace": {"metric": "ray-cell steps/s", "value": r["rsteps"] / (sum(r["t_ray"]) / 1e3),
                             "ray_cell_steps_per_step": r["rsteps"] // K, "roofline": r["ray_roofline"]},
                "stats_per_step": {k: v // K for k, v in S.items() if not k.startswith("n_")},
                "roofline": roof, "gather_probe": gp, "cpu_baseline": cpu, "e2e": r.get("e2e"),
                "clocks": r["clocks"], "gpu_launches": r["launches"], "schedule_tuning": r["tuned"],
                "shell_128": shell}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
