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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--packets", type=float, default=1e7)
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--tau", type=float, default=10.0)
    ap.add_argument("--npix", type=int, default=256)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
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
    return {"value": r["stats"]["crossings"] / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n} packets of the {N:.0e}-packet B&W emission (packet ids 0..{n - 1}), "
                      f"{r['stats']['crossings']} crossings in {dt:.1f} s"}


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
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": None, "kernel": "transport_kernel<float,1>", "peak_source": peak_src,
            "bytes_per_launch": bytes_alg, "launch_ms": t_tr_s * 1e3}

    # end to end through the public API with host buffers
    e2e = None
    if not a.no_e2e:
        rho_h = torch.from_numpy(m.rho.copy()).pin_memory()
        E_h = torch.empty((1, grid.ncell), dtype=torch.float64).pin_memory()
        T_h = torch.empty((1, grid.ncell), dtype=torch.float64).pin_memory()
        img_h = torch.empty((len(cams), len(fidx), a.npix, a.npix), dtype=torch.float32).pin_memory()
        sed_h = torch.empty((len(cams), len(fidx)), dtype=torch.float64).pin_memory()
        st_h = torch.empty(16, dtype=torch.int64).pin_memory()
        e2e_out = rt.TransportOut(grid.ncell, 1, opac.nf, event_cap=ev_cap)
        cross_e2e = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(a.steps):
            g2 = rt.Grid(ctx, rho_h, m.box_min, m.cell)           # H2D of the density grid
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
            del g2
        dt = time.perf_counter() - t0
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
