"""Parity at the benchmark's full size (r^-2 shell, 128^3 cells, tau(1 um) = 10,
64 frequencies, 1e7 packets, B&W, FP32 with FP64 accumulators, Lucy in thin
cells, event store), in the launch configuration the benchmark times.  The
oracle cannot run 1e7 B&W packets, so the checks are ones it can make one by
one or that hold at any size:

* exact conservation and counts (every packet escapes once, the escaped SED
  sums to L, absorption counts match the absorption events);
* Eq. 4 temperatures of sampled cells against the oracle's per-cell solve;
* FP64 trajectories of a sample of packet ids of the same 1e7-packet
  emission on the full grid (order-independent frozen-T mode);
* the FP32 production transport of all 1e7 packets in the frozen-T mode
  against the oracle's own 1e7-packet frozen-T run on every host core:
  per-cell absorbed energies within max(3 sigma, 1e-3 E) (binomial outlier
  allowance and chi-square of statcheck), the escaped SED per bin within
  3 sigma, and Eq. 4 temperatures within max(0.5 %, 3 sigma_T) on cells whose
  energy both runs sample to 1 % (binomial allowance for the 3-sigma part);
* the ray-traced images of one full-size camera at two image frequencies,
  from the GPU's temperatures and stored events, against the oracle's.
"""
import math

import numpy as np
import pytest

import workloads as W
from imgcheck import assert_images_close
from statcheck import assert_outliers, assert_same_energies, assert_same_sed

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    import __graft_entry__ as g
    g.build()
    import paper_1203_2941_gb300 as rt
    return rt


@pytest.fixture(scope="module")
def setup(rt):
    import torch
    ctx = rt.Context(0)
    m = W.r2_shell(n=128, tau_1um=10.0, nf=64)
    grid, opac, srcs = ctx.grid(m), ctx.opacity(m), rt.Sources(m.sources)
    N = 10 ** 7
    out = rt.transport(ctx, grid, opac, srcs, N, event_cap=6 * N, record_events=True, seed=7)
    T = rt.temperatures(ctx, grid, opac, out.E_abs)
    torch.cuda.synchronize()
    return ctx, m, grid, opac, srcs, N, out, T


def test_full_size_conservation_and_counts(setup):
    ctx, m, grid, opac, srcs, N, out, T = setup
    g = out.numpy()
    st = out.stats_dict()
    assert st["emitted"] == N and st["escaped"] == N and st["stuck"] == 0
    assert abs(g["sed_esc"].sum() / m.luminosity - 1) < 1e-9
    assert int(g["sed_cnt"].sum()) == N
    assert int(g["count"].sum()) == st["absorptions"]
    assert st["n_events"] == st["scatters"] and st["events_dropped"] == 0
    assert np.all(np.isfinite(g["E_abs"])) and np.all(g["E_abs"] >= 0)
    assert st["crossings"] > 100 * N and st["lucy_deposits"] > 0


def test_full_size_temperatures_on_sampled_cells(setup, O):
    ctx, m, grid, opac, srcs, N, out, T = setup
    E = out.E_abs.cpu().numpy()[0]
    Tg = T.cpu().numpy()[0]
    rho = m.rho.reshape(-1).astype(np.float64)
    V = m.cell ** 3
    cells = np.nonzero((E > 0) & (rho > 0))[0]
    sample = np.random.default_rng(5).choice(cells, size=300, replace=False)
    for c in sample:
        Tr = O.solve_temperature(m, 0, E[c] / (rho[c] * V))
        assert abs(Tg[c] / Tr - 1) < 1e-10, (c, Tg[c], Tr)


def test_full_size_fp64_trajectories_of_sampled_packets(rt, setup, O):
    import torch
    ctx, m, grid, opac, srcs, N, out, T = setup
    T0 = O.temperature_guess(m)
    b, e = 5_000_000, 5_000_300                   # packet ids of the 1e7 emission
    g = rt.transport(ctx, grid, opac, srcs, N, mode=rt.rtgb.RT_MODE_FROZEN_T,
                     precision=rt.rtgb.RT_PREC_FP64, T_prev=torch.tensor(T0, device="cuda"),
                     pid_begin=b, pid_end=e, traj_cap=400000, seed=7)
    torch.cuda.synchronize()
    ref = O.transport(m, N, seed=7, mode=O.MODE_FROZEN_T, T_prev=T0, pid_begin=b, pid_end=e,
                      traj_cap=400000)
    tg = np.sort(g.traj_numpy(), order=["pid", "seq"])
    tr = np.sort(ref["traj"], order=["pid", "seq"])
    assert len(tg) == len(tr) > 0
    for f in ("pid", "seq", "type", "cell", "nu"):
        np.testing.assert_array_equal(tg[f], tr[f])
    scale = m.cell * 128
    assert np.max(np.abs(tg["x"] - tr["x"])) <= 1e-9 * scale
    assert np.max(np.abs(tg["k"] - tr["k"])) <= 1e-8
    st = g.stats_dict()
    for k in ("crossings", "interactions", "absorptions", "escaped", "lucy_deposits"):
        assert st[k] == ref["stats"][k], k


def test_full_size_images_of_one_camera(rt, setup, O):
    import torch
    ctx, m, grid, opac, srcs, N, out, T = setup
    fidx_all = W.nearest_freq_indices(m.nu, W.image_wavelengths_um())
    fidx = [fidx_all[0], fidx_all[6]]              # 0.55 and 10 micron
    cam = [W.Camera(math.radians(W.inclinations_deg()[2]), 0.0, 256, 140 * W.PC)]
    img, sed = rt.raytrace(ctx, grid, opac, T, out, out.xi, srcs, cam, fidx)
    torch.cuda.synchronize()
    ev = out.events_numpy()
    ir, sr = O.raytrace(m, T.cpu().numpy(), ev, out.xi, cam, fidx)
    assert_images_close(img.cpu().numpy(), ir, rtol=1e-5, floor=1e-3)
    np.testing.assert_allclose(sed.cpu().numpy(), sr, rtol=1e-5)


def test_full_size_fp32_frozen_transport_matches_oracle(rt, setup, O):
    import os

    import torch
    ctx, m, grid, opac, srcs, N, out, T = setup
    T0 = O.temperature_guess(m)
    g = rt.transport(ctx, grid, opac, srcs, N, mode=rt.rtgb.RT_MODE_FROZEN_T,
                     T_prev=torch.tensor(T0, device="cuda"), seed=9)
    torch.cuda.synchronize()
    g = g.numpy()
    cores = os.cpu_count() or 1
    ref = O.transport(m, N, seed=10, mode=O.MODE_FROZEN_T, T_prev=T0, n_threads=cores)
    ref2 = O.transport(m, N, seed=11, mode=O.MODE_FROZEN_T, T_prev=T0, n_threads=cores)
    xi = m.luminosity / N
    assert g["stats"]["escaped"] == N and abs(g["sed_esc"].sum() / m.luminosity - 1) < 1e-9
    # 64 spatial blocks of 32^3 cells for the paired chi-square test
    i = np.arange(m.ncell)
    blocks = ((i // (128 * 128)) // 32) * 16 + (((i // 128) % 128) // 32) * 4 + (i % 128) // 32
    phi, ncell = assert_same_energies(g, ref, ref2, xi, blocks=blocks)
    assert ncell > 10000
    assert assert_same_sed(g, ref, xi) > 300
    # Eq. 4 temperatures where both runs sample the cell's energy to 1 %
    E, Er = g["E_abs"][0], ref["E_abs"][0]
    with np.errstate(divide="ignore", invalid="ignore"):
        rg = np.sqrt(g["esq"][0]) / E
        rr = np.sqrt(ref["esq"][0]) / Er
    rho = m.rho.reshape(-1).astype(np.float64)
    good = np.nonzero((E > 0) & (Er > 0) & (rho > 0) & (rg < 0.01) & (rr < 0.01))[0]
    assert good.size >= 20
    pick = np.random.default_rng(3).choice(good, size=min(good.size, 1500), replace=False)
    V = m.cell ** 3
    # within 0.5 %, or within 3 sigma_T where the sampling noise of both runs
    # exceeds that (sigma_T / T = sqrt(rg^2 + rr^2) / 4 is up to 0.35 % at 1 %),
    # with the binomial allowance for the 3-sigma part
    n_bad = 0
    for c in pick:
        Tg = O.solve_temperature(m, 0, E[c] / (rho[c] * V))
        Tr = O.solve_temperature(m, 0, Er[c] / (rho[c] * V))
        sT = 0.25 * math.sqrt(phi * (rg[c] ** 2 + rr[c] ** 2))
        n_bad += abs(Tg / Tr - 1) > max(0.005, 3 * sT)
    assert_outliers(n_bad, len(pick), "temperatures")
