"""GPU transport against the FP64 CPU oracle (run on a GB300).

* Philox on the device is bit-exact with the oracle's.
* FP64 debug build: per-packet trajectories (event types, cells, frequencies,
  positions, directions) agree with the oracle to 1e-9 relative on small
  irregular grids, for frozen-temperature transport on all SMs, Bjorkman &
  Wood transport in the one-lane serial schedule, 1-3 species, the Lucy
  variants and the modified random walk; accumulated energies agree to 1e-9.
* FP32 production build: per-cell absorbed energy within
  max(3 sigma, 1e-3 E) and escaped SED within 3 sigma, with the binomial
  outlier allowance and chi-square bound of statcheck (false-alarm rate
  1e-6 each); temperatures within 0.5% where the relative sigma of E is below
  1%; exact energy conservation.
* Edge cases: empty grid, source on a cell face, empty packet range, event
  and PAH buffer overflow, the per-packet event cap, ragged grid shapes.
"""
import copy
import math

import numpy as np
import pytest
import torch

import workloads as W
from statcheck import assert_outliers, assert_same_energies, assert_same_sed

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    import __graft_entry__ as g
    g.build()
    import paper_1203_2941_gb300 as rt
    return rt


@pytest.fixture(scope="module")
def ctx(rt):
    return rt.Context(0)


def _setup(rt, ctx, m):
    return ctx.grid(m), ctx.opacity(m), rt.Sources(m.sources)


def _traj_compare(tg, tr, scale, rtol=1e-9):
    tg = np.sort(tg, order=["pid", "seq"])
    tr = np.sort(tr, order=["pid", "seq"])
    assert len(tg) == len(tr), (len(tg), len(tr))
    for f in ("pid", "seq", "type", "cell", "nu"):
        bad = np.nonzero(tg[f] != tr[f])[0]
        assert bad.size == 0, (f, bad[:5], tg[bad[:3]], tr[bad[:3]])
    assert np.max(np.abs(tg["x"] - tr["x"])) <= rtol * scale
    assert np.max(np.abs(tg["k"] - tr["k"])) <= rtol * 10


def test_philox_bit_exact(rt, ctx, O):
    rng = np.random.default_rng(0)
    for _ in range(4):
        ctr = [int(v) for v in rng.integers(0, 2**32 - 5000, 4)]
        key = [int(v) for v in rng.integers(0, 2**32, 2)]
        out = rt.philox(ctx, ctr, key, 4096).reshape(-1, 4)
        for i in (0, 1, 77, 4095):
            c = [ctr[0] + i, ctr[1], ctr[2], ctr[3]]
            np.testing.assert_array_equal(out[i], O.philox(c, key))


@pytest.mark.parametrize("ns,lucy", [(1, 1), (2, 0), (3, 2), (1, 2)])
def test_fp64_frozen_trajectories_match_oracle(rt, ctx, O, ns, lucy):
    m = W.random_grid(n=(7, 5, 6), ns=ns, seed=10 + ns, tau_scale=2.0, albedo=(0.3, 0.8))
    grid, opac, srcs = _setup(rt, ctx, m)
    rng = np.random.default_rng(ns)
    T0 = rng.uniform(30, 900, size=(ns, m.ncell))
    N = 600
    out = rt.transport(ctx, grid, opac, srcs, N, mode=rt.rtgb.RT_MODE_FROZEN_T, lucy_mode=lucy,
                       precision=rt.rtgb.RT_PREC_FP64, T_prev=torch.tensor(T0, device="cuda"),
                       traj_cap=400 * N, event_cap=100 * N, record_events=True, seed=77)
    torch.cuda.synchronize()
    ref = O.transport(m, N, seed=77, mode=O.MODE_FROZEN_T, lucy_mode=lucy, T_prev=T0,
                      traj_cap=400 * N, event_cap=100 * N, record_events=True)
    st = out.stats_dict()
    assert st["traj_dropped"] == 0 and ref["stats"]["traj_dropped"] == 0
    _traj_compare(out.traj_numpy(), ref["traj"], m.cell * 7)
    for k in ("crossings", "interactions", "scatters", "absorptions", "escaped", "lucy_deposits"):
        assert st[k] == ref["stats"][k], k
    g = out.numpy()
    np.testing.assert_array_equal(g["count"], ref["count"])
    np.testing.assert_allclose(g["E_abs"], ref["E_abs"], rtol=1e-9, atol=1e-12 * ref["E_abs"].max())
    np.testing.assert_allclose(g["sed_esc"], ref["sed_esc"], rtol=1e-9, atol=0)
    ev = out.events_numpy()
    assert len(ev) == len(ref["events"])
    key = lambda e: np.lexsort((e["nu"], e["cell"]))
    a, b = ev[key(ev)], ref["events"][key(ref["events"])]
    np.testing.assert_array_equal(a["cell"], b["cell"])


def test_fp64_bw_serial_trajectories_match_oracle(rt, ctx, O):
    m = W.random_grid(n=(5, 6, 4), ns=2, seed=21, tau_scale=3.0, albedo=(0.1, 0.5))
    grid, opac, srcs = _setup(rt, ctx, m)
    N = 300
    out = rt.transport(ctx, grid, opac, srcs, N, mode=rt.rtgb.RT_MODE_BW,
                       precision=rt.rtgb.RT_PREC_FP64, schedule=rt.rtgb.RT_SCHED_SERIAL,
                       traj_cap=400 * N, seed=3)
    torch.cuda.synchronize()
    ref = O.transport(m, N, seed=3, mode=O.MODE_BW, traj_cap=400 * N)
    _traj_compare(out.traj_numpy(), ref["traj"], m.cell * 6)
    g = out.numpy()
    np.testing.assert_allclose(g["E_abs"], ref["E_abs"], rtol=1e-9, atol=1e-12 * ref["E_abs"].max())
    assert abs(g["sed_esc"].sum() / m.luminosity - 1) < 1e-12


def test_fp64_mrw_trajectories_match_oracle(rt, ctx, O):
    m = W.uniform_cube(n=3, tau_cell=14.0, nf=5, albedo=0.5)
    grid, opac, srcs = _setup(rt, ctx, m)
    T0 = np.full((1, m.ncell), 300.0)
    N = 120
    out = rt.transport(ctx, grid, opac, srcs, N, mode=rt.rtgb.RT_MODE_FROZEN_T, mrw=True,
                       precision=rt.rtgb.RT_PREC_FP64, T_prev=torch.tensor(T0, device="cuda"),
                       traj_cap=5000 * N, seed=9)
    torch.cuda.synchronize()
    ref = O.transport(m, N, seed=9, mode=O.MODE_FROZEN_T, mrw=True, T_prev=T0, traj_cap=5000 * N)
    assert ref["stats"]["mrw_steps"] > 0
    _traj_compare(out.traj_numpy(), ref["traj"], m.cell * 3)
    assert out.stats_dict()["mrw_steps"] == ref["stats"]["mrw_steps"]


@pytest.mark.parametrize("schedule", ["persistent", "serial"])
def test_deferred_packets_keep_their_trajectories(rt, ctx, O, schedule):
    """defer_events sets packets aside at a flight start and finishes them in
    a second pass: in the order-independent frozen-T mode (FP64) every
    trajectory, count and energy still equals the oracle's, with and without
    MRW steps; in FP32 B&W every packet still escapes exactly once."""
    sch = rt.rtgb.RT_SCHED_PERSISTENT if schedule == "persistent" else rt.rtgb.RT_SCHED_SERIAL
    for m, mrw, N in ((W.random_grid(n=(7, 5, 6), ns=2, seed=12, tau_scale=3.0, albedo=(0.3, 0.8)), False, 400),
                      (W.uniform_cube(n=5, tau_cell=12.0, nf=8, albedo=0.4, gray=True), True, 200)):
        grid, opac, srcs = _setup(rt, ctx, m)
        T0 = np.random.default_rng(3).uniform(30, 900, size=(m.ns, m.ncell))
        out = rt.transport(ctx, grid, opac, srcs, N, mode=rt.rtgb.RT_MODE_FROZEN_T, mrw=mrw,
                           precision=rt.rtgb.RT_PREC_FP64, T_prev=torch.tensor(T0, device="cuda"),
                           schedule=sch, traj_cap=1500 * N, seed=78, defer_events=2)
        torch.cuda.synchronize()
        ref = O.transport(m, N, seed=78, mode=O.MODE_FROZEN_T, mrw=mrw, T_prev=T0, traj_cap=1500 * N)
        st = out.stats_dict()
        assert st["deferred"] > 0 and st["traj_dropped"] == 0
        # the same run without deferral: bit-identical trajectories
        plain = rt.transport(ctx, grid, opac, srcs, N, mode=rt.rtgb.RT_MODE_FROZEN_T, mrw=mrw,
                             precision=rt.rtgb.RT_PREC_FP64, T_prev=torch.tensor(T0, device="cuda"),
                             schedule=sch, traj_cap=1500 * N, seed=78)
        torch.cuda.synchronize()
        a = np.sort(out.traj_numpy(), order=["pid", "seq"])
        b = np.sort(plain.traj_numpy(), order=["pid", "seq"])
        assert len(a) == len(b)
        for f in ("pid", "seq", "type", "cell", "nu", "x", "k"):
            np.testing.assert_array_equal(a[f], b[f])
        # and the oracle's (long MRW walks accumulate rounding: 1e-8 of the grid)
        _traj_compare(out.traj_numpy(), ref["traj"], m.cell * 7, rtol=1e-9 if not mrw else 1e-8)
        for k in ("crossings", "interactions", "absorptions", "escaped", "lucy_deposits", "mrw_steps",
                  "emitted"):
            assert st[k] == ref["stats"][k], k
        g = out.numpy()
        np.testing.assert_array_equal(g["count"], ref["count"])
        np.testing.assert_allclose(g["E_abs"], ref["E_abs"], rtol=1e-9, atol=1e-12 * ref["E_abs"].max())
    m = W.r2_shell(n=16, tau_1um=10.0, nf=24)
    grid, opac, srcs = _setup(rt, ctx, m)
    out = rt.transport(ctx, grid, opac, srcs, 20000, schedule=sch, defer_events=1, seed=5)
    torch.cuda.synchronize()
    st = out.stats_dict()
    assert st["deferred"] > 0 and st["escaped"] == 20000 and st["stuck"] == 0
    assert abs(out.numpy()["sed_esc"].sum() / m.luminosity - 1) < 1e-9


def test_fp64_several_sources_random_bins_match_oracle(rt, ctx, O):
    """Several sources with random frequency bins (Sect. 2): each packet's
    source is drawn by luminosity, then its bin from that source's own
    spectrum.  FP64 trajectories of three blackbody sources of different
    luminosity and temperature equal the oracle's to 1e-9."""
    m = W.random_grid(n=(6, 5, 4), ns=2, seed=16, tau_scale=1.5, albedo=(0.3, 0.7))
    p0 = np.asarray(m.sources[0].pos)
    m.sources = [W.Source(tuple(p0), 2.0 * W.LSUN, 5800.0),
                 W.Source(tuple(0.5 * p0), 1.0 * W.LSUN, 3500.0),
                 W.Source(tuple(0.3 * p0), 0.5 * W.LSUN, 900.0)]
    grid, opac, srcs = _setup(rt, ctx, m)
    T0 = np.random.default_rng(5).uniform(50, 800, size=(m.ns, m.ncell))
    N = 1500
    out = rt.transport(ctx, grid, opac, srcs, N, mode=rt.rtgb.RT_MODE_FROZEN_T,
                       precision=rt.rtgb.RT_PREC_FP64, T_prev=torch.tensor(T0, device="cuda"),
                       traj_cap=600 * N, seed=23)
    torch.cuda.synchronize()
    ref = O.transport(m, N, seed=23, mode=O.MODE_FROZEN_T, T_prev=T0, traj_cap=600 * N)
    tg = out.traj_numpy()
    _traj_compare(tg, ref["traj"], m.cell * 7)
    em = tg[tg["type"] == O.T_EMIT]
    starts = {tuple(np.round(x / m.cell, 6)) for x in em["x"]}
    assert len(starts) == 3                      # every source emitted


def test_equal_energy_source_bins_match_oracle(rt, ctx, O):
    """Eq. 1 source grid (source_bins = m): FP64 trajectories equal the
    oracle's; in FP32 the emission histogram (empty grid, every packet escapes
    at its emission frequency) equals the oracle's bin by bin."""
    m = W.random_grid(n=(6, 5, 4), ns=2, seed=15, tau_scale=1.5, albedo=(0.3, 0.7))
    m.sources = [W.Source(m.sources[0].pos, 2.0 * W.LSUN, 5800.0),
                 W.Source(tuple(0.5 * np.asarray(m.sources[0].pos)), 1.0 * W.LSUN, 3500.0)]
    grid, opac, srcs = _setup(rt, ctx, m)
    T0 = np.random.default_rng(4).uniform(50, 800, size=(m.ns, m.ncell))
    N = 1200
    out = rt.transport(ctx, grid, opac, srcs, N, mode=rt.rtgb.RT_MODE_FROZEN_T,
                       precision=rt.rtgb.RT_PREC_FP64, T_prev=torch.tensor(T0, device="cuda"),
                       traj_cap=600 * N, seed=21, source_bins=120)
    torch.cuda.synchronize()
    ref = O.transport(m, N, seed=21, mode=O.MODE_FROZEN_T, T_prev=T0, traj_cap=600 * N,
                      source_bins=120)
    _traj_compare(out.traj_numpy(), ref["traj"], m.cell * 7)
    e = copy.deepcopy(m)
    e.rho = np.zeros_like(m.rho)
    g0, o0, s0 = _setup(rt, ctx, e)
    N = 240000
    out = rt.transport(ctx, g0, o0, s0, N, mode=rt.rtgb.RT_MODE_NOREEMIT, seed=3, source_bins=4000)
    torch.cuda.synchronize()
    ref = O.transport(e, N, seed=3, mode=O.MODE_NOREEMIT, source_bins=4000)
    hg = out.numpy()["sed_cnt"].sum(axis=0)
    hr = ref["sed_cnt"].sum(axis=0)
    assert hg.sum() == hr.sum() == N
    # FP32 bin searches may move a source bin across a frequency-bin edge only
    # where its midpoint lies within FP32 rounding of the edge
    assert np.abs(hg - hr).sum() <= 2 * (N // 4000)
    with pytest.raises(rt.RtError):
        rt.transport(ctx, g0, o0, s0, 100, source_bins=101)


def test_separate_source_grid_matches_oracle(rt, ctx, O):
    """The separate source grid of Eq. 1 (rt_source_grid, equal-energy bins on
    the sources' continuous spectra): the library's table (an independent
    quadrature) equals the oracle's (series) bin for bin and its frequencies
    to 1e-11; FP64 trajectories of the transport emitting from it equal the
    oracle's; in FP32 the emission histogram (empty grid, every packet
    escapes at its emission frequency) is exactly N/m packets per source bin
    in its model bin; bad tables are refused."""
    m = W.random_grid(n=(6, 5, 4), ns=2, seed=15, tau_scale=1.5, albedo=(0.3, 0.7), nf=40)
    lnu = np.zeros(m.nf)
    lnu[5:30] = np.linspace(2.0, 0.5, 25)
    m.sources = [W.Source(m.sources[0].pos, 2.0 * W.LSUN, 5800.0),
                 W.Source(tuple(0.5 * np.asarray(m.sources[0].pos)), 1.0 * W.LSUN, 0.0, lnu),
                 W.Source(tuple(0.3 * np.asarray(m.sources[0].pos)), 0.5 * W.LSUN, 900.0)]
    grid, opac, srcs = _setup(rt, ctx, m)
    mb = 350
    nu_g, src_g, f_g = rt.source_grid(opac, srcs, mb)
    nu_o, src_o, f_o = O.source_grid(m, mb)
    np.testing.assert_array_equal(src_g, src_o)
    np.testing.assert_array_equal(nu_g, nu_o)
    np.testing.assert_allclose(f_g, f_o, rtol=1e-11)
    T0 = np.random.default_rng(4).uniform(50, 800, size=(m.ns, m.ncell))
    N = 1400
    out = rt.transport(ctx, grid, opac, srcs, N, mode=rt.rtgb.RT_MODE_FROZEN_T,
                       precision=rt.rtgb.RT_PREC_FP64, T_prev=torch.tensor(T0, device="cuda"),
                       traj_cap=600 * N, seed=22, source_bins=mb, source_grid=(nu_g, src_g))
    torch.cuda.synchronize()
    ref = O.transport(m, N, seed=22, mode=O.MODE_FROZEN_T, T_prev=T0, traj_cap=600 * N,
                      source_bins=mb, source_grid=(nu_o, src_o))
    _traj_compare(out.traj_numpy(), ref["traj"], m.cell * 7)
    e = copy.deepcopy(m)
    e.rho = np.zeros_like(m.rho)
    g0, o0, s0 = _setup(rt, ctx, e)
    N = 100 * mb
    out = rt.transport(ctx, g0, o0, s0, N, mode=rt.rtgb.RT_MODE_NOREEMIT, seed=3, source_bins=mb,
                       source_grid=(nu_g, src_g))
    torch.cuda.synchronize()
    hg = out.numpy()["sed_cnt"].sum(axis=0)
    np.testing.assert_array_equal(hg, 100 * np.bincount(nu_g, minlength=m.nf))
    bad = nu_g.copy()
    bad[7] = m.nf
    with pytest.raises(rt.RtError):
        rt.transport(ctx, g0, o0, s0, N, source_bins=mb, source_grid=(bad, src_g))


def test_fp64_pah_and_noreemit_match_oracle(rt, ctx, O):
    m = W.clumpy_torus(n=12, n_clump=40, seed=5, nf=20)
    grid, opac, srcs = _setup(rt, ctx, m)
    N = 300
    out = rt.transport(ctx, grid, opac, srcs, N, mode=rt.rtgb.RT_MODE_BW,
                       precision=rt.rtgb.RT_PREC_FP64, schedule=rt.rtgb.RT_SCHED_SERIAL,
                       traj_cap=300 * N, pah_cap=N, seed=4)
    torch.cuda.synchronize()
    ref = O.transport(m, N, seed=4, mode=O.MODE_BW, traj_cap=300 * N, pah_cap=N)
    _traj_compare(out.traj_numpy(), ref["traj"], m.cell * 12)
    assert out.stats_dict()["pah"] == ref["stats"]["pah"] > 0
    m2 = W.random_grid(n=(4, 4, 5), seed=2, tau_scale=2.0)
    grid2, opac2, srcs2 = _setup(rt, ctx, m2)
    out2 = rt.transport(ctx, grid2, opac2, srcs2, 500, mode=rt.rtgb.RT_MODE_NOREEMIT,
                        precision=rt.rtgb.RT_PREC_FP64, traj_cap=100000, seed=8)
    torch.cuda.synchronize()
    ref2 = O.transport(m2, 500, seed=8, mode=O.MODE_NOREEMIT, traj_cap=100000)
    _traj_compare(out2.traj_numpy(), ref2["traj"], m2.cell * 5)


def test_fp32_bw_statistics_match_oracle_homogeneous_sphere(rt, ctx, O):
    """Homogeneous sphere (32^3 in the full-size configuration; 16^3 here so
    the B&W oracle finishes in seconds), B&W, Lucy in thin cells: per-cell
    E_abs within max(3 sigma, 1e-3 E) with the binomial allowance of
    statcheck, the chi-square of the per-cell differences, the escaped SED
    per bin within 3 sigma, exact conservation, and temperatures within
    3 sigma_T + 0.5 % where both runs sample the energy to 10 %."""
    m = W.homogeneous_sphere(n=16, tau_v=1.0)
    grid, opac, srcs = _setup(rt, ctx, m)
    N = 400000
    out = rt.transport(ctx, grid, opac, srcs, N, seed=11)
    torch.cuda.synchronize()
    ref = O.transport(m, N, seed=12, mode=O.MODE_BW)
    ref2 = O.transport(m, N, seed=13, mode=O.MODE_BW)
    g = out.numpy()
    xi = m.luminosity / N
    assert abs(g["sed_esc"].sum() / m.luminosity - 1) < 1e-12
    assert g["stats"]["escaped"] == N
    phi, ncell = assert_same_energies(g, ref, ref2, xi)
    assert ncell > 800
    assert assert_same_sed(g, ref, xi) > 100
    # total absorbed energy (cells of one packet are correlated: phi-scaled)
    sig = np.sqrt(g["esq"] + ref["esq"])
    tot_sig = math.sqrt(phi * (sig ** 2).sum())
    assert abs(g["E_abs"].sum() - ref["E_abs"].sum()) < 3 * tot_sig + 1e-3 * ref["E_abs"].sum()
    # temperatures (T ~ E^(1/4)) within 3 sigma_T + 0.5 % where both runs'
    # energies are sampled to 10 % (the full-size test holds cells sampled to
    # 1 %, where the stated 0.5 % applies on its own)
    Tg = O.temperatures(m, g["E_abs"])
    Tr = O.temperatures(m, ref["E_abs"])
    with np.errstate(divide="ignore", invalid="ignore"):
        rg = np.sqrt(g["esq"]) / g["E_abs"]
        rr = np.sqrt(ref["esq"]) / ref["E_abs"]
    good = (g["E_abs"] > 0) & (ref["E_abs"] > 0) & (rg < 0.1) & (rr < 0.1)
    assert good.sum() > 100
    sT = 0.25 * np.sqrt(phi * (rg[good] ** 2 + rr[good] ** 2))
    dT = np.abs(Tg[good] / Tr[good] - 1)
    assert_outliers(int((dT > 3 * sT + 0.005).sum()), int(good.sum()), "temperatures")


def test_fp32_frozen_statistics_and_packet_ranges(rt, ctx, O):
    m = W.r2_shell(n=16, tau_1um=10.0, nf=32)
    grid, opac, srcs = _setup(rt, ctx, m)
    T0 = O.temperature_guess(m)
    N = 300000
    Tt = torch.tensor(T0, device="cuda")
    out = rt.transport(ctx, grid, opac, srcs, N, mode=rt.rtgb.RT_MODE_FROZEN_T, T_prev=Tt, seed=2)
    # the same emission split into two packet ranges accumulates identically
    out2 = rt.transport(ctx, grid, opac, srcs, N, mode=rt.rtgb.RT_MODE_FROZEN_T, T_prev=Tt, seed=2,
                        pid_begin=0, pid_end=N // 3)
    rt.transport(ctx, grid, opac, srcs, N, out=out2, mode=rt.rtgb.RT_MODE_FROZEN_T, T_prev=Tt,
                 seed=2, pid_begin=N // 3, pid_end=N)
    torch.cuda.synchronize()
    g, g2 = out.numpy(), out2.numpy()
    np.testing.assert_array_equal(g["count"], g2["count"])
    assert g["stats"]["crossings"] == g2["stats"]["crossings"]
    np.testing.assert_allclose(g["E_abs"], g2["E_abs"], rtol=1e-9, atol=1e-9 * g["E_abs"].max())
    ref = O.transport(m, N, seed=3, mode=O.MODE_FROZEN_T, T_prev=T0, n_threads=8)
    ref2 = O.transport(m, N, seed=4, mode=O.MODE_FROZEN_T, T_prev=T0, n_threads=8)
    xi = m.luminosity / N
    assert assert_same_energies(g, ref, ref2, xi)[1] > 100
    assert assert_same_sed(g, ref, xi) > 100
    assert abs(g["sed_esc"].sum() / m.luminosity - 1) < 1e-12


def test_fp32_mrw_path_lengths_match_the_series(rt, ctx, O):
    """The FP32 transport's MRW path-length draws (Sect. 3.2) against the
    oracle's FP64 inversion of the survival series, for uniforms on the FP32
    grid the kernel draws ((k + 1) 2^-24, k < 2^24), including both ends.
    Pointwise: within 1e-5 in y where u <= 0.9 (|S'(y)| > 0.05 there, so the
    table's FP32 rounding and linear interpolation stay far below that) and
    within 2e-4 everywhere (towards u = 1 the slope of S vanishes and the
    FP32 rounding of S, 6e-8, maps to up to ~1e-4 in y); <y> = 1/6 of the
    series.  Distribution: a KS test of 1e6 draws against 1 - S(y)."""
    from scipy import stats
    m = W.uniform_cube(n=2, tau_cell=20.0, nf=4)
    opac = ctx.opacity(m)
    rng = np.random.default_rng(7)
    k = rng.integers(0, 2 ** 24, 10 ** 6)
    ends = np.array([0, 1, 2, 3, 2 ** 24 - 4, 2 ** 24 - 3, 2 ** 24 - 2, 2 ** 24 - 1])
    k = np.concatenate([ends, k])
    u = ((k + 1).astype(np.float64) * 2.0 ** -24).astype(np.float32)
    y = rt.mrw_sample(ctx, opac, u).astype(np.float64)
    assert np.all(np.isfinite(y)) and np.all(y >= 0)
    assert y[ends.size - 1] == 0.0                         # u = 1: no path
    npt = 30000
    yr = np.array([O.mrw_sample_y(float(v)) for v in u[:npt]])
    err = np.abs(y[:npt] - yr)
    low = u[:npt] <= 0.9
    assert err[low].max() <= 1e-5, err[low].max()
    assert err.max() <= 2e-4, err.max()
    body = y[ends.size:]
    assert abs(body.mean() - 1.0 / 6.0) < 5 * math.sqrt(1.0 / 90.0 / body.size)
    F = 1.0 - np.array([O.mrw_survival(float(v)) for v in body])
    assert stats.kstest(F, "uniform").pvalue > 1e-6


def _batches(run, N, nb):
    """Per-cell energies, escaped SEDs and MRW step counts of N packets run as
    nb packet-id batches; totals with standard errors from the batches'
    spread (the batches are independent packet streams)."""
    E, S, Cn, M = [], [], [], []
    for b in range(nb):
        r = run(b * N // nb, (b + 1) * N // nb)
        E.append(np.asarray(r["E_abs"], dtype=np.float64).ravel())
        S.append(np.asarray(r["sed_esc"], dtype=np.float64).sum(0))
        M.append(float(r["stats"]["mrw_steps"]))
    E, S, M = np.array(E), np.array(S), np.array(M)
    k = math.sqrt(nb)
    return dict(E=E.sum(0), sE=E.std(0, ddof=1) * k, S=S.sum(0), sS=S.std(0, ddof=1) * k,
                M=M.sum(), sM=M.std(ddof=1) * k)


def test_fp32_mrw_transport_matches_oracle(rt, ctx, O):
    """The production FP32 transport with the modified random walk (Sect.
    3.2) on a uniform cube of tau_cell = 20 against the FP64 oracle, frozen
    temperatures (order-independent): absorbed energy per cell and in total,
    the escaped SED per frequency and the number of MRW steps within 3 sigma
    + 2 % (sigma from 20 independent packet batches of each run; per cell,
    where that sigma has about 38 degrees of freedom, |z| < 5 and a mean z^2
    below 2)."""
    m = W.uniform_cube(n=4, tau_cell=20.0, nf=4, albedo=0.5)
    grid, opac, srcs = _setup(rt, ctx, m)
    T0 = np.full((1, m.ncell), 300.0)
    Tt = torch.tensor(T0, device="cuda")
    N, nb = 200000, 20

    def gpu(b, e):
        out = rt.transport(ctx, grid, opac, srcs, N, mode=rt.rtgb.RT_MODE_FROZEN_T, T_prev=Tt,
                           mrw=True, seed=41, pid_begin=b, pid_end=e)
        torch.cuda.synchronize()
        return out.numpy()

    def ref(b, e):
        return O.transport(m, N, seed=42, mode=O.MODE_FROZEN_T, T_prev=T0, mrw=True, n_threads=8,
                           pid_begin=b, pid_end=e)

    g, r = _batches(gpu, N, nb), _batches(ref, N, nb)
    assert g["M"] > N and r["M"] > N                       # many MRW steps per packet
    assert abs(g["M"] - r["M"]) < 3 * math.hypot(g["sM"], r["sM"]) + 0.02 * r["M"]
    assert abs(g["E"].sum() - r["E"].sum()) < 3 * math.hypot(
        math.sqrt((g["sE"] ** 2).sum()), math.sqrt((r["sE"] ** 2).sum())) + 0.02 * r["E"].sum()
    z = (g["E"] - r["E"]) / np.sqrt(g["sE"] ** 2 + r["sE"] ** 2 + (0.02 * r["E"]) ** 2)
    assert np.all(np.abs(z) < 5.0) and (z ** 2).mean() < 2.0, (np.abs(z).max(), (z ** 2).mean())
    lit = r["S"] > 0
    assert np.all((np.abs(g["S"] - r["S"]) <= 3 * np.hypot(g["sS"], r["sS"]) + 0.02 * r["S"])[lit])
    assert np.all(g["S"][~lit] == 0)


@pytest.mark.parametrize("mrw", [False, True])
def test_compaction_keeps_every_packet_history(rt, ctx, O, mrw):
    """Per-warp packet compaction (RT_SCHED_COMPACT) moves packets between
    lanes and a shared-memory stash; each packet's registers are restored
    exactly, so in the frozen-T mode (order-independent) the counts of every
    kind, the per-cell absorption counts and the escaped-packet counts equal
    those of the persistent schedule bit for bit, and the FP64 energies agree
    to the order of the atomic additions.  B&W with compaction conserves
    energy exactly."""
    m = W.r2_shell(n=24, tau_1um=10.0, nf=32) if not mrw else W.uniform_cube(n=6, tau_cell=25.0, nf=8, albedo=0.4)
    grid, opac, srcs = _setup(rt, ctx, m)
    T0 = torch.tensor(O.temperature_guess(m) if not mrw else np.full((1, m.ncell), 300.0), device="cuda")
    N = 200000 if not mrw else 50000
    res, evs = {}, {}
    for name, sched in (("persistent", rt.rtgb.RT_SCHED_PERSISTENT), ("compact", rt.rtgb.RT_SCHED_COMPACT)):
        o = rt.transport(ctx, grid, opac, srcs, N, mode=rt.rtgb.RT_MODE_FROZEN_T, T_prev=T0, seed=13,
                         schedule=sched, mrw=mrw, event_cap=(40 if not mrw else 1000) * N,
                         record_events=True)
        torch.cuda.synchronize()
        res[name] = o.numpy()
        evs[name] = o.events_numpy()
    a, b = res["persistent"], res["compact"]
    for k in ("crossings", "interactions", "scatters", "absorptions", "mrw_steps", "escaped",
              "lucy_deposits", "emitted", "stuck", "n_events"):
        assert a["stats"][k] == b["stats"][k], k
    assert b["stats"]["escaped"] + b["stats"]["stuck"] == N
    np.testing.assert_array_equal(a["count"], b["count"])
    np.testing.assert_array_equal(a["sed_cnt"], b["sed_cnt"])
    np.testing.assert_allclose(b["E_abs"], a["E_abs"], rtol=1e-9, atol=1e-12 * a["E_abs"].max())
    np.testing.assert_allclose(b["esq"], a["esq"], rtol=1e-9, atol=1e-12 * a["esq"].max())
    np.testing.assert_allclose(b["sed_esc"], a["sed_esc"], rtol=1e-12, atol=0)
    if mrw:
        assert b["stats"]["mrw_steps"] > N // 2
    # the same event records (as a multiset: the order of appends differs)
    assert a["stats"]["events_dropped"] == 0 and b["stats"]["events_dropped"] == 0
    ea = np.sort(evs["persistent"], order=["cell", "nu", "species"])
    eb = np.sort(evs["compact"], order=["cell", "nu", "species"])
    assert len(ea) == len(eb) > 0
    for f in ("cell", "nu", "species"):
        np.testing.assert_array_equal(ea[f], eb[f])
    # B&W with compaction: every packet escapes, the escaped SED sums to L
    o = rt.transport(ctx, grid, opac, srcs, N, seed=14, schedule=rt.rtgb.RT_SCHED_COMPACT, mrw=mrw)
    torch.cuda.synchronize()
    g = o.numpy()
    assert g["stats"]["escaped"] + g["stats"]["stuck"] == N
    assert abs(g["sed_esc"].sum() / (m.luminosity * g["stats"]["escaped"] / N) - 1) < 1e-9


def test_edge_cases(rt, ctx, O):
    # empty grid: every packet escapes on its first flight, no interaction
    m = W.uniform_cube(n=5, tau_cell=0.5)
    m.rho[:] = 0.0
    grid, opac, srcs = _setup(rt, ctx, m)
    out = rt.transport(ctx, grid, opac, srcs, 2000, seed=1)
    torch.cuda.synchronize()
    st = out.stats_dict()
    assert st["escaped"] == 2000 and st["interactions"] == 0 and st["lucy_deposits"] == 0
    # source exactly on cell faces and corners (even grid, centre source)
    m = W.uniform_cube(n=4, tau_cell=0.7, albedo=0.4)
    grid, opac, srcs = _setup(rt, ctx, m)
    out = rt.transport(ctx, grid, opac, srcs, 400, precision=rt.rtgb.RT_PREC_FP64,
                       schedule=rt.rtgb.RT_SCHED_SERIAL, traj_cap=100000, seed=4)
    torch.cuda.synchronize()
    ref = O.transport(m, 400, seed=4, mode=O.MODE_BW, traj_cap=100000)
    _traj_compare(out.traj_numpy(), ref["traj"], m.cell * 4)
    # empty packet range launches nothing
    out = rt.transport(ctx, grid, opac, srcs, 100, pid_begin=50, pid_end=50)
    torch.cuda.synchronize()
    assert out.stats_dict()["emitted"] == 0
    # event buffer overflow is counted, never written past the capacity
    m = W.uniform_cube(n=4, tau_cell=2.0, albedo=0.9)
    grid, opac, srcs = _setup(rt, ctx, m)
    out = rt.transport(ctx, grid, opac, srcs, 500, event_cap=10, record_events=True, seed=2)
    torch.cuda.synchronize()
    st = out.stats_dict()
    assert st["n_events"] == st["scatters"] > 10 and st["events_dropped"] == st["scatters"] - 10
    # per-packet event cap
    out = rt.transport(ctx, grid, opac, srcs, 500, max_events=2, seed=2)
    torch.cuda.synchronize()
    st = out.stats_dict()
    assert st["stuck"] > 0 and st["stuck"] + st["escaped"] == 500
    # argument errors are synchronous and leave nothing launched
    with pytest.raises(rt.RtError):
        rt.transport(ctx, grid, opac, srcs, 0)
    with pytest.raises(rt.RtError):
        rt.transport(ctx, grid, opac, srcs, 10, mode=rt.rtgb.RT_MODE_FROZEN_T)
    bad = W.uniform_cube(n=4)
    bad.sources[0].pos = (10 * bad.cell * 4, 0.0, 0.0)
    with pytest.raises(rt.RtError):
        rt.transport(ctx, grid, opac, rt.Sources(bad.sources), 10)
    neg = W.uniform_cube(n=3)
    neg.rho[0, 1, 1, 1] = -1.0
    with pytest.raises(rt.RtError):
        ctx.grid(neg)


# ------------------------------------------------------- photon counting (Sect. 4)
def _pc_cams(rt, m):
    return [rt.PcCamera(0.0, 0.0, 12, 0.8), rt.PcCamera(1.1, 0.4, 9, -1.0),
            rt.PcCamera(2.2, -0.7, 5, 0.3, pixel=0.5 * m.cell), rt.PcCamera(0.6, 2.5, 33, 0.9)]


def test_fp64_photon_counting_matches_oracle(rt, ctx, O):
    m = W.random_grid(n=(6, 5, 4), ns=2, seed=4, tau_scale=1.5, albedo=(0.3, 0.8))
    grid, opac, srcs = _setup(rt, ctx, m)
    T0 = np.random.default_rng(2).uniform(40, 600, size=(m.ns, m.ncell))
    cams = _pc_cams(rt, m)
    N = 3000
    out = rt.transport(ctx, grid, opac, srcs, N, mode=rt.rtgb.RT_MODE_FROZEN_T,
                       precision=rt.rtgb.RT_PREC_FP64, T_prev=torch.tensor(T0, device="cuda"),
                       pc_cams=cams, seed=9)
    torch.cuda.synchronize()
    ref = O.transport(m, N, seed=9, mode=O.MODE_FROZEN_T, T_prev=T0, n_threads=4,
                      pc_cameras=[(c.theta, c.phi, c.npix, c.pixel, c.cos_accept) for c in cams])
    for g, r in zip(out.pc_images(), ref["pc_img"]):
        g = g.cpu().numpy()
        assert g.shape == r.shape and r.sum() > 0
        np.testing.assert_allclose(g, r, rtol=1e-10, atol=1e-10 * r.max())


def test_fp32_photon_counting_invariants(rt, ctx, O):
    """FP32 B&W run: the +z camera of acceptance 0.8 holds the top bin of the
    escape SED, the all-sky camera every escaped packet (per frequency; a
    packet with k_z within rounding of 0.8 may fall on either side), also
    after a second call accumulates into the same images."""
    m = W.r2_shell(n=24, tau_1um=3.0, nf=16)
    grid, opac, srcs = _setup(rt, ctx, m)
    cams = [rt.PcCamera(0.0, 0.0, 32, 0.8), rt.PcCamera(0.9, 0.3, 16, -1.0)]
    N = 200_000
    out = rt.transport(ctx, grid, opac, srcs, N, pc_cams=cams, seed=5)
    torch.cuda.synchronize()
    top, full = [g.cpu().numpy() for g in out.pc_images()]
    sed = out.sed_esc.cpu().numpy()
    xi = out.xi
    assert np.all(np.abs(top.sum(axis=(1, 2)) - sed[9]) <= 2 * xi)
    np.testing.assert_allclose(full.sum(axis=(1, 2)), sed.sum(axis=0), rtol=1e-12, atol=2 * xi)
    assert full.sum() == pytest.approx(m.luminosity, rel=1e-9, abs=0)
    rt.transport(ctx, grid, opac, srcs, N, out=out, pc_cams=cams, seed=6)
    torch.cuda.synchronize()
    top, full = [g.cpu().numpy() for g in out.pc_images()]
    sed = out.sed_esc.cpu().numpy()
    assert np.all(np.abs(top.sum(axis=(1, 2)) - sed[9]) <= 4 * xi)
    assert full.sum() == pytest.approx(2 * m.luminosity, rel=1e-9, abs=0)


def test_photon_counting_rejections(rt, ctx):
    m = W.uniform_cube(n=4, tau_cell=0.1)
    grid, opac, srcs = _setup(rt, ctx, m)
    with pytest.raises(rt.RtError):
        rt.transport(ctx, grid, opac, srcs, 100, pc_cams=[rt.PcCamera(0.0, 0.0, 0, 0.5)])
    with pytest.raises(rt.RtError):
        rt.transport(ctx, grid, opac, srcs, 100, pc_cams=[rt.PcCamera(0.0, 0.0, 8, 1.5)])
    with pytest.raises(rt.RtError):
        rt.transport(ctx, grid, opac, srcs, 100, pc_cams=[rt.PcCamera(0.0, 0.0, 8, 0.5)] * 17)


# ------------------------------------------------ PAH re-emission pass (Sect. 2.1)
def test_fp64_pah_reemission_matches_oracle(rt, ctx, O):
    """Records stored by the oracle's B&W pass of the torus, re-emitted on both
    sides (frozen T): per-packet trajectories equal to 1e-9, the same
    absorbed energies, escape tallies and re-stored PAH records."""
    m = W.clumpy_torus(n=16, n_clump=60, seed=3, nf=24)
    eps, cls = W.pah_emissivity(m)
    r1 = O.transport(m, 3000, seed=4, mode=O.MODE_BW, pah_cap=3000)
    rec, xi = r1["pah"], r1["xi"]
    n = len(rec)
    assert n > 20
    grid, opac, _ = _setup(rt, ctx, m)
    T0 = np.random.default_rng(3).uniform(30, 700, size=(m.ns, m.ncell))
    out = rt.pah_reemit(ctx, grid, opac, rec, xi, eps, torch.tensor(cls, device="cuda"),
                        mode=rt.rtgb.RT_MODE_FROZEN_T, precision=rt.rtgb.RT_PREC_FP64,
                        T_prev=torch.tensor(T0, device="cuda"), traj_cap=400 * n, pah_cap=n,
                        seed=21, model_id=1)
    torch.cuda.synchronize()
    ref = O.pah_reemit(m, rec, xi, eps, cls, seed=21, model_id=1, mode=O.MODE_FROZEN_T, T_prev=T0,
                       traj_cap=400 * n, pah_cap=n, n_threads=4)
    st = out.stats_dict()
    assert st["traj_dropped"] == 0 and ref["stats"]["traj_dropped"] == 0
    _traj_compare(out.traj_numpy(), ref["traj"], m.cell * 16)
    for k in ("emitted", "escaped", "pah", "absorptions", "crossings", "scatters", "lucy_deposits"):
        assert st[k] == ref["stats"][k], k
    g = out.numpy()
    np.testing.assert_allclose(g["E_abs"], ref["E_abs"], rtol=1e-9, atol=1e-9 * ref["E_abs"].max())
    np.testing.assert_allclose(g["sed_esc"], ref["sed_esc"], rtol=1e-9, atol=1e-12 * xi)
    assert sorted(out.pah_numpy()["cell"].tolist()) == sorted(ref["pah"]["cell"].tolist())


def test_fp32_pah_reemission_conserves_energy(rt, ctx):
    """FP32 B&W: the GPU's own stored PAH absorptions re-emitted with the same
    xi; first-pass escapes + second-pass escapes + second-pass stores = L."""
    m = W.clumpy_torus(n=32, n_clump=200, seed=5, nf=32)
    eps, cls = W.pah_emissivity(m)
    grid, opac, srcs = _setup(rt, ctx, m)
    N = 400_000
    o1 = rt.transport(ctx, grid, opac, srcs, N, pah_cap=N, seed=8)
    torch.cuda.synchronize()
    n1 = o1.stats_dict()["pah"]
    assert n1 > 1000 and o1.stats_dict()["pah_dropped"] == 0
    o2 = rt.pah_reemit(ctx, grid, opac, o1, o1.xi, eps, torch.tensor(cls, device="cuda"),
                       pah_cap=n1, seed=8, model_id=1)
    torch.cuda.synchronize()
    s2 = o2.stats_dict()
    assert s2["emitted"] == n1 and s2["escaped"] + s2["pah"] == n1 and s2["stuck"] == 0
    e1, e2 = o1.sed_esc.sum().item(), o2.sed_esc.sum().item()
    assert e1 + e2 + s2["pah"] * o1.xi == pytest.approx(m.luminosity, rel=1e-9, abs=0)


def test_fp32_pah_reemission_frequency_law(rt, ctx):
    """Eq. 6 in the FP32 build: dust-free grid, records in class-0 cells; the
    escape counts per bin are a multinomial sample of eps_0 dnu."""
    m = W.uniform_cube(n=6, tau_cell=0.0, nf=40)
    m.rho[:] = 0.0
    eps, cls = W.pah_emissivity(m, n_classes=3)
    cells = np.nonzero(cls == 0)[0]
    rec = np.zeros(300_000, rt.rtgb.PAH_DTYPE)
    rec["cell"] = np.resize(cells, len(rec))
    grid, opac, _ = _setup(rt, ctx, m)
    out = rt.pah_reemit(ctx, grid, opac, rec, 1.0, eps, torch.tensor(cls, device="cuda"),
                        mode=rt.rtgb.RT_MODE_NOREEMIT, seed=3)
    torch.cuda.synchronize()
    cnt = out.sed_cnt.cpu().numpy().sum(axis=0).astype(np.float64)
    w = eps[0] * m.dnu
    expect = len(rec) * w / w.sum()
    keep = expect > 0
    c2 = ((cnt[keep] - expect[keep]) ** 2 / expect[keep]).sum()
    dof = keep.sum() - 1
    assert abs(c2 - dof) <= 5 * math.sqrt(2 * dof), (c2, dof)


def test_pah_reemission_bad_inputs(rt, ctx):
    m = W.uniform_cube(n=3, tau_cell=0.1)
    grid, opac, _ = _setup(rt, ctx, m)
    rec = np.zeros(8, rt.rtgb.PAH_DTYPE)
    with pytest.raises(rt.RtError):
        rt.pah_reemit(ctx, grid, opac, rec, 1.0, np.zeros((1, m.nf)))
    with pytest.raises(rt.RtError):
        rt.pah_reemit(ctx, grid, opac, rec, 0.0, np.ones((1, m.nf)))
    rec["cell"][:3] = [m.ncell, 2 ** 31, 5]                 # outside the grid: counted as stuck
    cls = torch.full((m.ncell,), 7, dtype=torch.int32, device="cuda")
    cls[1:] = 0                                              # cell 0's class is out of range
    out = rt.pah_reemit(ctx, grid, opac, rec, 1.0, np.ones((1, m.nf)), cls,
                        mode=rt.rtgb.RT_MODE_NOREEMIT)
    torch.cuda.synchronize()
    st = out.stats_dict()
    assert st["emitted"] == 8 and st["stuck"] == 2 + 5 and st["escaped"] + st["absorptions"] >= 1


def test_photon_counting_edge_cases(rt, ctx):
    """Acceptance cosine 1 counts nothing (no direction is exactly k_obs in
    practice); one all-sky pixel holds every escaped packet."""
    m = W.uniform_cube(n=5, tau_cell=0.3, albedo=0.5)
    grid, opac, srcs = _setup(rt, ctx, m)
    cams = [rt.PcCamera(0.3, 0.1, 4, 1.0), rt.PcCamera(0.0, 0.0, 1, -1.0)]
    out = rt.transport(ctx, grid, opac, srcs, 50_000, pc_cams=cams, seed=4)
    torch.cuda.synchronize()
    none, one = [g.cpu().numpy() for g in out.pc_images()]
    assert none.sum() == 0.0
    assert one.shape == (m.nf, 1, 1)
    assert one.sum() == pytest.approx(m.luminosity, rel=1e-9, abs=0)


def test_pah_reemission_without_records(rt, ctx):
    """No stored records: the wrapper launches nothing, the C entry refuses
    an empty pass."""
    m = W.uniform_cube(n=3, tau_cell=0.1)
    grid, opac, _ = _setup(rt, ctx, m)
    out = rt.pah_reemit(ctx, grid, opac, np.zeros(0, rt.rtgb.PAH_DTYPE), 1.0, np.ones((1, m.nf)))
    torch.cuda.synchronize()
    assert out.stats_dict()["emitted"] == 0 and out.E_abs.abs().sum().item() == 0.0
    p = rt.make_params(1)
    with pytest.raises(rt.RtError):
        rt.rtgb.rt_pah_reemit(ctx.h, grid.h, opac.h, None, 0, 1.0,
                              np.ones(m.nf).ctypes.data_as(__import__("ctypes").c_void_p), 1, None, p,
                              None, out.c_struct(), 0)


def test_grid_update_reuses_the_grid(rt, ctx, O):
    """New densities through rt_grid_update give the same FP64 transport as
    a grid uploaded with them; a bad density is refused and the grid then
    refuses to be used until a good update."""
    m = W.random_grid(n=(6, 5, 4), ns=2, seed=31, tau_scale=1.5, albedo=(0.3, 0.8))
    m2 = W.random_grid(n=(6, 5, 4), ns=2, seed=31, tau_scale=3.0, albedo=(0.3, 0.8))
    grid, opac, srcs = _setup(rt, ctx, m)
    T0 = torch.full((m.ns, m.ncell), 200.0, dtype=torch.float64, device="cuda")
    kw = dict(mode=rt.rtgb.RT_MODE_FROZEN_T, precision=rt.rtgb.RT_PREC_FP64, T_prev=T0, seed=4)
    rt.transport(ctx, grid, opac, srcs, 300, **kw)               # packs the first density
    grid.update(m2.rho)
    a = rt.transport(ctx, grid, opac, srcs, 300, **kw)
    b = rt.transport(ctx, ctx.grid(m2), opac, srcs, 300, **kw)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(a.count.cpu().numpy(), b.count.cpu().numpy())
    np.testing.assert_allclose(a.E_abs.cpu().numpy(), b.E_abs.cpu().numpy(), rtol=1e-12, atol=0)
    bad = m2.rho.copy()
    bad.reshape(-1)[7] = np.nan
    with pytest.raises(rt.RtError):
        grid.update(bad)
    with pytest.raises(rt.RtError):
        rt.transport(ctx, grid, opac, srcs, 10, **kw)
    grid.update(m.rho)
    rt.transport(ctx, grid, opac, srcs, 10, **kw)
    torch.cuda.synchronize()


def test_plain_fp32_form(rt, ctx):
    """FP32 per-cell accumulators (the plain-FP32 comparison form): the
    same packets as the production form (same Philox streams), energy
    conservation exact in the FP64 escape tally, per-cell energies within
    the Monte Carlo noise of the production run (the two differ only by the
    accumulators' rounding and the order of B&W updates); refused where it
    is not served."""
    m = W.r2_shell(n=24, tau_1um=3.0, nf=24)
    grid, opac, srcs = _setup(rt, ctx, m)
    N = 400_000
    a = rt.transport(ctx, grid, opac, srcs, N, seed=12)
    b = rt.transport(ctx, grid, opac, srcs, N, seed=12, precision=rt.rtgb.RT_PREC_FP32_ACC32)
    torch.cuda.synchronize()
    sb = b.stats_dict()
    assert sb["escaped"] == N and sb["stuck"] == 0
    assert b.sed_esc.sum().item() == pytest.approx(m.luminosity, rel=1e-9, abs=0)
    Ea, Eb = a.E_abs.cpu().numpy()[0], b.E_abs.cpu().numpy()[0]
    sig = np.sqrt(a.esq.cpu().numpy()[0] + b.esq.cpu().numpy()[0])
    on = Ea > 0
    assert np.all(np.abs(Eb[on] - Ea[on]) <= 5 * sig[on] + 2e-3 * Ea[on])
    assert Eb.sum() == pytest.approx(Ea.sum(), rel=2e-3, abs=0)
    with pytest.raises(rt.RtError):
        rt.transport(ctx, grid, opac, srcs, 100, precision=rt.rtgb.RT_PREC_FP32_ACC32, traj_cap=1000)
