"""One level of sub-cube refinement (Sect. 2) on the GPU against the FP64
oracle (run on a GB300).

* FP64 transport on randomly refined grids whose sub-cubes have their own
  densities: per-packet trajectories (cells are sub-cubes) equal to 1e-9,
  frozen T on all SMs and B&W in the serial schedule, with Lucy cells and
  the modified random walk in thick sub-cubes; energies, tallies equal.
* FP32: per-cell energies against the oracle within the Monte Carlo noise
  (statcheck) on refined grids with and without the modified random walk;
  energy conservation, and a grid whose sub-cubes inherit their cube's
  density gives the unrefined grid's cube energies within the noise.
* Temperatures (sub-cube volumes), the initial guess, the PAH pass and the
  ray tracer (emissivity tables per sub-cube, two-level ray and starlight
  walks, scattering events in sub-cubes) against the oracle.
* The ray-tracer adjoint on a refined grid against the oracle's FP64
  adjoint, directly and through the autograd wrapper.
* The batched launch (refined and uniform grids mixed) and the no-alloc
  entry serve refined grids; bad refinement factors are refused.
"""
import numpy as np
import pytest
import torch

import workloads as W
from imgcheck import assert_images_close
from statcheck import assert_same_energies

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


def _refined(ns=2, seed=3, r=3, n=(6, 5, 4), tau_scale=2.0, frac=0.5, jitter=0.6):
    m = W.random_grid(n=n, ns=ns, seed=seed, tau_scale=tau_scale, albedo=(0.3, 0.8))
    mask = np.random.default_rng(seed + 100).random(m.rho.shape[1:]) < frac
    return W.refine_cubes(m, mask, r=r, jitter=jitter, seed=seed)


def _traj_compare(tg, tr, scale, rtol=1e-9):
    tg = np.sort(tg, order=["pid", "seq"])
    tr = np.sort(tr, order=["pid", "seq"])
    assert len(tg) == len(tr), (len(tg), len(tr))
    for f in ("pid", "seq", "type", "cell", "nu"):
        bad = np.nonzero(tg[f] != tr[f])[0]
        assert bad.size == 0, (f, bad[:5], tg[bad[:3]], tr[bad[:3]])
    assert np.max(np.abs(tg["x"] - tr["x"])) <= rtol * scale
    assert np.max(np.abs(tg["k"] - tr["k"])) <= rtol * 10


@pytest.mark.parametrize("ns,r,lucy", [(1, 2, 1), (2, 3, 2), (3, 4, 0)])
def test_fp64_frozen_trajectories_on_refined_grid(rt, ctx, O, ns, r, lucy):
    m = _refined(ns=ns, r=r, seed=10 + ns)
    grid, opac, srcs = ctx.grid(m), ctx.opacity(m), rt.Sources(m.sources)
    T0 = np.random.default_rng(ns).uniform(30, 900, size=(m.ns, m.ncell))
    N = 500
    kw = dict(mode=rt.rtgb.RT_MODE_FROZEN_T, lucy_mode=lucy, seed=77)
    out = rt.transport(ctx, grid, opac, srcs, N, precision=rt.rtgb.RT_PREC_FP64,
                       T_prev=torch.tensor(T0, device="cuda"), traj_cap=600 * N,
                       event_cap=200 * N, record_events=True, **kw)
    torch.cuda.synchronize()
    ref = O.transport(m, N, T_prev=T0, traj_cap=600 * N, event_cap=200 * N, record_events=True,
                      n_threads=4, seed=77, mode=O.MODE_FROZEN_T, lucy_mode=lucy)
    st = out.stats_dict()
    assert st["traj_dropped"] == 0
    _traj_compare(out.traj_numpy(), ref["traj"], m.cell * 6)
    for k in ("crossings", "interactions", "absorptions", "escaped", "lucy_deposits", "scatters"):
        assert st[k] == ref["stats"][k], k
    g = out.numpy()
    np.testing.assert_allclose(g["E_abs"], ref["E_abs"], rtol=1e-9, atol=1e-9 * ref["E_abs"].max())
    assert sorted(out.events_numpy()["cell"].tolist()) == sorted(ref["events"]["cell"].tolist())


def test_fp64_bw_serial_and_mrw_on_refined_grid(rt, ctx, O):
    """B&W in the one-lane schedule (sub-cube volumes in the temperature
    update) and the modified random walk in thick sub-cubes."""
    m = _refined(ns=1, r=2, seed=21, tau_scale=40.0, frac=0.6)
    grid, opac, srcs = ctx.grid(m), ctx.opacity(m), rt.Sources(m.sources)
    N = 150
    out = rt.transport(ctx, grid, opac, srcs, N, precision=rt.rtgb.RT_PREC_FP64,
                       schedule=rt.rtgb.RT_SCHED_SERIAL, mrw=True, mrw_tau_cell=3.0, mrw_gamma=1.0,
                       traj_cap=20000 * N, seed=5)
    torch.cuda.synchronize()
    ref = O.transport(m, N, seed=5, mode=O.MODE_BW, mrw=True, mrw_tau_cell=3.0, mrw_gamma=1.0,
                      traj_cap=20000 * N)
    st = out.stats_dict()
    assert st["mrw_steps"] > 0 and st["traj_dropped"] == 0
    _traj_compare(out.traj_numpy(), ref["traj"], m.cell * 6)
    for k in ("crossings", "mrw_steps", "absorptions", "escaped"):
        assert st[k] == ref["stats"][k], k
    g = out.numpy()
    np.testing.assert_allclose(g["E_abs"], ref["E_abs"], rtol=1e-9, atol=1e-9 * ref["E_abs"].max())


def _shell_refined(r, tau_1um=100.0):
    m = W.r2_shell(n=16, tau_1um=tau_1um, nf=32)
    c = np.arange(16) + 0.5 - 8
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    return W.refine_cubes(m, np.sqrt(X * X + Y * Y + Z * Z) < 5, r=r, jitter=0.5, seed=4)


@pytest.mark.parametrize("case", ["random_ns2_r3", "shell_r4_mrw"])
def test_fp32_refined_statistics_match_oracle(rt, ctx, O, case):
    """The FP32 two-level traversal (the next sub-cube or cube and its density
    fetched one crossing ahead) against the FP64 oracle, frozen T: per-cell
    E_abs within max(3 sigma, 1e-3 E) with the binomial allowance and the
    chi-square bound of statcheck, the dispersion calibrated by a second
    oracle run; the same counts of escapes.  Cases: a random grid of two
    species with half its cubes divided into 3^3 sub-cubes of their own
    densities, and an r^-2 shell whose central cubes are divided into 4^3
    with the modified random walk in its thick sub-cubes."""
    if case == "random_ns2_r3":
        m = _refined(ns=2, r=3, seed=31, tau_scale=6.0, frac=0.5, n=(8, 7, 6))
        kw = dict(mrw=False)
        N = 300_000
    else:
        m = _shell_refined(4)
        kw = dict(mrw=True, mrw_tau_cell=2.0, mrw_gamma=1.0)
        N = 600_000
    grid, opac, srcs = ctx.grid(m), ctx.opacity(m), rt.Sources(m.sources)
    T0 = O.temperature_guess(m)
    out = rt.transport(ctx, grid, opac, srcs, N, mode=rt.rtgb.RT_MODE_FROZEN_T,
                       T_prev=torch.tensor(T0, device="cuda"), seed=41, **kw)
    torch.cuda.synchronize()
    g = out.numpy()
    st = out.stats_dict()
    assert st["escaped"] == N and st["stuck"] == 0
    if kw["mrw"]:
        assert st["mrw_steps"] > 0
    ref = O.transport(m, N, seed=42, mode=O.MODE_FROZEN_T, T_prev=T0, n_threads=8, **kw)
    ref2 = O.transport(m, N, seed=43, mode=O.MODE_FROZEN_T, T_prev=T0, n_threads=8, **kw)
    xi = m.luminosity / N
    phi, ncell = assert_same_energies(g, ref, ref2, xi)
    assert ncell > 500
    assert g["E_abs"].sum() == pytest.approx(ref["E_abs"].sum(), rel=0.02, abs=0)


def test_fp32_refined_conservation_and_inherited_density(rt, ctx):
    """FP32 B&W on a refined grid conserves energy; with sub-cubes of their
    cube's density (frozen T, Lucy in every dust cell) the cube sums of the
    absorbed energy match the unrefined grid's within the noise."""
    m = W.r2_shell(n=24, tau_1um=3.0, nf=24)
    c = np.arange(24) + 0.5 - 12
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    mask = np.sqrt(X * X + Y * Y + Z * Z) < 6
    mr = W.refine_cubes(m, mask, r=2)
    per = np.where(mr.refined.reshape(-1) > 0, 8, 1)
    N = 400_000
    g_r, opac, srcs = ctx.grid(mr), ctx.opacity(m), rt.Sources(m.sources)
    o = rt.transport(ctx, g_r, opac, srcs, N, seed=3)
    torch.cuda.synchronize()
    st = o.stats_dict()
    assert st["escaped"] == N and st["stuck"] == 0
    assert o.sed_esc.sum().item() == pytest.approx(m.luminosity, rel=1e-9, abs=0)
    T0 = np.full((1, m.ncell), 150.0)
    g_u = ctx.grid(m)
    kw = dict(mode=rt.rtgb.RT_MODE_FROZEN_T, lucy_mode=rt.rtgb.RT_LUCY_ALL, seed=9)
    a = rt.transport(ctx, g_u, opac, srcs, N, T_prev=torch.tensor(T0, device="cuda"), **kw)
    b = rt.transport(ctx, g_r, opac, srcs, N, T_prev=torch.tensor(np.repeat(T0, per, axis=1),
                                                                   device="cuda"), **kw)
    torch.cuda.synchronize()
    Ea, qa = a.E_abs.cpu().numpy()[0], a.esq.cpu().numpy()[0]
    Eb = np.zeros(m.ncell)
    np.add.at(Eb, np.repeat(np.arange(m.ncell), per), b.E_abs.cpu().numpy()[0])
    sig = np.sqrt(qa)
    on = Ea > 0
    assert np.all(np.abs(Eb[on] - Ea[on]) <= 5 * sig[on] + 2e-3 * Ea[on])
    assert b.stats_dict()["crossings"] > a.stats_dict()["crossings"]


def test_refined_temperatures_and_guess(rt, ctx, O):
    m = _refined(ns=2, r=3, seed=4)
    grid, opac = ctx.grid(m), ctx.opacity(m)
    E = np.random.default_rng(2).uniform(1e26, 1e31, size=(m.ns, m.ncell))
    E[:, ::9] = 0.0
    T = rt.temperatures(ctx, grid, opac, torch.tensor(E, device="cuda"))
    torch.cuda.synchronize()
    np.testing.assert_allclose(T.cpu().numpy(), O.temperatures(m, E), rtol=1e-10, atol=0)
    Tg = rt.temperature_guess(ctx, grid, rt.Sources(m.sources))
    torch.cuda.synchronize()
    np.testing.assert_allclose(Tg.cpu().numpy(), O.temperature_guess(m), rtol=1e-12)


def test_refined_raytrace_matches_oracle(rt, ctx, O):
    m = _refined(ns=2, r=3, seed=6, n=(7, 6, 5), tau_scale=1.5)
    cams = [W.Camera(0.8, 0.3, 20, 1e17), W.Camera(2.3, -1.7, 20, 1e17, 0.4 * m.cell)]
    fidx = [0, 3, 6]
    grid, opac, srcs = ctx.grid(m), ctx.opacity(m), rt.Sources(m.sources)
    rng = np.random.default_rng(0)
    T = rng.uniform(20, 1500, size=(m.ns, m.ncell))
    ev = np.zeros(4000, dtype=[("cell", "<u4"), ("nu", "<u4"), ("species", "<u4"), ("pad", "<u4"),
                               ("k", "<f8", (3,))])
    ev["cell"] = rng.integers(0, m.ncell, len(ev))
    ev["nu"] = rng.choice(fidx, len(ev))
    ev["species"] = rng.integers(0, m.ns, len(ev))
    k = rng.normal(size=(len(ev), 3))
    ev["k"] = (k / np.linalg.norm(k, axis=1, keepdims=True)).astype(np.float32)
    xi = m.luminosity / 1e5
    img, sed = rt.raytrace(ctx, grid, opac, torch.tensor(T, device="cuda"), ev, xi, srcs, cams, fidx)
    torch.cuda.synchronize()
    ir, sr = O.raytrace(m, T, ev, xi, cams, fidx)
    assert_images_close(img.cpu().numpy(), ir, rtol=1e-5, floor=1e-3)
    np.testing.assert_allclose(sed.cpu().numpy(), sr, rtol=1e-5)


def test_fp64_pah_pass_on_refined_grid(rt, ctx, O):
    m0 = W.clumpy_torus(n=12, n_clump=40, seed=3, nf=24)
    c = np.arange(12) + 0.5 - 6
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    m = W.refine_cubes(m0, np.sqrt(X * X + Y * Y + Z * Z) < 4, r=2, jitter=0.3, seed=1)
    eps, cls = W.pah_emissivity(m)
    r1 = O.transport(m, 2000, seed=4, mode=O.MODE_BW, pah_cap=2000)
    rec, xi = r1["pah"], r1["xi"]
    n = len(rec)
    assert n > 10
    grid, opac = ctx.grid(m), ctx.opacity(m)
    T0 = np.random.default_rng(3).uniform(30, 700, size=(m.ns, m.ncell))
    out = rt.pah_reemit(ctx, grid, opac, rec, xi, eps, torch.tensor(cls, device="cuda"),
                        mode=rt.rtgb.RT_MODE_FROZEN_T, precision=rt.rtgb.RT_PREC_FP64,
                        T_prev=torch.tensor(T0, device="cuda"), traj_cap=600 * n, seed=2, model_id=1)
    torch.cuda.synchronize()
    ref = O.pah_reemit(m, rec, xi, eps, cls, seed=2, model_id=1, mode=O.MODE_FROZEN_T, T_prev=T0,
                       traj_cap=600 * n, n_threads=4)
    _traj_compare(out.traj_numpy(), ref["traj"], m.cell * 12)
    np.testing.assert_allclose(out.E_abs.cpu().numpy(), ref["E_abs"], rtol=1e-9,
                               atol=1e-9 * ref["E_abs"].max())


def test_refined_grid_bad_inputs(rt, ctx):
    m = _refined(ns=1, r=2, seed=30)
    with pytest.raises(ValueError):
        rt.sim.Grid(ctx, m.rho[:, :-1], m.box_min, m.cell, refine=2, refined=m.refined)
    with pytest.raises(rt.RtError):
        rt.sim.Grid(ctx, m.rho, m.box_min, m.cell, refine=17, refined=m.refined)
    with pytest.raises(rt.RtError):
        rt.sim.Grid(ctx, m.rho, m.box_min, m.cell, refine=1, refined=m.refined)


def test_refined_degenerate_grids(rt, ctx, O):
    """No cube divided: the refined grid is the uniform one (same cell
    numbers, identical FP64 trajectories and energies).  Every cube divided
    with the cube's density: identical paths, cube sums of the energies."""
    m = W.random_grid(n=(5, 4, 3), ns=2, seed=12, tau_scale=2.0, albedo=(0.3, 0.8))
    T0 = np.random.default_rng(1).uniform(40, 600, size=(m.ns, m.ncell))
    opac, srcs = ctx.opacity(m), rt.Sources(m.sources)
    kw = dict(mode=rt.rtgb.RT_MODE_FROZEN_T, lucy_mode=rt.rtgb.RT_LUCY_ALL,
              precision=rt.rtgb.RT_PREC_FP64, traj_cap=400 * 400, seed=3)
    base = rt.transport(ctx, ctx.grid(m), opac, srcs, 400, T_prev=torch.tensor(T0, device="cuda"), **kw)
    none = W.refine_cubes(m, np.zeros(m.shape, bool), r=2)
    a = rt.transport(ctx, ctx.grid(none), opac, srcs, 400, T_prev=torch.tensor(T0, device="cuda"), **kw)
    allm = W.refine_cubes(m, np.ones(m.shape, bool), r=2)
    b = rt.transport(ctx, ctx.grid(allm), opac, srcs, 400,
                     T_prev=torch.tensor(np.repeat(T0, 8, axis=1), device="cuda"), **kw)
    torch.cuda.synchronize()
    t0 = np.sort(base.traj_numpy(), order=["pid", "seq"])
    ta = np.sort(a.traj_numpy(), order=["pid", "seq"])
    tb = np.sort(b.traj_numpy(), order=["pid", "seq"])
    for f in ("pid", "seq", "type", "cell", "nu"):
        np.testing.assert_array_equal(ta[f], t0[f])
    np.testing.assert_allclose(ta["x"], t0["x"], rtol=0, atol=1e-12 * m.cell * 5)
    np.testing.assert_allclose(a.E_abs.cpu().numpy(), base.E_abs.cpu().numpy(), rtol=1e-12)
    for f in ("pid", "seq", "type", "nu"):
        np.testing.assert_array_equal(tb[f], t0[f])
    np.testing.assert_allclose(tb["x"], t0["x"], rtol=0, atol=1e-9 * m.cell * 5)
    Eb = b.E_abs.cpu().numpy().reshape(m.ns, m.ncell, 8).sum(axis=2)
    E0 = base.E_abs.cpu().numpy()
    np.testing.assert_allclose(Eb, E0, rtol=1e-9, atol=1e-12 * E0.max())


def test_largest_refinement_factor(rt, ctx, O):
    """r = 16 (the largest factor): 4096 sub-cubes per divided cube."""
    m0 = W.uniform_cube(n=3, tau_cell=0.4, nf=8, albedo=0.5)
    mask = np.zeros(m0.shape, bool)
    mask[1, 1, 1] = mask[0, 2, 1] = True
    m = W.refine_cubes(m0, mask, r=16, jitter=0.4, seed=2)
    assert m.ncell == 25 + 2 * 4096
    grid, opac, srcs = ctx.grid(m), ctx.opacity(m), rt.Sources(m.sources)
    T0 = np.full((1, m.ncell), 200.0)
    out = rt.transport(ctx, grid, opac, srcs, 300, mode=rt.rtgb.RT_MODE_FROZEN_T,
                       precision=rt.rtgb.RT_PREC_FP64, T_prev=torch.tensor(T0, device="cuda"),
                       traj_cap=300 * 400, seed=8)
    torch.cuda.synchronize()
    ref = O.transport(m, 300, seed=8, mode=O.MODE_FROZEN_T, T_prev=T0, traj_cap=300 * 400)
    _traj_compare(out.traj_numpy(), ref["traj"], m.cell * 3)
    o32 = rt.transport(ctx, grid, opac, srcs, 100_000, seed=9)
    torch.cuda.synchronize()
    assert o32.stats_dict()["escaped"] == 100_000
    assert o32.sed_esc.sum().item() == pytest.approx(m.luminosity, rel=1e-9, abs=0)


def test_refined_raytrace_adjoint_matches_oracle(rt, ctx, O):
    m = _refined(ns=2, r=2, seed=14, n=(6, 5, 4), tau_scale=1.2)
    grid, opac, srcs = ctx.grid(m), ctx.opacity(m), rt.Sources(m.sources)
    rng = np.random.default_rng(2)
    T = rng.uniform(50, 900, size=(m.ns, m.ncell))
    fidx = [2, 6]
    ev = np.zeros(600, dtype=[("cell", "<u4"), ("nu", "<u4"), ("species", "<u4"), ("pad", "<u4"),
                              ("k", "<f8", (3,))])
    ev["cell"] = rng.integers(0, m.ncell, len(ev))
    ev["nu"] = rng.choice(fidx, len(ev))
    ev["species"] = rng.integers(0, m.ns, len(ev))
    k = rng.normal(size=(len(ev), 3))
    ev["k"] = (k / np.linalg.norm(k, axis=1, keepdims=True)).astype(np.float32)
    cams = [W.Camera(0.6, 0.2, 12, 3e16), W.Camera(2.1, -1.3, 12, 3e16)]
    wi = rng.normal(size=(2, 2, 12, 12))
    ws = rng.normal(size=(2, 2)) * 1e32
    xi = 1e28
    Tt = torch.tensor(T, device="cuda")
    drho, dscale = rt.raytrace_backward(ctx, grid, opac, Tt, ev, xi, srcs, cams, fidx,
                                        torch.tensor(wi, device="cuda"), torch.tensor(ws, device="cuda"))
    torch.cuda.synchronize()
    gr, gsr = O.raytrace_backward(m, T, ev, xi, cams, fidx, wi, ws)
    g = drho.cpu().numpy().astype(np.float64)
    scale = np.abs(gr).max()
    assert np.all(np.abs(g - gr) <= 1e-2 * np.abs(gr) + 1e-4 * scale)
    assert dscale.item() == pytest.approx(gsr, rel=1e-3, abs=0)
    rho = torch.tensor(m.rho, device="cuda", requires_grad=True)
    sc = torch.tensor(1.0, dtype=torch.float64, device="cuda", requires_grad=True)
    img, sed = rt.RayTrace.apply(rho, sc, ctx, m.box_min, m.cell, opac, Tt, ev, xi, srcs, cams, fidx,
                                 m.refine, m.refined)
    L = (img * torch.tensor(wi, device="cuda", dtype=torch.float32)).sum() + \
        (sed * torch.tensor(ws, device="cuda")).sum()
    L.backward()
    ga = rho.grad.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(ga - gr) <= 1e-2 * np.abs(gr) + 1e-4 * scale)


def test_refined_and_uniform_grids_in_one_batch(rt, ctx, O):
    """A batch mixing refined and uniform grids: every model's FP64
    frozen-T run equals the oracle's (Philox model id = base + index)."""
    def torus(n, k, s):
        return W.clumpy_torus(n=n, n_clump=k, seed=s, nf=24, with_pah=False)
    m1 = torus(8, 20, 1)
    c = np.arange(8) + 0.5 - 4
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    m1 = W.refine_cubes(m1, np.sqrt(X * X + Y * Y + Z * Z) < 3, r=2, jitter=0.3, seed=1)
    m2 = torus(12, 35, 3)
    m3 = W.refine_cubes(torus(10, 30, 2), np.random.default_rng(3).random((10, 10, 10)) < 0.3, r=3,
                        jitter=0.3, seed=2)
    models = [m1, m2, m3]
    opac = ctx.opacity(m2)
    N = [150, 200, 150]
    T0 = [torch.full((2, m.ncell), 250.0, dtype=torch.float64, device="cuda") for m in models]
    b = rt.Batch(ctx, opac, models, N, T_prev=T0, mode=rt.rtgb.RT_MODE_FROZEN_T,
                 precision=rt.rtgb.RT_PREC_FP64, seed=9, model_id=100)
    b.run()
    torch.cuda.synchronize()
    for i, m in enumerate(models):
        ref = O.transport(m, N[i], seed=9, model_id=100 + i, mode=O.MODE_FROZEN_T,
                          T_prev=T0[i].cpu().numpy(), n_threads=4)
        g = b.outs[i].numpy()
        np.testing.assert_array_equal(g["count"], ref["count"])
        np.testing.assert_allclose(g["E_abs"], ref["E_abs"], rtol=1e-9, atol=1e-12 * ref["E_abs"].max())
        assert g["stats"]["crossings"] == ref["stats"]["crossings"]


def test_refined_shell_at_bench_size(rt, ctx, O):
    """The refined-shell bench workload at its full size (64^3 cubes, 912
    divided into 4^3, 1e7 packets, the bench's launch configuration):
    exact conservation and counts, and FP64 trajectories of 300 packet ids
    of the same emission against the oracle on the full refined grid."""
    m = W.r2_shell_refined(n=64, tau_1um=10.0, nf=64, r=4, refine_radius=6.0)
    grid, opac, srcs = ctx.grid(m), ctx.opacity(m), rt.Sources(m.sources)
    N = 10 ** 7
    out = rt.transport(ctx, grid, opac, srcs, N, event_cap=6 * N, record_events=True, seed=5)
    torch.cuda.synchronize()
    st = out.stats_dict()
    assert st["emitted"] == N and st["escaped"] == N and st["stuck"] == 0
    assert abs(out.sed_esc.sum().item() / m.luminosity - 1) < 1e-9
    assert int(out.count.sum().item()) == st["absorptions"]
    assert st["n_events"] == st["scatters"] and st["events_dropped"] == 0
    T0 = O.temperature_guess(m)
    b, e = 5_000_000, 5_000_300
    g = rt.transport(ctx, grid, opac, srcs, N, mode=rt.rtgb.RT_MODE_FROZEN_T,
                     precision=rt.rtgb.RT_PREC_FP64, T_prev=torch.tensor(T0, device="cuda"),
                     pid_begin=b, pid_end=e, traj_cap=400000, seed=5)
    torch.cuda.synchronize()
    ref = O.transport(m, N, seed=5, mode=O.MODE_FROZEN_T, T_prev=T0, pid_begin=b, pid_end=e,
                      traj_cap=400000, n_threads=4)
    _traj_compare(g.traj_numpy(), ref["traj"], m.cell * 64)
    for k in ("crossings", "interactions", "absorptions", "escaped", "lucy_deposits"):
        assert g.stats_dict()[k] == ref["stats"][k], k
