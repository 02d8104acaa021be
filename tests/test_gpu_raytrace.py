"""GPU temperature solve, ray tracer, adjoint and batched transport against
the FP64 CPU oracle (run on a GB300).

* rt_temperatures (Eq. 4) on the same absorbed energies: 1e-10 relative.
* rt_raytrace (Eqs. 11-17): images within 1e-5 relative on every pixel above
  1e-3 of the image maximum (1e-5 of the maximum below), SEDs within 1e-5
  relative, with thermal
  emission, stored scattering events and direct starlight, 1 and 3 species,
  several cameras, ragged image sizes.
* rt_raytrace_backward: dL/drho within 1e-2 of the oracle's FP64 adjoint on
  the cells that matter, dL/dscale within 1e-3; the autograd wrapper agrees.
* rt_batch_*: a batch of uneven models reproduces the single-model runs
  packet by packet (FP64) and conserves energy (FP32), also when replayed
  from a CUDA graph.
"""
import math

import numpy as np
import pytest
import torch

import workloads as W
from imgcheck import assert_images_close

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


def test_temperatures_match_oracle(rt, ctx, O):
    for m in (W.r2_shell(n=12, nf=64), W.clumpy_torus(n=12, n_clump=30, nf=40, seed=2)):
        grid, opac = ctx.grid(m), ctx.opacity(m)
        rng = np.random.default_rng(1)
        rv = m.rho.reshape(m.ns, -1).astype(np.float64) * m.cell ** 3
        # temperatures log-uniform over 0.2 K .. 5e5 K (the whole fine table,
        # including its steep Wien end); every 11th cell off the 0.1 K .. 1e6 K
        # table (0.02 .. 0.1 K or 1e6 .. 1e10 K: bisection fallback); every 7th
        # cell empty
        Tset = np.exp(rng.uniform(np.log(0.2), np.log(5e5), size=rv.shape))
        off = Tset[:, 3::11]
        lowside = rng.random(off.shape) < 0.5
        Tset[:, 3::11] = np.where(lowside, np.exp(rng.uniform(np.log(0.02), np.log(0.1), off.shape)),
                                  np.exp(rng.uniform(np.log(1e6), np.log(1e10), off.shape)))
        E = np.zeros_like(rv)
        for s_ in range(m.ns):
            for c in range(rv.shape[1]):
                E[s_, c] = rv[s_, c] * 4 * np.pi * O.planck_mean(m, s_, Tset[s_, c])
        E[:, ::7] = 0.0
        T = rt.temperatures(ctx, grid, opac, torch.tensor(E, device="cuda"))
        torch.cuda.synchronize()
        Tr = O.temperatures(m, E)
        np.testing.assert_allclose(T.cpu().numpy(), Tr, rtol=1e-10, atol=0)
        on = (E > 0) & (Tset > 0.1) & (Tset < 1e6)
        np.testing.assert_allclose(T.cpu().numpy()[on], Tset[on], rtol=1e-9)
    # the optically thin starting guess
    m = W.r2_shell(n=10, nf=16)
    grid = ctx.grid(m)
    Tg = rt.temperature_guess(ctx, grid, rt.Sources(m.sources))
    torch.cuda.synchronize()
    np.testing.assert_allclose(Tg.cpu().numpy(), O.temperature_guess(m), rtol=1e-12)


def _events(m, n, seed, nus):
    rng = np.random.default_rng(seed)
    ev = np.zeros(n, dtype=[("cell", "<u4"), ("nu", "<u4"), ("species", "<u4"), ("pad", "<u4"),
                            ("k", "<f8", (3,))])
    ev["cell"] = rng.integers(0, m.ncell, n)
    ev["nu"] = rng.choice(nus, n)
    ev["species"] = rng.integers(0, m.ns, n)
    k = rng.normal(size=(n, 3))
    ev["k"] = (k / np.linalg.norm(k, axis=1, keepdims=True)).astype(np.float32)
    return ev


def _compare_images(img, ref):
    assert_images_close(img, ref, rtol=1e-5, floor=1e-3)


@pytest.mark.parametrize("case", ["shell", "torus", "ragged"])
def test_raytrace_matches_oracle(rt, ctx, O, case):
    if case == "shell":
        m = W.r2_shell(n=16, nf=32, tau_1um=10.0)
        cams = [W.Camera(np.radians(t), 0.3, 24, 3e19) for t in (0.0, 45.0, 90.0)]
        fidx = [3, 10, 17, 25, 31]
    elif case == "torus":
        m = W.clumpy_torus(n=16, n_clump=80, nf=40, seed=3)
        cams = [W.Camera(np.radians(t), 1.0, 20, 1e26) for t in (12.5, 77.5)]
        fidx = list(range(0, 40, 4))
    else:
        m = W.random_grid(n=(9, 5, 7), ns=2, nf=12, seed=4, tau_scale=2.0)
        cams = [W.Camera(0.9, -0.4, 13, 1e17), W.Camera(2.5, 2.0, 13, 1e17, 0.3 * m.cell)]
        fidx = [0, 5, 5, 11]          # a repeated frequency slot
    grid, opac, srcs = ctx.grid(m), ctx.opacity(m), rt.Sources(m.sources)
    rng = np.random.default_rng(0)
    T = rng.uniform(20, 1500, size=(m.ns, m.ncell))
    ev = _events(m, 3000, 1, sorted(set(fidx)))
    xi = m.luminosity / 1e5
    img, sed = rt.raytrace(ctx, grid, opac, torch.tensor(T, device="cuda"), ev, xi, srcs, cams, fidx)
    torch.cuda.synchronize()
    ir, sr = O.raytrace(m, T, ev, xi, cams, fidx)
    _compare_images(img.cpu().numpy(), ir)
    np.testing.assert_allclose(sed.cpu().numpy(), sr, rtol=1e-5)


def test_raytrace_reads_event_count_on_device(rt, ctx, O):
    """Events straight from a transport output: the count is read on the
    device (capacity above and below the number stored) and the images equal
    those from the same events passed with a host count, and the oracle's."""
    m = W.r2_shell(n=12, nf=24, tau_1um=5.0)
    grid, opac, srcs = ctx.grid(m), ctx.opacity(m), rt.Sources(m.sources)
    cams = [W.Camera(np.radians(30.0), 0.2, 16, 3e19), W.Camera(np.radians(80.0), 1.1, 16, 3e19)]
    fidx = [2, 9, 15]
    T = torch.full((m.ns, m.ncell), 300.0, dtype=torch.float64, device="cuda")
    for cap in (200000, 500):
        out = rt.transport(ctx, grid, opac, srcs, 20000, event_cap=cap, seed=7, record_events=True)
        torch.cuda.synchronize()
        stored = int(out.stats[13].item())
        assert stored > 0 and (cap > stored or cap == 500)
        xi = m.luminosity / 20000
        img_d, sed_d = rt.raytrace(ctx, grid, opac, T, out, xi, srcs, cams, fidx)
        ev = out.events_numpy()
        assert len(ev) == min(stored, cap)
        img_h, sed_h = rt.raytrace(ctx, grid, opac, T, ev, xi, srcs, cams, fidx)
        torch.cuda.synchronize()
        np.testing.assert_allclose(img_d.cpu().numpy(), img_h.cpu().numpy(), rtol=1e-6,
                                   atol=1e-6 * float(img_h.abs().max()))
        np.testing.assert_allclose(sed_d.cpu().numpy(), sed_h.cpu().numpy(), rtol=1e-6)
        ir, sr = O.raytrace(m, T.cpu().numpy(), ev, xi, cams, fidx)
        _compare_images(img_d.cpu().numpy(), ir)
        np.testing.assert_allclose(sed_d.cpu().numpy(), sr, rtol=1e-5)


def test_visibilities_match_oracle(rt, ctx, O):
    """Visibilities of ray-traced images against the oracle's definition on
    the same images; V(0, 0) equals the images' share of the SED."""
    m = W.r2_shell(n=16, nf=24, tau_1um=5.0)
    grid, opac, srcs = ctx.grid(m), ctx.opacity(m), rt.Sources(m.sources)
    T = torch.tensor(np.random.default_rng(3).uniform(30, 900, size=(m.ns, m.ncell)), device="cuda")
    cams = [W.Camera(np.radians(t), 0.4, 48, 3e19) for t in (20.0, 70.0)]
    fidx = [4, 11, 18]
    img, sed = rt.raytrace(ctx, grid, opac, T, None, 0.0, None, cams, fidx)
    diag = m.cell * math.sqrt(3.0) * 16
    lam_over_res = 1.0 / (diag / 3e19)                  # cycles per radian of one field width
    uv = np.array([[0.0, 0.0], [0.5, 0.0], [0.0, 1.5], [3.0, -2.0], [-7.5, 4.0], [20.0, 11.0]]) * lam_over_res
    V = rt.visibilities(ctx, grid, cams, img, uv)
    torch.cuda.synchronize()
    Vr = O.visibilities(m, img.cpu().numpy(), cams, uv)
    Vg = V.cpu().numpy()
    scale = np.abs(Vr[:, :, :1])
    assert np.all(np.abs(Vg - Vr) <= 1e-6 * scale + 1e-300)
    np.testing.assert_allclose(Vg[:, :, 0].real, sed.cpu().numpy(), rtol=1e-6)   # no star in sed here
    with pytest.raises(rt.RtError):
        rt.visibilities(ctx, grid, cams, img, np.array([[np.nan, 0.0]]))


@pytest.mark.parametrize("ns", [2, 3])
def test_raytrace_adjoint_matches_oracle(rt, ctx, O, ns):
    # ns = 3 runs the float4-padded kernels (a fourth, empty species slot)
    m = W.random_grid(n=(8, 7, 6), ns=ns, nf=10, seed=6, tau_scale=1.5, albedo=(0.2, 0.7))
    grid, opac, srcs = ctx.grid(m), ctx.opacity(m), rt.Sources(m.sources)
    rng = np.random.default_rng(2)
    T = rng.uniform(50, 900, size=(m.ns, m.ncell))
    fidx = [2, 7]
    ev = _events(m, 800, 3, fidx)
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
    scale = np.abs(gr).max(axis=1, keepdims=True)          # each species on its own scale
    assert np.all(scale > 0)
    assert np.all(np.abs(g - gr) <= 1e-2 * np.abs(gr) + 1e-4 * scale)
    assert dscale.item() == pytest.approx(gsr, rel=1e-3, abs=0)
    # autograd wrapper: d(sum w * img + sum ws * sed)/d(rho, scale)
    rho = torch.tensor(m.rho, device="cuda", requires_grad=True)
    sc = torch.tensor(1.0, dtype=torch.float64, device="cuda", requires_grad=True)
    img, sed = rt.RayTrace.apply(rho, sc, ctx, m.box_min, m.cell, opac, Tt, ev, xi, srcs, cams, fidx)
    L = (img * torch.tensor(wi, device="cuda", dtype=torch.float32)).sum() + \
        (sed * torch.tensor(ws, device="cuda")).sum()
    L.backward()
    ga = rho.grad.cpu().numpy().reshape(ns, -1).astype(np.float64)
    assert np.all(np.abs(ga - gr) <= 1e-2 * np.abs(gr) + 1e-4 * scale)
    assert sc.grad.item() == pytest.approx(gsr, rel=1e-3, abs=0)


def test_batch_matches_single_model_runs(rt, ctx, O):
    models = [W.clumpy_torus(n=n, n_clump=k, seed=s, nf=24, with_pah=False)
              for n, k, s in ((8, 20, 1), (16, 60, 2), (12, 35, 3))]
    opac = ctx.opacity(models[0])
    N = [150, 300, 200]
    T0 = [torch.full((2, m.ncell), 250.0, dtype=torch.float64, device="cuda") for m in models]
    b = rt.Batch(ctx, opac, models, N, T_prev=T0, mode=rt.rtgb.RT_MODE_FROZEN_T,
                 precision=rt.rtgb.RT_PREC_FP64, seed=9, model_id=100)
    b.run()
    torch.cuda.synchronize()
    for i, m in enumerate(models):
        ref = O.transport(m, N[i], seed=9, model_id=100 + i, mode=O.MODE_FROZEN_T,
                          T_prev=T0[i].cpu().numpy())
        g = b.outs[i].numpy()
        np.testing.assert_array_equal(g["count"], ref["count"])
        np.testing.assert_allclose(g["E_abs"], ref["E_abs"], rtol=1e-9, atol=1e-12 * ref["E_abs"].max())
        assert g["stats"]["crossings"] == ref["stats"]["crossings"]
    # FP32 batch in a CUDA graph: replays conserve energy per model
    b32 = rt.Batch(ctx, opac, models, [4000, 8000, 6000], seed=1)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b32.run(s)                       # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    for o in b32.outs:
        o.zero_()
    gr = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gr):
        b32.run(torch.cuda.current_stream())
    for o in b32.outs:
        o.zero_()
    gr.replay()
    gr.replay()
    torch.cuda.synchronize()
    for i, m in enumerate(models):
        g = b32.outs[i].numpy()
        assert g["stats"]["emitted"] == 2 * [4000, 8000, 6000][i]
        assert abs(g["sed_esc"].sum() / (2 * m.luminosity) - 1) < 1e-9


def test_visibilities_ragged_image_and_single_uv(rt, ctx, O):
    """An odd image size (7 x 7 pixels, explicit pixel size) and a single
    (u, v) point, against the oracle's sum."""
    m = W.random_grid(n=(5, 4, 6), ns=2, nf=8, seed=8, tau_scale=1.0)
    grid, opac = ctx.grid(m), ctx.opacity(m)
    T = torch.tensor(np.random.default_rng(1).uniform(40, 800, size=(m.ns, m.ncell)), device="cuda")
    cams = [W.Camera(1.1, -0.6, 7, 2e17, 0.9 * m.cell)]
    img, sed = rt.raytrace(ctx, grid, opac, T, None, 0.0, None, cams, [3])
    uv = np.array([[1.3e3, -2.2e3]])
    V = rt.visibilities(ctx, grid, cams, img, uv).cpu().numpy()
    Vr = O.visibilities(m, img.cpu().numpy(), cams, uv)
    assert V.shape == (1, 1, 1)
    assert abs(V[0, 0, 0] - Vr[0, 0, 0]) <= 1e-6 * np.abs(img.cpu().numpy()).sum() * (0.9 * m.cell / 2e17) ** 2
