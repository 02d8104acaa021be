"""Pins of the oracle's primitives against mathematics and independent
implementations (CPU only).

* Philox4x32-10 against cuRAND's host-side generator (a library routine that
  runs on the CPU), including a counter that carries into the second word.
* Uniform stream: range (0, 1], moments, no lag-1 correlation.
* Henyey-Greenstein sampler (Eq. 15): <mu> = g, <mu^2> = (1 + 2 g^2)/3 and a
  Kolmogorov-Smirnov test against the analytic CDF.
* Direction rotation: k_new . k_old = mu, unit length, uniform azimuth.
* Modified random walk law (Sect. 3.2): the two series forms agree, sampled
  y has mean 1/6 and variance 1/90, KS against S(y), and a brute-force
  random walk in a sphere reproduces the diffusion-limit mean path.
* DDA cell traversal: segment sum equals the closed-form distance to the box
  boundary; per-cell chords agree with brute-force fine stepping; segment
  lengths are invariant under the cube's 48 isometries.
"""
import ctypes
import itertools
import math
import os

import numpy as np
import pytest

import workloads as W


def _curand():
    for p in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            return ctypes.CDLL(p)
        except OSError:
            continue
    return None


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF0, 2**64 - 1])
def test_philox_matches_curand_host_generator(O, seed):
    """cuRAND's host generator lays out 65536 interleaved sub-streams: output
    block b is Philox4x32-10 of counter (b >> 16 as a 64-bit value in words
    0-1, b & 0xffff in word 2, 0) under key (seed_lo, seed_hi).  Offsets reach
    counters that carry into the second word."""
    cr = _curand()
    if cr is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    if cr.curandCreateGeneratorHost(ctypes.byref(gen), 161) != 0:   # PHILOX4_32_10
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert cr.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for first in (0, 65530, 2**48 - 3, 2**50 + 77):
            assert cr.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(4 * first)) == 0
            nblk = 16
            out = np.zeros(4 * nblk, np.uint32)
            assert cr.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p),
                                     ctypes.c_size_t(out.size)) == 0
            for i in range(nblk):
                b = first + i
                hi = b >> 16
                ctr = [hi & 0xFFFFFFFF, hi >> 32, b & 0xFFFF, 0]
                np.testing.assert_array_equal(O.philox(ctr, key), out[4 * i:4 * i + 4])
    finally:
        cr.curandDestroyGenerator(gen)


def test_uniform_stream_statistics(O):
    u = np.concatenate([O.uniforms(7, 3, pid, 64) for pid in range(2000)])
    assert u.min() > 0.0 and u.max() <= 1.0
    n = u.size
    assert abs(u.mean() - 0.5) < 4 * math.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 4 * math.sqrt(1 / 180 / n)
    v = u.reshape(2000, 64)
    r = np.corrcoef(v[:, :-1].ravel(), v[:, 1:].ravel())[0, 1]
    assert abs(r) < 4 / math.sqrt(v[:, :-1].size)
    # different packets and different model ids give different streams
    assert not np.array_equal(O.uniforms(7, 3, 0, 8), O.uniforms(7, 3, 1, 8))
    assert not np.array_equal(O.uniforms(7, 3, 0, 8), O.uniforms(7, 4, 0, 8))


def _hg_cdf(mu, g):
    if abs(g) < 1e-12:
        return 0.5 * (1 + mu)
    return (1 - g * g) / (2 * g) * (1 / np.sqrt(1 + g * g - 2 * g * mu) - 1 / (1 + g))


@pytest.mark.parametrize("g", [-0.5, 0.0, 0.5, 0.9])
def test_hg_sampler_moments_and_ks(O, g):
    u = O.uniforms(11, 0, 5, 40000)
    mu = np.array([O.hg_mu(g, x) for x in u])
    n = mu.size
    s1 = math.sqrt((1 + 2 * g * g) / 3 - g * g)
    assert abs(mu.mean() - g) < 4 * s1 / math.sqrt(n)
    m2 = (1 + 2 * g * g) / 3
    assert abs((mu ** 2).mean() - m2) < 4 * math.sqrt(0.2) / math.sqrt(n)
    xs = np.sort(mu)
    F = _hg_cdf(xs, g)
    D = max(np.max(np.arange(1, n + 1) / n - F), np.max(F - np.arange(n) / n))
    assert D < 1.63 / math.sqrt(n)          # KS at 1%
    assert O.hg_mu(g, 1.0) == pytest.approx(-1.0, abs=1e-12)


def test_rotation_preserves_scattering_angle(O):
    rng = np.random.default_rng(3)
    phis = []
    for i in range(3000):
        k = rng.normal(size=3)
        if i % 10 == 0:
            k = np.array([0.0, 0.0, 1.0 if i % 20 == 0 else -1.0]) + 1e-7 * rng.normal(size=3)
        k /= np.linalg.norm(k)
        mu, phi = rng.uniform(-1, 1), rng.uniform(0, 2 * math.pi)
        kn = O.rotate(k, mu, phi)
        assert np.linalg.norm(kn) == pytest.approx(1.0, abs=1e-12)
        assert float(kn @ k) == pytest.approx(mu, abs=1e-6)
        # azimuth of the new direction about k, measured from a fixed reference
        ref = np.cross(k, [1.0, 0.0, 0.0]) if abs(k[0]) < 0.9 else np.cross(k, [0.0, 1.0, 0.0])
        ref /= np.linalg.norm(ref)
        perp = kn - (kn @ k) * k
        if np.linalg.norm(perp) > 1e-6:
            phis.append(math.atan2(np.cross(ref, perp) @ k, ref @ perp))
    # rotation by a uniform phi gives a uniform azimuth
    h, _ = np.histogram(phis, bins=12, range=(-math.pi, math.pi))
    e = len(phis) / 12
    assert ((h - e) ** 2 / e).sum() < 35.0      # chi2(11) at ~1e-4


def test_mrw_series_forms_agree(O):
    # the small-time image series and the large-time Fourier series are the
    # same function (Jacobi theta transformation); the oracle switches at 0.1
    for y in [0.02, 0.05, 0.09, 0.0999, 0.1, 0.1001, 0.2, 0.5]:
        large = 2 * sum((-1) ** (n + 1) * math.exp(-n * n * math.pi ** 2 * y) for n in range(1, 400))
        small = 1 - 2 / math.sqrt(math.pi * y) * sum(math.exp(-(m + 0.5) ** 2 / y) for m in range(60))
        assert large == pytest.approx(small, rel=1e-10, abs=1e-13)
        assert O.mrw_survival(y) == pytest.approx(large, rel=1e-10, abs=1e-13)
    ys = np.linspace(0, 2, 400)
    S = np.array([O.mrw_survival(y) for y in ys])
    assert S[0] == 1.0 and np.all(np.diff(S) <= 1e-15) and S[-1] < 1e-8


def test_mrw_sampler_moments_and_ks(O):
    u = O.uniforms(5, 1, 9, 20000)
    y = np.array([O.mrw_sample_y(x) for x in u])
    n = y.size
    # E[y] = int S dy = 1/6 ; E[y^2] = 2 int y S dy = 7/180 ; var = 1/90
    assert abs(y.mean() - 1 / 6) < 4 * math.sqrt(1 / 90 / n)
    assert abs(y.var() - 1 / 90) < 0.06 / 90 * 10
    xs = np.sort(y)
    F = 1 - np.array([O.mrw_survival(v) for v in xs])
    D = max(np.max(np.arange(1, n + 1) / n - F), np.max(F - np.arange(n) / n))
    assert D < 1.63 / math.sqrt(n)
    for x in u[:50]:
        assert O.mrw_survival(O.mrw_sample_y(x)) == pytest.approx(x, rel=1e-9, abs=1e-14)


def test_mrw_mean_path_matches_brute_force_walk():
    """Isotropic random walk (unit mean free path) from the centre of a sphere
    of radius tau0: the mean total path to the boundary approaches the
    diffusion value tau0^2/2 that the MRW law gives (<y> = 1/6, l = 3 tau0^2 y
    in units of the mean free path); the walk exceeds it by the boundary
    layer, O(tau0)."""
    rng = np.random.default_rng(12)
    tau0, nw = 30.0, 1500
    pos = np.zeros((nw, 3))
    path = np.zeros(nw)
    alive = np.ones(nw, bool)
    while alive.any():
        idx = np.nonzero(alive)[0]
        s = rng.exponential(1.0, idx.size)
        mu = rng.uniform(-1, 1, idx.size)
        ph = rng.uniform(0, 2 * math.pi, idx.size)
        st = np.sqrt(1 - mu * mu)
        d = np.stack([st * np.cos(ph), st * np.sin(ph), mu], 1)
        p0 = pos[idx]
        # distance to the sphere along d
        b = (p0 * d).sum(1)
        c = (p0 * p0).sum(1) - tau0 * tau0
        t_exit = -b + np.sqrt(b * b - c)
        hit = s >= t_exit
        path[idx] += np.where(hit, t_exit, s)
        pos[idx] = p0 + d * np.where(hit, t_exit, s)[:, None]
        alive[idx[hit]] = False
    ratio = path.mean() / (tau0 * tau0 / 2)
    assert 0.95 < ratio < 1.12, ratio


def _box_exit(x, k, lo, hi):
    t = np.inf
    for a in range(3):
        if k[a] > 0:
            t = min(t, (hi[a] - x[a]) / k[a])
        elif k[a] < 0:
            t = min(t, (lo[a] - x[a]) / k[a])
    return t


def test_dda_segment_sum_equals_box_exit(O):
    m = W.random_grid(n=(7, 5, 4), seed=1)
    lo = m.box_min
    hi = lo + m.cell * np.array([7, 5, 4])
    rng = np.random.default_rng(4)
    for _ in range(300):
        x = lo + (hi - lo) * rng.uniform(0.001, 0.999, 3)
        k = rng.normal(size=3)
        k /= np.linalg.norm(k)
        cells, lens = O.dda_segments(m, x, k)
        assert lens.sum() == pytest.approx(_box_exit(x, k, lo, hi), rel=1e-12, abs=0)
        assert np.all(lens >= 0)
        # consecutive cells share a face
        iz, rem = np.divmod(cells, 5 * 7)
        iy, ix = np.divmod(rem, 7)
        steps = np.abs(np.diff(ix)) + np.abs(np.diff(iy)) + np.abs(np.diff(iz))
        assert np.all(steps == 1)


def test_dda_chords_match_brute_force(O):
    m = W.random_grid(n=(4, 4, 4), seed=2)
    rng = np.random.default_rng(5)
    h = 2e-5 * m.cell
    for _ in range(12):
        x = m.box_min + m.cell * 4 * rng.uniform(0.05, 0.95, 3)
        k = rng.normal(size=3)
        k /= np.linalg.norm(k)
        cells, lens = O.dda_segments(m, x, k)
        L = lens.sum()
        s = (np.arange(int(L / h)) + 0.5) * h
        pts = x[None, :] + s[:, None] * k[None, :]
        ijk = np.floor((pts - m.box_min) / m.cell).astype(int)
        lin = (ijk[:, 2] * 4 + ijk[:, 1]) * 4 + ijk[:, 0]
        for c, l in zip(cells, lens):
            assert (lin == c).sum() * h == pytest.approx(l, abs=3 * h)


def test_dda_invariant_under_cube_isometries(O):
    m = W.uniform_cube(n=5)
    rng = np.random.default_rng(6)
    x = m.box_min + m.cell * 5 * rng.uniform(0.1, 0.9, 3)
    ctr = m.box_min + 2.5 * m.cell
    k = rng.normal(size=3)
    k /= np.linalg.norm(k)
    ref = np.sort(O.dda_segments(m, x, k)[1])
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product([1, -1], repeat=3):
            P = np.zeros((3, 3))
            for i, j in enumerate(perm):
                P[i, j] = signs[i]
            x2 = ctr + P @ (x - ctr)
            k2 = P @ k
            got = np.sort(O.dda_segments(m, x2, k2)[1])
            np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-9 * m.cell)


# ------------------------------------------------ one level of refinement (Sect. 2)
def _refined_grid(seed=3, r=3):
    m = W.random_grid(n=(5, 4, 3), seed=seed)
    mask = np.random.default_rng(seed).random(m.rho.shape[1:]) < 0.5
    return W.refine_cubes(m, mask, r=r, jitter=0.5, seed=seed)


def _leaf_of_points(m, pts):
    """Cell number of each point by direct computation (numbering of the
    model's docstring): cube by floor, sub-cube by floor within the cube."""
    nz, ny, nx = m.shape
    r = m.refine
    ijk = np.floor((pts - m.box_min) / m.cell).astype(np.int64)
    cube = (ijk[:, 2] * ny + ijk[:, 1]) * nx + ijk[:, 0]
    base = m.leaf_base[cube]
    fine = m.refined.reshape(-1)[cube] > 0
    sub = np.floor((pts - m.box_min - ijk * m.cell) / (m.cell / r)).astype(np.int64)
    sub = np.clip(sub, 0, r - 1)
    return np.where(fine, base + (sub[:, 2] * r + sub[:, 1]) * r + sub[:, 0], base)


def test_refined_dda_chords_match_brute_force(O):
    """Cells and chord lengths of rays through a grid with one level of
    refinement against dense point sampling classified cell by cell."""
    m = _refined_grid()
    nz, ny, nx = m.shape
    ext = m.cell * np.array([nx, ny, nz])
    rng = np.random.default_rng(7)
    h = 2e-5 * m.cell
    for _ in range(16):
        x = m.box_min + ext * rng.uniform(0.05, 0.95, 3)
        k = rng.normal(size=3)
        k /= np.linalg.norm(k)
        cells, lens = O.dda_segments(m, x, k)
        assert lens.sum() == pytest.approx(_box_exit(x, k, m.box_min, m.box_min + ext), rel=1e-12, abs=0)
        s = (np.arange(int(lens.sum() / h)) + 0.5) * h
        lin = _leaf_of_points(m, x[None, :] + s[:, None] * k[None, :])
        # the sampled sequence of distinct cells is the DDA's (cells shorter
        # than the sampling step may be missed by the samples)
        seq = lin[np.concatenate([[True], lin[1:] != lin[:-1]])]
        assert list(seq) == [c for c, l in zip(cells, lens) if l > 3 * h]
        for c, l in zip(cells, lens):
            assert (lin == c).sum() * h == pytest.approx(l, abs=3 * h)
        assert len(set(cells.tolist())) == len(cells)      # a straight ray visits a cell once


def test_refined_grid_with_inherited_density_changes_no_physics(O):
    """Dividing cubes into sub-cubes of the cube's own density changes no
    path: frozen-T trajectories (no MRW, Lucy in every dust cell, linear
    form) are identical, and each divided cube's energy is the sum over its
    sub-cubes."""
    m = W.random_grid(n=(5, 4, 3), ns=2, seed=8, tau_scale=2.0, albedo=(0.3, 0.8))
    mask = np.random.default_rng(2).random(m.rho.shape[1:]) < 0.5
    mr = W.refine_cubes(m, mask, r=2)
    T0 = np.random.default_rng(4).uniform(40, 500, size=(m.ns, m.ncell))
    per = np.where(mr.refined.reshape(-1) > 0, 8, 1)
    T0r = np.repeat(T0, per, axis=1)
    kw = dict(seed=5, mode=O.MODE_FROZEN_T, lucy_mode=O.LUCY_ALL, traj_cap=200000, n_threads=4)
    a = O.transport(m, 800, T_prev=T0, **kw)
    b = O.transport(mr, 800, T_prev=T0r, **kw)
    ta, tb = np.sort(a["traj"], order=["pid", "seq"]), np.sort(b["traj"], order=["pid", "seq"])
    assert len(ta) == len(tb) > 0
    for f in ("pid", "seq", "type", "nu"):
        np.testing.assert_array_equal(ta[f], tb[f])
    np.testing.assert_allclose(ta["x"], tb["x"], rtol=0, atol=1e-9 * m.cell)
    np.testing.assert_allclose(ta["k"], tb["k"], rtol=0, atol=1e-9)
    cube_of_leaf = np.repeat(np.arange(m.ncell), per)
    Eb = np.zeros_like(a["E_abs"])
    for s in range(m.ns):
        np.add.at(Eb[s], cube_of_leaf, b["E_abs"][s])
    np.testing.assert_allclose(Eb, a["E_abs"], rtol=1e-9, atol=1e-12 * a["E_abs"].max())
    assert b["stats"]["crossings"] > a["stats"]["crossings"]
    np.testing.assert_array_equal(a["sed_cnt"], b["sed_cnt"])


def test_refined_temperatures_use_sub_cube_volumes(O):
    """Eq. 4 per cell with the cell's own volume: a sub-cube holding 1/r^3 of
    its cube's energy at the same density has the cube's temperature."""
    m = W.random_grid(n=(3, 3, 2), seed=1)
    mask = np.zeros(m.rho.shape[1:], bool)
    mask[0, 1, 2] = mask[1, 0, 0] = True
    mr = W.refine_cubes(m, mask, r=2)
    E = np.random.default_rng(3).uniform(1e28, 1e31, size=(1, m.ncell))
    T = O.temperatures(m, E)
    per = np.where(mr.refined.reshape(-1) > 0, 8, 1)
    Tr = O.temperatures(mr, np.repeat(E / per, per, axis=1))
    np.testing.assert_allclose(Tr, np.repeat(T, per, axis=1), rtol=1e-12)


def test_refined_images_equal_unrefined_for_inherited_fields(O):
    """Formal solution (Eqs. 11-14, 17) over a cube split into sub-cubes of
    the same emissivity and opacity equals the unsplit one."""
    m = W.random_grid(n=(4, 4, 3), ns=1, seed=6, tau_scale=1.0, albedo=(0.0, 0.0))
    mask = np.random.default_rng(9).random(m.rho.shape[1:]) < 0.5
    mr = W.refine_cubes(m, mask, r=3)
    per = np.where(mr.refined.reshape(-1) > 0, 27, 1)
    T = np.random.default_rng(1).uniform(30, 900, size=(1, m.ncell))
    cams = [W.Camera(0.7, 0.3, 12, 100 * W.AU), W.Camera(2.0, -1.1, 12, 100 * W.AU)]
    ev = np.zeros(0, O.EVENT_DTYPE)
    ia, sa = O.raytrace(m, T, ev, 1.0, cams, [1, 4, 6])
    ib, sb = O.raytrace(mr, np.repeat(T, per, axis=1), ev, 1.0, cams, [1, 4, 6])
    np.testing.assert_allclose(ib, ia, rtol=1e-9, atol=1e-12 * np.abs(ia).max())
    np.testing.assert_allclose(sb, sa, rtol=1e-9)


def test_refined_mrw_sphere_stays_in_the_sub_cube(O):
    """Modified random walk on a refined grid (Sect. 3.2 with sub-cubes):
    every MRW step ends inside the cell it started in -- the sphere is the
    largest one inside the sub-cube, not inside its cube -- and the walk is
    taken in thick sub-cubes."""
    m0 = W.uniform_cube(n=4, tau_cell=60.0, nf=6, albedo=0.3)
    mask = np.zeros(m0.shape, bool)
    mask[1:3, 1:3, 1:3] = True
    m = W.refine_cubes(m0, mask, r=2)
    r = O.transport(m, 60, seed=3, mode=O.MODE_BW, mrw=True, mrw_tau_cell=3.0, mrw_gamma=1.0,
                    traj_cap=2_000_000)
    t = r["traj"]
    assert r["stats"]["mrw_steps"] > 0 and r["stats"]["traj_dropped"] == 0
    nz, ny, nx = m.shape
    lo_all, h_all = [], []
    for q in range(nx * ny * nz):
        cz, cy, cx = q // (nx * ny), (q // nx) % ny, q % nx
        base = m.box_min + m.cell * np.array([cx, cy, cz])
        if m.refined[cz, cy, cx]:
            h = m.cell / 2
            for sz in range(2):
                for sy in range(2):
                    for sx in range(2):
                        lo_all.append(base + h * np.array([sx, sy, sz]))
                        h_all.append(h)
        else:
            lo_all.append(base)
            h_all.append(m.cell)
    lo_all, h_all = np.array(lo_all), np.array(h_all)
    mrw = t[t["type"] == O.T_MRW]
    fine = h_all[mrw["cell"]] < m.cell
    assert fine.sum() > 0 and (~fine).sum() > 0
    f = (mrw["x"] - lo_all[mrw["cell"]]) / h_all[mrw["cell"]][:, None]
    assert np.all((f >= -1e-12) & (f <= 1 + 1e-12))
