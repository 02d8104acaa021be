"""Pins of the oracle's transport, temperature and ray-tracing results against
closed forms, conservation laws, brute force and independent quadrature
(CPU only)."""
import math

import numpy as np
import pytest

import workloads as W

SIGMA = 5.670374419e-5          # CODATA Stefan-Boltzmann constant, CGS
H, K = 6.62607015e-27, 1.380649e-16


def gray_fine_model(n=4, tau_cell=1e-3, nf=400, albedo=0.0, side_au=1.0, src=None):
    """Uniform gray cube with a fine frequency grid (0.01 um - 1 cm), so that
    sum_j B(nu_j, T) dnu_j matches sigma T^4 / pi closely."""
    m = W.uniform_cube(n=n, tau_cell=tau_cell, nf=8, albedo=albedo, side_au=side_au,
                       source_pos=src)
    nu, dnu = W.log_frequency_grid(nf, 0.01, 1.0e4)
    m.nu, m.dnu = nu, dnu
    m.kabs = np.full((1, nf), 1.0 - albedo)
    m.ksca = np.full((1, nf), albedo)
    m.g = np.zeros((1, nf))
    m.rho = np.full_like(m.rho, tau_cell / m.cell)
    return m


# ---------------------------------------------------------------- Planck / Eq. 4
def test_planck_sum_matches_stefan_boltzmann(O):
    m = gray_fine_model()
    for T in (20.0, 300.0, 2500.0, 5800.0):
        s = sum(O.planck_B(nu, T) * d for nu, d in zip(m.nu, m.dnu))
        assert s == pytest.approx(SIGMA * T ** 4 / math.pi, rel=2e-4, abs=0)


def test_planck_peak_and_derivative(O):
    T = 5000.0
    nus = np.geomspace(1e13, 1e16, 20001)
    B = np.array([O.planck_B(v, T) for v in nus])
    # Wien displacement in frequency: x_peak = 3 + W0(-3 e^-3) = 2.82143937212
    assert nus[np.argmax(B)] == pytest.approx(2.82143937212 * K * T / H, rel=5e-4, abs=0)
    for nu in (1e12, 3e13, 6e14, 3e15):
        for T in (30.0, 800.0, 6000.0):
            h = 1e-6 * T
            fd = (O.planck_B(nu, T + h) - O.planck_B(nu, T - h)) / (2 * h)
            assert O.planck_dBdT(nu, T) == pytest.approx(fd, rel=1e-6, abs=0)


def test_temperature_solve_gray_closed_form(O):
    m = gray_fine_model()
    # 4 pi kappa sigma T^4 / pi = E / (rho V)  =>  T = (target / (4 kappa sigma))^(1/4)
    for T0 in (15.0, 150.0, 1500.0):
        target = 4.0 * SIGMA * T0 ** 4
        T = O.solve_temperature(m, 0, target)
        assert T == pytest.approx(T0, rel=1e-4, abs=0)
    assert O.solve_temperature(m, 0, 0.0) == 0.0


def test_temperature_solve_inverts_planck_mean(O):
    m = W.r2_shell(n=8, nf=64)
    for T0 in (3.0, 47.0, 812.0, 1.6e4, 3.0e5):
        target = 4 * math.pi * O.planck_mean(m, 0, T0)
        assert O.solve_temperature(m, 0, target) == pytest.approx(T0, rel=1e-10, abs=0)


# ---------------------------------------------------------------- emission
def test_empty_grid_emission_spectrum_and_isotropy(O):
    m = W.r2_shell(n=8, nf=24)
    m.rho[:] = 0.0
    N = 40000
    r = O.transport(m, N, seed=3, mode=O.MODE_BW, traj_cap=2 * N)
    assert r["stats"]["escaped"] == N and r["stats"]["interactions"] == 0
    assert r["sed_esc"].sum() == pytest.approx(m.luminosity, rel=1e-12, abs=0)
    # frequency histogram vs L_nu dnu / L (chi^2); the weights are the
    # blackbody written out here from Planck's law, independent of the oracle
    x = H * m.nu / (K * 2500.0)
    w = m.nu ** 3 / np.expm1(x) * m.dnu
    p = w / w.sum()
    cnt = r["sed_cnt"].sum(0).astype(float)
    keep = p * N > 20
    chi2 = ((cnt[keep] - N * p[keep]) ** 2 / (N * p[keep])).sum()
    assert chi2 < keep.sum() + 6 * math.sqrt(2 * keep.sum())
    # isotropy: emission directions from the trajectory log
    tr = r["traj"]
    k = tr["k"][tr["type"] == O.T_EMIT]
    assert np.abs(k.mean(0)).max() < 4 / math.sqrt(3 * N)
    kk = (k[:, :, None] * k[:, None, :]).mean(0)
    assert np.abs(kk - np.eye(3) / 3).max() < 4 * math.sqrt(0.1 / N)
    # cos(theta) bins are equally populated
    h = r["sed_cnt"].sum(1)
    assert ((h - N / 10) ** 2 / (N / 10)).sum() < 30


# ---------------------------------------------------------------- pure absorber
def _fib_sphere(n):
    i = np.arange(n) + 0.5
    mu = 1 - 2 * i / n
    ph = math.pi * (1 + 5 ** 0.5) * i
    st = np.sqrt(1 - mu * mu)
    return np.stack([st * np.cos(ph), st * np.sin(ph), mu], 1)


def test_pure_absorber_escape_fraction_closed_form(O):
    """Uniform gray cube, source at the centre, no scattering, no re-emission:
    the escaped fraction is (1/4 pi) int exp(-chi d(Omega)) dOmega with the
    distance to the cube face d = (L/2) / max|k_a|; the integral is done here
    by quadrature of that closed form."""
    n, tau_cell = 6, 0.4
    m = W.uniform_cube(n=n, tau_cell=tau_cell, nf=6, albedo=0.0)
    N = 60000
    r = O.transport(m, N, seed=5, mode=O.MODE_NOREEMIT, lucy_mode=O.LUCY_OFF)
    k = _fib_sphere(400000)
    d = (n / 2) / np.abs(k).max(1)           # in cells
    f = np.exp(-tau_cell * d).mean()
    fe = r["stats"]["escaped"] / N
    assert abs(fe - f) < 4 * math.sqrt(f * (1 - f) / N)
    # energy: L = escaped + absorbed (count estimator), exactly
    xi = m.luminosity / N
    assert r["sed_esc"].sum() + r["count"].sum() * xi == pytest.approx(m.luminosity, rel=1e-12, abs=0)
    assert r["E_abs"].sum() == pytest.approx(r["count"].sum() * xi, rel=1e-12, abs=0)


def _absorbed_fraction_quadrature(O, m, ndir=60000):
    """(1/4 pi) int exp(-tau_before) (1 - exp(-tau_cell)) dOmega per cell for a
    gray pure absorber, from the oracle's DDA along a Fibonacci sphere."""
    chi = m.rho[0].reshape(-1).astype(np.float64) * (m.kabs[0, 0] + m.ksca[0, 0])
    frac = np.zeros(chi.size)
    src = np.array(m.sources[0].pos)
    for k in _fib_sphere(ndir):
        cells, lens = O.dda_segments(m, src, k)
        t = chi[cells] * lens
        before = np.concatenate([[0.0], np.cumsum(t)[:-1]])
        frac[cells] += np.exp(-before) * (-np.expm1(-t))
    return frac / ndir


def test_pure_absorber_cell_energies_match_quadrature(O):
    """Per-cell absorbed energy of both estimators (absorption counts and the
    Lucy path-length form) equals the deterministic quadrature on a small
    irregular grid."""
    m = W.random_grid(n=(4, 4, 4), seed=7, tau_scale=0.6, albedo=(0.0, 0.0))
    m.kabs[:] = 1.0
    m.ksca[:] = 0.0
    m.rho = (m.rho * (0.6 / (m.cell * m.rho.mean()))).astype(np.float32)
    N = 200000
    f = _absorbed_fraction_quadrature(O, m) * m.luminosity
    xi = m.luminosity / N
    rc = O.transport(m, N, seed=9, mode=O.MODE_NOREEMIT, lucy_mode=O.LUCY_OFF)
    Ec = rc["E_abs"][0]
    sig = xi * np.sqrt(np.maximum(rc["count"][0], 1))
    assert np.all(np.abs(Ec - f) < 4.5 * sig + 1e-9 * m.luminosity)
    rl = O.transport(m, N, seed=10, mode=O.MODE_NOREEMIT, lucy_mode=O.LUCY_ALL)
    El = rl["E_abs"][0]
    sl = np.sqrt(rl["esq"][0]) + 1e-12
    assert np.all(np.abs(El - f) < 4.5 * np.maximum(sl, 0.02 * f) + 1e-9 * m.luminosity)
    # the path-length estimator has the smaller variance in thin cells
    thin = (m.rho[0].reshape(-1) * m.cell < 0.1) & (f > 0)
    assert (sl[thin] < sig[thin]).mean() > 0.8


def test_source_spectrum_is_the_normalised_blackbody(O):
    """A stellar source's L_nu on the model grid is the blackbody B_nu(T_eff),
    written out here from Planck's law, scaled so that sum_j L_nu,j dnu_j is
    the source's luminosity L (Sect. 2: packets of equal energy L/N)."""
    m = W.uniform_cube(n=2, tau_cell=0.1, nf=12, albedo=0.0)
    lnu = O.source_lnu(m)
    src = m.sources[0]
    B = np.array([2 * H * nu ** 3 / 2.99792458e10 ** 2 / math.expm1(H * nu / (K * src.T_eff))
                  for nu in m.nu])
    assert (lnu * m.dnu).sum() == pytest.approx(src.L, rel=1e-12, abs=0)
    np.testing.assert_allclose(lnu, B * src.L / (B * m.dnu).sum(), rtol=1e-12)


def test_sources_emit_in_proportion_to_their_luminosity(O):
    """Packets of equal energy L/N (Sect. 2): with several sources and random
    frequency bins, each packet's source is drawn with probability L_i / L,
    so the packets leaving each source follow a binomial law with that mean
    (within 4 sigma), and each source's packets follow its own spectrum."""
    m = W.uniform_cube(n=3, tau_cell=0.5, nf=24, gray=False)
    m.rho[:] = 0.0
    m.sources = [W.Source((0.1 * m.cell, 0.2 * m.cell, 0.0), 2.0 * W.LSUN, 5800.0),
                 W.Source((-0.3 * m.cell, 0.0, 0.1 * m.cell), 1.0 * W.LSUN, 3000.0)]
    N = 30000
    r = O.transport(m, N, seed=8, mode=O.MODE_NOREEMIT, traj_cap=3 * N)
    em = r["traj"][r["traj"]["type"] == O.T_EMIT]
    assert len(em) == N
    first = np.abs(em["x"][:, 0] - m.sources[0].pos[0]) < 1e-3 * m.cell
    p = 2.0 / 3.0
    assert abs(first.sum() - N * p) < 4 * math.sqrt(N * p * (1 - p)), first.sum()
    # the 3000 K source's packets sit at longer wavelengths than the 5800 K one's
    assert em["nu"][~first].mean() < em["nu"][first].mean()


def test_lucy_and_count_estimators_agree_per_species(O):
    """The path-length (Lucy) estimator and the absorption-count estimator of a
    cell's absorbed energy have the same expectation, because absorptions
    happen at the rate rho_s kappa^abs_s per unit path (Sect. 3.1).  This holds
    with scattering and with two species of opposite albedo, where a deposit
    by extinction instead of absorption, or a species drawn by the wrong
    cross-section, shows as a per-species bias.  sigma from 10 independent
    packet batches of each run; every (species, cell) within 4.5 sigma, the
    mean z^2 below 2."""
    m = W.random_grid(n=(4, 4, 4), ns=2, nf=4, seed=13, tau_scale=1.5, empty_frac=0.1)
    m.kabs = np.array([[0.8] * 4, [0.2] * 4])
    m.ksca = np.array([[0.2] * 4, [0.8] * 4])
    m.g[:] = 0.5
    kmax = 1.0
    m.rho = (m.rho * (1.5 / (kmax * m.cell * m.rho.reshape(2, -1).mean()))).astype(np.float32)
    N, nb = 200000, 10
    kw = dict(mode=O.MODE_NOREEMIT)
    el, ec = [], []
    for b in range(nb):
        rng = dict(pid_begin=b * N // nb, pid_end=(b + 1) * N // nb)
        el.append(O.transport(m, N, seed=41, lucy_mode=O.LUCY_ALL, **rng, **kw)["E_abs"])
        ec.append(O.transport(m, N, seed=42, lucy_mode=O.LUCY_OFF, **rng, **kw)["E_abs"])
    el, ec = np.array(el), np.array(ec)
    El, Ec = el.sum(0), ec.sum(0)
    s2 = (el.var(0, ddof=1) + ec.var(0, ddof=1)) * nb
    lit = (Ec > 0) & (El > 0)
    assert lit.sum() > 100
    z = (El - Ec)[lit] / np.sqrt(s2[lit])
    assert np.all(np.abs(z) < 4.5) and (z ** 2).mean() < 2.0, (np.abs(z).max(), (z ** 2).mean())
    for s in range(2):
        assert El[s].sum() == pytest.approx(Ec[s].sum(), rel=0.02, abs=0)


# ---------------------------------------------------------------- conservation
def test_bw_conserves_energy_exactly(O):
    m = W.homogeneous_sphere(n=12, tau_v=3.0)
    N = 4000
    r = O.transport(m, N, seed=2, mode=O.MODE_BW)
    assert r["stats"]["escaped"] == N
    assert r["sed_esc"].sum() == pytest.approx(m.luminosity, rel=1e-12, abs=0)


def test_pah_packets_are_stored_and_counted(O):
    m = W.clumpy_torus(n=16, n_clump=60, seed=3, nf=24)
    N = 3000
    r = O.transport(m, N, seed=4, mode=O.MODE_BW, pah_cap=N)
    st = r["stats"]
    assert st["pah"] > 0 and st["escaped"] + st["pah"] == N
    xi = m.luminosity / N
    assert r["sed_esc"].sum() + st["pah"] * xi == pytest.approx(m.luminosity, rel=1e-12, abs=0)
    assert len(r["pah"]) == st["pah"]


def test_event_cap_terminates_packets(O):
    m = W.uniform_cube(n=4, tau_cell=5.0, albedo=0.9)
    r = O.transport(m, 500, seed=1, mode=O.MODE_BW, max_events=3)
    st = r["stats"]
    assert st["stuck"] > 0 and st["escaped"] + st["stuck"] == 500


def test_lucy_cells_are_those_below_the_face_to_face_threshold(O):
    """Reading 2 of Sect. 3.1: with the thin-cell mode a cell takes
    path-length deposits when its largest face-to-face optical depth over the
    frequency grid is below lucy_tau = 1e-2.  Gray uniform cubes just below
    and just above the threshold: every crossing deposits, or none does."""
    for tau_cell, lucy in ((0.009, True), (0.011, False)):
        m = W.uniform_cube(n=4, tau_cell=tau_cell, nf=4, albedo=0.5)
        r = O.transport(m, 3000, seed=3, mode=O.MODE_BW, lucy_mode=O.LUCY_THIN)
        st = r["stats"]
        assert st["crossings"] > 0
        if lucy:
            assert st["lucy_deposits"] >= st["crossings"]
        else:
            assert st["lucy_deposits"] == 0


def test_stored_events_carry_the_incoming_direction(O):
    """The scattering source of Eq. 16 weighs each stored event by the angle
    between the observer and the packet's direction before it scattered, so
    the event store keeps the incoming direction.  In an optically thin,
    purely scattering cube (tau 0.08 from the central source to a face) almost
    every event is a first scattering, whose incoming direction points from
    the source to the event: against the direction to the cell centre, for
    cells at least two cells from the source, the cosines have a median above
    0.97 and a mean above 0.9.  The outgoing (isotropic, g = 0) direction
    would give a mean near 0, the reversed one near -1."""
    n = 8
    m = W.uniform_cube(n=n, tau_cell=0.02, nf=4, albedo=1.0, g=0.0)
    N = 60000
    r = O.transport(m, N, seed=12, mode=O.MODE_BW, record_events=True, event_cap=N)
    ev = r["events"]
    assert len(ev) == r["stats"]["scatters"] > 2000
    c = ev["cell"].astype(np.int64)
    ctr = m.box_min + m.cell * (np.stack([c % n, (c // n) % n, c // (n * n)], 1) + 0.5)
    d = ctr - np.array(m.sources[0].pos)
    dist = np.linalg.norm(d, axis=1)
    far = dist >= 2 * m.cell
    cosv = (ev["k"][far] * d[far]).sum(1) / dist[far]
    assert far.sum() > 1000
    assert np.median(cosv) > 0.97 and cosv.mean() > 0.9, (np.median(cosv), cosv.mean())


def test_scattering_only_matches_brute_force_walk(O):
    """Albedo 1, isotropic scattering in a uniform gray cube with the source at
    the centre: the mean number of scatterings per packet equals that of a
    brute-force random walk (exponential steps, isotropic turns) in a cube of
    the same optical half-width, written here independently."""
    n, tau_cell = 4, 2.5
    m = W.uniform_cube(n=n, tau_cell=tau_cell, nf=4, albedo=1.0, g=0.0)
    N = 6000
    r = O.transport(m, N, seed=6, mode=O.MODE_BW)
    assert r["stats"]["escaped"] == N and r["stats"]["absorptions"] == 0
    assert r["sed_esc"].sum() == pytest.approx(m.luminosity, rel=1e-12, abs=0)
    mc = r["stats"]["scatters"] / N
    rng = np.random.default_rng(1)
    half = n * tau_cell / 2
    nw = 20000
    pos = np.zeros((nw, 3))
    cnt = np.zeros(nw)
    alive = np.ones(nw, bool)

    def iso(k):
        mu = rng.uniform(-1, 1, k)
        ph = rng.uniform(0, 2 * math.pi, k)
        st = np.sqrt(1 - mu * mu)
        return np.stack([st * np.cos(ph), st * np.sin(ph), mu], 1)

    d = iso(nw)
    while alive.any():
        idx = np.nonzero(alive)[0]
        s = rng.exponential(1.0, idx.size)
        p = pos[idx] + d[idx] * s[:, None]
        out = np.abs(p).max(1) > half
        alive[idx[out]] = False
        keep = idx[~out]
        pos[keep] = p[~out]
        cnt[keep] += 1
        d[keep] = iso(keep.size)
    bf = cnt.mean()
    err = math.sqrt(cnt.var() / nw + (r["stats"]["scatters"] / N) / N * 4)
    assert abs(mc - bf) < 4 * err + 0.01 * bf, (mc, bf)


def test_optically_thin_equilibrium_temperature(O):
    """Gray optically thin dust around a point source: T^4 = L <1/r^2> /
    (16 pi sigma) cell by cell, with <1/r^2> averaged over the cell volume by
    quadrature (Lucy estimator, frozen temperatures, no re-emission needed at
    tau ~ 1e-3)."""
    n = 8
    m = gray_fine_model(n=n, tau_cell=2e-4, nf=160)
    N = 60000
    r = O.transport(m, N, seed=8, mode=O.MODE_NOREEMIT, lucy_mode=O.LUCY_ALL)
    T = O.temperatures(m, r["E_abs"])[0].reshape(n, n, n)
    sub = (np.arange(6) + 0.5) / 6
    Tref = np.zeros((n, n, n))
    for iz in range(n):
        for iy in range(n):
            for ix in range(n):
                pts = m.box_min + m.cell * (np.array([ix, iy, iz])[None, :] +
                                            np.stack(np.meshgrid(sub, sub, sub), -1).reshape(-1, 3))
                inv = (1.0 / (pts ** 2).sum(1)).mean()
                Tref[iz, iy, ix] = (m.luminosity * inv / (16 * math.pi * SIGMA)) ** 0.25
    E = r["E_abs"][0].reshape(n, n, n)
    relE = np.sqrt(r["esq"][0].reshape(n, n, n)) / E
    c = (np.arange(n) + 0.5 - n / 2)
    R = np.sqrt(c[:, None, None] ** 2 + c[None, :, None] ** 2 + c[None, None, :] ** 2)
    sel = R > 2.0
    err = np.abs(T[sel] / Tref[sel] - 1)
    # Sigma e^2 per deposit underestimates the per-packet variance; 6 sigma
    assert np.all(err < 6 * relE[sel] / 4 + 2e-3), err.max()


def test_bw_and_iterative_reach_the_same_temperatures(O):
    """Bjorkman & Wood (Eq. 10) and the iterative scheme (Eq. 5 with frozen
    temperatures, Eq. 4 between iterations) converge to the same equilibrium
    (Sect. 3.3): per cell within 3 sigma + 0.5 %, sigma the temperature
    noise of both runs' absorption counts (T ~ E^(1/4), so sigma_T / T =
    sqrt(1/n_bw + 1/n_it) / 4); the cells' mean deviation within 3 sigma of
    the mean + 0.5 %."""
    m = W.homogeneous_sphere(n=6, tau_v=2.0, nf=20)
    N = 250000
    rb = O.transport(m, N, seed=21, mode=O.MODE_BW, n_threads=1)
    Tb = O.temperatures(m, rb["E_abs"])
    Tp = O.temperature_guess(m)
    for it in range(5):
        ri = O.transport(m, N, seed=100 + it, mode=O.MODE_FROZEN_T, T_prev=Tp, n_threads=4)
        Tp = O.temperatures(m, ri["E_abs"])
    nb, ni = rb["count"][0].astype(float), ri["count"][0].astype(float)
    good = (nb > 400) & (ni > 400)
    assert good.sum() >= 40
    sig = 0.25 * np.sqrt(1 / nb[good] + 1 / ni[good])
    d = Tb[0][good] / Tp[0][good] - 1
    assert np.all(np.abs(d) < 3 * sig + 0.005), (np.abs(d) / sig).max()
    assert abs(d.mean()) < 3 * math.sqrt((sig ** 2).sum()) / good.sum() + 0.005, d.mean()
    # the escaped spectrum: B&W's re-emission from the difference spectrum
    # (Eq. 10, dB/dT) leaves the equilibrium SED of the converged iterative
    # scheme, frequency by frequency (sigma from both runs' escape counts)
    xi = m.luminosity / N
    Sb, Si = rb["sed_esc"].sum(0), ri["sed_esc"].sum(0)
    sS = xi * np.sqrt(rb["sed_cnt"].sum(0) + ri["sed_cnt"].sum(0))
    lit = sS > 0
    z = (Sb - Si)[lit] / (sS[lit] + 0.005 * np.maximum(Sb, Si)[lit])
    assert np.all(np.abs(z) < 4.0) and (z ** 2).mean() < 2.0, (np.abs(z).max(), (z ** 2).mean())


def _batch_sums(O, m, N, nb, **kw):
    """Totals of N packets run as nb packet-id batches, with the standard
    error of each total from the spread of the batches (independent packet
    streams, so batch means give an honest sigma for correlated tallies)."""
    E, S, C = [], [], []
    for b in range(nb):
        r = O.transport(m, N, pid_begin=b * N // nb, pid_end=(b + 1) * N // nb, **kw)
        E.append(r["E_abs"].sum())
        S.append(r["sed_esc"].sum(0))
        C.append(r["E_abs"][0].copy())
        last = r
    E, S, C = np.array(E), np.array(S), np.array(C)
    k = math.sqrt(nb)
    return (E.sum(), E.std(ddof=1) * k, S.sum(0), S.std(0, ddof=1) * k, C.sum(0),
            C.std(0, ddof=1) * k, last)


@pytest.mark.parametrize("n,albedo", [(4, 0.5), (2, 0.999)])
def test_mrw_on_and_off_agree(O, n, albedo):
    """A uniform gray cube with tau_cell = 20: the modified random walk
    (Sect. 3.2) reproduces the absorbed energy (total and per cell) and the
    escaped spectrum of plain transport within 3 sigma + 2 % (sigma from 10
    independent packet batches of each run), while taking fewer
    interactions.  At albedo 0.999 most packets leave the cube before their
    first absorption, so the escaped spectrum (source frequencies against the
    re-emitted ones) also weighs how often a walk ends in an absorption."""
    m = W.uniform_cube(n=n, tau_cell=20.0, nf=4, albedo=albedo)
    T0 = np.full((1, m.ncell), 300.0)
    N = 20000
    kw = dict(mode=O.MODE_FROZEN_T, T_prev=T0, n_threads=4)
    Ea, sEa, Sa, sSa, Ca, sCa, ron = _batch_sums(O, m, N, 10, seed=31, mrw=True, **kw)
    Eb, sEb, Sb, sSb, Cb, sCb, roff = _batch_sums(O, m, N, 10, seed=32, mrw=False, **kw)
    assert ron["stats"]["mrw_steps"] > 0 and roff["stats"]["mrw_steps"] == 0
    assert abs(Ea - Eb) < 3 * math.hypot(sEa, sEb) + 0.02 * Eb
    lit = Sb > 0
    assert np.all(np.abs(Sa - Sb)[lit] <= (3 * np.hypot(sSa, sSb) + 0.02 * Sb)[lit])
    assert np.all(Sa[~lit] == 0)
    z = (Ca - Cb) / np.sqrt(sCa ** 2 + sCb ** 2 + (0.02 * Cb) ** 2)
    assert np.all(np.abs(z) < 4.0) and (z ** 2).mean() < 2.0, (np.abs(z).max(), (z ** 2).mean())
    assert ron["stats"]["interactions"] < 0.7 * roff["stats"]["interactions"]


@pytest.mark.xfail(strict=True, reason="reading 6: a walk draws at most one absorption, so PAH "
                   "terminations inside walks are undercounted when chi_abs * l is not small")
def test_mrw_keeps_pah_absorptions(O):
    """A walk that ends in an absorption by a PAH species stores the packet
    for the PAH pass, as an absorption at the end of a plain flight does
    (Sects. 2.1, 3.2): in a gray tau_cell = 20 cube of two species, one of
    them a PAH species (pure absorber, 0.2 % of the dust), the fraction of
    packets stored as PAH absorptions with the modified random walk should
    equal that of plain transport within 4 sigma + 2 % (sigma from 10 packet
    batches of each run).  It does not under the walk's absorption rule of
    reading 6 (one absorption test per walk, the species then drawn by
    rho_s kappa^abs_s): a walk of path l really holds a Poisson number of
    absorptions, any of which may be a PAH one, so the walk stores with
    probability (1 - e^{-chi_abs l}) q instead of 1 - e^{-chi_pah l}
    (q = chi_pah / chi_abs).  Measured: 0.352 of the packets stored with the
    walk against 0.402 without (sigma 0.004).  Strict: the test fails once
    the rule is changed, so that this marker is removed with it."""
    m = W.uniform_cube(n=2, tau_cell=20.0, nf=4, albedo=0.9)
    m.rho = np.concatenate([m.rho, 0.002 * m.rho]).astype(np.float32)
    m.kabs = np.vstack([m.kabs, np.ones(m.nf)])
    m.ksca = np.vstack([m.ksca, np.zeros(m.nf)])
    m.g = np.vstack([m.g, np.zeros(m.nf)])
    m.is_pah = np.array([0, 1], np.int32)
    T0 = np.full((2, m.ncell), 300.0)
    N, nb = 20000, 10

    def fractions(seed, mrw):
        f = []
        for b in range(nb):
            r = O.transport(m, N, seed=seed, mode=O.MODE_FROZEN_T, T_prev=T0, mrw=mrw,
                            pid_begin=b * N // nb, pid_end=(b + 1) * N // nb, pah_cap=N, n_threads=4)
            f.append(r["stats"]["pah"] / (N // nb))
            last = r
        return np.array(f), last

    fa, ron = fractions(51, True)
    fb, roff = fractions(52, False)
    assert ron["stats"]["mrw_steps"] > 0 and roff["stats"]["mrw_steps"] == 0
    assert 0.05 < fb.mean() < 0.95
    sig = math.hypot(fa.std(ddof=1), fb.std(ddof=1)) / math.sqrt(nb)
    assert abs(fa.mean() - fb.mean()) < 4 * sig + 0.02 * fb.mean(), (fa.mean(), fb.mean(), sig)


def test_packet_range_sharding_is_exact(O):
    m = W.random_grid(n=(5, 4, 3), ns=2, seed=11, tau_scale=2.0)
    T0 = np.full((2, m.ncell), 200.0)
    N = 2000
    kw = dict(seed=4, mode=O.MODE_FROZEN_T, T_prev=T0, record_events=True, event_cap=20 * N)
    full = O.transport(m, N, **kw)
    a = O.transport(m, N, pid_begin=0, pid_end=700, **kw)
    b = O.transport(m, N, pid_begin=700, pid_end=N, **kw)
    thr = O.transport(m, N, n_threads=3, **kw)
    np.testing.assert_array_equal(a["count"] + b["count"], full["count"])
    np.testing.assert_allclose(a["E_abs"] + b["E_abs"], full["E_abs"], rtol=1e-12, atol=0)
    np.testing.assert_array_equal(np.concatenate([a["events"], b["events"]]), full["events"])
    np.testing.assert_array_equal(thr["events"], full["events"])
    np.testing.assert_allclose(thr["E_abs"], full["E_abs"], rtol=1e-12, atol=0)


# ---------------------------------------------------------------- ray tracer
def test_raytrace_axis_view_of_uniform_cube(O):
    """Uniform cube viewed along +z with pixels equal to cells: every pixel
    sees I = S (1 - exp(-tau)) with S = eta / chi (Eqs. 12-14, R9)."""
    n = 4
    m = W.uniform_cube(n=n, tau_cell=0.3, nf=6, albedo=0.0)
    T = np.full((1, m.ncell), 300.0)
    cam = W.Camera(0.0, 0.0, n, 1e20, m.cell)
    fidx = [1, 4]
    img, sed = O.raytrace(m, T, None, 0.0, [cam], fidx)
    chi = m.rho[0, 0, 0, 0] * (m.kabs[0] + m.ksca[0])
    for f, j in enumerate(fidx):
        x = H * m.nu[j] / (K * 300.0)
        B = 2 * H * m.nu[j] ** 3 / 2.99792458e10 ** 2 / math.expm1(x)
        S = m.rho[0, 0, 0, 0] * m.kabs[0, j] * B / chi[j]
        I = S * (1 - math.exp(-chi[j] * n * m.cell))
        np.testing.assert_allclose(img[0, f], I, rtol=1e-10)


def test_raytrace_image_symmetry(O):
    """A voxelised sphere is symmetric under the cube's reflections and axis
    swaps, and so is its image along a grid axis about the image centre: one
    ray through each pixel centre, pixels placed symmetrically about the
    line of sight through the box centre (reading 9).  The image is therefore
    unchanged by flipping either pixel index and by transposition."""
    m = W.homogeneous_sphere(n=8, tau_v=3.0, nf=6)
    T = np.full((1, m.ncell), 400.0)
    for npix in (9, 12):
        for th, ph in [(0.0, 0.0), (math.pi / 2, 0.0), (math.pi / 2, math.pi / 2)]:
            img, _ = O.raytrace(m, T, None, 0.0, [W.Camera(th, ph, npix, 1e20)], [2, 5])
            im = img[0]
            assert im.max() > 0
            np.testing.assert_allclose(im, im[:, ::-1, :], rtol=1e-9, atol=0)
            np.testing.assert_allclose(im, im[:, :, ::-1], rtol=1e-9, atol=0)
            np.testing.assert_allclose(im, im.transpose(0, 2, 1), rtol=1e-9, atol=0)


def test_raytrace_optically_thin_flux_and_star(O):
    n = 4
    m = W.uniform_cube(n=n, tau_cell=1e-9, nf=6, albedo=0.0)
    T = np.full((1, m.ncell), 500.0)
    D = 1e20
    cam = W.Camera(0.0, 0.0, n, D, m.cell)
    fidx = [0, 3, 5]
    _, sed = O.raytrace(m, T, None, 0.0, [cam], fidx)
    lnu = O.source_lnu(m)
    V = m.cell ** 3
    for f, j in enumerate(fidx):
        x = H * m.nu[j] / (K * 500.0)
        B = 2 * H * m.nu[j] ** 3 / 2.99792458e10 ** 2 / math.expm1(x)
        eta = m.rho[0, 0, 0, 0] * m.kabs[0, j] * B
        star = lnu[j] / (4 * math.pi * D * D)
        assert sed[0, f] == pytest.approx(m.ncell * eta * V / D ** 2 + star, rel=1e-6, abs=0)
    # dark screen: cold dust, only the attenuated star; tau along +z from the
    # centre to the face is chi * (n/2) cells
    m2 = W.uniform_cube(n=n, tau_cell=0.7, nf=6, albedo=0.0)
    T0 = np.zeros((1, m2.ncell))
    for th, ph, dist in [(0.0, 0.0, n / 2), (math.pi / 2, 0.0, n / 2),
                         (math.acos(1 / math.sqrt(3)), math.pi / 4, n / 2 * math.sqrt(3))]:
        _, sd = O.raytrace(m2, T0, None, 0.0, [W.Camera(th, ph, 4, D)], fidx)
        for f, j in enumerate(fidx):
            tau = m2.rho[0, 0, 0, 0] * (m2.kabs[0, j] + m2.ksca[0, j]) * dist * m2.cell
            assert sd[0, f] == pytest.approx(lnu[j] * math.exp(-tau) / (4 * math.pi * D * D),
                                             rel=1e-9, abs=0)


def test_scattering_source_normalisation(O):
    """Eq. 16 with the HG phase function normalised per steradian: the same
    scattering event in every cell of an optically thin cube, seen from many
    directions, integrates to N xi / dnu; with g = 0 every direction sees
    N xi / (4 pi dnu D^2) (thermal emission and direct light off)."""
    n = 3
    m = W.uniform_cube(n=n, tau_cell=1e-10, nf=5, albedo=1.0, g=0.6)
    T0 = np.zeros((1, m.ncell))
    ev = np.zeros(m.ncell, dtype=O.EVENT_DTYPE)
    ev["cell"] = np.arange(m.ncell)
    ev["nu"] = 2
    ev["k"] = [0.0, 0.6, 0.8]
    m.sources[0].L = 1e-300            # no direct light
    xi, D = 3.0e20, 1e18
    npix = 48
    dirs = _fib_sphere(300)
    tot = 0.0
    for k in dirs:
        th, ph = math.acos(np.clip(k[2], -1, 1)), math.atan2(k[1], k[0])
        _, sd = O.raytrace(m, T0, ev, xi, [W.Camera(th, ph, npix, D)], [2])
        tot += sd[0, 0]
    integral = tot / len(dirs) * 4 * math.pi * D * D     # int F D^2 dOmega
    assert integral == pytest.approx(m.ncell * xi / m.dnu[2], rel=1e-2, abs=0)
    m.g[:] = 0.0
    for k in dirs[:6]:
        th, ph = math.acos(np.clip(k[2], -1, 1)), math.atan2(k[1], k[0])
        _, sd = O.raytrace(m, T0, ev, xi, [W.Camera(th, ph, npix, D)], [2])
        assert sd[0, 0] == pytest.approx(m.ncell * xi / (4 * math.pi * m.dnu[2] * D * D), rel=3e-3, abs=0)
    # axis view with pixels equal to cells: the pixel sum is exact
    _, sd = O.raytrace(m, T0, ev, xi, [W.Camera(0.0, 0.0, n, D, m.cell)], [2])
    assert sd[0, 0] == pytest.approx(m.ncell * xi / (4 * math.pi * m.dnu[2] * D * D), rel=1e-8, abs=0)


def _loss(O, m, T, ev, xi, cams, fidx, wi, ws):
    img, sed = O.raytrace(m, T, ev, xi, cams, fidx)
    return float((wi * img).sum() + (ws * sed).sum())


def test_adjoint_matches_central_differences(O):
    m = W.random_grid(n=(5, 4, 3), ns=2, nf=6, seed=3, tau_scale=1.5, albedo=(0.2, 0.6))
    rng = np.random.default_rng(0)
    T = rng.uniform(50, 900, size=(2, m.ncell))
    ev = np.zeros(40, dtype=O.EVENT_DTYPE)
    ev["cell"] = rng.integers(0, m.ncell, 40)
    ev["nu"] = rng.choice([1, 4], 40)
    ev["species"] = rng.integers(0, 2, 40)
    kk = rng.normal(size=(40, 3))
    ev["k"] = kk / np.linalg.norm(kk, axis=1, keepdims=True)
    cams = [W.Camera(0.7, 0.3, 5, 3e16), W.Camera(2.0, -1.1, 5, 3e16)]
    fidx = [1, 4]
    wi = rng.normal(size=(2, 2, 5, 5))
    ws = rng.normal(size=(2, 2)) * 1e32
    xi = 1e28
    g, gs = O.raytrace_backward(m, T, ev, xi, cams, fidx, wi, ws)
    base = m.rho.copy()
    for s, c in [(0, 0), (1, 7), (0, 23), (1, 31), (0, 44), (1, 59)]:
        flat = base.reshape(2, -1)
        if flat[s, c] == 0:
            continue
        rp, rm = flat.copy(), flat.copy()
        rp[s, c] = np.float32(flat[s, c] * (1 + 1e-3))
        rm[s, c] = np.float32(flat[s, c] * (1 - 1e-3))
        m.rho = rp.reshape(base.shape)
        Lp = _loss(O, m, T, ev, xi, cams, fidx, wi, ws)
        m.rho = rm.reshape(base.shape)
        Lm = _loss(O, m, T, ev, xi, cams, fidx, wi, ws)
        m.rho = base
        fd = (Lp - Lm) / (float(rp[s, c]) - float(rm[s, c]))
        assert g[s, c] == pytest.approx(fd, rel=2e-5, abs=1e-9 * np.abs(g).max())
    # global scale: dL/dscale from FD on rho * (1 +- h)
    h = 1e-3
    m.rho = (base.astype(np.float64) * (1 + h)).astype(np.float32)
    Lp = _loss(O, m, T, ev, xi, cams, fidx, wi, ws)
    m.rho = (base.astype(np.float64) * (1 - h)).astype(np.float32)
    Lm = _loss(O, m, T, ev, xi, cams, fidx, wi, ws)
    m.rho = base
    assert gs == pytest.approx((Lp - Lm) / (2 * h), rel=1e-3, abs=0)
    assert gs == pytest.approx(float((base.reshape(2, -1).astype(np.float64) * g).sum()), rel=1e-12, abs=0)


def test_adjoint_zero_where_no_ray_passes(O):
    m = W.uniform_cube(n=6, tau_cell=0.5, nf=4)
    T = np.full((1, m.ncell), 400.0)
    cam = W.Camera(0.0, 0.0, 2, 1e20, 0.5 * m.cell)    # tiny image on the axis
    g, _ = O.raytrace_backward(m, T, None, 0.0, [cam], [1], np.ones((1, 1, 2, 2)), np.zeros((1, 1)))
    g = g.reshape(6, 6, 6)
    assert np.all(g[:, 0, :] == 0) and np.all(g[:, :, 0] == 0)
    assert np.abs(g[:, 2:4, 2:4]).sum() > 0


def test_equal_energy_source_bins(O):
    """Eq. 1 source grid: with the sources' luminosity cut into m bins of
    equal energy and N/m packets per bin, the packets emitted into each model
    frequency bin carry its energy sum_s L_nu,s dnu to within one source bin
    (L/m) per source, and each source receives its share of L to within one
    source bin.  An
    empty grid with re-emission off lets every packet escape at its emission
    frequency, so the escape tallies are the emission histogram."""
    m = W.uniform_cube(n=3, tau_cell=0.5, nf=24, gray=False)
    m.rho[:] = 0.0
    m.sources = [W.Source((0.1 * m.cell, 0.2 * m.cell, 0.0), 2.0 * W.LSUN, 5800.0),
                 W.Source((-0.3 * m.cell, 0.0, 0.1 * m.cell), 1.0 * W.LSUN, 3000.0)]
    Ltot = 3.0 * W.LSUN
    for mbins in (60, 600):
        N = 30 * mbins
        r = O.transport(m, N, seed=3, mode=O.MODE_NOREEMIT, source_bins=mbins)
        assert r["stats"]["escaped"] == N
        counts = r["sed_cnt"].sum(axis=0)
        E_emit = counts * (Ltot / N)
        E_true = np.zeros(m.nf)
        for s in m.sources:
            lnu = O.source_lnu(m, m.sources.index(s))
            E_true += lnu * m.dnu
        assert np.all(np.abs(E_emit - E_true) <= len(m.sources) * Ltot / mbins * (1 + 1e-9))
        assert np.abs(E_emit - E_true).max() > 0                 # not trivially exact
        # each source's packets (told apart by position at emission) carry its L
        r_t = O.transport(m, N, seed=3, mode=O.MODE_NOREEMIT, source_bins=mbins, traj_cap=3 * N)
        em = r_t["traj"][r_t["traj"]["type"] == O.T_EMIT]
        n0 = int(np.sum(np.abs(em["x"][:, 0] - m.sources[0].pos[0]) < 1e-3 * m.cell))
        assert abs(n0 * Ltot / N - m.sources[0].L) <= Ltot / mbins * (1 + 1e-9)
    # stratification: packet ids of one source bin share one frequency bin,
    # independent of the seed
    r1 = O.transport(m, 600, seed=1, mode=O.MODE_NOREEMIT, source_bins=60, traj_cap=10000)
    r2 = O.transport(m, 600, seed=9, mode=O.MODE_NOREEMIT, source_bins=60, traj_cap=10000)
    e1 = np.sort(r1["traj"][r1["traj"]["type"] == O.T_EMIT], order="pid")
    e2 = np.sort(r2["traj"][r2["traj"]["type"] == O.T_EMIT], order="pid")
    np.testing.assert_array_equal(e1["nu"], e2["nu"])
    nu = e1["nu"].reshape(60, 10)
    assert np.all(nu == nu[:, :1])
    # frequency bins where the sources emit nothing receive no packet, also
    # at the ends of the cumulative luminosity (the first and last source bins)
    lz = np.array([O.planck_B(v, 5800.0) for v in m.nu])
    lz[:3] = 0.0
    lz[-3:] = 0.0
    m.sources = [W.Source((0.0, 0.0, 0.0), W.LSUN, 0.0, lz)]
    for mbins in (7, 60):
        r = O.transport(m, 20 * mbins, seed=5, mode=O.MODE_NOREEMIT, source_bins=mbins)
        cnt = r["sed_cnt"].sum(0)
        assert cnt[:3].sum() == 0 and cnt[-3:].sum() == 0 and cnt.sum() == 20 * mbins


def _model_edges(nu):
    # model frequency bin edges: geometric means of neighbours, outer ones mirrored
    e = np.empty(len(nu) + 1)
    e[1:-1] = np.sqrt(nu[:-1] * nu[1:])
    e[0] = nu[0] ** 2 / e[1]
    e[-1] = nu[-1] ** 2 / e[-2]
    return e


def test_separate_source_grid_has_equal_energy_bins(O):
    """The source frequency grid of Eq. 1 on the sources' own continuous
    spectra: each bin holds the energy L/m, i.e. the cumulative luminosity at
    the frequency of bin b is (b + 1/2) L/m, checked by adaptive quadrature of
    the Planck function (scipy, independent of the oracle's series); the
    model frequency bins receive the exact integral of the spectrum over
    their frequency range to within one source bin per source; a tabulated
    spectrum (constant over each model bin) receives its L_nu dnu per bin the
    same way; with two sources the first L_1/L of the bins belong to the
    first; the transport emits source bin b's packets in its model bin."""
    from scipy import integrate
    h, k = 6.62607015e-27, 1.380649e-16
    m = W.r2_shell(n=4, nf=64)
    e = _model_edges(m.nu)
    T = m.sources[0].T_eff
    B = lambda nu: nu ** 3 / np.expm1(h * nu / (k * T))

    def cum(a, b):
        # in ln nu, split at the model edges so quad sees smooth pieces
        tot = 0.0
        pts = np.concatenate([[a], e[(e > a) & (e < b)], [b]])
        for lo, hi in zip(pts[:-1], pts[1:]):
            tot += integrate.quad(lambda t: B(np.exp(t)) * np.exp(t), np.log(lo), np.log(hi),
                                  epsabs=0, epsrel=1e-12, limit=200)[0]
        return tot

    total = cum(e[0], e[-1])
    mb = 200
    nu_i, src_i, fr = O.source_grid(m, mb)
    assert np.all(src_i == 0) and np.all(np.diff(fr) > 0)
    for b in range(0, mb, 7):
        assert abs(cum(e[0], fr[b]) / total - (b + 0.5) / mb) < 1e-9, b
    # each frequency bin index is the model bin holding the frequency
    assert np.all((fr >= e[nu_i]) & (fr < e[nu_i + 1]))
    # energy per model bin within one source bin
    E_bins = np.bincount(nu_i, minlength=m.nf) / mb
    E_true = np.array([cum(e[j], e[j + 1]) for j in range(m.nf)]) / total
    assert np.all(np.abs(E_bins - E_true) <= 1.0 / mb * (1 + 1e-9))
    # a tabulated spectrum, constant over each model bin
    lnu = np.zeros(m.nf)
    lnu[20:40] = np.linspace(1.0, 3.0, 20)
    mt = W.r2_shell(n=4, nf=64)
    mt.sources = [W.Source(mt.sources[0].pos, mt.sources[0].L, 0.0, lnu)]
    nt, _, _ = O.source_grid(mt, mb)
    w = lnu * np.diff(e)
    assert np.all(np.abs(np.bincount(nt, minlength=m.nf) / mb - w / w.sum()) <= 1.0 / mb * (1 + 1e-9))
    # two sources: bins in order of the sources, each with its share
    m2 = W.r2_shell(n=4, nf=64)
    m2.sources = [W.Source((0.0, 0.0, 0.0), 3.0 * W.LSUN, 5800.0), W.Source((0.0, 0.0, 0.0), 1.0 * W.LSUN, 2500.0)]
    n2, s2, f2 = O.source_grid(m2, 400)
    assert np.all(s2[:300] == 0) and np.all(s2[300:] == 1)
    # the transport: source bin b's packets are emitted in model bin nu_i[b]
    N = 4 * mb
    r = O.transport(m, N, seed=5, mode=O.MODE_NOREEMIT, source_bins=mb, source_grid=(nu_i, src_i),
                    traj_cap=40 * N)
    em = np.sort(r["traj"][r["traj"]["type"] == O.T_EMIT], order="pid")
    assert len(em) == N
    np.testing.assert_array_equal(em["nu"], nu_i[(em["pid"] * mb) // N])


def test_visibility_definition_pins(O):
    """Visibilities of images (oracle): a single bright pixel gives |V| = its
    flux with the phase of its sky offset; a Gaussian image gives the
    Gaussian transform exp(-2 pi^2 s^2 (u^2 + v^2)); real images are
    Hermitian, V(-u, -v) = conj V(u, v); a one-pixel shift multiplies V by
    exp(-2 pi i u dalpha)."""
    m = W.uniform_cube(n=4, tau_cell=0.5)
    npix, D = 64, 1e19
    cam = W.Camera(0.3, 0.2, npix, D, 0.05 * m.cell)
    pix = cam.pixel
    a = (np.arange(npix) + 0.5 - 0.5 * npix) * pix / D
    uv = np.array([[0.0, 0.0], [3e4, -1e4], [-2e5, 7e4], [5e5, 5e5]]) * (D / (npix * pix)) / 3e4
    img = np.zeros((1, 1, npix, npix))
    img[0, 0, 40, 13] = 2.5
    V = O.visibilities(m, img, [cam], uv)[0, 0]
    F = 2.5 * pix * pix / (D * D)
    np.testing.assert_allclose(np.abs(V), F, rtol=1e-12)
    np.testing.assert_allclose(V, F * np.exp(-2j * np.pi * (uv[:, 0] * a[13] + uv[:, 1] * a[40])),
                               rtol=1e-12, atol=1e-12 * F)
    # Gaussian of rms s (radians) much wider than a pixel and much narrower than the field
    s = 5 * pix / D
    g = np.exp(-(a[None, :] ** 2 + a[:, None] ** 2) / (2 * s * s))[None, None]
    ug = np.array([[0.0, 0.0], [0.05 / s, 0.0], [0.1 / s, 0.05 / s], [0.0, 0.15 / s]])
    Vg = O.visibilities(m, g, [cam], ug)[0, 0]
    expect = np.exp(-2 * np.pi ** 2 * s * s * (ug[:, 0] ** 2 + ug[:, 1] ** 2))
    np.testing.assert_allclose((Vg / Vg[0]).real, expect, rtol=1e-6)
    assert np.all(np.abs((Vg / Vg[0]).imag) < 1e-9)
    # Hermitian symmetry of a random real image, and the shift theorem
    rnd = np.random.default_rng(4).random((1, 1, npix, npix))
    Vp = O.visibilities(m, rnd, [cam], uv)[0, 0]
    Vm = O.visibilities(m, rnd, [cam], -uv)[0, 0]
    np.testing.assert_allclose(Vm, np.conj(Vp), rtol=1e-12, atol=1e-14 * abs(Vp[0]))
    sh = np.zeros_like(rnd)
    sh[..., 1:] = rnd[..., :-1]
    sh[..., 0] = 0.0
    rnd0 = rnd.copy()
    rnd0[..., -1] = 0.0                                 # the column shifted out
    V0 = O.visibilities(m, rnd0, [cam], uv)[0, 0]
    Vs = O.visibilities(m, sh, [cam], uv)[0, 0]
    np.testing.assert_allclose(Vs, V0 * np.exp(-2j * np.pi * uv[:, 0] * pix / D), rtol=1e-10,
                               atol=1e-12 * abs(V0[0]))


# ------------------------------------------------------- photon counting (Sect. 4)
def test_photon_counting_geometry_closed_forms(O):
    """Dust-free cube, point source off the centre, camera looking down +x
    with acceptance cosine c: every accepted packet leaves through the face
    x = h at (y0 + h ky/kx, z0 + h kz/kx).  Closed forms for isotropic
    emission: accepted fraction (1 - c)/2; image centroid (y0, z0); per-axis
    variance h^2 (1/c - 1)/2 plus the pixel's p^2/12."""
    side = W.AU
    h = side / 2
    y0, z0, c = 0.2 * h, -0.15 * h, 0.8
    m = W.uniform_cube(n=4, tau_cell=0.0, nf=6, source_pos=(0.0, y0, z0))
    m.rho[:] = 0.0
    npix = 64
    pix = side / npix
    N = 200_000
    r = O.transport(m, N, seed=3, mode=O.MODE_NOREEMIT, n_threads=4,
                    pc_cameras=[(math.pi / 2, 0.0, npix, pix, c)])
    img = r["pc_img"][0].sum(axis=0)                 # [iy, ix]
    xi = r["xi"]
    L = m.luminosity
    p = (1 - c) / 2
    assert abs(img.sum() - L * p) <= 5 * xi * math.sqrt(N * p * (1 - p))
    n_acc = img.sum() / xi
    ctr = (np.arange(npix) + 0.5 - npix / 2) * pix
    wy, wx = img.sum(axis=1), img.sum(axis=0)        # y' (rows) and x' (columns)
    mx, my = (wx * ctr).sum() / img.sum(), (wy * ctr).sum() / img.sum()
    sd = h * math.sqrt((1 / c - 1) / 2)
    assert abs(mx - y0) <= 5 * sd / math.sqrt(n_acc)
    assert abs(my - z0) <= 5 * sd / math.sqrt(n_acc)
    for w, mu in ((wx, y0), (wy, z0)):
        var = (w * (ctr - mu) ** 2).sum() / img.sum()
        assert var == pytest.approx(sd ** 2 + pix ** 2 / 12, rel=0.05, abs=0)


def test_photon_counting_matches_escape_tallies(O):
    """With dust: a camera on the +z axis with acceptance cosine 0.8 counts
    exactly the packets of the top cos(theta) bin of the escape SED, and a
    camera accepting every direction (c = -1, field = box diagonal) counts
    every escaped packet, per frequency; the threaded run merges the images
    in the same order as the serial one."""
    m = W.random_grid(n=(6, 5, 4), ns=2, seed=4, tau_scale=1.5, albedo=(0.3, 0.8))
    cams = [(0.0, 0.0, 12, 0.0, 0.8), (1.1, 0.4, 9, 0.0, -1.0), (2.2, -0.7, 5, 0.5 * m.cell, 0.3)]
    T0 = np.random.default_rng(2).uniform(40, 600, size=(m.ns, m.ncell))
    kw = dict(seed=9, mode=O.MODE_FROZEN_T, T_prev=T0, pc_cameras=cams)
    r1 = O.transport(m, 4000, n_threads=1, **kw)
    r4 = O.transport(m, 4000, n_threads=4, **kw)
    top, full, part = r1["pc_img"]
    assert r1["stats"]["escaped"] == 4000
    np.testing.assert_allclose(top.sum(axis=(1, 2)), r1["sed_esc"][9], rtol=1e-12, atol=0)
    np.testing.assert_allclose(full.sum(axis=(1, 2)), r1["sed_esc"].sum(axis=0), rtol=1e-12, atol=0)
    assert 0 < part.sum() < full.sum()
    for a, b in zip(r1["pc_img"], r4["pc_img"]):
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=0)


# ------------------------------------------------ PAH re-emission pass (Sect. 2.1)
def _chi2_ok(counts, expect, z=5.0):
    """chi^2 of a multinomial histogram within z sigma of its mean."""
    keep = expect > 0
    assert np.all(counts[~keep] == 0)
    c2 = ((counts[keep] - expect[keep]) ** 2 / expect[keep]).sum()
    dof = keep.sum() - 1
    return abs(c2 - dof) <= z * math.sqrt(2 * dof), (c2, dof)


def test_pah_reemission_frequency_law_per_class(O):
    """Eq. 6 with the class's eps_n: in a dust-free grid every re-emitted
    packet escapes at its emitted bin, so the escape counts per bin are a
    multinomial sample of eps_n(nu_j) dnu_j / sum; records in class-0 and
    class-2 cells are checked separately against their own table."""
    m = W.uniform_cube(n=6, tau_cell=0.0, nf=40)
    m.rho[:] = 0.0
    eps, cls = W.pah_emissivity(m, n_classes=3)
    for want in (0, 2):
        cells = np.nonzero(cls == want)[0]
        rec = np.zeros(20000, O.PAH_DTYPE)
        rec["cell"] = np.resize(cells, len(rec))
        r = O.pah_reemit(m, rec, 1.0, eps, cls, seed=11, mode=O.MODE_NOREEMIT, n_threads=4)
        assert r["stats"]["escaped"] == len(rec) and r["stats"]["emitted"] == len(rec)
        cnt = r["sed_cnt"].sum(axis=0).astype(np.float64)
        w = eps[want] * m.dnu
        ok, info = _chi2_ok(cnt, len(rec) * w / w.sum())
        assert ok, info
        other = eps[2 - want] * m.dnu
        assert not _chi2_ok(cnt, len(rec) * other / other.sum())[0]
        assert r["sed_esc"].sum() == pytest.approx(len(rec) * 1.0, rel=1e-12, abs=0)


@pytest.mark.parametrize("refined", [False, True])
def test_pah_reemission_positions_and_directions(O, refined):
    """Emission points lie in the record's cell (a sub-cube on a refined
    grid), uniform per axis (mean 1/2, variance 1/12 of the cell edge);
    directions isotropic (<k> = 0, <k_a^2> = 1/3)."""
    m = W.random_grid(n=(5, 4, 3), ns=1, seed=2)
    m.rho[:] = 0.0
    if refined:
        mask = np.zeros(m.rho.shape[1:], bool)
        mask[1, 2, 3] = mask[2, 0, 0] = True
        m = W.refine_cubes(m, mask, r=3)
    eps, _ = W.pah_emissivity(m, n_classes=1)
    rng = np.random.default_rng(1)
    rec = np.zeros(6000, O.PAH_DTYPE)
    rec["cell"] = rng.integers(0, m.ncell, len(rec))
    r = O.pah_reemit(m, rec, 2.0, eps, None, seed=5, mode=O.MODE_NOREEMIT, traj_cap=3 * len(rec))
    t = r["traj"]
    em = np.sort(t[t["type"] == 0], order="pid")
    assert len(em) == len(rec)
    c = rec["cell"][em["pid"]].astype(np.int64)
    nz, ny, nx = m.shape
    # lower corner and edge of every cell, from the model's cell numbering
    lo_all, h_all = [], []
    for q in range(nx * ny * nz):
        cz, cy, cx = q // (nx * ny), (q // nx) % ny, q % nx
        base = m.box_min + m.cell * np.array([cx, cy, cz])
        if refined and m.refined[cz, cy, cx]:
            h = m.cell / m.refine
            for sz in range(m.refine):
                for sy in range(m.refine):
                    for sx in range(m.refine):
                        lo_all.append(base + h * np.array([sx, sy, sz]))
                        h_all.append(h)
        else:
            lo_all.append(base)
            h_all.append(m.cell)
    lo_all, h_all = np.array(lo_all), np.array(h_all)
    assert len(h_all) == m.ncell
    f = (em["x"] - lo_all[c]) / h_all[c][:, None]
    assert np.all((f >= 0) & (f <= 1))
    n = len(f)
    assert np.all(np.abs(f.mean(axis=0) - 0.5) <= 5 * math.sqrt(1 / 12 / n))
    assert np.all(np.abs(f.var(axis=0) - 1 / 12) <= 5 * math.sqrt(1 / 180 / n))
    k = em["k"]
    assert np.all(np.abs(k.mean(axis=0)) <= 5 * math.sqrt(1 / 3 / n))
    assert np.all(np.abs((k ** 2).mean(axis=0) - 1 / 3) <= 5 * math.sqrt(4 / 45 / n))


def test_pah_reemission_conserves_the_stored_energy(O):
    """B&W transport of the torus stores PAH absorptions; the re-emission pass
    sends one packet of the same xi per record: it escapes or is stored
    again, so first-pass escapes + second-pass escapes + second-pass stores
    add up to L exactly; frozen-T passes split across threads agree."""
    m = W.clumpy_torus(n=16, n_clump=60, seed=3, nf=24)
    eps, cls = W.pah_emissivity(m)
    N = 3000
    r1 = O.transport(m, N, seed=4, mode=O.MODE_BW, pah_cap=N)
    xi = r1["xi"]
    n1 = r1["stats"]["pah"]
    assert n1 > 20 and len(r1["pah"]) == n1
    r2 = O.pah_reemit(m, r1["pah"], xi, eps, cls, seed=4, model_id=1, mode=O.MODE_BW,
                      pah_cap=n1, accumulate=r1)
    st2 = r2["stats"]
    assert st2["emitted"] == n1 and st2["escaped"] + st2["pah"] == n1
    esc2 = r2["sed_esc"].sum() - r1["sed_esc"].sum()
    assert r1["sed_esc"].sum() + esc2 + st2["pah"] * xi == pytest.approx(m.luminosity, rel=1e-12, abs=0)
    T0 = np.full((m.ns, m.ncell), 80.0)
    a = O.pah_reemit(m, r1["pah"], xi, eps, cls, seed=4, mode=O.MODE_FROZEN_T, T_prev=T0,
                     n_threads=1)
    b = O.pah_reemit(m, r1["pah"], xi, eps, cls, seed=4, mode=O.MODE_FROZEN_T, T_prev=T0,
                     n_threads=4)
    np.testing.assert_allclose(a["E_abs"], b["E_abs"], rtol=1e-12, atol=0)
    np.testing.assert_array_equal(a["sed_cnt"], b["sed_cnt"])


def test_pah_reemission_rejects_bad_inputs(O):
    m = W.uniform_cube(n=3, tau_cell=0.1)
    eps = np.ones((1, m.nf))
    rec = np.zeros(4, O.PAH_DTYPE)
    with pytest.raises(ValueError):
        O.pah_reemit(m, rec, 1.0, np.zeros((1, m.nf)), None)           # eps sums to 0
    rec["cell"][0] = m.ncell
    with pytest.raises(ValueError):
        O.pah_reemit(m, rec, 1.0, eps, None)                           # cell out of range
    rec["cell"][0] = 0
    with pytest.raises(ValueError):
        O.pah_reemit(m, rec, 1.0, eps, np.full(m.ncell, 1))            # class out of range


def test_refined_adjoint_matches_central_differences(O):
    """The adjoint on a grid with one level of refinement, against central
    differences of the forward ray tracer, for cells in divided cubes
    (sub-cubes) and undivided ones."""
    m0 = W.random_grid(n=(4, 3, 3), ns=1, nf=6, seed=5, tau_scale=1.5, albedo=(0.2, 0.6))
    mask = np.zeros(m0.rho.shape[1:], bool)
    mask[1, 1, 1] = mask[2, 0, 2] = mask[0, 2, 0] = True
    m = W.refine_cubes(m0, mask, r=2, jitter=0.5, seed=3)
    rng = np.random.default_rng(4)
    T = rng.uniform(50, 900, size=(1, m.ncell))
    ev = np.zeros(30, dtype=O.EVENT_DTYPE)
    ev["cell"] = rng.integers(0, m.ncell, 30)
    ev["nu"] = rng.choice([1, 4], 30)
    kk = rng.normal(size=(30, 3))
    ev["k"] = kk / np.linalg.norm(kk, axis=1, keepdims=True)
    cams = [W.Camera(0.7, 0.3, 6, 3e16), W.Camera(2.0, -1.1, 6, 3e16)]
    fidx = [1, 4]
    wi = rng.normal(size=(2, 2, 6, 6))
    ws = rng.normal(size=(2, 2)) * 1e32
    xi = 1e28
    g, gs = O.raytrace_backward(m, T, ev, xi, cams, fidx, wi, ws)
    base = m.rho.copy()
    fine = np.nonzero(np.repeat(mask.reshape(-1), np.where(mask.reshape(-1), 8, 1)))[0]
    picks = [int(fine[0]), int(fine[5]), int(fine[13]), int(fine[22]), 0, m.ncell - 1]
    tested = 0
    for c in picks:
        if base[0, c] == 0 or g[0, c] == 0:
            continue
        rp, rm = base.copy(), base.copy()
        rp[0, c] = np.float32(base[0, c] * (1 + 1e-3))
        rm[0, c] = np.float32(base[0, c] * (1 - 1e-3))
        m.rho = rp
        Lp = _loss(O, m, T, ev, xi, cams, fidx, wi, ws)
        m.rho = rm
        Lm = _loss(O, m, T, ev, xi, cams, fidx, wi, ws)
        m.rho = base
        fd = (Lp - Lm) / (float(rp[0, c]) - float(rm[0, c]))
        assert g[0, c] == pytest.approx(fd, rel=2e-5, abs=1e-9 * np.abs(g).max())
        tested += 1
    assert tested >= 3
    assert gs == pytest.approx(float((base.astype(np.float64) * g).sum()), rel=1e-12, abs=0)


def test_temperature_guess_closed_form(O):
    """The optically thin starting guess: T^4 = sum_i L_i / (16 pi sigma r_i^2)
    at each cell centre (sigma from CODATA, not from the oracle's Planck
    constants), capped at 2000 K; on a refined grid at each sub-cube centre."""
    m = W.uniform_cube(n=5, tau_cell=0.1, side_au=40.0, source_pos=(0.3 * W.AU, -0.2 * W.AU, 0.1 * W.AU))
    m.sources.append(W.Source((-6.0 * W.AU, 5.0 * W.AU, 2.0 * W.AU), 3.0 * W.LSUN, 4000.0))
    mask = np.zeros(m.shape, bool)
    mask[2, 2, 2] = mask[0, 4, 1] = True
    mr = W.refine_cubes(m, mask, r=3)
    for mm in (m, mr):
        T = O.temperature_guess(mm)
        nz, ny, nx = mm.shape
        centres = []
        for cz in range(nz):
            for cy in range(ny):
                for cx in range(nx):
                    lo = mm.box_min + mm.cell * np.array([cx, cy, cz])
                    if mm.refine and mm.refined[cz, cy, cx]:
                        h = mm.cell / mm.refine
                        for sz in range(mm.refine):
                            for sy in range(mm.refine):
                                for sx in range(mm.refine):
                                    centres.append(lo + h * (np.array([sx, sy, sz]) + 0.5))
                    else:
                        centres.append(lo + 0.5 * mm.cell)
        centres = np.array(centres)
        assert len(centres) == mm.ncell
        q = np.zeros(mm.ncell)
        for s in mm.sources:
            r2 = ((centres - np.asarray(s.pos)) ** 2).sum(axis=1)
            q += s.L / (16 * math.pi * SIGMA * r2)
        expect = np.minimum(q ** 0.25, 2000.0)
        np.testing.assert_allclose(T[0], expect, rtol=1e-9)
    # the cap: a hot source close to a cell centre (unit cube of 0.05 AU)
    h = W.uniform_cube(n=4, tau_cell=0.1, side_au=0.05, source_pos=(0.01 * W.AU, 0.0, 0.0))
    h.sources[0] = W.Source(h.sources[0].pos, 1e4 * W.LSUN, 5800.0)
    T = O.temperature_guess(h)[0]
    assert T.max() == 2000.0 and (T == 2000.0).sum() >= 8
