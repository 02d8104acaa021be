"""Seeded synthetic inputs shaped like the paper's models.

This module only *builds inputs*: frequency grids, synthetic dust opacities,
voxelised density grids, source descriptors and cameras.  It holds none of the
transport, temperature or ray-tracing arithmetic, and it is the one module that
both the FP64 CPU oracle (``oracle/``) and the CUDA library consume.

Geometries follow the paper's models:

* homogeneous sphere (Sect. 5.1 test geometry, constant density),
* r^-2 spherical shell with r_out = 1000 r_in (Sect. 5.1, Ivezic benchmark
  radii 3.14/3.15/3.20 AU for tau = 1/10/100),
* flared disk rho ~ (r/r_d)^-1 exp(-z^2 / 2h^2), h = z_d (r/r_d)^1.125
  (Sect. 5.2, Table 2 radii; Gaussian written in the exp(-z^2/2h^2) form),
* clumpy AGN torus (Sect. 6, Eq. 21 clump placement with r offset by r_in,
  Eq. 20 broken power-law source spectrum).

The dust optical data of the paper (Mie/Bruggeman composites, Draine
silicates) are not available, so opacities are smooth synthetic laws with the
same qualitative features (a flat UV/optical plateau, a lambda^-1 IR fall-off,
9.7 and 18 micron silicate bumps, PAH-like bands).

Every density is voxelised by averaging the analytic profile over sub-samples
of each cell and stored as float32; the optical depth is normalised on the
voxelised grid by summing rho * cell * kappa_ref along the cell row that starts
at the box centre and runs along +x.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

# CGS constants used to *place* the models (not the radiative-transfer math).
AU = 1.495978707e13          # cm
PC = 3.0856775814913673e18   # cm
LSUN = 3.828e33              # erg/s
C_LIGHT = 2.99792458e10      # cm/s
UM = 1.0e-4                  # cm


@dataclasses.dataclass
class Source:
    """A point source.  ``L_nu`` (erg/s/Hz on the model grid) gives the spectral
    shape; when it is None the source is a blackbody of temperature ``T_eff``.
    ``L`` is the bolometric luminosity (erg/s) that the spectrum is scaled to."""
    pos: Sequence[float]
    L: float
    T_eff: float = 0.0
    L_nu: Optional[np.ndarray] = None


@dataclasses.dataclass
class Camera:
    """Observer direction (theta, phi in radians, measured from +z), square
    image of ``npix`` pixels, distance ``D`` (cm), pixel size in cm (0 = the
    library's default: the box diagonal divided by npix)."""
    theta: float
    phi: float
    npix: int
    D: float
    pixel: float = 0.0


@dataclasses.dataclass
class Model:
    """One dust model on a Cartesian grid of cubes (Sect. 2).

    rho      float32 [ns, nz, ny, nx]  g/cm^3 per species (uniform grid), or
             float32 [ns, ncell]       per cell of a refined grid
    nu, dnu  float64 [nf]              Hz, ascending, bin widths
    kabs, ksca, g  float64 [ns, nf]    cm^2/g, cm^2/g, HG asymmetry
    is_pah   int32 [ns]                1 for stochastically heated species
    refine   int                       r >= 2 for one level of refinement, else 0
    refined  uint8 [nz, ny, nx]        1 = cube divided into r^3 sub-cubes

    Cells of a refined grid are numbered cube by cube (z, y, x order), a
    divided cube's r^3 sub-cubes consecutively, again in z, y, x order.
    """
    rho: np.ndarray
    box_min: np.ndarray
    cell: float
    nu: np.ndarray
    dnu: np.ndarray
    kabs: np.ndarray
    ksca: np.ndarray
    g: np.ndarray
    is_pah: np.ndarray
    sources: List[Source]
    name: str = ""
    refine: int = 0
    refined: Optional[np.ndarray] = None

    @property
    def shape(self):
        """Cube counts (nz, ny, nx)."""
        return self.refined.shape if self.refine else self.rho.shape[1:]

    @property
    def ns(self):
        return self.rho.shape[0]

    @property
    def nf(self):
        return self.nu.shape[0]

    @property
    def ncell(self):
        """Cells (leaves of a refined grid)."""
        return int(self.rho.shape[1]) if self.refine else int(np.prod(self.rho.shape[1:]))

    @property
    def leaf_base(self):
        """int64 [nz*ny*nx]: first cell of each cube (refined grids)."""
        per = np.where(self.refined.reshape(-1) > 0, self.refine ** 3, 1).astype(np.int64)
        return np.concatenate([[0], np.cumsum(per)[:-1]]).astype(np.int64)

    @property
    def luminosity(self):
        return float(sum(s.L for s in self.sources))


# --------------------------------------------------------------------------
# frequency grids and synthetic opacities
# --------------------------------------------------------------------------

def log_frequency_grid(n: int, lam_min_um: float, lam_max_um: float):
    """n log-spaced wavelengths; returns ascending nu (Hz) and bin widths whose
    edges sit at the geometric midpoints (outer edges half a log step out)."""
    lam = np.geomspace(lam_max_um, lam_min_um, n) * UM      # descending lambda
    nu = C_LIGHT / lam                                      # ascending nu
    r = (lam_max_um / lam_min_um) ** (1.0 / (n - 1))
    dnu = nu * (math.sqrt(r) - 1.0 / math.sqrt(r))
    return nu.astype(np.float64), dnu.astype(np.float64)


def wavelength_um(nu):
    return C_LIGHT / np.asarray(nu) / UM


def opacity_powerlaw(nu, kext_ref: float, lam_ref_um: float, slope: float,
                     albedo: float, g: float):
    """kappa_ext ~ nu^slope normalised to kext_ref at lam_ref, constant albedo
    and asymmetry (the homogeneous-sphere dust)."""
    nu_ref = C_LIGHT / (lam_ref_um * UM)
    kext = kext_ref * (np.asarray(nu) / nu_ref) ** slope
    return kext * (1.0 - albedo), kext * albedo, np.full_like(kext, g)


def _gauss(x, mu, sig):
    return np.exp(-0.5 * ((x - mu) / sig) ** 2)


def opacity_silicate_like(nu, kabs_uv: float = 1.0):
    """Synthetic silicate-like grain: kappa_abs flat below 1 micron and ~1/lambda
    above, times (1 + 4 G(9.7um, 1.0) + 1.5 G(18um, 2.5)); albedo
    0.6 (lambda/0.55um)^-1 and g = 0.6 (lambda/0.55um)^-0.5, both clipped to
    [0, 0.6]."""
    lam = wavelength_um(nu)
    base = np.where(lam < 1.0, 1.0, 1.0 / lam)
    kabs = kabs_uv * base * (1.0 + 4.0 * _gauss(lam, 9.7, 1.0) + 1.5 * _gauss(lam, 18.0, 2.5))
    alb = np.clip(0.6 * (lam / 0.55) ** -1.0, 0.0, 0.6)
    g = np.clip(0.6 * (lam / 0.55) ** -0.5, 0.0, 0.6)
    ksca = kabs * alb / (1.0 - alb)
    return kabs, ksca, g


def opacity_carbon_like(nu, kabs_uv: float = 1.0):
    """Synthetic amorphous-carbon-like grain: kappa_abs flat below 1 micron and
    ~1/lambda above, albedo 0.3, g 0.5."""
    lam = wavelength_um(nu)
    kabs = kabs_uv * np.where(lam < 1.0, 1.0, 1.0 / lam)
    ksca = kabs * 0.3 / 0.7
    return kabs, ksca, np.full_like(kabs, 0.5)


def opacity_pah_like(nu, kabs_uv: float = 1.0):
    """Absorption-only PAH-like cross-section: a UV continuum falling off past
    0.3 micron plus Drude-like bands at 3.3, 6.2, 7.7, 8.6 and 11.3 micron."""
    lam = wavelength_um(nu)
    cont = np.where(lam < 0.3, 1.0, (0.3 / lam) ** 3)
    bands = [(3.3, 0.05, 0.02), (6.2, 0.2, 0.05), (7.7, 0.4, 0.08), (8.6, 0.3, 0.05), (11.3, 0.2, 0.06)]
    b = np.zeros_like(lam)
    for lc, wid, amp in bands:
        gam = wid / lc
        x = lam / lc
        b += amp * gam ** 2 / ((x - 1.0 / x) ** 2 + gam ** 2)
    kabs = kabs_uv * (cont + b)
    return kabs, np.zeros_like(kabs), np.zeros_like(kabs)


def extinction_at(kabs, ksca, nu, lam_um: float):
    """Interpolate kappa_ext of one species (log-log in nu) at a wavelength."""
    x = np.log(C_LIGHT / (lam_um * UM))
    return float(np.exp(np.interp(x, np.log(nu), np.log(kabs + ksca))))


# --------------------------------------------------------------------------
# voxelisation helpers
# --------------------------------------------------------------------------

def cell_centres(n: int, lo: float, cell: float):
    return lo + (np.arange(n) + 0.5) * cell


def voxelise(profile, n: Sequence[int], box_min, cell: float, sub: int = 4,
             slab: int = 4) -> np.ndarray:
    """Average ``profile(x, y, z)`` over sub^3 regular sub-samples per cell.
    Returns float64 [nz, ny, nx]; evaluated slab by slab to bound memory."""
    nx, ny, nz = n
    off = (np.arange(sub) + 0.5) / sub
    xs = (box_min[0] + (np.arange(nx)[:, None] + off[None, :]) * cell).reshape(-1)
    ys = (box_min[1] + (np.arange(ny)[:, None] + off[None, :]) * cell).reshape(-1)
    out = np.empty((nz, ny, nx), dtype=np.float64)
    for k0 in range(0, nz, slab):
        k1 = min(nz, k0 + slab)
        zs = (box_min[2] + (np.arange(k0, k1)[:, None] + off[None, :]) * cell).reshape(-1)
        Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
        v = profile(X, Y, Z)
        v = v.reshape(k1 - k0, sub, ny, sub, nx, sub).mean(axis=(1, 3, 5))
        out[k0:k1] = v
    return out


def tau_row_plus_x(rho_kext: np.ndarray, cell: float) -> float:
    """Optical depth summed along the +x cell row that starts at the box centre
    (the row (j, k) = (ny//2, nz//2), cells i >= nx//2)."""
    nz, ny, nx = rho_kext.shape
    return float(rho_kext[nz // 2, ny // 2, nx // 2:].sum() * cell)


def _finish(rho_unit: np.ndarray, kext_ref: float, cell: float, tau: float) -> np.ndarray:
    t = tau_row_plus_x(rho_unit * kext_ref, cell)
    return (rho_unit * (tau / t)).astype(np.float32)


# --------------------------------------------------------------------------
# the models
# --------------------------------------------------------------------------

def homogeneous_sphere(n: int = 32, tau_v: float = 1.0, side_au: float = 2.0,
                       nf: int = 30, T_star: float = 5800.0, sub: int = 4) -> Model:
    """Uniform dust sphere of radius side/2 in a cube, central 5800 K star,
    kappa_ext ~ nu^1.5, albedo 0.5, g 0.5, 30 frequencies 0.1-100 micron."""
    side = side_au * AU
    cell = side / n
    bmin = np.array([-side / 2] * 3)
    nu, dnu = log_frequency_grid(nf, 0.1, 100.0)
    kabs, ksca, g = opacity_powerlaw(nu, 1.0, 0.55, 1.5, 0.5, 0.5)
    R = side / 2
    prof = lambda X, Y, Z: (X * X + Y * Y + Z * Z <= R * R).astype(np.float64)
    rho = _finish(voxelise(prof, (n, n, n), bmin, cell, sub), 1.0, cell, tau_v)
    return Model(rho[None], bmin, cell, nu, dnu, kabs[None], ksca[None], g[None],
                 np.zeros(1, np.int32), [Source((0.0, 0.0, 0.0), LSUN, T_star)],
                 name=f"homogeneous sphere {n}^3 tauV={tau_v:g}")


SHELL_RIN_AU = {1.0: 3.14, 10.0: 3.15, 100.0: 3.20, 1000.0: 3.52}


def r2_shell(n: int = 128, tau_1um: float = 10.0, nf: int = 64, T_star: float = 2500.0,
             sub: int = 4) -> Model:
    """rho ~ r^-2 between r_in and 1000 r_in, box half-side r_out, central
    2500 K 1 Lsun star, silicate-like dust, 64 frequencies 0.1-1000 micron,
    tau normalised at 1 micron on the voxelised grid."""
    r_in = SHELL_RIN_AU.get(float(tau_1um), 3.15) * AU
    r_out = 1000.0 * r_in
    cell = 2 * r_out / n
    bmin = np.array([-r_out] * 3)
    nu, dnu = log_frequency_grid(nf, 0.1, 1000.0)
    kabs, ksca, g = opacity_silicate_like(nu)
    kref = extinction_at(kabs, ksca, nu, 1.0)

    def prof(X, Y, Z):
        r2 = X * X + Y * Y + Z * Z
        inside = (r2 >= r_in * r_in) & (r2 <= r_out * r_out)
        return np.where(inside, (r_in * r_in) / np.maximum(r2, 1e-300), 0.0)

    rho = _finish(voxelise(prof, (n, n, n), bmin, cell, sub), kref, cell, tau_1um)
    return Model(rho[None], bmin, cell, nu, dnu, kabs[None], ksca[None], g[None],
                 np.zeros(1, np.int32), [Source((0.0, 0.0, 0.0), LSUN, T_star)],
                 name=f"r^-2 shell {n}^3 tau1um={tau_1um:g}")


def flared_disk(n: int = 256, tau_v: float = 100.0, nf: int = 100, T_star: float = 5800.0,
                sub: int = 2) -> Model:
    """Flared disk rho ~ (r/r_d)^-1 exp(-z^2/2h^2), h = z_d (r/r_d)^1.125,
    r_in 1 AU, r_out 1000 AU, r_d 500 AU, z_d 125 AU (Table 2), zero inside
    r_in and outside r_out; midplane tau at 0.55 micron on the voxelised
    grid; central 5800 K star."""
    r_in, r_out, r_d, z_d = 1.0 * AU, 1000.0 * AU, 500.0 * AU, 125.0 * AU
    cell = 2 * r_out / n
    bmin = np.array([-r_out] * 3)
    nu, dnu = log_frequency_grid(nf, 0.1, 1000.0)
    kabs, ksca, g = opacity_silicate_like(nu)
    kref = extinction_at(kabs, ksca, nu, 0.55)

    def prof(X, Y, Z):
        r = np.sqrt(X * X + Y * Y)
        rr = np.maximum(r, r_in) / r_d
        h = z_d * rr ** 1.125
        v = np.exp(-0.5 * (Z / h) ** 2) / rr
        return np.where((r >= r_in) & (r <= r_out), v, 0.0)

    rho = _finish(voxelise(prof, (n, n, n), bmin, cell, sub), kref, cell, tau_v)
    return Model(rho[None], bmin, cell, nu, dnu, kabs[None], ksca[None], g[None],
                 np.zeros(1, np.int32), [Source((0.0, 0.0, 0.0), LSUN, T_star)],
                 name=f"flared disk {n}^3 tauV={tau_v:g}")


def agn_broken_powerlaw_Lnu(nu):
    """Eq. 20 shape: lambda F_lambda ~ lambda^1.2 below 0.01 micron, constant to
    0.1 micron, lambda^-0.5 to 1 micron, lambda^-3 beyond (continuous at the
    breaks).  Returns L_nu up to a constant (lambda F_lambda = nu F_nu)."""
    lam = wavelength_um(nu)
    lfl = np.where(lam < 0.01, (lam / 0.01) ** 1.2,
          np.where(lam < 0.1, 1.0,
          np.where(lam < 1.0, (lam / 0.1) ** -0.5, (0.1) ** 0.5 * lam ** -3.0)))
    return lfl / np.asarray(nu)


def torus_grid_size(m: int) -> int:
    return int(min(192, max(64, 8 * ((64 + 2 * (m % 65)) // 8))))


def torus_clump_count(m: int) -> int:
    return 200 + (m * 76) % 4801


def clumpy_torus(n: int = 128, n_clump: int = 1000, seed: int = 77, nf: int = 100,
                 tau_clump_v: float = 30.0, contrast: float = 100.0,
                 half_open_deg: float = 30.0, L: float = 1e45,
                 r_in_pc: float = 0.4, r_out_pc: float = 6.0,
                 clump_r_frac=(0.005, 0.02), with_pah: bool = True, sub: int = 2) -> Model:
    """Clumpy AGN torus (Sect. 6).  Clump centres from Eq. 21 with the radius
    offset by r_in; clump radii uniform in clump_r_frac * r_out; constant
    clump density giving tau_V = tau_clump_v through a clump of the mean radius;
    inter-clump medium at 1/contrast of the clump density inside the torus
    envelope; overlaps keep the clump density (max).  Species: silicate and
    carbon (mass fractions 0.68/0.32) plus PAH at 0.05 of the total."""
    rng = np.random.default_rng(seed)
    r_in, r_out = r_in_pc * PC, r_out_pc * PC
    cell = 2 * r_out / n
    bmin = np.array([-r_out] * 3)
    nu, dnu = log_frequency_grid(nf, 0.01, 1000.0)
    ka_s, ks_s, g_s = opacity_silicate_like(nu)
    ka_c, ks_c, g_c = opacity_carbon_like(nu)
    fr = np.array([0.68, 0.32])
    species = [(ka_s, ks_s, g_s), (ka_c, ks_c, g_c)]
    if with_pah:
        species.append(opacity_pah_like(nu))
        fr = np.array([0.68, 0.32, 0.05])
    # mixture extinction at V of the large grains sets the clump density
    kv = fr[0] * extinction_at(ka_s, ks_s, nu, 0.55) + fr[1] * extinction_at(ka_c, ks_c, nu, 0.55)
    th1 = math.radians(half_open_deg)
    z1, z2, z3 = rng.random(n_clump), rng.random(n_clump), rng.random(n_clump)
    rc = r_in + z1 * (r_out - r_in)
    ph = 2 * math.pi * z2
    th = math.pi / 2 + (2 * z3 - 1) * th1
    cx, cy, cz = rc * np.sin(th) * np.cos(ph), rc * np.sin(th) * np.sin(ph), rc * np.cos(th)
    rad = r_out * (clump_r_frac[0] + rng.random(n_clump) * (clump_r_frac[1] - clump_r_frac[0]))
    rho_c = tau_clump_v / (2.0 * r_out * 0.5 * sum(clump_r_frac) * kv)

    ns = n * sub
    fine = cell / sub
    inside = np.zeros((ns, ns, ns), dtype=bool)
    for x, y, z, r in zip(cx, cy, cz, rad):
        lo = np.floor((np.array([x, y, z]) - r - bmin) / fine).astype(int)
        hi = np.ceil((np.array([x, y, z]) + r - bmin) / fine).astype(int)
        lo = np.clip(lo, 0, ns)
        hi = np.clip(hi, 0, ns)
        if np.any(hi <= lo):
            continue
        gx = bmin[0] + (np.arange(lo[0], hi[0]) + 0.5) * fine - x
        gy = bmin[1] + (np.arange(lo[1], hi[1]) + 0.5) * fine - y
        gz = bmin[2] + (np.arange(lo[2], hi[2]) + 0.5) * fine - z
        d2 = gz[:, None, None] ** 2 + gy[None, :, None] ** 2 + gx[None, None, :] ** 2
        inside[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] |= d2 <= r * r
    c = bmin[0] + (np.arange(ns) + 0.5) * fine
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij", sparse=True)
    R = np.sqrt(X * X + Y * Y + Z * Z)
    cos_t = np.abs(Z) / np.maximum(R, 1e-300)
    env = (R >= r_in) & (R <= r_out) & (cos_t <= math.sin(th1))
    fine_rho = np.where(inside, rho_c, np.where(env, rho_c / contrast, 0.0))
    rho_tot = fine_rho.reshape(n, sub, n, sub, n, sub).mean(axis=(1, 3, 5))
    rho = np.stack([(f * rho_tot) for f in fr]).astype(np.float32)
    kabs = np.stack([s[0] for s in species])
    ksca = np.stack([s[1] for s in species])
    g = np.stack([s[2] for s in species])
    is_pah = np.array([0, 0, 1][:len(species)], dtype=np.int32)
    Lnu = agn_broken_powerlaw_Lnu(nu)
    return Model(rho, bmin, cell, nu, dnu, kabs, ksca, g, is_pah,
                 [Source((0.0, 0.0, 0.0), L, 0.0, Lnu)],
                 name=f"clumpy torus {n}^3 N_clump={n_clump} seed={seed}")


def batched_tori(n_models: int = 64, base_seed: int = 1000, scale: float = 1.0, **kw) -> List[Model]:
    """The batch of clumpy-torus realisations: model m has grid
    torus_grid_size(m) (64^3-192^3, scaled by ``scale`` for small test
    batches) and torus_clump_count(m) clumps, seed base_seed + m."""
    out = []
    for m in range(n_models):
        n = max(8, int(round(torus_grid_size(m) * scale / 8)) * 8)
        out.append(clumpy_torus(n=n, n_clump=torus_clump_count(m), seed=base_seed + m, **kw))
    return out


def uniform_cube(n: int = 8, tau_cell: float = 0.5, nf: int = 8, albedo: float = 0.0,
                 g: float = 0.0, T_star: float = 5800.0, side_au: float = 1.0,
                 source_pos=None, gray: bool = True) -> Model:
    """Small uniform cube for closed-form checks: every cell has the same
    density; tau_cell is the optical depth across one cell at every frequency
    when ``gray`` (kappa_ext independent of nu)."""
    side = side_au * AU
    cell = side / n
    bmin = np.array([-side / 2] * 3)
    nu, dnu = log_frequency_grid(nf, 0.1, 100.0)
    kext = np.ones(nf) if gray else (nu / nu[-1]) ** 1.0 + 0.05
    kabs, ksca = kext * (1 - albedo), kext * albedo
    rho = np.full((1, n, n, n), tau_cell / (kext.max() * cell), dtype=np.float32)
    pos = (0.0, 0.0, 0.0) if source_pos is None else tuple(source_pos)
    return Model(rho, bmin, cell, nu, dnu, kabs[None], ksca[None], np.full((1, nf), g),
                 np.zeros(1, np.int32), [Source(pos, LSUN, T_star)],
                 name=f"uniform cube {n}^3 tau_cell={tau_cell:g}")


def random_grid(n=(6, 5, 4), ns: int = 1, nf: int = 8, seed: int = 0, tau_scale: float = 1.0,
                empty_frac: float = 0.2, albedo=(0.0, 0.8), T_star: float = 5800.0) -> Model:
    """Small irregular grid with log-normal cell densities, some empty cells,
    random smooth opacities per species; for parity tests on ragged shapes."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = n
    cell = AU
    bmin = -0.5 * cell * np.array([nx, ny, nz], dtype=np.float64)
    nu, dnu = log_frequency_grid(nf, 0.1, 300.0)
    lam = wavelength_um(nu)
    kabs = np.empty((ns, nf)); ksca = np.empty((ns, nf)); gg = np.empty((ns, nf))
    for s in range(ns):
        a = rng.uniform(*albedo)
        base = np.where(lam < 1.0, 1.0, lam ** -rng.uniform(0.5, 1.5))
        kabs[s] = base * (1 - a) * rng.uniform(0.5, 2.0)
        ksca[s] = base * a * rng.uniform(0.5, 2.0)
        gg[s] = np.clip(rng.uniform(-0.3, 0.8) * np.ones(nf), -0.9, 0.9)
    rho = rng.lognormal(0.0, 1.0, size=(ns, nz, ny, nx))
    rho[:, rng.random((nz, ny, nx)) < empty_frac] = 0.0
    kmax = (kabs + ksca).max()
    rho = rho * tau_scale / (kmax * cell * max(rho.mean(), 1e-30))
    pos = tuple(bmin + cell * np.array([nx, ny, nz]) * rng.uniform(0.2, 0.8, 3))
    return Model(rho.astype(np.float32), bmin, cell, nu, dnu, kabs, ksca, gg,
                 np.zeros(ns, np.int32), [Source(pos, LSUN, T_star)],
                 name=f"random grid {n} ns={ns} seed={seed}")


def refine_cubes(model: Model, mask: np.ndarray, r: int = 2, fine_rho=None, jitter: float = 0.0,
                 seed: int = 0) -> Model:
    """One level of refinement (Sect. 2) of a uniform model: the cubes where
    ``mask`` [nz, ny, nx] is true are divided into r^3 sub-cubes.  Sub-cube
    densities come from ``fine_rho`` [ns, r nz, r ny, r nx] (e.g. the profile
    voxelised at r times the resolution) or inherit the cube's density;
    ``jitter`` > 0 multiplies them by seeded log-normal factors."""
    rng = np.random.default_rng(seed)
    ns = model.ns
    nz, ny, nx = model.rho.shape[1:]
    mask = np.asarray(mask, dtype=bool).reshape(nz, ny, nx)
    cols = []
    for cz in range(nz):
        for cy in range(ny):
            for cx in range(nx):
                if not mask[cz, cy, cx]:
                    cols.append(model.rho[:, cz, cy, cx][:, None])
                    continue
                if fine_rho is not None:
                    blk = fine_rho[:, cz * r:(cz + 1) * r, cy * r:(cy + 1) * r, cx * r:(cx + 1) * r]
                    leaf = blk.reshape(ns, r ** 3)
                else:
                    leaf = np.repeat(model.rho[:, cz, cy, cx][:, None], r ** 3, axis=1)
                if jitter > 0:
                    leaf = leaf * np.exp(jitter * rng.standard_normal(leaf.shape))
                cols.append(leaf)
    rho = np.concatenate(cols, axis=1).astype(np.float32)
    out = dataclasses.replace(model, rho=rho, refine=int(r), refined=mask.astype(np.uint8),
                              name=f"{model.name} refined r={r} ({int(mask.sum())} cubes)")
    return out


def r2_shell_refined(n: int = 64, tau_1um: float = 10.0, nf: int = 64, r: int = 4,
                     refine_radius: float = 4.0) -> Model:
    """The r^-2 shell on n^3 cubes with the cubes within ``refine_radius``
    cube edges of the centre divided into r^3 sub-cubes -- finer sampling
    near the dust evaporation zone, where the paper refines; sub-cube
    densities from the profile voxelised at r times the resolution with the
    same tau normalisation."""
    coarse = r2_shell(n=n, tau_1um=tau_1um, nf=nf)
    fine = r2_shell(n=n * r, tau_1um=tau_1um, nf=nf, sub=1)
    c = np.arange(n) + 0.5 - n / 2
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    mask = np.sqrt(X * X + Y * Y + Z * Z) <= refine_radius
    return refine_cubes(coarse, mask, r=r, fine_rho=fine.rho)


def pah_emissivity(model: Model, n_classes: int = 4):
    """Synthetic PAH emissivity classes for the re-emission pass: eps_n(nu) =
    K_PAH(nu) * s_n(nu), s_n a log-normal band in wavelength whose peak moves
    from 5 to 40 micron with the class (standing in for the band-weighted
    temperature distributions of cells in weaker radiation fields), and each
    cell's class set by its distance from the box centre (inner cells class
    0).  Returns eps [n_classes][nf] and eps_class int32 [ncell]."""
    pah = [s for s in range(model.ns) if model.is_pah[s]]
    kabs = model.kabs[pah[0]] if pah else model.kabs[0]
    lam = wavelength_um(model.nu)
    peaks = np.geomspace(5.0, 40.0, n_classes)
    eps = np.stack([kabs * np.exp(-0.5 * (np.log(lam / p) / 0.6) ** 2) for p in peaks])
    nz, ny, nx = model.shape
    z, y, x = np.meshgrid(np.arange(nz) + 0.5 - nz / 2, np.arange(ny) + 0.5 - ny / 2,
                          np.arange(nx) + 0.5 - nx / 2, indexing="ij")
    r = np.sqrt(x * x + y * y + z * z) / (0.5 * math.sqrt(nx * nx + ny * ny + nz * nz))
    cls = np.minimum((r * n_classes).astype(np.int32), n_classes - 1).reshape(-1)
    if model.refine:                       # sub-cubes take their cube's class
        per = np.where(model.refined.reshape(-1) > 0, model.refine ** 3, 1)
        cls = np.repeat(cls, per)
    return eps, cls


def inclinations_deg():
    return [12.5, 30.0, 45.0, 60.0, 77.5]


def image_wavelengths_um():
    return [0.55, 1.0, 2.2, 3.5, 5.0, 8.0, 10.0, 12.0, 18.0, 24.0, 70.0, 160.0]


def nearest_freq_indices(nu, lam_um: Sequence[float]):
    lam = wavelength_um(nu)
    return [int(np.argmin(np.abs(np.log(lam / l)))) for l in lam_um]


# --------------------------------------------------------------------------
# Synthetic observation for the ray-tracer adjoint (a density fit): the
# SED wavelengths, the eight viewing angles and the "true" density that the
# synthetic observation is made from, all seeded.

def adjoint_sed_wavelengths_um(n: int = 40) -> List[float]:
    """n log-spaced SED wavelengths over 0.3-500 um, the one nearest 10 um
    replaced by 10 um."""
    lam = np.geomspace(0.3, 500.0, n)
    lam[int(np.argmin(np.abs(np.log(lam / 10.0))))] = 10.0
    return [float(v) for v in lam]


def adjoint_view_angles():
    """Eight viewing directions (theta, phi in radians) of the image part of
    the fit: inclinations 10-150 degrees, azimuths 45 degrees apart."""
    return [(math.radians(th), math.radians(45.0 * k))
            for k, th in enumerate((10, 30, 50, 70, 90, 110, 130, 150))]


def perturbed_density(model: Model, sigma: float = 0.3, seed: int = 78) -> np.ndarray:
    """The density a synthetic observation is made from: rho (1 + sigma n),
    n a standard normal field smoothed over 3^3 cells and rescaled to unit
    variance, the factor clipped at 0.05 (same factor for every species)."""
    rng = np.random.default_rng(seed)
    shape = model.rho.shape[1:]
    g = rng.normal(size=shape)
    s = np.zeros_like(g)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                s += np.roll(g, (dz, dy, dx), axis=(0, 1, 2))
    s /= s.std()
    f = np.clip(1.0 + sigma * s, 0.05, None)
    return (model.rho * f[None]).astype(np.float32)
