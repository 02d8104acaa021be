"""Statistical comparison of two Monte Carlo transport results.

Per-cell absorbed energies of the FP32 GPU transport and of the FP64 oracle
are noisy estimates of the same expectation.  The check follows the stated
tolerance: per cell |E_gpu - E_ref| <= max(3 sigma, 1e-3 E), sigma from both
runs' sums of squared deposits.  Three refinements make it a test with a
known false-alarm rate instead of a hand-picked allowance:

* only well-sampled cells are tested (at least `min_n` equal-weight deposits
  in both runs, n_eff = E^2 / sum e^2), where the sums are close to Gaussian;
* deposits of one packet in one cell are correlated (a packet re-absorbed in
  a thick cell deposits there many times), so sum e^2 underestimates the
  variance by a workload-dependent factor phi.  phi is measured by comparing
  two independent oracle runs with each other (mean square of their z-scores;
  never below 1), so the null distribution is calibrated without the GPU;
* the number of cells outside 3 sigma may not exceed the binomial tail of
  the Gaussian 3-sigma rate (0.27 %) at probability 1e-6, and the sum of the
  squared z-scores may not exceed the chi-square tail at 1e-6;
* on large grids the cells are not independent: one packet's long flight
  through optically thin cells deposits in hundreds of them, and the
  mean squared z-score of a million cells then varies by about 1 % from run
  to run, far more than the chi-square law of independent cells allows.
  There the chi-square bound is replaced by a paired test against the
  oracle's own spread: the mean squared z of GPU against oracle minus that
  of the second oracle run against the same first run, over the same cells,
  judged by the scatter of that difference over large spatial blocks (t
  below 5, one-sided).
"""
import math

import numpy as np
from scipy import stats

P_FAIL = 1e-6


def _sigma(r, xi):
    if r.get("esq") is not None:
        return np.sqrt(np.asarray(r["esq"], dtype=np.float64))
    return xi * np.sqrt(np.asarray(r["count"], dtype=np.float64))


def _neff(r, xi):
    E = np.asarray(r["E_abs"], dtype=np.float64)
    s = _sigma(r, xi)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(s > 0, (E / np.where(s > 0, s, 1.0)) ** 2, 0.0)


def cell_z(a, b, xi, E_rel=1e-3, min_n=25):
    """z-scores of per-cell E_abs differences of runs a and b and the mask of
    cells well sampled in both."""
    Ea = np.asarray(a["E_abs"], dtype=np.float64).ravel()
    Eb = np.asarray(b["E_abs"], dtype=np.float64).ravel()
    sa, sb = _sigma(a, xi).ravel(), _sigma(b, xi).ravel()
    den = np.sqrt(sa ** 2 + sb ** 2 + (E_rel * np.maximum(Ea, Eb)) ** 2)
    mask = (_neff(a, xi).ravel() >= min_n) & (_neff(b, xi).ravel() >= min_n) & (den > 0)
    z = np.zeros_like(Ea)
    z[mask] = (Ea[mask] - Eb[mask]) / den[mask]
    return z, mask


def assert_z_scores(z, label, nsig=3.0):
    n = z.size
    assert n > 0, f"{label}: no well-sampled cells"
    p = 2.0 * stats.norm.sf(nsig)
    kmax = int(stats.binom.isf(P_FAIL, n, p))
    out = int((np.abs(z) > nsig).sum())
    assert out <= kmax, f"{label}: {out} of {n} outside {nsig} sigma (allowed {kmax}); worst {np.abs(z).max():.2f}"
    chi2 = float((z ** 2).sum())
    lim = float(stats.chi2.isf(P_FAIL, n))
    assert chi2 <= lim, f"{label}: chi2 {chi2:.1f} over {n} cells above {lim:.1f}"


def assert_outliers(n_bad, n, label, nsig=3.0):
    """n_bad of n independent checks failed at the Gaussian nsig rate: no
    more than the binomial tail allows at probability 1e-6."""
    kmax = int(stats.binom.isf(P_FAIL, n, 2.0 * stats.norm.sf(nsig)))
    assert n_bad <= kmax, f"{label}: {n_bad} of {n} outside {nsig} sigma (allowed {kmax})"


def assert_same_energies(g, ref, ref2, xi, E_rel=1e-3, min_n=25, phi_max=4.0, blocks=None):
    """GPU run g against oracle run ref; ref2 is a second, independent
    oracle run of the same workload that calibrates the dispersion phi.
    `blocks` (a block label per cell) selects the paired block test instead
    of the chi-square bound for grids whose cells are strongly correlated.
    Returns (phi, number of cells tested)."""
    z0, m0 = cell_z(ref2, ref, xi, E_rel, min_n)
    phi = max(1.0, float((z0[m0] ** 2).mean())) if m0.any() else 1.0
    assert phi < phi_max, f"oracle-vs-oracle dispersion {phi:.2f}: sum e^2 misstates the variance"
    z, m = cell_z(g, ref, xi, E_rel, min_n)
    if blocks is None:
        assert_z_scores(z[m] / math.sqrt(phi), "E_abs per cell")
        return phi, int(m.sum())
    zs = z[m] / math.sqrt(phi)
    out = int((np.abs(zs) > 3.0).sum())
    assert_outliers(out, int(m.sum()), "E_abs per cell")
    both = m & m0
    lab = np.asarray(blocks).ravel()[both]
    nb = int(lab.max()) + 1
    a = np.bincount(lab, (z[both] ** 2), nb)
    b = np.bincount(lab, (z0[both] ** 2), nb)
    cnt = np.bincount(lab, None, nb)
    use = cnt > 0
    d = (a[use] - b[use]) / cnt.sum()
    diff = float(d.sum())
    se = float(d.std(ddof=1) * math.sqrt(use.sum()))
    assert diff < 5.0 * se, (f"E_abs per cell: mean z^2 {a.sum() / cnt.sum():.4f} against the oracle's "
                             f"own {b.sum() / cnt.sum():.4f} (difference {diff:+.4f}, block error {se:.4f})")
    return phi, int(m.sum())


def assert_same_sed(g, ref, xi, min_n=25):
    """Escaped SED per (direction bin, frequency): each packet escapes once,
    so a bin's count is binomial and its sigma at most xi sqrt(count)."""
    cg = np.asarray(g["sed_cnt"], dtype=np.float64).ravel()
    cr = np.asarray(ref["sed_cnt"], dtype=np.float64).ravel()
    Sg = np.asarray(g["sed_esc"], dtype=np.float64).ravel()
    Sr = np.asarray(ref["sed_esc"], dtype=np.float64).ravel()
    m = (cg >= min_n) & (cr >= min_n)
    z = (Sg[m] - Sr[m]) / (xi * np.sqrt(cg[m] + cr[m]))
    assert_z_scores(z, "escaped SED per bin")
    return int(m.sum())
