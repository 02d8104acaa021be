/*
 * FP64 CPU oracle for Monte Carlo dust radiative transfer
 * (Heymann & Siebenmorgen 2012, arXiv:1203.2941).
 *
 * TEST INFRASTRUCTURE ONLY: the plain, slow, obviously-correct restatement of
 * the method that the CUDA library is checked against.  Only tests, the smoke
 * check and the benchmark's CPU-baseline leg load it.  Nothing here is shared
 * with the CUDA library (no header, helper, table or constant generator).
 *
 * Every quantity is double precision.  The packet algorithm follows the
 * paper's order (Sect. 2): equal-energy packets xi = L/N, isotropic emission,
 * one optical depth tau = -ln(u) per flight (the footnote of Sect. 2 states
 * the per-cell redraw is equivalent), the cell test tau_i = (k_abs+k_sca) rho l
 * (Eq. 2), the interaction distance (Eq. 3), albedo choice, Henyey-Greenstein
 * scattering (Eq. 15) with the event store (cell, frequency, incoming
 * direction), absorption with re-emission from Eq. 5 (iterative scheme, frozen
 * temperatures) or Eq. 10 (Bjorkman & Wood, temperature from Eq. 4 after every
 * absorption), the Lucy path-length estimator in optically thin cells
 * (Sect. 3.1, Eq. 9) and the modified random walk in very thick cells
 * (Sect. 3.2).  The ray tracer follows Sect. 4 (Eqs. 11-17).
 *
 * Each function is pinned by the CPU tests against closed forms, brute
 * force, invariants or the paper's printed values, with one exception marked
 * "parity unpinned": the modified random walk's absorption by a PAH species
 * (run_packet, MRW branch).  The walk tests for one absorption along its
 * path and then draws the species, so a PAH species terminates fewer walks
 * than the Poisson number of absorptions along the path would; the pin
 * written for it (MRW on and off store the same fraction of packets as PAH
 * absorptions) records that bias as an expected failure.
 */
#define _POSIX_C_SOURCE 199309L   /* clock_gettime for the loop timer */
#include "rt_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* CGS physical constants (exact SI-derived values). */
static const double OR_H = 6.62607015e-27;     /* erg s */
static const double OR_K = 1.380649e-16;       /* erg / K */
static const double OR_C = 2.99792458e10;      /* cm / s */
static const double OR_PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator, from its published definition      */
/* (Salmon, Moraes, Dror & Shaw 2011): ten rounds of two 32x32->64 products, */
/* word permutation and xor with a Weyl-sequence key schedule.               */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Per-packet stream: key = (seed_lo, seed_hi ^ model_id), counter =
 * (block, 0, pid_lo, pid_hi).  Draw d uses block d/2; even draws take the
 * 64-bit word (x1:x0), odd draws (x3:x2); u = ((w >> 11) + 1) 2^-53 in (0,1]. */
typedef struct {
    uint32_t key[2];
    uint64_t pid;
    uint32_t draw;
    uint32_t blk[4];
} or_rng;

static void rng_init(or_rng* r, uint64_t seed, uint32_t model_id, uint64_t pid)
{
    r->key[0] = (uint32_t)seed;
    r->key[1] = (uint32_t)(seed >> 32) ^ model_id;
    r->pid = pid;
    r->draw = 0;
}

static double rng_u(or_rng* r)
{
    uint32_t d = r->draw++;
    if ((d & 1u) == 0) {
        uint32_t ctr[4] = { d >> 1, 0u, (uint32_t)r->pid, (uint32_t)(r->pid >> 32) };
        or_philox4x32_10(ctr, r->key, r->blk);
    }
    uint64_t w = (d & 1u) ? (((uint64_t)r->blk[3] << 32) | r->blk[2])
                          : (((uint64_t)r->blk[1] << 32) | r->blk[0]);
    return (double)((w >> 11) + 1u) * 0x1p-53;
}

void or_uniforms(uint64_t seed, uint32_t model_id, uint64_t pid, uint32_t n, double* out)
{
    or_rng r;
    rng_init(&r, seed, model_id, pid);
    for (uint32_t i = 0; i < n; ++i) out[i] = rng_u(&r);
}

/* ------------------------------------------------------------------------ */
/* Planck function and its temperature derivative                           */
/* ------------------------------------------------------------------------ */
double or_planck_B(double nu, double T)
{
    if (T <= 0.0) return 0.0;
    double x = OR_H * nu / (OR_K * T);
    return 2.0 * OR_H * nu * nu * nu / (OR_C * OR_C) / expm1(x);
}

double or_planck_dBdT(double nu, double T)
{
    /* dB/dT = B * x e^x / ((e^x - 1) T); written as x / (T (e^x-1)(1-e^-x)). */
    if (T <= 0.0) return 0.0;
    double x = OR_H * nu / (OR_K * T);
    double pre = 2.0 * OR_H * nu * nu * nu / (OR_C * OR_C);
    return pre * (x / T) / (expm1(x) * (-expm1(-x)));
}

/* Left-hand side of Eq. 4 for species s: sum_j kabs_j B(nu_j, T) dnu_j. */
double or_planck_mean(const or_model* m, int s, double T)
{
    double acc = 0.0;
    for (int j = 0; j < m->nf; ++j)
        acc += m->kabs[s * m->nf + j] * or_planck_B(m->nu[j], T) * m->dnu[j];
    return acc;
}

/* Eq. 4: the T with 4 pi sum_j kabs B(nu_j,T) dnu_j = target (target =
 * E / (rho V)); bisection to 1e-12 relative.  target <= 0 gives T = 0. */
double or_solve_temperature(const or_model* m, int s, double target)
{
    if (!(target > 0.0)) return 0.0;
    double lo = 0.0, hi = 1.0e5;
    while (4.0 * OR_PI * or_planck_mean(m, s, hi) < target && hi < 1e12) hi *= 2.0;
    while (hi - lo > 1e-12 * hi) {
        double mid = 0.5 * (lo + hi);
        if (4.0 * OR_PI * or_planck_mean(m, s, mid) < target) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* ------------------------------------------------------------------------ */
/* Sources: L_nu on the model grid normalised so sum_j L_nu,j dnu_j = L     */
/* (equal-energy packets, Eq. 1 in expectation).                            */
/* ------------------------------------------------------------------------ */
void or_source_lnu(const or_model* m, const or_source* src, double* lnu)
{
    double tot = 0.0;
    for (int j = 0; j < m->nf; ++j) {
        lnu[j] = src->L_nu ? src->L_nu[j] : or_planck_B(m->nu[j], src->T_eff);
        tot += lnu[j] * m->dnu[j];
    }
    for (int j = 0; j < m->nf; ++j) lnu[j] = tot > 0.0 ? src->L * lnu[j] / tot : 0.0;
}

/* ------------------------------------------------------------------------ */
/* Source frequency grid of Eq. 1                                            */
/* ------------------------------------------------------------------------ */
/* G(x) = int_0^x t^3 / (e^t - 1) dt, the blackbody's cumulative in
 * x = h nu / k T: for x >= 2 the exponential series
 *   G(x) = pi^4 / 15 - sum_k e^{-k x} (x^3/k + 3 x^2/k^2 + 6 x/k^3 + 6/k^4),
 * for x < 2 the power series from t / (e^t - 1) = sum_n B_n t^n / n!,
 *   G(x) = sum_n B_n x^(n+3) / (n! (n + 3))   (converges for x < 2 pi). */
static double bb_cumulative(double x)
{
    if (x <= 0.0) return 0.0;
    if (x >= 2.0) {
        double s = 0.0;
        for (int k = 1; k < 200; ++k) {
            const double e = exp(-k * x);
            const double t = e * (x * x * x / k + 3.0 * x * x / ((double)k * k) +
                                  6.0 * x / ((double)k * k * k) + 6.0 / ((double)k * k * k * k));
            s += t;
            if (t < 1e-18 * s) break;
        }
        return OR_PI * OR_PI * OR_PI * OR_PI / 15.0 - s;
    }
    /* Bernoulli numbers B_0, B_1, B_2, B_4, ..., B_30 (odd ones above 1 vanish) */
    static const double Bn[17] = { 1.0, -0.5, 1.0 / 6.0, -1.0 / 30.0, 1.0 / 42.0, -1.0 / 30.0,
                                   5.0 / 66.0, -691.0 / 2730.0, 7.0 / 6.0, -3617.0 / 510.0,
                                   43867.0 / 798.0, -174611.0 / 330.0, 854513.0 / 138.0,
                                   -236364091.0 / 2730.0, 8553103.0 / 6.0,
                                   -23749461029.0 / 870.0, 8615841276005.0 / 14322.0 };
    double s = x * x * x / 3.0 - 0.5 * x * x * x * x / 4.0;   /* n = 0, 1 */
    double fact = 1.0;                                          /* n! */
    double xp = x * x * x;                                      /* x^(n+3) at n = 0 */
    int nprev = 0;
    for (int i = 2; i < 17; ++i) {
        const int n = 2 * (i - 1);
        for (int q = nprev + 1; q <= n; ++q) { fact *= q; xp *= x; }
        nprev = n;
        s += Bn[i] * xp / (fact * (n + 3));
    }
    return s;
}

/* edges of the model frequency bins: geometric means of neighbouring
 * frequencies, the outer edges mirrored in ln nu */
static void model_edges(const or_model* m, double* e)
{
    for (int j = 1; j < m->nf; ++j) e[j] = sqrt(m->nu[j - 1] * m->nu[j]);
    e[0] = m->nf > 1 ? m->nu[0] * m->nu[0] / e[1] : 0.5 * m->nu[0];
    e[m->nf] = m->nf > 1 ? m->nu[m->nf - 1] * m->nu[m->nf - 1] / e[m->nf - 1] : 2.0 * m->nu[0];
}

/* cumulative luminosity of source s from the lower model edge to nu, in
 * units of its total over the model range (continuous spectrum) */
static double src_cumulative(const or_model* m, const or_source* s, const double* e, double nu)
{
    if (nu <= e[0]) return 0.0;
    if (nu >= e[m->nf]) return 1.0;
    if (s->L_nu) {
        double tot = 0.0, below = 0.0;
        for (int j = 0; j < m->nf; ++j) {
            const double w = s->L_nu[j] * (e[j + 1] - e[j]);
            if (nu >= e[j + 1]) below += w;
            else if (nu > e[j]) below += s->L_nu[j] * (nu - e[j]);
            tot += w;
        }
        return tot > 0.0 ? below / tot : 0.0;
    }
    const double a = OR_H / (OR_K * s->T_eff);
    const double g0 = bb_cumulative(a * e[0]), g1 = bb_cumulative(a * e[m->nf]);
    return (bb_cumulative(a * nu) - g0) / (g1 - g0);
}

int or_source_grid(const or_model* m, const or_source* src, int nsrc, uint32_t mbins,
                   int32_t* nu_idx, int32_t* src_idx, double* nu_star)
{
    if (nsrc < 1 || mbins < 1 || m->nf < 1) return 1;
    double* e = (double*)malloc(sizeof(double) * (m->nf + 1));
    model_edges(m, e);
    double Ltot = 0.0;
    for (int i = 0; i < nsrc; ++i) Ltot += src[i].L;
    for (uint32_t b = 0; b < mbins; ++b) {
        /* the source where the running sum of the L_i first reaches the
         * point, then the frequency within it */
        const double target = ((double)b + 0.5) / (double)mbins * Ltot;
        double below = 0.0;
        int si = 0;
        for (; si < nsrc - 1; ++si) {
            if (below + src[si].L >= target) break;
            below += src[si].L;
        }
        const double f = src[si].L > 0.0 ? (target - below) / src[si].L : 0.5;
        /* bisection in ln nu on the continuous cumulative */
        double lo = log(e[0]), hi = log(e[m->nf]);
        for (int it = 0; it < 200 && hi - lo > 1e-15 * fabs(hi); ++it) {
            const double mid = 0.5 * (lo + hi);
            if (src_cumulative(m, &src[si], e, exp(mid)) < f) lo = mid; else hi = mid;
        }
        const double nus = exp(0.5 * (lo + hi));
        int j = 0;
        while (j < m->nf - 1 && nus >= e[j + 1]) ++j;
        nu_idx[b] = j;
        src_idx[b] = si;
        if (nu_star) nu_star[b] = nus;
    }
    free(e);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Grid helpers                                                              */
/* ------------------------------------------------------------------------ */
static int64_t ncube_of(const or_model* m) { return (int64_t)m->nx * m->ny * m->nz; }
static int64_t ncell_of(const or_model* m) { return m->refine > 0 ? m->nleaf : ncube_of(m); }

/* A cell of the grid: cube i[3]; inside a refined cube (f = 1) also its
 * sub-cube s[3], each index in [0, r). */
typedef struct { int i[3]; int s[3]; int f; } or_pos;

static int64_t cube_lin(const or_model* m, const int i[3])
{
    return ((int64_t)i[2] * m->ny + i[1]) * m->nx + i[0];
}

static int inside(const or_model* m, const or_pos* p)
{
    return p->i[0] >= 0 && p->i[0] < m->nx && p->i[1] >= 0 && p->i[1] < m->ny &&
           p->i[2] >= 0 && p->i[2] < m->nz;
}

static int cube_refined(const or_model* m, const int i[3])
{
    return m->refine > 0 && m->refined[cube_lin(m, i)];
}

/* cell number of p (see or_model) */
static int64_t lin(const or_model* m, const or_pos* p)
{
    int64_t c = cube_lin(m, p->i);
    if (m->refine <= 0) return c;
    int64_t b = m->leaf_base[c];
    if (!p->f) return b;
    int r = m->refine;
    return b + ((int64_t)p->s[2] * r + p->s[1]) * r + p->s[0];
}

/* edge of cell p and its lower corner along axis a */
static double pos_size(const or_model* m, const or_pos* p)
{
    return p->f ? m->cell / m->refine : m->cell;
}

static double pos_lo(const or_model* m, const or_pos* p, int a)
{
    double lo = m->box_min[a] + p->i[a] * m->cell;
    return p->f ? lo + p->s[a] * (m->cell / m->refine) : lo;
}

static double rho_of(const or_model* m, int s, int64_t c)
{
    return (double)m->rho[(int64_t)s * ncell_of(m) + c];
}

/* Sub-cube of refined cube p->i holding x (face rule of locate), clamped to
 * the cube. */
static void descend(const or_model* m, const double x[3], const double k[3], or_pos* p)
{
    int r = m->refine;
    double h = m->cell / r;
    for (int a = 0; a < 3; ++a) {
        double u = (x[a] - (m->box_min[a] + p->i[a] * m->cell)) / h;
        double f = floor(u);
        int sa = (int)f;
        if (f == u && k[a] < 0.0) sa -= 1;
        if (sa < 0) sa = 0;
        if (sa > r - 1) sa = r - 1;
        p->s[a] = sa;
    }
    p->f = 1;
}

/* Cell containing x; a coordinate exactly on a face belongs to the lower cell
 * when the packet moves towards -axis, otherwise to the upper cell. */
static void locate(const or_model* m, const double x[3], const double k[3], or_pos* p)
{
    for (int a = 0; a < 3; ++a) {
        double u = (x[a] - m->box_min[a]) / m->cell;
        double f = floor(u);
        int i = (int)f;
        if (f == u && k[a] < 0.0) i -= 1;
        p->i[a] = i;
        p->s[a] = 0;
    }
    p->f = 0;
    if (inside(m, p) && cube_refined(m, p->i)) descend(m, x, k, p);
}

/* Distance to the exit face of cell p along k; axis of that face returned
 * in *axis (ties go to the lowest axis). */
static double exit_distance(const or_model* m, const double x[3], const double k[3],
                            const or_pos* p, int* axis)
{
    double best = INFINITY, h = pos_size(m, p);
    int ba = 0;
    for (int a = 0; a < 3; ++a) {
        double t, lo = pos_lo(m, p, a);
        if (k[a] > 0.0) t = (lo + h - x[a]) / k[a];
        else if (k[a] < 0.0) t = (lo - x[a]) / k[a];
        else t = INFINITY;
        if (t < 0.0) t = 0.0;
        if (t < best) { best = t; ba = a; }
    }
    *axis = ba;
    return best;
}

/* Move to the face found by exit_distance and step into the neighbour: the
 * next sub-cube of the same cube, else the next cube -- descending into its
 * sub-cube at the entry point when it is refined. */
static void cross_face(const or_model* m, double x[3], const double k[3], or_pos* p,
                       double t, int a)
{
    double lo = pos_lo(m, p, a), h = pos_size(m, p);
    int step = k[a] > 0.0 ? 1 : -1;
    for (int b = 0; b < 3; ++b) x[b] += t * k[b];
    x[a] = step > 0 ? lo + h : lo;
    if (p->f) {
        p->s[a] += step;
        if (p->s[a] >= 0 && p->s[a] < m->refine) return;
        p->f = 0;
    }
    p->i[a] += step;
    for (int b = 0; b < 3; ++b) p->s[b] = 0;
    if (inside(m, p) && cube_refined(m, p->i)) {
        descend(m, x, k, p);
        p->s[a] = step > 0 ? 0 : m->refine - 1;      /* entered through face a */
    }
}

/* Cell p of cell number c. */
static void pos_of(const or_model* m, int64_t c, or_pos* p)
{
    int64_t cube = c;
    p->f = 0;
    p->s[0] = p->s[1] = p->s[2] = 0;
    if (m->refine > 0) {
        /* the last cube whose first cell is <= c */
        int64_t lo = 0, hi = ncube_of(m) - 1;
        while (lo < hi) {
            int64_t mid = (lo + hi + 1) / 2;
            if (m->leaf_base[mid] <= c) lo = mid; else hi = mid - 1;
        }
        cube = lo;
        if (m->refined[cube]) {
            int r = m->refine;
            int64_t off = c - m->leaf_base[cube];
            p->s[0] = (int)(off % r);
            p->s[1] = (int)((off / r) % r);
            p->s[2] = (int)(off / ((int64_t)r * r));
            p->f = 1;
        }
    }
    p->i[0] = (int)(cube % m->nx);
    p->i[1] = (int)((cube / m->nx) % m->ny);
    p->i[2] = (int)(cube / ((int64_t)m->nx * m->ny));
}

/* Edge length of every cell (cube edge, or cube edge / r in refined cubes). */
static void cell_sizes(const or_model* m, double* h)
{
    int64_t nc = ncell_of(m);
    for (int64_t c = 0; c < nc; ++c) {
        or_pos p;
        pos_of(m, c, &p);
        h[c] = pos_size(m, &p);
    }
}

int or_dda_segments(const or_model* m, const double x0[3], const double k[3], int max,
                    int64_t* cells, double* lens)
{
    double x[3] = { x0[0], x0[1], x0[2] };
    or_pos p;
    locate(m, x, k, &p);
    int n = 0;
    while (inside(m, &p) && n < max) {
        int a;
        double t = exit_distance(m, x, k, &p, &a);
        cells[n] = lin(m, &p);
        lens[n] = t;
        ++n;
        cross_face(m, x, k, &p, t, a);
    }
    return n;
}

/* ------------------------------------------------------------------------ */
/* Sampling primitives                                                       */
/* ------------------------------------------------------------------------ */
/* Isotropic direction: phi = 2 pi zeta1, cos(theta) = 1 - 2 zeta2, zeta = 1-u. */
static void iso_dir(double u1, double u2, double k[3])
{
    double phi = 2.0 * OR_PI * (1.0 - u1);
    double mu = 1.0 - 2.0 * (1.0 - u2);
    double st = sqrt(fmax(0.0, 1.0 - mu * mu));
    k[0] = st * cos(phi);
    k[1] = st * sin(phi);
    k[2] = mu;
}

/* Henyey-Greenstein (Eq. 15) inverse CDF for cos(beta), zeta = 1 - u. */
double or_hg_mu(double g, double u)
{
    double z = 1.0 - u;
    double mu;
    if (fabs(g) > 1e-6) {
        double t = (1.0 - g * g) / (1.0 - g + 2.0 * g * z);
        mu = (1.0 + g * g - t * t) / (2.0 * g);
    } else {
        mu = 2.0 * z - 1.0;
    }
    if (mu > 1.0) mu = 1.0;
    if (mu < -1.0) mu = -1.0;
    return mu;
}

/* Turn direction k by polar angle acos(mu) and azimuth phi about itself. */
void or_rotate(double k[3], double mu, double phi)
{
    double st = sqrt(fmax(0.0, 1.0 - mu * mu));
    double cp = cos(phi), sp = sin(phi);
    double n[3];
    if (fabs(k[2]) > 0.99999) {
        n[0] = st * cp;
        n[1] = st * sp;
        n[2] = k[2] > 0.0 ? mu : -mu;
    } else {
        double t = sqrt(1.0 - k[2] * k[2]);
        n[0] = st * (k[0] * k[2] * cp - k[1] * sp) / t + k[0] * mu;
        n[1] = st * (k[1] * k[2] * cp + k[0] * sp) / t + k[1] * mu;
        n[2] = -st * cp * t + k[2] * mu;
    }
    double l = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    k[0] = n[0] / l; k[1] = n[1] / l; k[2] = n[2] / l;
}

/* Modified random walk: survival probability of a diffusing packet started
 * at the centre of an absorbing sphere, y = D t / R0^2 with D = 1/(3 chi) in
 * path-length units: S(y) = 2 sum_n (-1)^(n+1) exp(-n^2 pi^2 y).  For small y
 * the equivalent image-series form 1 - 2/sqrt(pi y) sum_m exp(-(m+1/2)^2/y) is
 * used (Jacobi theta transformation). */
double or_mrw_survival(double y)
{
    if (y <= 0.0) return 1.0;
    if (y < 0.1) {
        double s = 0.0;
        for (int mm = 0; mm < 60; ++mm) {
            double t = exp(-(mm + 0.5) * (mm + 0.5) / y);
            s += t;
            if (t < 1e-300) break;
        }
        return 1.0 - 2.0 / sqrt(OR_PI * y) * s;
    }
    double s = 0.0;
    for (int n = 1; n < 200; ++n) {
        double t = exp(-(double)n * n * OR_PI * OR_PI * y);
        s += (n & 1) ? t : -t;
        if (t < 1e-22) break;
    }
    return 2.0 * s;
}

/* Solve S(y) = u by bisection (S decreases from 1 to 0). */
double or_mrw_sample_y(double u)
{
    if (u >= 1.0) return 0.0;
    double lo = 0.0, hi = fmax(log(2.0 / u) / (OR_PI * OR_PI), 1e-3);
    while (or_mrw_survival(hi) > u) hi *= 2.0;
    for (int it = 0; it < 200 && hi - lo > 1e-15 * hi; ++it) {
        double mid = 0.5 * (lo + hi);
        if (or_mrw_survival(mid) > u) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* Smallest j with C_j >= u C_{n-1} for the running sum C of w. */
static int pick_cdf(const double* w, int n, double u)
{
    double tot = 0.0;
    for (int j = 0; j < n; ++j) tot += w[j];
    double target = u * tot, acc = 0.0;
    for (int j = 0; j < n; ++j) {
        acc += w[j];
        if (acc >= target) return j;
    }
    return n - 1;
}

/* ------------------------------------------------------------------------ */
/* Transport                                                                 */
/* ------------------------------------------------------------------------ */
typedef struct {
    const or_model* m;
    const or_params* p;
    const double* T_prev;
    double xi;
    int nsrc;
    const or_source* src;
    double* src_w;      /* [nsrc][nf] emission weights L_nu dnu */
    double* src_L;      /* [nsrc] */
    unsigned char* lucy;/* [ncell] */
    double* h;          /* [ncell] cell edge */
    const or_pah_src* ps;  /* PAH re-emission pass, or NULL */
    double* eps_w;      /* [n_eps][nf] eps_n(nu_j) dnu_j */
} or_ctx;

static double chi_ext(const or_model* m, int64_t c, int j)
{
    double chi = 0.0;
    for (int s = 0; s < m->ns; ++s)
        chi += rho_of(m, s, c) * (m->kabs[s * m->nf + j] + m->ksca[s * m->nf + j]);
    return chi;
}

static double chi_abs(const or_model* m, int64_t c, int j)
{
    double chi = 0.0;
    for (int s = 0; s < m->ns; ++s) chi += rho_of(m, s, c) * m->kabs[s * m->nf + j];
    return chi;
}

static void log_event(or_out* o, uint64_t pid, uint32_t* seq, uint32_t type, int64_t cell,
                      int nu, const double x[3], const double k[3])
{
    uint32_t q = (*seq)++;
    if (!o->traj || o->traj_cap == 0) return;
    if (o->n_traj >= o->traj_cap) { o->stats[OR_S_TRAJ_DROP]++; return; }
    or_traj* t = &o->traj[o->n_traj++];
    t->pid = pid; t->seq = q; t->type = type; t->cell = (uint32_t)cell; t->nu = (uint32_t)nu;
    for (int a = 0; a < 3; ++a) { t->x[a] = x[a]; t->k[a] = k[a]; }
}

/* Energy deposited along a path of length l in a Lucy cell (Sect. 3.1). */
static void lucy_deposit(const or_ctx* C, or_out* o, int64_t c, int j, double l)
{
    const or_model* m = C->m;
    for (int s = 0; s < m->ns; ++s) {
        double ta = m->kabs[s * m->nf + j] * rho_of(m, s, c) * l;
        double e = (C->p->lucy_form == OR_LUCY_EXPM1) ? -expm1(-ta) * C->xi : ta * C->xi;
        o->E_abs[s * ncell_of(m) + c] += e;
        if (o->esq) o->esq[s * ncell_of(m) + c] += e * e;
    }
    o->stats[OR_S_LUCY]++;
}

/* Re-emission frequency (Eq. 5 frozen temperature, Eq. 10 Bjorkman & Wood). */
static int reemit_bin(const or_ctx* C, const or_out* o, int s, int64_t c, double u)
{
    const or_model* m = C->m;
    double T;
    if (C->p->mode == OR_MODE_BW) {
        double rv = rho_of(m, s, c) * C->h[c] * C->h[c] * C->h[c];
        double E = o->E_abs[s * ncell_of(m) + c];
        T = (rv > 0.0) ? or_solve_temperature(m, s, E / rv) : 0.0;
    } else {
        T = C->T_prev ? C->T_prev[s * ncell_of(m) + c] : 0.0;
    }
    double w[1024];
    double* wp = m->nf <= 1024 ? w : (double*)malloc(sizeof(double) * m->nf);
    for (int l = 0; l < m->nf; ++l) {
        double b = (C->p->mode == OR_MODE_BW) ? or_planck_dBdT(m->nu[l], T)
                                               : or_planck_B(m->nu[l], T);
        wp[l] = m->kabs[s * m->nf + l] * b * m->dnu[l];
    }
    int j = pick_cdf(wp, m->nf, u);
    if (wp != w) free(wp);
    return j;
}

/* Species picked with probability proportional to rho_s kappa_s (abs or sca). */
static int pick_species(const or_model* m, int64_t c, int j, int sca, double u)
{
    double w[64];
    for (int s = 0; s < m->ns; ++s)
        w[s] = rho_of(m, s, c) * (sca ? m->ksca[s * m->nf + j] : m->kabs[s * m->nf + j]);
    return pick_cdf(w, m->ns, u);
}

/* Observer direction k_obs (from the model towards the observer) for
 * (theta, phi); image axes e_x' = (-sin phi, cos phi, 0) and
 * e_y' = (-cos theta cos phi, -cos theta sin phi, sin theta), so that
 * (e_x', e_y', k_obs) is right handed and e_y' follows +z. */
static void obs_frame(double theta, double phi, double kobs[3], double ex[3], double ey[3])
{
    double st = sin(theta), ct = cos(theta), sp = sin(phi), cp = cos(phi);
    kobs[0] = st * cp; kobs[1] = st * sp; kobs[2] = ct;
    ex[0] = -sp; ex[1] = cp; ex[2] = 0.0;
    ey[0] = -ct * cp; ey[1] = -ct * sp; ey[2] = st;
}

/* Photon counting (Sect. 4): an escaping packet whose direction lies in a
 * camera's acceptance cone, k . k_obs >= cos_accept, adds its power xi to the
 * pixel that holds its exit point x projected on the image plane,
 * x' = (x - centre) . e_x', y' = (x - centre) . e_y', pixel
 * (floor(x'/p + npix/2), floor(y'/p + npix/2)); points outside the image
 * are not counted. */
static void pc_count(const or_model* m, const or_params* p, or_out* o, const double x[3],
                     const double k[3], int j, double xi)
{
    if (!p->pc || !o->pc_img) return;
    int nn[3] = { m->nx, m->ny, m->nz };
    double rel[3];
    for (int a = 0; a < 3; ++a) rel[a] = x[a] - (m->box_min[a] + 0.5 * nn[a] * m->cell);
    size_t off = 0;
    for (int c = 0; c < p->n_pc; ++c) {
        const or_pc_camera* cam = &p->pc[c];
        const int n = cam->npix;
        double kobs[3], ex[3], ey[3];
        obs_frame(cam->theta, cam->phi, kobs, ex, ey);
        double pix = cam->pixel;
        if (!(pix > 0.0))
            pix = m->cell * sqrt((double)nn[0] * nn[0] + (double)nn[1] * nn[1] + (double)nn[2] * nn[2]) / n;
        double kd = k[0] * kobs[0] + k[1] * kobs[1] + k[2] * kobs[2];
        if (kd >= cam->cos_accept) {
            double xp = rel[0] * ex[0] + rel[1] * ex[1] + rel[2] * ex[2];
            double yp = rel[0] * ey[0] + rel[1] * ey[1] + rel[2] * ey[2];
            double fx = floor(xp / pix + 0.5 * n), fy = floor(yp / pix + 0.5 * n);
            if (fx >= 0.0 && fx < n && fy >= 0.0 && fy < n)
                o->pc_img[off + ((size_t)j * n + (size_t)fy) * n + (size_t)fx] += xi;
        }
        off += (size_t)m->nf * n * n;
    }
}

/* One packet, from emission to escape (or termination). */
static void run_packet(const or_ctx* C, or_out* o, uint64_t pid)
{
    const or_model* m = C->m;
    const or_params* p = C->p;
    const int64_t nc = ncell_of(m);
    or_rng r;
    rng_init(&r, p->seed, p->model_id, pid);
    uint32_t seq = 0;

    int si = 0, j = 0;
    double k[3], x[3];
    or_pos idx;
    if (C->ps) {
        /* PAH re-emission (Sect. 2.1): the record's cell is the source; the
         * bin follows Eq. 6 with the cell's emissivity class, the position is
         * uniform in the cell (one draw per axis), the direction isotropic */
        const int64_t c = (int64_t)C->ps->rec[pid].cell;
        const int n = C->ps->eps_class ? C->ps->eps_class[c] : 0;
        j = pick_cdf(C->eps_w + (size_t)n * m->nf, m->nf, rng_u(&r));
        pos_of(m, c, &idx);
        const double h = pos_size(m, &idx);
        for (int a = 0; a < 3; ++a) x[a] = pos_lo(m, &idx, a) + rng_u(&r) * h;
        { double u1 = rng_u(&r), u2 = rng_u(&r); iso_dir(u1, u2, k); }
    } else {
        /* emission (Sect. 2): source, frequency bin, isotropic direction */
        if (p->source_bins == 0) {
            if (C->nsrc > 1) si = pick_cdf(C->src_L, C->nsrc, rng_u(&r));
            j = pick_cdf(C->src_w + (size_t)si * m->nf, m->nf, rng_u(&r));
        } else {
            /* Eq. 1: the sources' combined luminosity is cut into m bins of
             * equal energy L/m, and N/m packets are emitted in each: packet
             * pid belongs to bin b = floor(pid m / N) and takes the point
             * u = (b + 1/2) / m of the cumulative luminosity -- the source
             * where the running sum of the L_i first reaches u L, then, by
             * the fraction of that source's luminosity below the point, its
             * frequency bin. */
            const uint64_t b = (pid * (uint64_t)p->source_bins) / p->n_packets;
            const double u = ((double)b + 0.5) / (double)p->source_bins;
            if (p->sg_nu) {
                /* the separate source grid of Eq. 1 (or_source_grid) */
                si = p->sg_src[b];
                j = p->sg_nu[b];
                goto emitted;
            }
            double tot = 0.0;
            for (int i = 0; i < C->nsrc; ++i) tot += C->src_L[i];
            const double target = u * tot;
            double below = 0.0, upto = 0.0;
            for (si = 0; si < C->nsrc; ++si) {
                upto = below + C->src_L[si];
                if (upto >= target || si == C->nsrc - 1) break;
                below = upto;
            }
            const double uf = (target - below) / (upto - below);
            j = pick_cdf(C->src_w + (size_t)si * m->nf, m->nf, uf);
        }
    emitted:
        { double u1 = rng_u(&r), u2 = rng_u(&r); iso_dir(u1, u2, k); }
        for (int a = 0; a < 3; ++a) x[a] = C->src[si].pos[a];
        locate(m, x, k, &idx);
    }
    o->stats[OR_S_EMIT]++;
    log_event(o, pid, &seq, OR_T_EMIT, inside(m, &idx) ? lin(m, &idx) : 0, j, x, k);
    uint64_t n_ev = 0;
    int64_t last_cell = inside(m, &idx) ? lin(m, &idx) : 0;

    for (;;) {
        if (!inside(m, &idx)) {
            /* escape: tally in 10 bins equal in cos(theta) */
            int b = (int)floor((k[2] + 1.0) * 5.0);
            if (b < 0) b = 0;
            if (b > 9) b = 9;
            o->sed_esc[b * m->nf + j] += C->xi;
            o->sed_cnt[b * m->nf + j] += 1;
            pc_count(m, p, o, x, k, j, C->xi);
            o->stats[OR_S_ESCAPE]++;
            log_event(o, pid, &seq, OR_T_ESCAPE, last_cell, j, x, k);
            return;
        }
        int64_t c = lin(m, &idx);
        last_cell = c;

        /* modified random walk in very thick cells (Sect. 3.2); the sphere
         * stays inside the current cell (sub-cube in refined cubes) */
        if (p->mrw && p->mode != OR_MODE_NOREEMIT) {
            double chi = chi_ext(m, c, j);
            double R0 = INFINITY, h = pos_size(m, &idx);
            for (int a = 0; a < 3; ++a) {
                double lo = pos_lo(m, &idx, a);
                double d1 = x[a] - lo, d2 = lo + h - x[a];
                if (d1 < R0) R0 = d1;
                if (d2 < R0) R0 = d2;
            }
            if (R0 < 0.0) R0 = 0.0;
            if (chi * h > p->mrw_tau_cell && R0 * chi >= p->mrw_gamma) {
                if (++n_ev > p->max_events) {
                    o->stats[OR_S_STUCK]++;
                    log_event(o, pid, &seq, OR_T_STUCK, c, j, x, k);
                    return;
                }
                double y = or_mrw_sample_y(rng_u(&r));
                double l = 3.0 * chi * R0 * R0 * y;
                double nh[3];
                { double u1 = rng_u(&r), u2 = rng_u(&r); iso_dir(u1, u2, nh); }
                for (int a = 0; a < 3; ++a) x[a] += R0 * nh[a];
                { double u3 = rng_u(&r), u4 = rng_u(&r); iso_dir(u3, u4, k); }
                for (int s = 0; s < m->ns; ++s) {
                    double e = C->xi * m->kabs[s * m->nf + j] * rho_of(m, s, c) * l;
                    o->E_abs[s * nc + c] += e;
                    if (o->esq) o->esq[s * nc + c] += e * e;
                }
                o->stats[OR_S_MRW]++;
                double ca = chi_abs(m, c, j);
                if (rng_u(&r) < -expm1(-ca * l)) {
                    int s = 0;
                    if (m->ns > 1) s = pick_species(m, c, j, 0, rng_u(&r));
                    if (m->is_pah && m->is_pah[s]) {
                        if (o->pah && o->n_pah < o->pah_cap) {
                            o->pah[o->n_pah].cell = (uint32_t)c;
                            o->pah[o->n_pah].nu = (uint32_t)j;
                            o->n_pah++;
                        } else {
                            o->stats[OR_S_PAH_DROP]++;
                        }
                        o->stats[OR_S_PAH]++;
                        log_event(o, pid, &seq, OR_T_PAH, c, j, x, k);
                        return;
                    }
                    j = reemit_bin(C, o, s, c, rng_u(&r));
                }
                log_event(o, pid, &seq, OR_T_MRW, c, j, x, k);
                continue;
            }
        }

        /* one flight: tau = -ln(u), march cells (Eq. 2) until tau is used up */
        double tau = -log(rng_u(&r));
        int interact = 0;
        while (inside(m, &idx)) {
            c = lin(m, &idx);
            last_cell = c;
            int a;
            double t = exit_distance(m, x, k, &idx, &a);
            double chi = chi_ext(m, c, j);
            double dtau = chi * t;
            if (dtau <= tau) {
                if (C->lucy[c]) lucy_deposit(C, o, c, j, t);
                tau -= dtau;
                cross_face(m, x, k, &idx, t, a);
                o->stats[OR_S_CROSS]++;
            } else {
                double d = tau / chi;          /* Eq. 3 */
                if (C->lucy[c]) lucy_deposit(C, o, c, j, d);
                for (int b = 0; b < 3; ++b) x[b] += d * k[b];
                interact = 1;
                break;
            }
        }
        if (!interact) continue;                /* left the grid: escape next */

        c = lin(m, &idx);
        if (++n_ev > p->max_events) {
            o->stats[OR_S_STUCK]++;
            log_event(o, pid, &seq, OR_T_STUCK, c, j, x, k);
            return;
        }
        o->stats[OR_S_INTERACT]++;
        double ce = chi_ext(m, c, j);
        double cs = 0.0;
        for (int s = 0; s < m->ns; ++s) cs += rho_of(m, s, c) * m->ksca[s * m->nf + j];
        double albedo = cs / ce;
        if (rng_u(&r) < albedo) {
            /* scattering: keep frequency, new direction from HG (Eq. 15) */
            int s = 0;
            if (m->ns > 1) s = pick_species(m, c, j, 1, rng_u(&r));
            double gg = m->g[s * m->nf + j];
            double mu = or_hg_mu(gg, rng_u(&r));
            double phi = 2.0 * OR_PI * (1.0 - rng_u(&r));
            if (p->record_events) {
                if (o->events && o->n_events < o->event_cap) {
                    or_event* e = &o->events[o->n_events++];
                    e->cell = (uint32_t)c; e->nu = (uint32_t)j; e->species = (uint32_t)s; e->pad = 0;
                    e->k[0] = k[0]; e->k[1] = k[1]; e->k[2] = k[2];
                } else {
                    o->stats[OR_S_EV_DROP]++;
                }
            }
            or_rotate(k, mu, phi);
            o->stats[OR_S_SCATTER]++;
            log_event(o, pid, &seq, OR_T_SCATTER, c, j, x, k);
            continue;
        }
        /* absorption (Sect. 2): species, energy tally, re-emission */
        o->stats[OR_S_ABSORB]++;
        int s = 0;
        if (m->ns > 1) s = pick_species(m, c, j, 0, rng_u(&r));
        if (m->is_pah && m->is_pah[s]) {
            if (o->pah && o->n_pah < o->pah_cap) {
                o->pah[o->n_pah].cell = (uint32_t)c;
                o->pah[o->n_pah].nu = (uint32_t)j;
                o->n_pah++;
            } else {
                o->stats[OR_S_PAH_DROP]++;
            }
            o->stats[OR_S_PAH]++;
            log_event(o, pid, &seq, OR_T_PAH, c, j, x, k);
            return;
        }
        if (!C->lucy[c]) {
            o->E_abs[s * nc + c] += C->xi;
            if (o->esq) o->esq[s * nc + c] += C->xi * C->xi;
        }
        o->count[s * nc + c] += 1;
        if (p->mode == OR_MODE_NOREEMIT) {
            log_event(o, pid, &seq, OR_T_ABSORB_END, c, j, x, k);
            return;
        }
        j = reemit_bin(C, o, s, c, rng_u(&r));
        { double u1 = rng_u(&r), u2 = rng_u(&r); iso_dir(u1, u2, k); }
        log_event(o, pid, &seq, OR_T_ABSORB, c, j, x, k);
    }
}

static void zero_out_counts(or_out* o)
{
    o->n_events = 0; o->n_pah = 0; o->n_traj = 0;
    memset(o->stats, 0, sizeof(o->stats));
}

static int transport_impl(const or_model* m, const or_source* src, int nsrc,
                          const or_pah_src* ps, const or_params* p, const double* T_prev,
                          or_out* out, int n_threads)
{
    if (m->nf < 1 || m->ns < 1 || m->ns > 64 || p->n_packets == 0) return 1;
    if (p->pid_end < p->pid_begin || p->pid_end > p->n_packets) return 1;
    if (p->sg_nu && p->source_bins > 0) {
        if (!p->sg_src) return 1;
        for (uint32_t b = 0; b < p->source_bins; ++b)
            if (p->sg_nu[b] < 0 || p->sg_nu[b] >= m->nf || p->sg_src[b] < 0 || p->sg_src[b] >= nsrc) return 1;
    }
    if (p->n_pc < 0 || (p->n_pc > 0 && !p->pc)) return 1;
    for (int c = 0; c < p->n_pc; ++c)
        if (p->pc[c].npix < 1) return 1;
    or_ctx C;
    C.m = m; C.p = p; C.T_prev = T_prev; C.nsrc = nsrc; C.src = src;
    C.h = (double*)malloc(sizeof(double) * ncell_of(m));
    cell_sizes(m, C.h);
    C.ps = ps;
    C.eps_w = NULL;
    C.src_w = (double*)malloc(sizeof(double) * (nsrc > 0 ? nsrc : 1) * m->nf);
    C.src_L = (double*)malloc(sizeof(double) * (nsrc > 0 ? nsrc : 1));
    double Ltot = 0.0;
    for (int i = 0; i < nsrc; ++i) {
        or_source_lnu(m, &src[i], C.src_w + (size_t)i * m->nf);
        for (int j = 0; j < m->nf; ++j) C.src_w[(size_t)i * m->nf + j] *= m->dnu[j];
        C.src_L[i] = src[i].L;
        Ltot += src[i].L;
    }
    C.xi = Ltot / (double)p->n_packets;
    if (ps) {
        /* Eq. 6 on the model's frequency bins: weights eps_n(nu_j) dnu_j */
        C.eps_w = (double*)malloc(sizeof(double) * (size_t)ps->n_eps * m->nf);
        for (int n = 0; n < ps->n_eps; ++n)
            for (int j = 0; j < m->nf; ++j)
                C.eps_w[(size_t)n * m->nf + j] = ps->eps[(size_t)n * m->nf + j] * m->dnu[j];
        C.xi = ps->xi;
    }
    int64_t nc = ncell_of(m);
    C.lucy = (unsigned char*)calloc((size_t)nc, 1);
    for (int64_t c = 0; c < nc; ++c) {
        /* a Lucy cell holds dust; THIN: its largest face-to-face optical depth
         * over the frequency grid is below lucy_tau (Sect. 3.1) */
        double dust = 0.0;
        for (int s = 0; s < m->ns; ++s) dust += rho_of(m, s, c);
        if (!(dust > 0.0)) continue;
        if (p->lucy_mode == OR_LUCY_ALL) { C.lucy[c] = 1; continue; }
        if (p->lucy_mode != OR_LUCY_THIN) continue;
        double mx = 0.0;
        for (int j = 0; j < m->nf; ++j) {
            double t = chi_ext(m, c, j) * C.h[c];
            if (t > mx) mx = t;
        }
        C.lucy[c] = mx < p->lucy_tau;
    }

    size_t n_pc_px = 0;
    if (p->pc && out->pc_img)
        for (int c = 0; c < p->n_pc; ++c)
            n_pc_px += (size_t)m->nf * p->pc[c].npix * p->pc[c].npix;
    int nt = n_threads < 1 ? 1 : n_threads;
    if (p->mode == OR_MODE_BW) nt = 1;      /* order-dependent: serial by definition */
    struct timespec t_loop0, t_loop1;
    clock_gettime(CLOCK_MONOTONIC, &t_loop0);
    uint64_t np = p->pid_end - p->pid_begin;
    if ((uint64_t)nt > np) nt = np > 0 ? (int)np : 1;
    if (nt == 1) {
        for (uint64_t pid = p->pid_begin; pid < p->pid_end; ++pid) run_packet(&C, out, pid);
    } else {
        /* contiguous pid chunks, merged in chunk order (same event order as serial) */
        or_out* parts = (or_out*)calloc((size_t)nt, sizeof(or_out));
        for (int t = 0; t < nt; ++t) {
            parts[t].E_abs = (double*)calloc((size_t)(m->ns * nc), sizeof(double));
            parts[t].count = (uint32_t*)calloc((size_t)(m->ns * nc), sizeof(uint32_t));
            parts[t].esq = out->esq ? (double*)calloc((size_t)(m->ns * nc), sizeof(double)) : NULL;
            parts[t].sed_esc = (double*)calloc((size_t)(10 * m->nf), sizeof(double));
            parts[t].sed_cnt = (uint64_t*)calloc((size_t)(10 * m->nf), sizeof(uint64_t));
            parts[t].pc_img = n_pc_px ? (double*)calloc(n_pc_px, sizeof(double)) : NULL;
            parts[t].event_cap = out->events ? out->event_cap : 0;
            parts[t].events = parts[t].event_cap ? (or_event*)malloc(sizeof(or_event) * parts[t].event_cap) : NULL;
            parts[t].pah_cap = out->pah ? out->pah_cap : 0;
            parts[t].pah = parts[t].pah_cap ? (or_pah*)malloc(sizeof(or_pah) * parts[t].pah_cap) : NULL;
            parts[t].traj_cap = out->traj ? out->traj_cap : 0;
            parts[t].traj = parts[t].traj_cap ? (or_traj*)malloc(sizeof(or_traj) * parts[t].traj_cap) : NULL;
            zero_out_counts(&parts[t]);
        }
#ifdef _OPENMP
#pragma omp parallel for schedule(static, 1) num_threads(nt)
#endif
        for (int t = 0; t < nt; ++t) {
            uint64_t b = p->pid_begin + np * (uint64_t)t / (uint64_t)nt;
            uint64_t e = p->pid_begin + np * (uint64_t)(t + 1) / (uint64_t)nt;
            for (uint64_t pid = b; pid < e; ++pid) run_packet(&C, &parts[t], pid);
        }
        for (int t = 0; t < nt; ++t) {
            or_out* q = &parts[t];
            for (int64_t i = 0; i < m->ns * nc; ++i) {
                out->E_abs[i] += q->E_abs[i];
                out->count[i] += q->count[i];
                if (out->esq) out->esq[i] += q->esq[i];
            }
            for (int i = 0; i < 10 * m->nf; ++i) {
                out->sed_esc[i] += q->sed_esc[i];
                out->sed_cnt[i] += q->sed_cnt[i];
            }
            for (size_t i = 0; i < n_pc_px; ++i) out->pc_img[i] += q->pc_img[i];
            for (uint64_t i = 0; i < q->n_events; ++i) {
                if (out->n_events < out->event_cap) out->events[out->n_events++] = q->events[i];
                else out->stats[OR_S_EV_DROP]++;
            }
            for (uint64_t i = 0; i < q->n_pah; ++i) {
                if (out->n_pah < out->pah_cap) out->pah[out->n_pah++] = q->pah[i];
                else out->stats[OR_S_PAH_DROP]++;
            }
            for (uint64_t i = 0; i < q->n_traj; ++i) {
                if (out->n_traj < out->traj_cap) out->traj[out->n_traj++] = q->traj[i];
                else out->stats[OR_S_TRAJ_DROP]++;
            }
            for (int i = 0; i < OR_S_N; ++i) out->stats[i] += q->stats[i];
            free(q->E_abs); free(q->count); free(q->esq); free(q->sed_esc); free(q->sed_cnt);
            free(q->events); free(q->pah); free(q->traj); free(q->pc_img);
        }
        free(parts);
    }
    clock_gettime(CLOCK_MONOTONIC, &t_loop1);
    out->loop_seconds += (double)(t_loop1.tv_sec - t_loop0.tv_sec) + 1e-9 * (double)(t_loop1.tv_nsec - t_loop0.tv_nsec);
    free(C.src_w); free(C.src_L); free(C.lucy); free(C.eps_w); free(C.h);
    return 0;
}

int or_transport(const or_model* m, const or_source* src, int nsrc, const or_params* p,
                 const double* T_prev, or_out* out, int n_threads)
{
    if (nsrc < 1) return 1;
    return transport_impl(m, src, nsrc, NULL, p, T_prev, out, n_threads);
}

int or_pah_reemit(const or_model* m, const or_pah_src* ps, const or_params* p,
                  const double* T_prev, or_out* out, int n_threads)
{
    if (!ps || !ps->rec || !ps->eps || ps->n_eps < 1 || ps->n_rec != p->n_packets) return 1;
    if (p->source_bins != 0 || !(ps->xi > 0.0)) return 1;
    const int64_t nc = ncell_of(m);
    for (uint64_t i = 0; i < ps->n_rec; ++i)
        if ((int64_t)ps->rec[i].cell >= nc) return 1;
    if (ps->eps_class)
        for (int64_t c = 0; c < nc; ++c)
            if (ps->eps_class[c] < 0 || ps->eps_class[c] >= ps->n_eps) return 1;
    for (int n = 0; n < ps->n_eps; ++n) {
        double tot = 0.0;
        for (int j = 0; j < m->nf; ++j) {
            if (!(ps->eps[(size_t)n * m->nf + j] >= 0.0)) return 1;
            tot += ps->eps[(size_t)n * m->nf + j];
        }
        if (!(tot > 0.0)) return 1;
    }
    return transport_impl(m, NULL, 0, ps, p, T_prev, out, n_threads);
}

/* ------------------------------------------------------------------------ */
/* Temperatures (Eq. 4) per species and cell                                */
/* ------------------------------------------------------------------------ */
void or_temperatures(const or_model* m, const double* E_abs, double* T)
{
    int64_t nc = ncell_of(m);
    double* h = (double*)malloc(sizeof(double) * nc);
    cell_sizes(m, h);
    for (int s = 0; s < m->ns; ++s)
        for (int64_t c = 0; c < nc; ++c) {
            double rv = rho_of(m, s, c) * h[c] * h[c] * h[c];
            double E = E_abs[s * nc + c];
            T[s * nc + c] = (rv > 0.0 && E > 0.0) ? or_solve_temperature(m, s, E / rv) : 0.0;
        }
    free(h);
}

/* Initial guess of the iterative scheme: optically thin gray dust around
 * the sources, T^4 = sum L / (16 pi sigma r^2), capped at 2000 K; cells at the
 * source position take the cap. */
void or_temperature_guess(const or_model* m, const or_source* src, int nsrc, double* T)
{
    const double sigma = 2.0 * pow(OR_PI, 5) * pow(OR_K, 4) / (15.0 * pow(OR_H, 3) * OR_C * OR_C);
    int64_t nc = ncell_of(m);
    for (int64_t c = 0; c < nc; ++c) {
        or_pos p;
        pos_of(m, c, &p);
        double h = pos_size(m, &p), ctr[3];
        for (int a = 0; a < 3; ++a) ctr[a] = pos_lo(m, &p, a) + 0.5 * h;
        double q = 0.0;
        for (int i = 0; i < nsrc; ++i) {
            double dx = ctr[0] - src[i].pos[0], dy = ctr[1] - src[i].pos[1], dz = ctr[2] - src[i].pos[2];
            double r2 = dx * dx + dy * dy + dz * dz;
            q += r2 > 0.0 ? src[i].L / (16.0 * OR_PI * sigma * r2) : INFINITY;
        }
        double t = pow(q, 0.25);
        if (!(t < 2000.0)) t = 2000.0;
        for (int s = 0; s < m->ns; ++s) T[s * nc + c] = t;
    }
}

/* ------------------------------------------------------------------------ */
/* Ray tracer (Sect. 4)                                                      */
/* ------------------------------------------------------------------------ */
/* camera frame of a ray-tracing camera (obs_frame) */
static void camera_frame(const or_camera* cam, double kobs[3], double ex[3], double ey[3])
{
    obs_frame(cam->theta, cam->phi, kobs, ex, ey);
}

static double pixel_size(const or_model* m, const or_camera* cam)
{
    if (cam->pixel > 0.0) return cam->pixel;
    double d = m->cell * sqrt((double)m->nx * m->nx + (double)m->ny * m->ny + (double)m->nz * m->nz);
    return d / cam->npix;
}

static double hg_phase(double g, double cb)
{
    double d = 1.0 + g * g - 2.0 * g * cb;
    return (1.0 - g * g) / (4.0 * OR_PI * d * sqrt(d));
}

/* (1 - exp(-x)) / x and its derivative, stable near x = 0 */
static double phi_f(double x)
{
    if (x < 1e-8) return 1.0 - 0.5 * x;
    return -expm1(-x) / x;
}
static double dphi_f(double x)
{
    if (x < 1e-3) return -0.5 + x / 3.0 - x * x / 8.0 + x * x * x / 30.0;
    return (exp(-x) * (1.0 + x) - 1.0) / (x * x);
}

/* Entry point of the line o + s k (s in R) into the box and its path length.
 * Returns 0 when the line misses the box. */
static int box_span(const or_model* m, const double o[3], const double k[3], double* s_lo,
                    double* s_hi)
{
    double lo = -INFINITY, hi = INFINITY;
    int n[3] = { m->nx, m->ny, m->nz };
    for (int a = 0; a < 3; ++a) {
        double bmin = m->box_min[a], bmax = m->box_min[a] + n[a] * m->cell;
        if (k[a] != 0.0) {
            double s1 = (bmin - o[a]) / k[a], s2 = (bmax - o[a]) / k[a];
            if (s1 > s2) { double t = s1; s1 = s2; s2 = t; }
            if (s1 > lo) lo = s1;
            if (s2 < hi) hi = s2;
        } else if (o[a] < bmin || o[a] > bmax) {
            return 0;
        }
    }
    if (!(lo < hi)) return 0;
    *s_lo = lo; *s_hi = hi;
    return 1;
}

/* Ray path through the grid from the box face nearest the observer, moving
 * along d = -k_obs.  Cells and chord lengths are written front to back. */
static int ray_path(const or_model* m, const double o[3], const double kobs[3], int max,
                    int64_t* cells, double* lens)
{
    double s_lo, s_hi;
    if (!box_span(m, o, kobs, &s_lo, &s_hi)) return 0;
    double d[3] = { -kobs[0], -kobs[1], -kobs[2] };
    double x[3];
    for (int a = 0; a < 3; ++a) x[a] = o[a] + s_hi * kobs[a];
    or_pos p;
    locate(m, x, d, &p);
    int nn[3] = { m->nx, m->ny, m->nz };
    for (int a = 0; a < 3; ++a) {              /* entry point on the box: clamp */
        if (p.i[a] < 0) p.i[a] = 0;
        if (p.i[a] >= nn[a]) p.i[a] = nn[a] - 1;
        p.s[a] = 0;
    }
    p.f = 0;
    if (cube_refined(m, p.i)) descend(m, x, d, &p);
    int n = 0;
    while (inside(m, &p) && n < max) {
        int a;
        double t = exit_distance(m, x, d, &p, &a);
        cells[n] = lin(m, &p);
        lens[n] = t;
        ++n;
        cross_face(m, x, d, &p, t, a);
    }
    return n;
}

/* Source functions of Eqs. 14 and 16 as volume emissivities:
 * eta_th[c][f] = sum_s rho_s kabs_s B(nu_f, T_s), and per camera
 * eta_sca[c][f] = xi_ev / (V dnu_f) sum_events P_HG(k_in . k_obs; g_s). */
static void emissivities(const or_model* m, const double* T, const or_event* ev, uint64_t nev,
                         double xi_ev, const or_camera* cam, const int* fidx, int nfi,
                         double* eta)
{
    int64_t nc = ncell_of(m);
    double* h = (double*)malloc(sizeof(double) * nc);
    cell_sizes(m, h);
    for (int64_t c = 0; c < nc; ++c)
        for (int f = 0; f < nfi; ++f) {
            int j = fidx[f];
            double e = 0.0;
            for (int s = 0; s < m->ns; ++s)
                e += rho_of(m, s, c) * m->kabs[s * m->nf + j] * or_planck_B(m->nu[j], T[s * nc + c]);
            eta[c * nfi + f] = e;
        }
    double kobs[3], ex[3], ey[3];
    camera_frame(cam, kobs, ex, ey);
    for (uint64_t i = 0; i < nev; ++i) {
        const or_event* e = &ev[i];
        for (int f = 0; f < nfi; ++f) {
            if ((int)e->nu != fidx[f]) continue;
            double cb = e->k[0] * kobs[0] + e->k[1] * kobs[1] + e->k[2] * kobs[2];
            double gg = m->g[e->species * m->nf + e->nu];
            double vol = h[e->cell] * h[e->cell] * h[e->cell];
            eta[(int64_t)e->cell * nfi + f] += xi_ev / (vol * m->dnu[e->nu]) * hg_phase(gg, cb);
        }
    }
    free(h);
}

static void pixel_origin(const or_model* m, const or_camera* cam, int ix, int iy, double o[3],
                         double* apix)
{
    double kobs[3], ex[3], ey[3];
    camera_frame(cam, kobs, ex, ey);
    double p = pixel_size(m, cam);
    double xp = (ix + 0.5 - 0.5 * cam->npix) * p;
    double yp = (iy + 0.5 - 0.5 * cam->npix) * p;
    int nn[3] = { m->nx, m->ny, m->nz };
    for (int a = 0; a < 3; ++a) {
        double ctr = m->box_min[a] + 0.5 * nn[a] * m->cell;
        o[a] = ctr + xp * ex[a] + yp * ey[a];
    }
    *apix = p * p;
}

void or_raytrace(const or_model* m, const double* T, const or_event* ev, uint64_t nev,
                 double xi_ev, const or_source* src, int nsrc, const or_camera* cams, int ncam,
                 const int* fidx, int nfi, double* images, double* sed)
{
    int64_t nc = ncell_of(m);
    int maxp = (m->nx + m->ny + m->nz) * (m->refine > 0 ? m->refine : 1) + 8;
    int64_t* cells = (int64_t*)malloc(sizeof(int64_t) * maxp);
    double* lens = (double*)malloc(sizeof(double) * maxp);
    double* eta = (double*)malloc(sizeof(double) * nc * nfi);
    double* lnu = (double*)malloc(sizeof(double) * m->nf);
    for (int ci = 0; ci < ncam; ++ci) {
        const or_camera* cam = &cams[ci];
        double kobs[3], ex[3], ey[3];
        camera_frame(cam, kobs, ex, ey);
        emissivities(m, T, ev, nev, xi_ev, cam, fidx, nfi, eta);
        int np = cam->npix;
        for (int f = 0; f < nfi; ++f) sed[ci * nfi + f] = 0.0;
        for (int iy = 0; iy < np; ++iy)
            for (int ix = 0; ix < np; ++ix) {
                double o[3], apix;
                pixel_origin(m, cam, ix, iy, o, &apix);
                int n = ray_path(m, o, kobs, maxp, cells, lens);
                for (int f = 0; f < nfi; ++f) {
                    int j = fidx[f];
                    double I = 0.0, tau = 0.0;
                    for (int q = 0; q < n; ++q) {
                        double chi = chi_ext(m, cells[q], j);
                        double dt = chi * lens[q];
                        /* S (1 - e^-dtau) e^-tau with S = eta / chi (Eqs. 12-14) */
                        I += eta[cells[q] * nfi + f] * lens[q] * phi_f(dt) * exp(-tau);
                        tau += dt;
                    }
                    images[(((int64_t)ci * nfi + f) * np + iy) * np + ix] = I;
                    sed[ci * nfi + f] += I * apix / (cam->D * cam->D);   /* Eq. 17 */
                }
            }
        /* direct light of each source attenuated along k_obs */
        for (int i = 0; i < nsrc; ++i) {
            or_source_lnu(m, &src[i], lnu);
            int n = or_dda_segments(m, src[i].pos, kobs, maxp, cells, lens);
            for (int f = 0; f < nfi; ++f) {
                int j = fidx[f];
                double tau = 0.0;
                for (int q = 0; q < n; ++q) tau += chi_ext(m, cells[q], j) * lens[q];
                sed[ci * nfi + f] += lnu[j] * exp(-tau) / (4.0 * OR_PI * cam->D * cam->D);
            }
        }
    }
    free(cells); free(lens); free(eta); free(lnu);
}

/* Adjoint of or_raytrace with T and the scattering events held fixed:
 * dL/drho_s for every cell and dL/dscale = sum rho dL/drho.  For a ray with
 * contributions c_q = eta_q l_q phi(dtau_q) exp(-tau_<q):
 *   dI/drho_s(q) = [kabs_s B_s l phi + eta l^2 kext_s phi'] exp(-tau_<q)
 *                  - kext_s l_q sum_{p>q} c_p                              */
void or_raytrace_backward(const or_model* m, const double* T, const or_event* ev, uint64_t nev,
                          double xi_ev, const or_source* src, int nsrc, const or_camera* cams,
                          int ncam, const int* fidx, int nfi, const double* dL_dimg,
                          const double* dL_dsed, double* dL_drho, double* dL_dscale)
{
    int64_t nc = ncell_of(m);
    int maxp = (m->nx + m->ny + m->nz) * (m->refine > 0 ? m->refine : 1) + 8;
    int64_t* cells = (int64_t*)malloc(sizeof(int64_t) * maxp);
    double* lens = (double*)malloc(sizeof(double) * maxp);
    double* contrib = (double*)malloc(sizeof(double) * maxp);
    double* att = (double*)malloc(sizeof(double) * maxp);
    double* eta = (double*)malloc(sizeof(double) * nc * nfi);
    double* lnu = (double*)malloc(sizeof(double) * m->nf);
    for (int ci = 0; ci < ncam; ++ci) {
        const or_camera* cam = &cams[ci];
        double kobs[3], ex[3], ey[3];
        camera_frame(cam, kobs, ex, ey);
        emissivities(m, T, ev, nev, xi_ev, cam, fidx, nfi, eta);
        int np = cam->npix;
        for (int iy = 0; iy < np; ++iy)
            for (int ix = 0; ix < np; ++ix) {
                double o[3], apix;
                pixel_origin(m, cam, ix, iy, o, &apix);
                int n = ray_path(m, o, kobs, maxp, cells, lens);
                for (int f = 0; f < nfi; ++f) {
                    int j = fidx[f];
                    double w = dL_dimg[(((int64_t)ci * nfi + f) * np + iy) * np + ix]
                             + dL_dsed[ci * nfi + f] * apix / (cam->D * cam->D);
                    if (w == 0.0) continue;
                    double tau = 0.0;
                    for (int q = 0; q < n; ++q) {
                        double chi = chi_ext(m, cells[q], j);
                        double dt = chi * lens[q];
                        att[q] = exp(-tau);
                        contrib[q] = eta[cells[q] * nfi + f] * lens[q] * phi_f(dt) * att[q];
                        tau += dt;
                    }
                    double behind = 0.0;   /* sum of contributions farther from the observer */
                    for (int q = n - 1; q >= 0; --q) {
                        int64_t c = cells[q];
                        double l = lens[q];
                        double chi = chi_ext(m, c, j);
                        double dt = chi * l;
                        double e = eta[c * nfi + f];
                        for (int s = 0; s < m->ns; ++s) {
                            double kext = m->kabs[s * m->nf + j] + m->ksca[s * m->nf + j];
                            double deta = m->kabs[s * m->nf + j] * or_planck_B(m->nu[j], T[s * nc + c]);
                            double g = (deta * l * phi_f(dt) + e * l * l * kext * dphi_f(dt)) * att[q]
                                     - kext * l * behind;
                            dL_drho[s * nc + c] += w * g;
                        }
                        behind += contrib[q];
                    }
                }
            }
        for (int i = 0; i < nsrc; ++i) {
            or_source_lnu(m, &src[i], lnu);
            int n = or_dda_segments(m, src[i].pos, kobs, maxp, cells, lens);
            for (int f = 0; f < nfi; ++f) {
                int j = fidx[f];
                double w = dL_dsed[ci * nfi + f];
                if (w == 0.0) continue;
                double tau = 0.0;
                for (int q = 0; q < n; ++q) tau += chi_ext(m, cells[q], j) * lens[q];
                double F = lnu[j] * exp(-tau) / (4.0 * OR_PI * cam->D * cam->D);
                for (int q = 0; q < n; ++q)
                    for (int s = 0; s < m->ns; ++s) {
                        double kext = m->kabs[s * m->nf + j] + m->ksca[s * m->nf + j];
                        dL_drho[s * nc + cells[q]] += -w * F * kext * lens[q];
                    }
            }
        }
    }
    double acc = 0.0;
    for (int s = 0; s < m->ns; ++s)
        for (int64_t c = 0; c < nc; ++c) acc += rho_of(m, s, c) * dL_drho[s * nc + c];
    *dL_dscale = acc;
    free(cells); free(lens); free(contrib); free(att); free(eta); free(lnu);
}
