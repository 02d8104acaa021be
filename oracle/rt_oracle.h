/*
 * FP64 CPU oracle for Monte Carlo dust radiative transfer
 * (Heymann & Siebenmorgen 2012, arXiv:1203.2941).
 *
 * TEST INFRASTRUCTURE ONLY.  This plain, slow, all-double-precision
 * implementation exists to check the CUDA library.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It shares
 * no code, header, table or constant with the CUDA library.
 */
#ifndef RT_ORACLE_H
#define RT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* The grid (Sect. 2): nx x ny x nz cubes of edge `cell`; with refine = r > 0
 * the cubes flagged in `refined` are divided into r^3 sub-cubes (one level
 * of refinement).  Cells ("leaves") are numbered cube by cube in z, y, x
 * order; a refined cube's r^3 sub-cubes take consecutive numbers from
 * leaf_base[cube], again in z, y, x order.  Per-cell arrays (rho, E_abs, T)
 * are [ns][ncell], ncell = nleaf (refined) or nx ny nz. */
typedef struct {
    int nx, ny, nz, ns, nf;
    double box_min[3];
    double cell;                 /* cubic cell edge, cm */
    const float* rho;            /* [ns][ncell] g/cm^3 */
    const double* nu;            /* [nf] Hz, ascending */
    const double* dnu;           /* [nf] Hz */
    const double* kabs;          /* [ns][nf] cm^2/g */
    const double* ksca;          /* [ns][nf] cm^2/g */
    const double* g;             /* [ns][nf] HG asymmetry */
    const int* is_pah;           /* [ns] */
    int refine;                  /* r >= 2, or 0 for a uniform grid */
    const unsigned char* refined;/* [nz][ny][nx] 1 = divided (refine > 0) */
    const int64_t* leaf_base;    /* [nz][ny][nx] first cell of each cube (refine > 0) */
    int64_t nleaf;               /* cells of a refined grid */
} or_model;

typedef struct {
    double pos[3];
    double L;                    /* erg/s */
    double T_eff;                /* blackbody temperature when L_nu == NULL */
    const double* L_nu;          /* [nf] spectral shape or NULL */
} or_source;

enum { OR_MODE_BW = 0, OR_MODE_FROZEN_T = 1, OR_MODE_NOREEMIT = 2 };
enum { OR_LUCY_OFF = 0, OR_LUCY_THIN = 1, OR_LUCY_ALL = 2 };
enum { OR_LUCY_LINEAR = 0, OR_LUCY_EXPM1 = 1 };

/* Photon-counting camera (Sect. 4): packets leaving the grid with
 * k . k_obs >= cos_accept are counted in the pixel of their exit point
 * projected on the image plane (frame and pixel size as for or_camera). */
typedef struct { double theta, phi; int npix; double pixel; double cos_accept; } or_pc_camera;

typedef struct {
    int mode, lucy_mode, lucy_form;
    double lucy_tau;
    int mrw;
    double mrw_tau_cell, mrw_gamma;
    uint64_t seed;
    uint32_t model_id;
    uint64_t n_packets, pid_begin, pid_end, max_events;
    int record_events;
    uint32_t source_bins;   /* 0: source and bin drawn at random (prob. ~ L_nu dnu);
                               m > 0: Eq. 1 equal-energy source bins, packet pid
                               from bin floor(pid m / N) (see or_transport) */
    const or_pc_camera* pc;  /* [n_pc] photon-counting cameras (or NULL) */
    int n_pc;
    const int32_t* sg_nu;    /* with source_bins = m: the source frequency grid of Eq. 1
                                (or_source_grid), source bin b's model frequency bin and */
    const int32_t* sg_src;   /* source ([m] each); NULL: bins on the model grid (reading 20) */
} or_params;

typedef struct { uint32_t cell, nu, species, pad; double k[3]; } or_event;
typedef struct { uint32_t cell, nu; } or_pah;

enum { OR_T_EMIT = 0, OR_T_SCATTER = 1, OR_T_ABSORB = 2, OR_T_MRW = 3, OR_T_ESCAPE = 4,
       OR_T_PAH = 5, OR_T_STUCK = 6, OR_T_ABSORB_END = 7 };
typedef struct { uint64_t pid; uint32_t seq, type, cell, nu; double x[3]; double k[3]; } or_traj;

enum { OR_S_CROSS = 0, OR_S_INTERACT, OR_S_SCATTER, OR_S_ABSORB, OR_S_MRW, OR_S_ESCAPE,
       OR_S_STUCK, OR_S_PAH, OR_S_EV_DROP, OR_S_LUCY, OR_S_EMIT, OR_S_PAH_DROP, OR_S_TRAJ_DROP,
       OR_S_N = 16 };

typedef struct {
    double* E_abs;               /* [ns][ncell] erg/s, accumulated */
    uint32_t* count;             /* [ns][ncell] absorption events */
    double* esq;                 /* [ns][ncell] sum of squared deposits (may be NULL) */
    double* sed_esc;             /* [10][nf] erg/s per cos(theta) bin */
    uint64_t* sed_cnt;           /* [10][nf] */
    or_event* events; uint64_t event_cap; uint64_t n_events;
    or_pah* pah; uint64_t pah_cap; uint64_t n_pah;
    or_traj* traj; uint64_t traj_cap; uint64_t n_traj;
    uint64_t stats[OR_S_N];
    double* pc_img;              /* camera c at offset sum_{c'<c} nf npix_c'^2: [nf][npix][npix] */
    double loop_seconds;         /* wall time of the packet loop alone (set-up excluded),
                                    a timing record for the CPU baseline, not a result */
} or_out;

typedef struct { double theta, phi; int npix; double D; double pixel; } or_camera;

/* PAH re-emission pass (Sect. 2.1): the stored PAH absorptions become the
 * sources, one packet of energy xi per record, emitted from a point drawn
 * uniformly in the record's cell, in the frequency bin drawn from Eq. 6 with
 * the emissivity eps_n(nu) of Eq. 7 supplied per class n. */
typedef struct {
    const or_pah* rec;           /* [n_rec] stored absorptions (cell used, nu ignored) */
    uint64_t n_rec;
    double xi;                   /* packet energy of the pass that stored them */
    const double* eps;           /* [n_eps][nf] eps_n(nu_j), >= 0 */
    int n_eps;
    const int* eps_class;        /* [ncell] class n of each cell, or NULL (class 0) */
} or_pah_src;

/* primitives exposed for the pins */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void or_uniforms(uint64_t seed, uint32_t model_id, uint64_t pid, uint32_t n, double* out);
double or_planck_B(double nu, double T);
double or_planck_dBdT(double nu, double T);
double or_planck_mean(const or_model* m, int s, double T);
double or_solve_temperature(const or_model* m, int s, double target);
double or_hg_mu(double g, double u);
void or_rotate(double k[3], double mu, double phi);
double or_mrw_survival(double y);
double or_mrw_sample_y(double u);
void or_source_lnu(const or_model* m, const or_source* src, double* lnu);
int or_dda_segments(const or_model* m, const double x[3], const double k[3], int max,
                    int64_t* cells, double* lens);

/* the path */
int or_transport(const or_model* m, const or_source* src, int nsrc, const or_params* p,
                 const double* T_prev, or_out* out, int n_threads);
/* The source frequency grid of Eq. 1 (Sect. 2): the sources' combined
 * luminosity cut into mbins bins of equal energy on each source's own
 * continuous spectrum (a blackbody of T_eff; a tabulated L_nu is constant over
 * each model frequency bin), between the outer edges of the model frequency
 * bins (bin edges at the geometric means of neighbouring frequencies, the
 * outer ones mirrored).  Bin b is monochromatic at nu_star[b], where the
 * cumulative luminosity reaches (b + 1/2) L / mbins; src_idx[b] is its source
 * and nu_idx[b] the model bin holding nu_star[b].  Returns 0, or 1 for bad
 * arguments. */
int or_source_grid(const or_model* m, const or_source* src, int nsrc, uint32_t mbins,
                   int32_t* nu_idx, int32_t* src_idx, double* nu_star);
/* Runs packets [pid_begin, pid_end) of the pass; p->n_packets must equal
 * ps->n_rec and p->source_bins must be 0.  Packet pid starts from rec[pid]. */
int or_pah_reemit(const or_model* m, const or_pah_src* ps, const or_params* p,
                  const double* T_prev, or_out* out, int n_threads);
void or_temperatures(const or_model* m, const double* E_abs, double* T);
void or_temperature_guess(const or_model* m, const or_source* src, int nsrc, double* T);
void or_raytrace(const or_model* m, const double* T, const or_event* ev, uint64_t nev,
                 double xi_ev, const or_source* src, int nsrc, const or_camera* cams, int ncam,
                 const int* fidx, int nfi, double* images, double* sed);
void or_raytrace_backward(const or_model* m, const double* T, const or_event* ev, uint64_t nev,
                          double xi_ev, const or_source* src, int nsrc, const or_camera* cams,
                          int ncam, const int* fidx, int nfi, const double* dL_dimg,
                          const double* dL_dsed, double* dL_drho, double* dL_dscale);

#ifdef __cplusplus
}
#endif
#endif
