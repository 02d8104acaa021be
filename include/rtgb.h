/*
 * rtgb — GB300-native Monte Carlo dust radiative transfer
 * (method of Heymann & Siebenmorgen 2012, arXiv:1203.2941).
 *
 * C ABI of librtgb.so.  Every entry point is callable from C; no C++ or
 * PyTorch type appears here.  Pointers documented as "device" must point to
 * memory of the context's GPU (cudaMalloc'd or equivalent); "host" pointers are
 * read during the call and may be released when it returns.
 *
 * Streams: every call that launches GPU work takes an rt_stream (a
 * cudaStream_t; NULL means the legacy default stream) and is asynchronous with
 * respect to the host unless stated otherwise.  Argument errors are reported
 * synchronously through the return value; rt_last_error() then holds a
 * message (thread-local, owned by the library, valid until the next call on
 * the same thread).  Device-side conditions (capacity overflow, event cap) are
 * reported through counters in the caller's stats array, readable after the
 * stream is synchronised.
 *
 * Units are CGS throughout: lengths in cm, densities in g/cm^3, opacities in
 * cm^2/g, frequencies in Hz, luminosities in erg/s, energies deposited per
 * unit time in erg/s, intensities in erg/s/cm^2/Hz/sr.
 */
#ifndef RTGB_H
#define RTGB_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RT_API __attribute__((visibility("default")))
#else
#define RT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* rt_stream;   /* identical to cudaStream_t */

typedef int rt_status;
enum {
    RT_OK = 0,
    RT_ERR_INVALID_ARG = 1,  /* a pointer, size or value was rejected; nothing was launched */
    RT_ERR_CUDA = 2,         /* a CUDA runtime call failed; message in rt_last_error() */
    RT_ERR_OOM = 3,          /* device allocation failed */
    RT_ERR_CAPACITY = 4,     /* a fixed-size buffer is too small for the request */
    RT_ERR_STUCK = 5,        /* reserved: packets hit the per-packet event cap (see stats) */
    RT_ERR_STATE = 6         /* handle used with the wrong context or after free */
};

typedef struct rt_ctx rt_ctx;
typedef struct rt_grid rt_grid;
typedef struct rt_opacity rt_opacity;
typedef struct rt_batch rt_batch;

/* Message for the last failing call on this thread ("" if none). */
RT_API const char* rt_last_error(void);
/* Library version string. */
RT_API const char* rt_version(void);

/* Create a context on CUDA device `device` (it becomes current for the calling
 * thread).  The context owns small scratch buffers (work counters).  Errors:
 * RT_ERR_INVALID_ARG (no such device / out == NULL), RT_ERR_CUDA. */
RT_API rt_status rt_ctx_create(int device, rt_ctx** out);
RT_API void rt_ctx_destroy(rt_ctx* ctx);

/* ---------------------------------------------------------------------------
 * Model space (paper Sect. 2: a Cartesian grid of cubes with constant density
 * per cube, several grain materials).
 *
 * rho: [n_species][nz][ny][nx] float32 g/cm^3, x fastest, host OR device
 * pointer (copied; the caller keeps ownership).  box_min: host [3] cm, lower
 * corner; cell_size: edge of the cubic cells (cm).  The library keeps its own
 * copy, re-packed per transport call into an interleaved per-cell layout.
 * Errors: RT_ERR_INVALID_ARG for non-positive sizes, n_species outside 1..4,
 * non-finite box or cell, negative or non-finite density (checked on the
 * device copy, synchronously on `stream`).
 * ------------------------------------------------------------------------- */
RT_API rt_status rt_grid_upload(rt_ctx* ctx, int nx, int ny, int nz, int n_species,
                         const double box_min[3], double cell_size, const float* rho,
                         rt_stream stream, rt_grid** out);
/* A grid with one level of refinement (Sect. 2: each cube may be divided
 * into sub-cubes of constant density).  nx x ny x nz cubes of edge
 * cell_size; the cubes with refined[cube] != 0 (host [nz][ny][nx] bytes) are
 * divided into r^3 sub-cubes (r = refine, 2..16).  Cells are numbered cube
 * by cube in z, y, x order; a divided cube's r^3 sub-cubes take consecutive
 * numbers, again in z, y, x order.  rho: [n_species][ncell] float32, host or
 * device, ncell = (cubes not divided) + r^3 (cubes divided) < 2^30.
 * Every per-cell array of the other calls (E_abs, count, esq, T, the cell of
 * events and PAH records) is indexed by this cell number.  Served by
 * every call that takes a grid (a batch may mix refined and uniform
 * grids).  Errors as rt_grid_upload, plus a bad refine factor. */
RT_API rt_status rt_grid_upload_refined(rt_ctx* ctx, int nx, int ny, int nz, int n_species,
                                        const double box_min[3], double cell_size, int refine,
                                        const unsigned char* refined, const float* rho,
                                        rt_stream stream, rt_grid** out);
/* New densities for an existing grid (same shape, species and refinement):
 * rho as for the upload (host or device, [n_species][ncell] float32), copied
 * on `stream` into the grid's own copy and checked there, synchronously
 * (finite, >= 0); no device memory is allocated or freed after the first
 * call.  The packed copy the kernels read is rebuilt by the next call that
 * uses the grid.  Errors: RT_ERR_INVALID_ARG for NULL or a bad density --
 * the grid then refuses every call (RT_ERR_STATE) until an update succeeds;
 * RT_ERR_CUDA. */
RT_API rt_status rt_grid_update(rt_grid* grid, const float* rho, rt_stream stream);
/* Cells of a grid (leaves of a refined one). */
RT_API uint64_t rt_grid_ncell(const rt_grid* grid);
RT_API void rt_grid_free(rt_grid* grid);

/* Dust cross sections per unit mass (paper Sect. 2 "absorption kappa_abs and
 * scattering kappa_sca cross-sections", Henyey-Greenstein g of Eq. 15),
 * tabulated on one frequency grid shared by the sources and the dust.
 * nu, dnu: host [n_freq] Hz, nu strictly ascending, dnu > 0 (bin widths).
 * kabs, ksca, g: host [n_species][n_freq]; kabs, ksca >= 0, |g| < 1.
 * is_pah: host [n_species] or NULL; a nonzero entry marks a stochastically
 * heated species (Sect. 2.1) whose absorptions end the packet and are stored.
 * All arrays are copied.  n_freq in 2..1024, n_species in 1..4. */
RT_API rt_status rt_opacity_upload(rt_ctx* ctx, int n_freq, const double* nu, const double* dnu,
                            int n_species, const double* kabs, const double* ksca,
                            const double* g, const int* is_pah, rt_opacity** out);
RT_API void rt_opacity_free(rt_opacity* opac);

/* A point source inside the grid.  L_nu: host [n_freq] spectral shape (erg/s/Hz,
 * any normalisation) or NULL for a blackbody of temperature T_eff.  The
 * spectrum is normalised so that sum_j L_nu,j dnu_j = L (equal-energy packets,
 * paper Eq. 1 in expectation). */
typedef struct {
    double pos[3];
    double L;
    double T_eff;
    const double* L_nu;
} rt_source;

/* ---------------------------------------------------------------------------
 * Photon-packet transport (paper Sects. 2 and 3.1-3.4).
 * ------------------------------------------------------------------------- */
enum { RT_MODE_BW = 0,        /* Bjorkman & Wood: T from Eq. 4 after each absorption,
                                 re-emission from Eq. 10 (Sect. 3.3) */
       RT_MODE_FROZEN_T = 1,  /* iterative scheme: re-emission from Eq. 5 at T_prev (Sect. 2) */
       RT_MODE_NOREEMIT = 2 };/* absorbed packets end (pure-absorber diagnostics) */
enum { RT_LUCY_OFF = 0, RT_LUCY_THIN = 1, RT_LUCY_ALL = 2 };   /* Sect. 3.1 cells */
enum { RT_LUCY_LINEAR = 0,    /* deposit xi kappa_abs rho l (unbiased path-length form) */
       RT_LUCY_EXPM1 = 1 };   /* deposit (1 - exp(-kappa_abs rho l)) xi (Eq. 9) */
enum { RT_PREC_FP32 = 0,      /* production: FP32 transport, FP64 accumulators */
       RT_PREC_FP64 = 1,      /* debug: every quantity in FP64 (trajectory parity) */
       RT_PREC_FP32_ACC32 = 2 };  /* plain FP32: FP32 transport and FP32 per-cell
                                 accumulators (a comparison form: sums of many
                                 deposits lose digits); rt_transport on uniform
                                 grids without trajectories, deferred queue,
                                 cameras or PAH sources only */
enum { RT_SCHED_PERSISTENT = 0, /* all SMs, dynamic packet refill */
       RT_SCHED_SERIAL = 1,     /* one GPU thread, packets in id order (debug) */
       RT_SCHED_COMPACT = 2 };  /* all SMs with per-warp packet compaction (Sect. 3.4
                                   load balancing): each warp parks packets in a
                                   shared-memory stash so that its lanes march
                                   together and serve interactions together;
                                   single-model FP32 launches on uniform grids
                                   without trajectories, the deferred queue or
                                   cameras (others run RT_SCHED_PERSISTENT) */

/* A photon-counting camera (the Monte Carlo image of Sect. 4, which the
 * paper sets against its ray tracer): packets that leave the grid with
 * k . k_obs >= cos_accept add their power xi to the pixel of their exit
 * point projected on the image plane.  Frame as in rt_raytrace: k_obs from
 * (theta, phi), image axes e_x' = (-sin phi, cos phi, 0), e_y' = (-cos theta
 * cos phi, -cos theta sin phi, sin theta), image centred on the box centre,
 * npix^2 pixels of `pixel` cm (0 = box diagonal / npix). */
typedef struct {
    double theta, phi;
    int npix;
    double pixel;
    double cos_accept;
} rt_pc_camera;

typedef struct {
    int mode;                 /* RT_MODE_* */
    int lucy_mode;            /* RT_LUCY_* */
    int lucy_form;            /* RT_LUCY_LINEAR / RT_LUCY_EXPM1 */
    double lucy_tau;          /* THIN: largest face-to-face tau below this (paper: 1e-2) */
    int mrw;                  /* modified random walk in thick cells (Sect. 3.2) */
    double mrw_tau_cell;      /* cell tau above which MRW is tried (10) */
    double mrw_gamma;         /* minimum sphere optical radius (2) */
    uint64_t seed;            /* Philox key = (seed_lo, seed_hi ^ model_id) */
    uint32_t model_id;
    uint64_t n_packets;       /* N; packet energy xi = L / N */
    uint64_t pid_begin, pid_end;  /* packets simulated: [pid_begin, pid_end) within [0, N) */
    uint64_t max_events;      /* per-packet interaction cap; capped packets are counted "stuck" */
    int record_events;        /* store scattering events for the ray tracer (Sect. 2) */
    int precision;            /* RT_PREC_* */
    int schedule;             /* RT_SCHED_* */
    int threads_per_block;    /* 0 = library default */
    int blocks_per_sm;        /* 0 = occupancy-derived */
    int march_min_active;     /* lanes still marching below which a warp serves its
                                 pending interactions (0..31; -1 = default, 16) */
    uint64_t defer_events;    /* 0 = off.  rt_transport only: a packet that starts a
                                 flight after this many interactions + MRW steps is
                                 queued (device memory, up to 2^20 packets per call)
                                 and finished by a second pass after every other
                                 packet, so slow packets do not hold up the warps
                                 (a full queue leaves the packet where it is) */
    uint32_t source_bins;     /* 0 = source and frequency bin drawn per packet with
                                 probability ~ L_nu dnu.  m > 0: the source grid of
                                 Eq. 1 -- the sources' combined luminosity is cut
                                 into m bins of equal energy L/m and packet pid is
                                 emitted from bin b = floor(pid m / N), at the point
                                 (b + 1/2) / m of the cumulative luminosity (its
                                 source, then its frequency bin); N/m packets per
                                 bin when m divides N */
    const rt_pc_camera* pc_cams;  /* host [n_pc_cams] photon-counting cameras
                                 (rt_transport only; NULL with 0 = none) */
    int n_pc_cams;            /* 0..16 (rt_transport only) */
    const uint32_t* record_nu_mask;  /* host bitmask over the frequency bins,
                                 bit j = (mask[j / 32] >> (j % 32)) & 1: with
                                 record_events, a scattering event is stored only
                                 when the packet's bin j is set (the image
                                 frequencies of the ray tracer, whose scattering
                                 source, Eq. 16, uses events at those frequencies
                                 alone); NULL = every bin.  (n_freq + 31) / 32 words */
    const int32_t* source_grid_nu;   /* with source_bins = m: host [m] model frequency bin
                                 of each bin of the separate source grid of Eq. 1
                                 (rt_source_grid); packet pid is emitted from source
                                 grid_src[b] in bin grid_nu[b], b = floor(pid m / N).
                                 NULL: bins on the model grid (see source_bins).
                                 rt_transport only */
    const int32_t* source_grid_src;  /* host [m] source index of each bin (with the above) */
    int compact_swap;         /* RT_SCHED_COMPACT: when at most this many lanes of a
                                 warp still march, its stopped lanes trade their
                                 packets for parked marching ones (0..31; -1 = 24) */
} rt_transport_params;

/* Fill p with the defaults: B&W, Lucy THIN at 1e-2, linear form, MRW off
 * (tau 10, gamma 2), seed 1, FP32, persistent, max_events 1e7. */
RT_API void rt_transport_params_default(rt_transport_params* p);

/* One stored scattering event (20 bytes): cell index, frequency index,
 * scattering species, model index in a batch, incoming direction. */
typedef struct {
    uint32_t cell;
    uint16_t nu;
    uint8_t species;
    uint8_t model;
    float k[3];
} rt_event;

/* One stored PAH absorption (Sect. 2.1): cell and frequency index. */
typedef struct {
    uint32_t cell;
    uint16_t nu;
    uint16_t model;
} rt_pah_event;

/* Trajectory record (debug/parity): packet id, event number within the
 * packet, type (RT_TRAJ_*), cell, frequency index after the event, position
 * (cm) and direction after the event. 72 bytes. */
typedef struct {
    uint64_t pid;
    uint32_t seq, type, cell, nu;
    double x[3];
    double k[3];
} rt_traj;
enum { RT_TRAJ_EMIT = 0, RT_TRAJ_SCATTER = 1, RT_TRAJ_ABSORB = 2, RT_TRAJ_MRW = 3,
       RT_TRAJ_ESCAPE = 4, RT_TRAJ_PAH = 5, RT_TRAJ_STUCK = 6, RT_TRAJ_ABSORB_END = 7 };

/* Indices of the uint64 stats array (RT_STAT_COUNT entries, device). */
enum {
    RT_STAT_CROSSINGS = 0,    /* packet cell-face crossings */
    RT_STAT_INTERACTIONS = 1, RT_STAT_SCATTERS = 2, RT_STAT_ABSORPTIONS = 3,
    RT_STAT_MRW = 4, RT_STAT_ESCAPED = 5, RT_STAT_STUCK = 6, RT_STAT_PAH = 7,
    RT_STAT_EVENTS_DROPPED = 8, RT_STAT_LUCY = 9, RT_STAT_EMITTED = 10,
    RT_STAT_PAH_DROPPED = 11, RT_STAT_TRAJ_DROPPED = 12,
    RT_STAT_N_EVENTS = 13,    /* cursor into events (also counts dropped ones) */
    RT_STAT_N_PAH = 14, RT_STAT_N_TRAJ = 15,
    RT_STAT_DEFERRED = 16,    /* packets queued by defer_events (finished later) */
    RT_STAT_COUNT = 17
};

/* Caller-owned device outputs.  All are ACCUMULATED into (zero them for a
 * fresh run); B&W temperatures see the accumulated E_abs, so a run split into
 * packet ranges continues exactly where the previous call stopped.
 *   E_abs   [n_species][ncell] double  absorbed power per species and cell
 *   count   [n_species][ncell] uint32  absorption events
 *   esq     [n_species][ncell] double  sum of squared deposits, or NULL
 *   sed_esc [10][n_freq] double        escaped power in 10 bins equal in cos(theta)
 *   sed_cnt [10][n_freq] uint64        escaped packets
 *   events/pah/traj: append buffers (NULL with cap 0 to disable); the cursor
 *           is stats[RT_STAT_N_*]; entries beyond the capacity are counted in
 *           the *_DROPPED stats and not written.
 *   stats   [RT_STAT_COUNT] uint64 (required).
 *   pc_img  device double, one [n_freq][npix][npix] block per photon-counting
 *           camera (camera c after the blocks of cameras 0..c-1): power
 *           (erg/s) of the packets it counted, per frequency bin and pixel
 *           (required when p->n_pc_cams > 0). */
typedef struct {
    double* E_abs;
    uint32_t* count;
    double* esq;
    double* sed_esc;
    uint64_t* sed_cnt;
    rt_event* events; uint64_t event_cap;
    rt_pah_event* pah; uint64_t pah_cap;
    rt_traj* traj; uint64_t traj_cap;
    uint64_t* stats;
    double* pc_img;
} rt_transport_out;

/* Transport N = p->n_packets equal-energy packets (packets [pid_begin,
 * pid_end)) from the sources through the grid: isotropic emission, one
 * optical depth -ln(u) per flight (Sect. 2 and its footnote), cell traversal
 * with tau_i = (kabs + ksca) rho l (Eq. 2), interaction distance (Eq. 3),
 * albedo choice, HG scattering (Eq. 15) with the event store, absorption with
 * B&W (Eq. 4 + Eq. 10) or frozen-T (Eq. 5) re-emission, Lucy deposits in thin
 * cells (Sect. 3.1, Eq. 9) and the modified random walk in thick cells
 * (Sect. 3.2).  T_prev: device [n_species][ncell] double, required in
 * RT_MODE_FROZEN_T, ignored otherwise.  Sources must lie inside the grid.
 * Random numbers: Philox4x32-10, key (seed_lo, seed_hi ^ model_id), counter
 * (draw/2, 0, pid_lo, pid_hi); the k-th draw of a packet is the uniform
 * ((w >> 11) + 1) 2^-53 (FP64) or ((w >> 40) + 1) 2^-24 (FP32) of 64-bit word
 * k mod 2 of block k/2.  Photon-counting cameras (p->pc_cams, Sect. 4) add
 * each escaping packet's power to out->pc_img (accumulated, not cleared).
 * Errors: RT_ERR_INVALID_ARG (ranges, pointers, precision/mode combinations),
 * RT_ERR_CUDA. */
RT_API rt_status rt_transport(rt_ctx* ctx, const rt_grid* grid, const rt_opacity* opac,
                       const rt_source* sources, int n_sources,
                       const rt_transport_params* p, const double* T_prev,
                       const rt_transport_out* out, rt_stream stream);

/* PAH re-emission pass (Sect. 2.1, Eqs. 6-7).  After the large grains'
 * temperatures are known, every cell with stored PAH absorptions becomes a
 * source that emits as many packets as it absorbed: packet pid (of
 * [p->pid_begin, p->pid_end), p->n_packets == n_records) starts in the cell
 * of records[pid], at a point drawn uniformly in the cell (one draw per axis
 * after the bin draw), in the frequency bin j of Eq. 6 -- the smallest j with
 * sum_{l<=j} eps_n(nu_l) dnu_l >= u sum_l eps_n(nu_l) dnu_l -- with n the
 * cell's emissivity class, in an isotropic direction, carrying energy xi
 * (that of the pass that stored the records).  The packets are then
 * transported exactly as by rt_transport with p (mode, Lucy, MRW, seed,
 * model_id, precision, schedule, photon-counting cameras); PAH absorptions
 * in this pass are stored again in out->pah for a further pass.
 *   records: device [n_records] (the records' nu and model fields are
 *            ignored); must not overlap out->pah.
 *   eps: host [n_eps][n_freq] double, eps_n(nu_j) of Eq. 7 (K_PAH times the
 *        P_n(T)-weighted Planck function, supplied by the caller), finite,
 *        >= 0, each class nonzero on the grid; n_eps 1..65535.
 *   eps_class: device int [ncell] class n of each cell, or NULL (class 0).
 *   A record whose cell is outside the grid, or whose class is out of
 *   range, emits nothing and is counted in RT_STAT_STUCK.
 * Errors: as rt_transport; RT_ERR_INVALID_ARG for n_records = 0,
 * n_packets != n_records, source_bins != 0, xi <= 0 or a bad eps table. */
RT_API rt_status rt_pah_reemit(rt_ctx* ctx, const rt_grid* grid, const rt_opacity* opac,
                               const rt_pah_event* records, uint64_t n_records, double xi,
                               const double* eps, int n_eps, const int* eps_class,
                               const rt_transport_params* p, const double* T_prev,
                               const rt_transport_out* out, rt_stream stream);

/* The separate source frequency grid of Eq. 1 (Sect. 2): the sources'
 * combined luminosity L cut into m bins of equal energy L/m on each source's
 * own continuous spectrum -- a blackbody of T_eff, or a tabulated L_nu taken
 * constant over each model frequency bin -- between the outer edges of the
 * model bins (edges at the geometric means of neighbouring frequencies, the
 * outer ones mirrored in ln nu).  Bin b is monochromatic at nu_star[b], where
 * the cumulative luminosity reaches (b + 1/2) L/m (the sources taken in
 * order, by their luminosities); src_idx[b] is its source and nu_idx[b] the
 * model bin holding nu_star[b] (the dust grid extends the source grid,
 * Sect. 2).  Pass nu_idx and src_idx as rt_transport_params.source_grid_nu /
 * source_grid_src with source_bins = m to emit N/m packets per bin.
 * Host arrays [m]; nu_star may be NULL.  FP64 on the host (the blackbody's
 * cumulative by Simpson's rule on 2^15 intervals in ln nu, targets solved by
 * Newton steps).  Errors: RT_ERR_INVALID_ARG for m = 0, no source or NULL
 * outputs. */
RT_API rt_status rt_source_grid(const rt_opacity* opac, const rt_source* sources, int n_sources,
                                uint32_t m, int32_t* nu_idx, int32_t* src_idx, double* nu_star);

/* Allocation-free variant of rt_transport (no counterpart in the paper; it
 * exists for callers that must not allocate device memory).  Same arguments,
 * semantics, outputs and errors as rt_transport, but the call itself never
 * allocates or frees device memory: its scratch (work counter, model and
 * source tables, a packed copy of the density grid, the FP64 energy scratch of
 * the FP32 build) lives in one 64 MiB statically allocated device array that
 * every GPU which loads the library holds until the process exits.  Callers
 * that need this: code running where a device allocation is not allowed or
 * not affordable -- e.g. a host whose device memory is entirely owned by
 * another allocator or pool with a fixed budget, or a loop that must not hit
 * the implicit device synchronisation that cudaMalloc/cudaFree may cause.
 * Limit: 1 MiB of staging plus ncell*4*vec bytes of packed density
 * (vec = 1, 2 or 4 floats for 1, 2 or 3-4 species) plus, in FP32,
 * n_species*ncell*8 bytes (16 with esq) must fit in 64 MiB - 64 KiB; larger
 * grids return RT_ERR_CAPACITY without launching anything.  The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress with
 * that device current) and should come before any stream capture.  All calls
 * share the one array: calls whose GPU work overlaps (different streams
 * without ordering, or several host threads) race and must not be issued;
 * calls ordered on one stream are safe (each rewrites what the previous call
 * left: the counters start at zero, the energy scratch at E_abs / xi).
 * Photon-counting cameras, the deferred-packet queue, the separate source
 * grid and the plain-FP32 form are not served here: n_pc_cams and
 * defer_events must be 0, source_grid_nu NULL and precision not
 * RT_PREC_FP32_ACC32, else RT_ERR_INVALID_ARG. */
RT_API rt_status rt_transport_noalloc(rt_ctx* ctx, const rt_grid* grid, const rt_opacity* opac,
                                      const rt_source* sources, int n_sources,
                                      const rt_transport_params* p, const double* T_prev,
                                      const rt_transport_out* out, rt_stream stream);

/* Dust temperatures from Eq. 4: for every species s and cell i, the T with
 * 4 pi sum_j kabs_s,j B_nu_j(T) dnu_j = E_abs[s][i] / (rho_s,i V); 0 where E or
 * rho is 0.  FP64 (table start, Newton polish to ~1e-13 relative).
 * E_abs, T: device [n_species][ncell] double. */
RT_API rt_status rt_temperatures(rt_ctx* ctx, const rt_grid* grid, const rt_opacity* opac,
                          const double* E_abs, double* T, rt_stream stream);

/* Initial guess of the iterative scheme (Sect. 2): optically thin gray dust,
 * T^4 = sum_src L / (16 pi sigma r^2) at the cell centre, capped at 2000 K.
 * T: device [n_species][ncell] double. */
RT_API rt_status rt_temperature_guess(rt_ctx* ctx, const rt_grid* grid, const rt_source* sources,
                               int n_sources, double* T, rt_stream stream);

/* ---------------------------------------------------------------------------
 * Ray tracer (paper Sect. 4).
 * ------------------------------------------------------------------------- */
/* Observer direction (theta, phi) from +z, square image npix x npix, distance
 * D (cm), pixel size (cm; <= 0: box diagonal / npix so any view fits).  Image
 * axes e_x' = (-sin phi, cos phi, 0), e_y' = (-cos theta cos phi,
 * -cos theta sin phi, sin theta); pixel (ix, iy) is centred at
 * ((ix + 0.5 - npix/2) p, (iy + 0.5 - npix/2) p) about the box centre (Eq. 11). */
typedef struct {
    double theta, phi;
    int npix;
    double D;
    double pixel;
} rt_camera;

/* Images and SEDs from the dust temperatures and the stored scattering events.
 * Per pixel ray (parallel projection, Eq. 11) marched front to back:
 * I = sum_k S_k (1 - exp(-dtau_k)) exp(-tau_<k) with dtau = (kabs+ksca) rho l
 * over the actual chord, S = (eta_th + eta_sca) / ((kabs+ksca) rho),
 * eta_th = sum_s rho_s kabs_s B_nu(T_s) (Eq. 14 source function),
 * eta_sca = xi_ev / (V dnu) sum_events P_HG(k_in . k_obs; g) (Eq. 16).
 * sed[c][f] = sum_pix I A_pix / D^2 (Eq. 17) + sum_src L_nu exp(-tau_src) / (4 pi D^2).
 *   T: device [n_species][ncell] double;  events: device [n_events] (may be
 *   NULL if n_events == 0);  n_events_dev: device uint64 or NULL; when given,
 *   the number of events used is min(*n_events_dev, n_events), read on the
 *   device, so n_events is the buffer's capacity and the call needs no host
 *   copy of a count that the transport writes (stats[RT_STAT_N_EVENTS]);
 *   xi_ev: power carried by one event (= L/N of the
 *   transport that stored them);  cams: host [n_cams], all with the same npix;
 *   freq_idx: host [n_f] indices into the opacity grid, n_f in 1..16;
 *   images: device [n_cams][n_f][npix][npix] float;  sed: device [n_cams][n_f]
 *   double;  ray_steps: device uint64 or NULL, incremented by the number of
 *   ray-cell steps marched.  Scratch: emissivity tables of n_cams * ncell *
 *   n_f floats are allocated by the context and kept for reuse. */
RT_API rt_status rt_raytrace(rt_ctx* ctx, const rt_grid* grid, const rt_opacity* opac,
                      const double* T, const rt_event* events, uint64_t n_events,
                      const uint64_t* n_events_dev, double xi_ev,
                      const rt_source* sources, int n_sources, const rt_camera* cams, int n_cams,
                      const int* freq_idx, int n_f, float* images, double* sed,
                      uint64_t* ray_steps, rt_stream stream);

/* Adjoint of rt_raytrace with T and the events held fixed (no counterpart in
 * the paper; added to differentiate images and SEDs with respect to density).
 * dL_dimg: device [n_cams][n_f][npix][npix] float; dL_dsed: device
 * [n_cams][n_f] double (either may be NULL = zero).  Accumulates
 * dL/drho_s,i into dL_drho (device [n_species][ncell] float) and
 * sum_s,i rho_s,i dL/drho_s,i (the derivative with respect to a global
 * density scale) into dL_dscale (device, one double).  Per ray the forward
 * march is recomputed (pass 1: totals, pass 2: gradients); no path is stored.
 * events, n_events and n_events_dev as for rt_raytrace.  ray_steps: device
 * uint64 or NULL, incremented by the ray-cell steps of both passes. */
RT_API rt_status rt_raytrace_backward(rt_ctx* ctx, const rt_grid* grid, const rt_opacity* opac,
                               const double* T, const rt_event* events, uint64_t n_events,
                               const uint64_t* n_events_dev, double xi_ev, const rt_source* sources, int n_sources,
                               const rt_camera* cams, int n_cams, const int* freq_idx, int n_f,
                               const float* dL_dimg, const double* dL_dsed, float* dL_drho,
                               double* dL_dscale, uint64_t* ray_steps, rt_stream stream);

/* Complex visibilities of ray-traced images.  Sect. 4 names visibilities
 * among the ray tracer's products without a formula; this is the plain
 * definition: for image (c, f) of rt_raytrace's output,
 *   V(u, v) = sum over pixels of I A_pix / D^2 exp(-2 pi i (u alpha + v beta)),
 * alpha, beta = the pixel centre's offsets along the image axes (e_x', e_y')
 * divided by D (small-angle sky coordinates, radians), so V(0, 0) is the
 * image's part of the SED.
 *   cams: host [n_cams], as passed to rt_raytrace for this grid (the default
 *   pixel size comes from the grid), 1..1024 cameras with one npix <= 8192;
 *   images: device [n_cams][n_f][npix][npix] float; n_f 1..16;
 *   uv: host [n_uv][2] doubles, cycles per radian along e_x', e_y' (a
 *   projected baseline divided by the wavelength), n_uv 1..65535;
 *   vis: device [n_cams][n_f][n_uv][2] double (real, imaginary part).
 * Errors: RT_ERR_INVALID_ARG on NULL pointers or sizes out of range. */
RT_API rt_status rt_visibilities(rt_ctx* ctx, const rt_grid* grid, const rt_camera* cams, int n_cams,
                                 const float* images, int n_f, const double* uv, int n_uv,
                                 double* vis, rt_stream stream);

/* ---------------------------------------------------------------------------
 * Batched transport: many models of uneven grid size in one persistent launch
 * (no counterpart in the paper; packets of all models share the warps).
 * Model m uses Philox model_id = p->model_id + m and packets [0, n_packets).
 * ------------------------------------------------------------------------- */
typedef struct {
    const rt_grid* grid;
    const rt_source* sources;   /* host [n_sources] */
    int n_sources;
    uint64_t n_packets;
    const double* T_prev;       /* device, frozen-T mode only */
    rt_transport_out out;
} rt_model;

/* Prepare a batch: packs every grid, uploads the model table and source
 * tables (host-synchronous).  The batch keeps pointers to the grids and the
 * output buffers; they must outlive it.  n_models in 1..4096; all grids share
 * `opac` and must have its species count (grids may be refined);
 * p->n_pc_cams must be 0. */
RT_API rt_status rt_batch_create(rt_ctx* ctx, const rt_opacity* opac, int n_models,
                          const rt_model* models, const rt_transport_params* p,
                          rt_batch** out);
/* Launch the batch on `stream`: one memset of the work counter and one
 * persistent kernel, nothing else (no host synchronisation, no allocation),
 * so the call can be recorded into a CUDA graph and replayed. */
RT_API rt_status rt_batch_run(rt_batch* batch, rt_stream stream);
RT_API void rt_batch_free(rt_batch* batch);

/* Convenience: rt_batch_create + rt_batch_run + release (stream-ordered). */
RT_API rt_status rt_transport_batched(rt_ctx* ctx, const rt_opacity* opac, int n_models,
                               const rt_model* models, const rt_transport_params* p,
                               rt_stream stream);

/* ---------------------------------------------------------------------------
 * Diagnostics and test hooks.
 * ------------------------------------------------------------------------- */
/* Number of CUDA kernel launches this process has issued through the library
 * (all contexts, all threads), for launch accounting in benchmarks. */
RT_API uint64_t rt_kernel_launches(void);

/* Philox4x32-10 on the device: for i < n, out[4i..4i+3] = Philox(ctr_i, key)
 * with ctr_i = (ctr0[0] + i, ctr0[1], ctr0[2], ctr0[3]) (no carry; the caller
 * keeps ctr0[0] + n below 2^32).  out: device uint32 [4n]. */
RT_API rt_status rt_philox(rt_ctx* ctx, const uint32_t ctr0[4], const uint32_t key[2], uint64_t n,
                    uint32_t* out, rt_stream stream);

/* The modified random walk's path-length law as the FP32 transport draws it
 * (Sect. 3.2; Fleck & Canfield 1984): for i < n, y[i] is the dimensionless
 * first-passage time the FP32 kernel takes for the uniform u[i] in (0, 1] --
 * the y with S(y) = u, S(y) = 2 sum_{k>=1} (-1)^(k+1) exp(-k^2 pi^2 y) the
 * probability that a walker started at the centre of a sphere has not yet
 * reached its surface, interpolated in the opacity's FP32 table of S
 * (2048 nodes on 0 <= y <= 2; beyond, the one-term tail ln(2/u)/pi^2); the
 * path length of an MRW step is l = 3 chi R0^2 y.  u, y: device float [n].
 * Test hook: lets the FP32 draws be checked against the series. */
RT_API rt_status rt_mrw_sample(rt_ctx* ctx, const rt_opacity* opac, const float* u, uint64_t n,
                               float* y, rt_stream stream);

/* Memory-level probe (no counterpart in the paper): n_reads reads of one
 * 4-byte word each, at pseudo-random 32-byte sectors of buf[0, bytes),
 * spread over every SM (8 blocks of 256 threads each, four independent reads
 * in flight per thread), the access pattern of the transport's per-crossing
 * density gathers.  Timed by the caller (CUDA
 * events on `stream`), n_reads * 32 bytes over the time is the sector
 * bandwidth that the memory level holding the buffer serves to such gathers:
 * the L2 for a buffer well inside it, HBM for one far larger.  buf: device,
 * 32-byte aligned, bytes >= 32 (and below 128 GiB); sink: device uint64 or
 * NULL, incremented only on an impossible checksum (keeps the reads live).
 * Errors: RT_ERR_INVALID_ARG for a bad buffer. */
RT_API rt_status rt_probe_gather(rt_ctx* ctx, const void* buf, size_t bytes, uint64_t n_reads,
                                 uint32_t seed, unsigned long long* sink, rt_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* RTGB_H */
