// Internal declarations of librtgb: handle layouts, kernel parameter blocks
// and small device helpers shared by the CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rtgb.h"

namespace rtgb {

// ----------------------------------------------------------------- errors
void set_error(const std::string& msg);
rt_status fail(rt_status code, const std::string& msg);
rt_status cuda_fail(cudaError_t e, const char* what);
#define RT_CUDA(call)                                          \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return ::rtgb::cuda_fail(e_, #call); \
    } while (0)

// ----------------------------------------------------------------- sizes
constexpr int kMaxSpecies = 4;
constexpr int kMaxFreq = 1024;
constexpr int kTinvN = 4096;      // FP32 temperature-inverse table entries per species
constexpr int kTz64N = 65536;     // FP64 table of ln(4 pi P(T)) and its slope on a ln T grid
constexpr int kZinvN = 16384;     // FP32 table: ln T grid position on a uniform ln(4 pi P) grid
constexpr int kReT = 4096;        // FP32 re-emission CDF rows on a uniform log2 T grid, 0.1 K .. 1e6 K
constexpr int kMrwN = 2048;       // MRW survival table entries on y in [0, kMrwYmax]
constexpr double kMrwYmax = 2.0;
constexpr int kSedBins = 10;
constexpr int kParamModels = 64;  // model descriptors carried in the transport launch parameters
constexpr int kPcMax = 16;        // photon-counting cameras of one transport call
constexpr int kMaxImgFreq = 16;

// Node j of the linear-space temperature table on the uniform ln T grid:
// W = 4 pi P(T_j), m = dW/du (u = position within the interval, in units of
// the grid step h), T = T_j, g = 1 / (d ln W / du).
struct alignas(32) TwNode {
    double W, m, T, g;
};

}  // namespace rtgb

// ----------------------------------------------------------------- handles
struct rt_ctx {
    int magic;
    int device;
    int num_sms;
    unsigned long long* d_counters;   // scratch: work counters [64]
    // ray-tracer scratch, grown on demand and reused
    float* d_eta;  size_t eta_cap;    // [ncam][ncell][nfp]
    float* d_bk;   size_t bk_cap;     // [ns][ncell][nfp] kabs_s B_nu(T_s)
    double* d_red; size_t red_cap;    // reduction scratch
};

struct rt_opacity {
    rt_ctx* ctx;
    int nf, ns;
    uint64_t serial;
    std::vector<double> nu, dnu, kabs, ksca, g;
    std::vector<int> is_pah;
    // device tables
    double* d_nu; double* d_dnu;           // [nf]
    double* d_kabs; double* d_ksca; double* d_g;  // [ns][nf]
    float4* d_opac32;                      // [ns][nf] {kext, kabs, ksca, g}
    uint32_t* d_realias;                   // [2][ns][kReT][nf] re-emission alias tables:
                                           // [0] Eq. 5 (kabs B dnu), [1] Eq. 10 (kabs dB/dT dnu)
    float re_lg0, re_inv_dlg;              // row k at log2 T = re_lg0 + k / re_inv_dlg
    float* d_tinv;                         // [ns][kTinvN] log2 T on uniform log2(P) grid
    double2* d_tz;                         // [ns][kTz64N] {ln(4 pi P), d/dlnT} on uniform ln T
    double tz_lnT0, tz_dlnT;
    rtgb::TwNode* d_tw;                    // [ns][kTz64N] linear-space nodes (same ln T grid)
    float* d_zinv;                         // [ns][kZinvN] grid position (lnT - lnT0) / dlnT
    float zinv_z0[rtgb::kMaxSpecies], zinv_idz[rtgb::kMaxSpecies];
    int tw_ok[rtgb::kMaxSpecies];          // species has a finite, increasing table
    float tinv_y0[rtgb::kMaxSpecies], tinv_inv_dy[rtgb::kMaxSpecies];
    float* d_mrwS;                         // [kMrwN] survival S(y)
};

struct rt_grid {
    rt_ctx* ctx;
    int nx, ny, nz, ns;
    double box_min[3];
    double cell;
    float* d_rho;                          // [ns][ncell] as uploaded
    // packed per-cell layout with the Lucy flag in the sign bit of species 0
    void* d_packed;
    int packed_vec;                        // 1, 2 or 4 floats per cell
    uint64_t packed_opac_serial;
    int packed_lucy_mode;
    double packed_lucy_tau;
    int packed_prec;
    int rho_bad;                           // the last density update was refused
    unsigned int* d_flag;                  // device word for the density check of updates
    // one level of refinement (refine = r >= 2; 0 = uniform grid)
    int refine;
    size_t nleaf;                          // cells of a refined grid
    int* d_cube;                           // [ncube] first cell, kCubeDivided if divided
    int* d_leaf_cube;                      // [ncell] cube of each cell
    unsigned char* d_leaf_fine;            // [ncell] 1 = sub-cube
    // refined grids: [ncube] packed density of each undivided cube (the
    // packed layout; zero for divided cubes), rebuilt with every packing
    void* d_cube_packed;
    size_t ncube() const { return (size_t)nx * ny * nz; }
    size_t ncell() const { return refine ? nleaf : ncube(); }
};
constexpr int kCubeDivided = 1 << 30;      // flag in rt_grid::d_cube

// ----------------------------------------------------------------- kernel parameter blocks
namespace rtgb {

struct ModelDev {
    const void* rho;           // packed cells (float, float2 or float4)
    int nx, ny, nz;
    int ncell;                 // cells (nx * ny * nz, or the leaves of a refined grid)
    uint32_t model_id;
    int model_index;
    int nsrc;
    double cell, vol, xi;
    double log2_4piV;          // log2(4 pi V / cell) for the packed FP32 density rho*cell
    double box_min[3];
    uint64_t pid_begin;
    uint64_t n_emit;           // N of the model's emission (packet ids 0..N-1)
    const double* src_pos;     // [nsrc][3] in cell units
    const double* src_Lcdf;    // [nsrc] cumulative luminosity
    const double* src_cdf64;   // [nsrc][nf] cumulative L_nu dnu
    const float* src_cdf32;    // [nsrc][nf] cumulative, normalised to 1
    double* E_abs; uint32_t* count; double* esq;
    const int* cube;           // refined grids: [ncube] first cell | kCubeDivided
    const int* leaf_cube;      // refined grids: [ncell] cube of each cell
    const void* cube_rho;      // refined grids: [ncube] packed density of undivided cubes
    int refine;                // r, or 0
    double inv_refine;         // 1 / r (exact for the power-of-two factors)
    float inv_refine32;        // the same in FP32 (no FP64 conversion in the FP32 walk)
    double* accE;              // FP32 build: this call's deposits in units of xi (float
                               // sums in the plain-FP32 form); with
    int acc_q;                 // acc_q = 1 each cell holds {sum, sum of squares} (xi, xi^2)
    double* sed_esc; unsigned long long* sed_cnt;
    const double* T_prev;
    rt_event* events; uint64_t event_cap;
    rt_pah_event* pah; uint64_t pah_cap;
    rt_traj* traj; uint64_t traj_cap;
    unsigned long long* stats;
};

// A packet set aside by defer_events: enough state to restart it at the
// start of its next flight (positions and directions in the build's
// precision, stored as doubles).
struct alignas(16) DeferRec {
    double x[3], k[3];
    uint64_t pid;
    uint32_t cell, j, m, nev, seq, draw, c_lo, c_hi;
};
constexpr uint64_t kDeferCap = 1ull << 20;   // queue records per call

// A photon-counting camera in the grid's cell units: observer direction,
// image axes, acceptance cosine, pixels per cell length, and the offset of
// its [nf][npix][npix] image in the output.
struct PcDev {
    double kobs[3], ex[3], ey[3];
    double cos_accept, pix_per_cell, half_npix;
    int npix;
    unsigned long long off;
};

struct TransportKP {
    const ModelDev* models;
    const unsigned long long* prefix;   // [n_models + 1] work-index prefix
    int n_models;
    unsigned long long total_work;
    unsigned long long* work_ctr;
    int nf;
    int ns;                             // species of the opacity (<= the kernel's padded NS)
    int mode, lucy_form, mrw, record_events;
    uint32_t ev_mask[kMaxFreq / 32];    // frequency bins whose scattering events are stored
    int pah_mask;
    int march_min_active;
    int want_traj;                      // some model logs trajectories
    int single;                         // one model, with packed grid rho0
    const void* rho0;
    int param_models;                   // models whose descriptors are in mp (0: only in models)
    ModelDev mp[kParamModels];          // descriptors read from the launch parameters
    int smem_sed;                       // single-model persistent launch: SED tallied per block
    int smem_cdf;                       // floats of model 0's source CDFs kept in shared memory
    // dynamic shared-memory layout (byte offsets, set by the launcher)
    int so_sed, so_cnt, so_op, so_mrw, so_cdf, so_ctr, so_claim, so_stash;
    int compact_swap;                   // compaction: swap stopped lanes at <= this many marching
    unsigned long long max_events;
    unsigned long long source_bins;     // 0: random source bins; m: Eq. 1 equal-energy bins
    const int* sg_nu;                   // with source_bins: the separate source grid's model bin
    const int* sg_src;                  // and source of each source bin (device), or NULL
    unsigned long long defer_events;    // 0 = off
    DeferRec* defer;                    // queue (main pass appends, resume pass reads)
    unsigned long long* defer_n;        // queue cursor (device)
    unsigned long long defer_cap;
    int resume;                         // 1: packets come from the queue, not from emission
    // PAH re-emission pass (single-model calls): packet pid starts in the
    // cell of record pid, its bin drawn from the cell's emissivity class
    const rt_pah_event* pah_src;        // NULL: emission from the sources
    const double* eps_cdf64;            // [n_eps][nf] cumulative eps dnu
    const float* eps_cdf32;             // [n_eps][nf] cumulative, normalised to 1
    const int* eps_class;               // [ncell] or NULL (class 0)
    int n_eps;
    int refined;                        // the model's grid has one level of refinement
    int acc32;                          // FP32 per-cell accumulators (plain-FP32 form)
    int n_pc;                           // photon-counting cameras (single-model calls)
    double* pc_img;
    double pc_ctr[3];                   // grid centre, cell units
    PcDev pc[kPcMax];
    uint64_t seed;
    double mrw_tau_cell, mrw_gamma;
    // opacity tables
    const float4* opac32;
    const uint32_t* realias;            // [ns][kReT][nf] re-emission alias tables of the call's mode
    float re_lg0, re_inv_dlg;
    const float* tinv;
    float tinv_y0[kMaxSpecies], tinv_inv_dy[kMaxSpecies];
    const float* mrwS;
    const double* nu; const double* dnu;
    const double* kabs; const double* ksca; const double* g;
};

// ----------------------------------------------------------------- device helpers
#ifdef __CUDACC__
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw 2011): ten rounds, each with two
// 32x32 products whose halves are permuted and xored with the counter words
// and a Weyl-sequence key.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t a = 0xD2511F53u * c.x, ah = __umulhi(0xD2511F53u, c.x);
        const uint32_t b = 0xCD9E8D57u * c.z, bh = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(bh ^ c.y ^ k.x, b, ah ^ c.w ^ k.y, a);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// log2 of a positive double using only integer work and an FP32 log2 of the
// top 23 mantissa bits (GB300 has little FP64 throughput)
__device__ __forceinline__ float log2_d(double v)
{
    const unsigned hi = (unsigned)__double2hiint(v);
    const unsigned lo = (unsigned)__double2loint(v);
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023;
    const float m = __uint_as_float(0x3f800000u | ((hi & 0xfffffu) << 3) | (lo >> 29));
    return (float)e + __log2f(m);
}

// Exact float -> double by re-biasing the exponent with integer operations
// (no FP64 pipe); zero and denormal inputs give 0.
__device__ __forceinline__ double f2d(float f)
{
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xffu;
    if (e == 0u) return 0.0;
    const unsigned hi = (b & 0x80000000u) | ((e + (1023u - 127u)) << 20) | ((b & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)((b & 7u) << 29));
}

// MRW y from the survival table (FP32 path): S decreases on the uniform y
// grid; below the table the tail S ~ 2 exp(-pi^2 y) is exact to 1e-7.
__device__ __forceinline__ float mrw_y32(const float* S, float u)
{
    if (u >= 1.0f) return 0.0f;
    const float s_last = S[kMrwN - 1];
    if (u <= s_last) return logf(2.0f / u) * (float)(1.0 / (3.14159265358979323846 * 3.14159265358979323846));
    int lo = 0, hi = kMrwN - 1;               // S[lo] >= u > S[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (S[mid] >= u) lo = mid; else hi = mid;
    }
    const float a = S[lo], b = S[hi];
    const float w = (a - u) / fmaxf(a - b, 1e-30f);
    return ((float)lo + w) * (float)(kMrwYmax / (kMrwN - 1));
}

// Hardware reciprocal estimate of a double (a Newton step needs no more)
__device__ __forceinline__ double rcp_approx(double x)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    return r;
}
#endif

}  // namespace rtgb

// ----------------------------------------------------------------- cross-TU host entry points
namespace rtgb {
rt_status build_opacity_tables(rt_opacity* op);
rt_status build_source_grid(const rt_opacity* op, const rt_source* src, int nsrc, uint32_t m,
                            int32_t* nu_idx, int32_t* src_idx, double* nu_star);
rt_status pack_grid(rt_grid* g, const rt_opacity* op, int lucy_mode, double lucy_tau, int prec,
                    cudaStream_t s);
rt_status pack_grid_into(const rt_grid* g, const rt_opacity* op, int lucy_mode, double lucy_tau,
                         int prec, double* kext, void* dst, void* cube_dst, cudaStream_t s);
rt_status visibilities_impl(rt_ctx* ctx, const rt_grid* g, const rt_camera* cams, int ncam,
                            const float* images, int nf, const double* uv, int nuv, double* vis,
                            cudaStream_t s);
template <int NS>
rt_status launch_transport_ns(rt_ctx* ctx, const TransportKP& kp, int prec, int schedule, int threads,
                              int blocks_per_sm, cudaStream_t s);
rt_status launch_transport(rt_ctx* ctx, const rt_opacity* op, const TransportKP& kp,
                           int ns, int prec, int schedule, int threads, int blocks_per_sm,
                           cudaStream_t s);
rt_status launch_finalize(const double* acc, int acc_q, size_t n, double xi, double* E_abs,
                          double* esq, cudaStream_t s);
rt_status launch_finalize32(const float* acc, int acc_q, size_t n, double xi, double* E_abs,
                            double* esq, cudaStream_t s);
rt_status launch_seed(double* acc, int acc_q, size_t n, double xi, const double* E_abs,
                      cudaStream_t s);
rt_status launch_temperatures(rt_ctx* ctx, const rt_grid* g, const rt_opacity* op,
                              const double* E, double* T, cudaStream_t s);
rt_status launch_temperature_guess(rt_ctx* ctx, const rt_grid* g, const double* src_pos,
                                   const double* src_L, int nsrc, double* T, cudaStream_t s);
rt_status raytrace_impl(rt_ctx* ctx, const rt_grid* g, const rt_opacity* op, const double* T,
                        const rt_event* ev, uint64_t nev, const uint64_t* nev_dev, double xi_ev,
                        const rt_source* src, int nsrc, const rt_camera* cams, int ncam, const int* fidx, int nfi,
                        float* images, double* sed, const float* dimg, const double* dsed,
                        float* drho, double* dscale, unsigned long long* ray_steps, bool backward,
                        cudaStream_t s);
rt_status launch_philox(const uint32_t ctr0[4], const uint32_t key[2], uint64_t n, uint32_t* out,
                        cudaStream_t s);
rt_status launch_mrw_sample(const float* table, const float* u, uint64_t n, float* y, cudaStream_t s);
rt_status launch_gather_probe(int num_sms, const void* buf, size_t bytes, uint64_t n_reads, uint32_t seed,
                              unsigned long long* sink, cudaStream_t s);
// launch accounting (rt_kernel_launches)
void count_launches(unsigned n = 1);
// host helpers
double planck_B_host(double nu, double T);
void source_spectrum(const rt_opacity* op, const rt_source& src, std::vector<double>& lnu);
}  // namespace rtgb
