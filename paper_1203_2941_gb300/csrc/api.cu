// C ABI of librtgb: handles, argument validation, per-call model tables and
// launches.  Every computation of the method runs in the kernels of
// transport.cu, temperature.cu and raytrace.cu; this file only marshals.
#include <math.h>

#include <atomic>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "rt_internal.cuh"

namespace rtgb {

static thread_local std::string g_err;
static std::atomic<uint64_t> g_serial{1};
static std::atomic<uint64_t> g_launches{0};

void count_launches(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
static const int kMagic = 0x72746762;   // "rtgb"

void set_error(const std::string& msg) { g_err = msg; }

rt_status fail(rt_status code, const std::string& msg)
{
    g_err = msg;
    return code;
}

rt_status cuda_fail(cudaError_t e, const char* what)
{
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA;
}

static bool isfin(double v) { return std::isfinite(v); }

__global__ void check_rho_kernel(const float* rho, size_t n, unsigned int* bad)
{
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) {
        const float v = rho[i];
        if (!(v >= 0.0f) || !isfinite(v)) atomicOr(bad, 1u);
    }
}

}  // namespace rtgb

using namespace rtgb;

extern "C" {

const char* rt_last_error(void) { return g_err.c_str(); }
const char* rt_version(void) { return "rtgb 0.1 (sm_103a)"; }
uint64_t rt_kernel_launches(void) { return g_launches.load(); }

rt_status rt_ctx_create(int device, rt_ctx** out)
{
    if (!out) return fail(RT_ERR_INVALID_ARG, "rt_ctx_create: out is NULL");
    int n = 0;
    RT_CUDA(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return fail(RT_ERR_INVALID_ARG, "rt_ctx_create: no such device");
    RT_CUDA(cudaSetDevice(device));
    rt_ctx* c = new rt_ctx();
    std::memset(c, 0, sizeof(*c));
    c->magic = kMagic;
    c->device = device;
    cudaError_t e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) { delete c; return cuda_fail(e, "cudaDeviceGetAttribute"); }
    e = cudaMalloc(&c->d_counters, 64 * sizeof(unsigned long long));
    if (e != cudaSuccess) { delete c; return cuda_fail(e, "cudaMalloc(counters)"); }
    *out = c;
    return RT_OK;
}

void rt_ctx_destroy(rt_ctx* c)
{
    if (!c || c->magic != kMagic) return;
    cudaSetDevice(c->device);
    cudaFree(c->d_counters);
    cudaFree(c->d_eta);
    cudaFree(c->d_bk);
    cudaFree(c->d_red);
    c->magic = 0;
    delete c;
}

rt_status rt_grid_upload(rt_ctx* ctx, int nx, int ny, int nz, int ns, const double box_min[3],
                         double cell, const float* rho, rt_stream stream, rt_grid** out)
{
    return rt_grid_upload_refined(ctx, nx, ny, nz, ns, box_min, cell, 0, nullptr, rho, stream, out);
}

uint64_t rt_grid_ncell(const rt_grid* g) { return g ? (uint64_t)g->ncell() : 0; }

rt_status rt_grid_upload_refined(rt_ctx* ctx, int nx, int ny, int nz, int ns, const double box_min[3],
                                 double cell, int refine, const unsigned char* refined,
                                 const float* rho, rt_stream stream, rt_grid** out)
{
    if (!ctx || ctx->magic != kMagic) return fail(RT_ERR_STATE, "rt_grid_upload: bad context");
    if (!out || !rho || !box_min) return fail(RT_ERR_INVALID_ARG, "rt_grid_upload: NULL pointer");
    if (nx <= 0 || ny <= 0 || nz <= 0) return fail(RT_ERR_INVALID_ARG, "rt_grid_upload: sizes must be positive");
    if ((double)nx * ny * nz > 2.0e9) return fail(RT_ERR_INVALID_ARG, "rt_grid_upload: more than 2e9 cells");
    if (ns < 1 || ns > kMaxSpecies) return fail(RT_ERR_INVALID_ARG, "rt_grid_upload: n_species must be 1..4");
    if (!(cell > 0.0) || !isfin(cell)) return fail(RT_ERR_INVALID_ARG, "rt_grid_upload: bad cell size");
    for (int a = 0; a < 3; ++a)
        if (!isfin(box_min[a])) return fail(RT_ERR_INVALID_ARG, "rt_grid_upload: non-finite box_min");
    if (refine != 0 && (refine < 2 || refine > 16 || !refined))
        return fail(RT_ERR_INVALID_ARG, "rt_grid_upload_refined: refine must be 2..16 with a refined mask");
    // one level of refinement: first cell of every cube, cube of every cell
    const size_t ncube = (size_t)nx * ny * nz;
    std::vector<int> cube, leaf_cube;
    std::vector<unsigned char> leaf_fine;
    size_t nleaf = ncube;
    if (refine) {
        const size_t r3 = (size_t)refine * refine * refine;
        nleaf = 0;
        for (size_t c = 0; c < ncube; ++c) nleaf += refined[c] ? r3 : 1;
        if ((double)nleaf > 2.0e9 || nleaf >= (size_t)kCubeDivided)
            return fail(RT_ERR_INVALID_ARG, "rt_grid_upload_refined: 2^30 cells or more");
        cube.resize(ncube);
        leaf_cube.resize(nleaf);
        leaf_fine.resize(nleaf);
        size_t b = 0;
        for (size_t c = 0; c < ncube; ++c) {
            const size_t m = refined[c] ? r3 : 1;
            cube[c] = (int)b | (refined[c] ? kCubeDivided : 0);
            for (size_t q = 0; q < m; ++q) {
                leaf_cube[b + q] = (int)c;
                leaf_fine[b + q] = refined[c] ? 1 : 0;
            }
            b += m;
        }
    }
    RT_CUDA(cudaSetDevice(ctx->device));
    rt_grid* g = new rt_grid();
    std::memset((void*)g, 0, sizeof(*g));
    g->ctx = ctx; g->nx = nx; g->ny = ny; g->nz = nz; g->ns = ns; g->cell = cell;
    for (int a = 0; a < 3; ++a) g->box_min[a] = box_min[a];
    g->refine = refine;
    g->nleaf = nleaf;
    const size_t n = g->ncell() * ns;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned int* bad = nullptr;
    cudaError_t e = cudaSuccess;
    if (refine) {
        e = cudaMalloc(&g->d_cube, ncube * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&g->d_leaf_cube, nleaf * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&g->d_leaf_fine, nleaf);
        if (e == cudaSuccess) e = cudaMemcpy(g->d_cube, cube.data(), ncube * sizeof(int), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(g->d_leaf_cube, leaf_cube.data(), nleaf * sizeof(int), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(g->d_leaf_fine, leaf_fine.data(), nleaf, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(g->d_cube); cudaFree(g->d_leaf_cube); cudaFree(g->d_leaf_fine);
            delete g;
            return cuda_fail(e, "rt_grid_upload_refined tables");
        }
    }
    e = cudaMalloc(&g->d_rho, n * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->d_rho, rho, n * sizeof(float), cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&bad, sizeof(unsigned int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(unsigned int), s);
    if (e == cudaSuccess) {
        check_rho_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g->d_rho, n, bad);
        count_launches();
        e = cudaGetLastError();
    }
    unsigned int hbad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
    if (bad) cudaFreeAsync(bad, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(g->d_rho); cudaFree(g->d_cube); cudaFree(g->d_leaf_cube); cudaFree(g->d_leaf_fine);
        delete g;
        return cuda_fail(e, "rt_grid_upload");
    }
    if (hbad) {
        cudaFree(g->d_rho); cudaFree(g->d_cube); cudaFree(g->d_leaf_cube); cudaFree(g->d_leaf_fine);
        delete g;
        return fail(RT_ERR_INVALID_ARG, "rt_grid_upload: density must be finite and >= 0");
    }
    *out = g;
    return RT_OK;
}

rt_status rt_grid_update(rt_grid* g, const float* rho, rt_stream stream)
{
    if (!g || !rho) return fail(RT_ERR_INVALID_ARG, "rt_grid_update: NULL pointer");
    rt_ctx* ctx = g->ctx;
    if (!ctx || ctx->magic != kMagic) return fail(RT_ERR_STATE, "rt_grid_update: bad context");
    RT_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = g->ncell() * g->ns;
    if (!g->d_flag) RT_CUDA(cudaMalloc(&g->d_flag, sizeof(unsigned int)));
    unsigned int* bad = g->d_flag;
    g->rho_bad = 1;                          // until the new values are checked
    g->packed_prec = -1;                     // the packed copy is stale: repacked on next use
    cudaError_t e = cudaMemcpyAsync(g->d_rho, rho, n * sizeof(float), cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(unsigned int), s);
    if (e == cudaSuccess) {
        check_rho_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g->d_rho, n, bad);
        count_launches();
        e = cudaGetLastError();
    }
    unsigned int hbad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "rt_grid_update");
    if (hbad) return fail(RT_ERR_INVALID_ARG, "rt_grid_update: density must be finite and >= 0");
    g->rho_bad = 0;
    return RT_OK;
}

void rt_grid_free(rt_grid* g)
{
    if (!g) return;
    cudaSetDevice(g->ctx->device);
    cudaFree(g->d_rho);
    cudaFree(g->d_packed);
    cudaFree(g->d_cube);
    cudaFree(g->d_leaf_cube);
    cudaFree(g->d_leaf_fine);
    cudaFree(g->d_cube_packed);
    cudaFree(g->d_flag);
    delete g;
}

rt_status rt_opacity_upload(rt_ctx* ctx, int nf, const double* nu, const double* dnu, int ns,
                            const double* kabs, const double* ksca, const double* g,
                            const int* is_pah, rt_opacity** out)
{
    if (!ctx || ctx->magic != kMagic) return fail(RT_ERR_STATE, "rt_opacity_upload: bad context");
    if (!out || !nu || !dnu || !kabs || !ksca || !g)
        return fail(RT_ERR_INVALID_ARG, "rt_opacity_upload: NULL pointer");
    if (nf < 2 || nf > kMaxFreq) return fail(RT_ERR_INVALID_ARG, "rt_opacity_upload: n_freq must be 2..1024");
    if (ns < 1 || ns > kMaxSpecies) return fail(RT_ERR_INVALID_ARG, "rt_opacity_upload: n_species must be 1..4");
    for (int j = 0; j < nf; ++j) {
        if (!(nu[j] > 0.0) || !isfin(nu[j]) || !(dnu[j] > 0.0) || !isfin(dnu[j]))
            return fail(RT_ERR_INVALID_ARG, "rt_opacity_upload: nu and dnu must be positive and finite");
        if (j > 0 && !(nu[j] > nu[j - 1]))
            return fail(RT_ERR_INVALID_ARG, "rt_opacity_upload: nu must be strictly ascending");
    }
    for (int i = 0; i < ns * nf; ++i) {
        if (!(kabs[i] >= 0.0) || !(ksca[i] >= 0.0) || !isfin(kabs[i]) || !isfin(ksca[i]))
            return fail(RT_ERR_INVALID_ARG, "rt_opacity_upload: kappa must be finite and >= 0");
        if (!(fabs(g[i]) < 1.0)) return fail(RT_ERR_INVALID_ARG, "rt_opacity_upload: |g| must be < 1");
    }
    RT_CUDA(cudaSetDevice(ctx->device));
    rt_opacity* op = new rt_opacity();
    op->ctx = ctx; op->nf = nf; op->ns = ns;
    op->serial = g_serial.fetch_add(1);
    op->nu.assign(nu, nu + nf);
    op->dnu.assign(dnu, dnu + nf);
    op->kabs.assign(kabs, kabs + ns * nf);
    op->ksca.assign(ksca, ksca + ns * nf);
    op->g.assign(g, g + ns * nf);
    op->is_pah.assign(ns, 0);
    if (is_pah)
        for (int s = 0; s < ns; ++s) op->is_pah[s] = is_pah[s] != 0;
    rt_status st = build_opacity_tables(op);
    if (st != RT_OK) {
        rt_opacity_free(op);
        return st;
    }
    *out = op;
    return RT_OK;
}

void rt_opacity_free(rt_opacity* op)
{
    if (!op) return;
    cudaSetDevice(op->ctx->device);
    cudaFree(op->d_nu); cudaFree(op->d_dnu); cudaFree(op->d_kabs); cudaFree(op->d_ksca);
    cudaFree(op->d_g); cudaFree(op->d_opac32); cudaFree(op->d_realias);
    cudaFree(op->d_tinv); cudaFree(op->d_tz); cudaFree(op->d_tw); cudaFree(op->d_zinv); cudaFree(op->d_mrwS);
    delete op;
}

void rt_transport_params_default(rt_transport_params* p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->mode = RT_MODE_BW;
    p->lucy_mode = RT_LUCY_THIN;
    p->lucy_form = RT_LUCY_LINEAR;
    p->lucy_tau = 1e-2;
    p->mrw = 0;
    p->mrw_tau_cell = 10.0;
    p->mrw_gamma = 2.0;
    p->seed = 1;
    p->model_id = 0;
    p->n_packets = 0;
    p->pid_begin = 0;
    p->pid_end = 0;
    p->max_events = 10000000ull;
    p->record_events = 0;
    p->precision = RT_PREC_FP32;
    p->schedule = RT_SCHED_PERSISTENT;
    p->threads_per_block = 0;
    p->blocks_per_sm = 0;
    p->march_min_active = -1;
    p->defer_events = 0;
    p->source_bins = 0;
    p->compact_swap = -1;
}

}  // extern "C"

namespace rtgb {

static rt_status check_params(const rt_transport_params* p)
{
    if (!p) return fail(RT_ERR_INVALID_ARG, "transport: params is NULL");
    if (p->mode < RT_MODE_BW || p->mode > RT_MODE_NOREEMIT) return fail(RT_ERR_INVALID_ARG, "transport: bad mode");
    if (p->lucy_mode < RT_LUCY_OFF || p->lucy_mode > RT_LUCY_ALL) return fail(RT_ERR_INVALID_ARG, "transport: bad lucy_mode");
    if (p->lucy_form != RT_LUCY_LINEAR && p->lucy_form != RT_LUCY_EXPM1) return fail(RT_ERR_INVALID_ARG, "transport: bad lucy_form");
    if (!(p->lucy_tau >= 0.0) || !isfin(p->lucy_tau)) return fail(RT_ERR_INVALID_ARG, "transport: bad lucy_tau");
    if (p->mrw && (!(p->mrw_tau_cell > 0.0) || !(p->mrw_gamma > 0.0)))
        return fail(RT_ERR_INVALID_ARG, "transport: MRW thresholds must be positive");
    if (p->precision != RT_PREC_FP32 && p->precision != RT_PREC_FP64 && p->precision != RT_PREC_FP32_ACC32)
        return fail(RT_ERR_INVALID_ARG, "transport: bad precision");
    if (p->schedule != RT_SCHED_PERSISTENT && p->schedule != RT_SCHED_SERIAL && p->schedule != RT_SCHED_COMPACT)
        return fail(RT_ERR_INVALID_ARG, "transport: bad schedule");
    if (p->compact_swap < -1 || p->compact_swap > 31) return fail(RT_ERR_INVALID_ARG, "transport: compact_swap must be -1..31");
    if (p->n_packets == 0) return fail(RT_ERR_INVALID_ARG, "transport: n_packets must be > 0");
    if (p->march_min_active < -1 || p->march_min_active > 31) return fail(RT_ERR_INVALID_ARG, "transport: march_min_active must be -1..31");
    if (p->threads_per_block != 0 && (p->threads_per_block % 32 != 0 || p->threads_per_block > 256 || p->threads_per_block < 32))
        return fail(RT_ERR_INVALID_ARG, "transport: threads_per_block must be a multiple of 32 in 32..256");
    if (p->blocks_per_sm < 0 || p->blocks_per_sm > 64) return fail(RT_ERR_INVALID_ARG, "transport: blocks_per_sm must be 0..64");
    if (p->max_events == 0) return fail(RT_ERR_INVALID_ARG, "transport: max_events must be > 0");
    if (p->source_bins > 0 && ((double)p->source_bins > (double)p->n_packets ||
                               (double)p->source_bins * (double)p->n_packets > 9.0e18))
        return fail(RT_ERR_INVALID_ARG, "transport: source_bins must be <= n_packets with n_packets * source_bins < 9e18");
    if (p->n_pc_cams < 0 || p->n_pc_cams > kPcMax)
        return fail(RT_ERR_INVALID_ARG, "transport: n_pc_cams must be 0..16");
    if (p->n_pc_cams > 0 && !p->pc_cams) return fail(RT_ERR_INVALID_ARG, "transport: pc_cams is NULL");
    for (int c = 0; c < p->n_pc_cams; ++c) {
        const rt_pc_camera& q = p->pc_cams[c];
        if (q.npix < 1 || q.npix > 4096 || !isfin(q.theta) || !isfin(q.phi) || !(q.pixel >= 0.0) ||
            !isfin(q.pixel) || !(q.cos_accept >= -1.0 && q.cos_accept <= 1.0))
            return fail(RT_ERR_INVALID_ARG, "transport: photon-counting camera needs npix 1..4096, finite angles, "
                                            "pixel >= 0 and cos_accept in [-1, 1]");
    }
    return RT_OK;
}

// Photon-counting cameras of a single-model call: frames in cell units, in
// the launch parameters.
static void fill_pc(TransportKP& kp, const rt_grid* g, const rt_transport_params* p,
                    const rt_transport_out* out)
{
    kp.n_pc = p->n_pc_cams;
    kp.pc_img = out->pc_img;
    const double n[3] = { (double)g->nx, (double)g->ny, (double)g->nz };
    for (int a = 0; a < 3; ++a) kp.pc_ctr[a] = 0.5 * n[a];
    unsigned long long off = 0;
    for (int c = 0; c < p->n_pc_cams; ++c) {
        const rt_pc_camera& q = p->pc_cams[c];
        PcDev& d = kp.pc[c];
        const double st = std::sin(q.theta), ct = std::cos(q.theta);
        const double sp = std::sin(q.phi), cp = std::cos(q.phi);
        d.kobs[0] = st * cp; d.kobs[1] = st * sp; d.kobs[2] = ct;
        d.ex[0] = -sp; d.ex[1] = cp; d.ex[2] = 0.0;
        d.ey[0] = -ct * cp; d.ey[1] = -ct * sp; d.ey[2] = st;
        const double pix = q.pixel > 0.0
            ? q.pixel
            : g->cell * std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]) / q.npix;
        d.cos_accept = q.cos_accept;
        d.pix_per_cell = g->cell / pix;
        d.half_npix = 0.5 * q.npix;
        d.npix = q.npix;
        d.off = off;
        off += (unsigned long long)kp.nf * q.npix * q.npix;
    }
}

static rt_status check_out(const rt_transport_out* o)
{
    if (!o) return fail(RT_ERR_INVALID_ARG, "transport: out is NULL");
    if (!o->E_abs || !o->count || !o->sed_esc || !o->sed_cnt || !o->stats)
        return fail(RT_ERR_INVALID_ARG, "transport: E_abs, count, sed_esc, sed_cnt and stats are required");
    if ((o->event_cap && !o->events) || (o->pah_cap && !o->pah) || (o->traj_cap && !o->traj))
        return fail(RT_ERR_INVALID_ARG, "transport: buffer with capacity but NULL pointer");
    return RT_OK;
}

// Host-side staging of one model: its descriptor and source tables.
struct HostModel {
    ModelDev md;
    std::vector<double> pos, Lcdf, cdf64;
    std::vector<float> cdf32;
};

// xi_fixed > 0: a pass without sources (PAH re-emission) whose packets carry
// that energy; otherwise xi = L / n_packets of the 1..64 sources.
static rt_status make_model(const rt_grid* g, const rt_opacity* op, const rt_source* src, int nsrc,
                            uint64_t n_packets, uint64_t pid_begin, uint32_t model_id, int model_index,
                            const double* T_prev, const rt_transport_out* o, HostModel& hm,
                            double xi_fixed = 0.0)
{
    if (xi_fixed > 0.0) nsrc = 0;
    else if (!src || nsrc < 1 || nsrc > 64) return fail(RT_ERR_INVALID_ARG, "transport: need 1..64 sources");
    const int nf = op->nf;
    double Ltot = 0.0;
    hm.pos.resize(3 * nsrc);
    hm.Lcdf.resize(nsrc);
    hm.cdf64.resize((size_t)nsrc * nf);
    hm.cdf32.resize((size_t)nsrc * nf);
    std::vector<double> lnu;
    const double hi[3] = { g->box_min[0] + g->nx * g->cell, g->box_min[1] + g->ny * g->cell,
                           g->box_min[2] + g->nz * g->cell };
    for (int i = 0; i < nsrc; ++i) {
        const rt_source& s = src[i];
        if (!(s.L >= 0.0) || !isfin(s.L)) return fail(RT_ERR_INVALID_ARG, "transport: source L must be >= 0");
        if (!s.L_nu && !(s.T_eff > 0.0)) return fail(RT_ERR_INVALID_ARG, "transport: blackbody source needs T_eff > 0");
        if (s.L_nu)
            for (int j = 0; j < nf; ++j)
                if (!(s.L_nu[j] >= 0.0) || !isfin(s.L_nu[j]))
                    return fail(RT_ERR_INVALID_ARG, "transport: L_nu must be finite and >= 0");
        for (int a = 0; a < 3; ++a) {
            if (!(s.pos[a] >= g->box_min[a] && s.pos[a] <= hi[a]))
                return fail(RT_ERR_INVALID_ARG, "transport: sources must lie inside the grid");
            hm.pos[3 * i + a] = (s.pos[a] - g->box_min[a]) / g->cell;
        }
        source_spectrum(op, s, lnu);
        double acc = 0.0;
        for (int j = 0; j < nf; ++j) {
            acc += lnu[j] * op->dnu[j];
            hm.cdf64[(size_t)i * nf + j] = acc;
        }
        if (!(acc > 0.0) && s.L > 0.0) return fail(RT_ERR_INVALID_ARG, "transport: source spectrum is zero on the grid");
        for (int j = 0; j < nf; ++j)
            hm.cdf32[(size_t)i * nf + j] = acc > 0.0 ? (float)(hm.cdf64[(size_t)i * nf + j] / acc) : 1.0f;
        hm.cdf32[(size_t)i * nf + nf - 1] = 1.0f;
        Ltot += s.L;
        hm.Lcdf[i] = Ltot;
    }
    if (!(Ltot > 0.0) && !(xi_fixed > 0.0)) return fail(RT_ERR_INVALID_ARG, "transport: total luminosity must be > 0");
    ModelDev& m = hm.md;
    std::memset(&m, 0, sizeof(m));
    m.rho = g->d_packed;
    m.nx = g->nx; m.ny = g->ny; m.nz = g->nz;
    m.ncell = (int)g->ncell();
    m.refine = g->refine;
    m.inv_refine = g->refine ? 1.0 / g->refine : 1.0;
    m.inv_refine32 = (float)m.inv_refine;
    m.cube = g->d_cube;
    m.leaf_cube = g->d_leaf_cube;
    m.cube_rho = g->d_cube_packed;
    m.model_id = model_id;
    m.model_index = model_index;
    m.nsrc = nsrc;
    m.cell = g->cell;
    m.vol = g->cell * g->cell * g->cell;
    m.xi = xi_fixed > 0.0 ? xi_fixed : Ltot / (double)n_packets;
    m.log2_4piV = 2.0 * log2(g->cell);
    for (int a = 0; a < 3; ++a) m.box_min[a] = g->box_min[a];
    m.pid_begin = pid_begin;
    m.n_emit = n_packets;
    m.E_abs = o->E_abs; m.count = o->count; m.esq = o->esq;
    m.sed_esc = o->sed_esc; m.sed_cnt = (unsigned long long*)o->sed_cnt;
    m.T_prev = T_prev;
    m.events = o->events; m.event_cap = o->event_cap;
    m.pah = o->pah; m.pah_cap = o->pah_cap;
    m.traj = o->traj; m.traj_cap = o->traj_cap;
    m.stats = (unsigned long long*)o->stats;
    return RT_OK;
}

// Device image of a set of models: descriptors, prefix sums and source tables
// in one allocation.
struct DeviceModels {
    void* buf = nullptr;
    size_t bytes = 0;
    ModelDev* models = nullptr;
    unsigned long long* prefix = nullptr;
    unsigned long long* work = nullptr;
    unsigned long long total = 0;
};

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

static rt_status stage_models(std::vector<HostModel>& hms, const std::vector<uint64_t>& nwork,
                              int nf, bool async, cudaStream_t s, DeviceModels& dm)
{
    const int n = (int)hms.size();
    size_t off = 0;
    const size_t o_models = off; off = align_up(off + sizeof(ModelDev) * n, 64);
    const size_t o_prefix = off; off = align_up(off + sizeof(unsigned long long) * (n + 1), 64);
    const size_t o_work = off; off = align_up(off + sizeof(unsigned long long) * 2, 64);
    std::vector<size_t> o_pos(n), o_L(n), o_c64(n), o_c32(n);
    for (int i = 0; i < n; ++i) {
        const int ns_ = hms[i].md.nsrc;
        o_pos[i] = off; off = align_up(off + sizeof(double) * 3 * ns_, 64);
        o_L[i] = off; off = align_up(off + sizeof(double) * ns_, 64);
        o_c64[i] = off; off = align_up(off + sizeof(double) * ns_ * nf, 64);
        o_c32[i] = off; off = align_up(off + sizeof(float) * ns_ * nf, 64);
    }
    std::vector<unsigned char> h(off, 0);
    std::vector<unsigned long long> prefix(n + 1, 0);
    for (int i = 0; i < n; ++i) prefix[i + 1] = prefix[i] + nwork[i];
    char* base = nullptr;
    if (async) RT_CUDA(cudaMallocAsync((void**)&base, off, s));
    else RT_CUDA(cudaMalloc((void**)&base, off));
    for (int i = 0; i < n; ++i) {
        ModelDev md = hms[i].md;
        std::memcpy(&h[o_pos[i]], hms[i].pos.data(), sizeof(double) * hms[i].pos.size());
        std::memcpy(&h[o_L[i]], hms[i].Lcdf.data(), sizeof(double) * hms[i].Lcdf.size());
        std::memcpy(&h[o_c64[i]], hms[i].cdf64.data(), sizeof(double) * hms[i].cdf64.size());
        std::memcpy(&h[o_c32[i]], hms[i].cdf32.data(), sizeof(float) * hms[i].cdf32.size());
        md.src_pos = (const double*)(base + o_pos[i]);
        md.src_Lcdf = (const double*)(base + o_L[i]);
        md.src_cdf64 = (const double*)(base + o_c64[i]);
        md.src_cdf32 = (const float*)(base + o_c32[i]);
        std::memcpy(&h[o_models + sizeof(ModelDev) * i], &md, sizeof(ModelDev));
        hms[i].md = md;                // the host copy now matches the device one
    }
    std::memcpy(&h[o_prefix], prefix.data(), sizeof(unsigned long long) * (n + 1));
    if (async) {
        cudaError_t e = cudaMemcpyAsync(base, h.data(), off, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) { cudaFreeAsync(base, s); return cuda_fail(e, "stage models"); }
    } else {
        cudaError_t e = cudaMemcpy(base, h.data(), off, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { cudaFree(base); return cuda_fail(e, "stage models"); }
    }
    dm.buf = base;
    dm.bytes = off;
    dm.models = (ModelDev*)(base + o_models);
    dm.prefix = (unsigned long long*)(base + o_prefix);
    dm.work = (unsigned long long*)(base + o_work);
    dm.total = prefix[n];
    return RT_OK;
}

static void fill_kp(TransportKP& kp, const rt_opacity* op, const rt_transport_params* p,
                    const DeviceModels& dm, int n_models)
{
    std::memset(&kp, 0, sizeof(kp));
    kp.models = dm.models;
    kp.prefix = dm.prefix;
    kp.n_models = n_models;
    kp.total_work = dm.total;
    kp.work_ctr = dm.work;
    kp.nf = op->nf;
    kp.mode = p->mode;
    kp.lucy_form = p->lucy_form;
    kp.mrw = p->mrw;
    kp.record_events = p->record_events;
    for (int w = 0; w < kMaxFreq / 32; ++w) {
        uint32_t bits = 0u;
        for (int b = 0; b < 32; ++b) {
            const int j = 32 * w + b;
            if (j < op->nf && (!p->record_nu_mask || ((p->record_nu_mask[j / 32] >> (j % 32)) & 1u)))
                bits |= 1u << b;
        }
        kp.ev_mask[w] = bits;
    }
    kp.pah_mask = 0;
    for (int s = 0; s < op->ns; ++s)
        if (op->is_pah[s]) kp.pah_mask |= 1 << s;
    kp.march_min_active = p->march_min_active < 0 ? 16 : p->march_min_active;
    kp.compact_swap = p->compact_swap < 0 ? 24 : p->compact_swap;
    kp.want_traj = 0;
    kp.single = 0;
    kp.rho0 = nullptr;
    kp.param_models = 0;
    kp.smem_sed = 0;
    kp.smem_cdf = 0;
    kp.max_events = p->max_events;
    kp.source_bins = p->source_bins;
    kp.sg_nu = nullptr;                // set by rt_transport for a separate source grid
    kp.sg_src = nullptr;
    kp.defer_events = 0;               // set by rt_transport when it allocates a queue
    kp.defer = nullptr;
    kp.defer_n = nullptr;
    kp.defer_cap = 0;
    kp.resume = 0;
    kp.seed = p->seed;
    kp.mrw_tau_cell = p->mrw_tau_cell;
    kp.mrw_gamma = p->mrw_gamma;
    kp.ns = op->ns;
    kp.opac32 = op->d_opac32;
    kp.realias = op->d_realias + (p->mode == RT_MODE_BW ? (size_t)op->ns * kReT * op->nf : 0);
    kp.re_lg0 = op->re_lg0;
    kp.re_inv_dlg = op->re_inv_dlg;
    kp.tinv = op->d_tinv;
    for (int s = 0; s < kMaxSpecies; ++s) {
        kp.tinv_y0[s] = s < op->ns ? op->tinv_y0[s] : 0.0f;
        kp.tinv_inv_dy[s] = s < op->ns ? op->tinv_inv_dy[s] : 0.0f;
    }
    kp.mrwS = op->d_mrwS;
    kp.nu = op->d_nu; kp.dnu = op->d_dnu;
    kp.kabs = op->d_kabs; kp.ksca = op->d_ksca; kp.g = op->d_g;
}

// Shared-memory options of a single-model launch: per-block escape SED (the
// 10 x nf tallies otherwise take heavily contended global atomics) and the
// source CDFs; trajectory logging selects the kernel variant that has it.
static rt_status single_model_options(TransportKP& kp, const rt_opacity* op,
                                      const rt_transport_params* p, const rt_transport_out* out,
                                      int n_sources, const ModelDev& m0)
{
    // the kernel reads this descriptor from its launch parameters: it must
    // be the staged one, with every device table in place
    if (!m0.rho || !m0.src_pos || !m0.src_Lcdf || !m0.src_cdf64 || !m0.src_cdf32 || !m0.stats)
        return fail(RT_ERR_STATE, "transport: model descriptor not staged");
    kp.want_traj = out->traj != nullptr && out->traj_cap > 0;
    kp.single = 1;
    kp.rho0 = m0.rho;
    kp.param_models = 1;
    kp.mp[0] = m0;
    const bool persistent = p->schedule != RT_SCHED_SERIAL && p->precision != RT_PREC_FP64;
    kp.smem_sed = persistent && op->nf <= 256 ? 1 : 0;
    kp.smem_cdf = persistent && n_sources * op->nf <= 4096 ? n_sources * op->nf : 0;
    return RT_OK;
}

// The stored absorptions and emissivity classes of a PAH re-emission pass.
struct PahPass {
    const rt_pah_event* rec;
    uint64_t n_rec;
    double xi;
    const double* eps;
    int n_eps;
    const int* eps_class;
};

static rt_status transport_one(rt_ctx* ctx, const rt_grid* grid, const rt_opacity* op,
                               const rt_source* sources, int n_sources, const rt_transport_params* p,
                               const double* T_prev, const rt_transport_out* out, cudaStream_t s,
                               const PahPass* pp);

}  // namespace rtgb

struct rt_batch {
    rt_ctx* ctx;
    const rt_opacity* op;
    rt_transport_params p;
    int n_models, ns;
    DeviceModels dm;
    TransportKP kp;
    double* acc;                       // FP32 build scratch for all models
    size_t acc_bytes;
    std::vector<rtgb::ModelDev> host;  // per-model descriptors (finalize arguments)
    std::vector<size_t> n_acc;
};

extern "C" {

rt_status rt_transport(rt_ctx* ctx, const rt_grid* grid, const rt_opacity* op,
                       const rt_source* sources, int n_sources, const rt_transport_params* p,
                       const double* T_prev, const rt_transport_out* out, rt_stream stream)
{
    return transport_one(ctx, grid, op, sources, n_sources, p, T_prev, out, (cudaStream_t)stream, nullptr);
}

rt_status rt_pah_reemit(rt_ctx* ctx, const rt_grid* grid, const rt_opacity* op,
                        const rt_pah_event* records, uint64_t n_records, double xi,
                        const double* eps, int n_eps, const int* eps_class,
                        const rt_transport_params* p, const double* T_prev,
                        const rt_transport_out* out, rt_stream stream)
{
    if (!op || !ctx || ctx->magic != kMagic) return fail(RT_ERR_INVALID_ARG, "rt_pah_reemit: bad context or NULL opacity");
    if (!records || n_records == 0) return fail(RT_ERR_INVALID_ARG, "rt_pah_reemit: need records");
    if (!p || p->n_packets != n_records)
        return fail(RT_ERR_INVALID_ARG, "rt_pah_reemit: p->n_packets must equal n_records");
    if (p->source_bins != 0) return fail(RT_ERR_INVALID_ARG, "rt_pah_reemit: source_bins must be 0");
    if (!(xi > 0.0) || !isfin(xi)) return fail(RT_ERR_INVALID_ARG, "rt_pah_reemit: xi must be finite and > 0");
    if (!eps || n_eps < 1 || n_eps > 65535)
        return fail(RT_ERR_INVALID_ARG, "rt_pah_reemit: need 1..65535 emissivity classes");
    for (int n = 0; n < n_eps; ++n) {
        double tot = 0.0;
        for (int j = 0; j < op->nf; ++j) {
            const double v = eps[(size_t)n * op->nf + j];
            if (!(v >= 0.0) || !isfin(v)) return fail(RT_ERR_INVALID_ARG, "rt_pah_reemit: eps must be finite and >= 0");
            tot += v * op->dnu[j];
        }
        if (!(tot > 0.0)) return fail(RT_ERR_INVALID_ARG, "rt_pah_reemit: an emissivity class is zero on the grid");
    }
    const PahPass pp{ records, n_records, xi, eps, n_eps, eps_class };
    return transport_one(ctx, grid, op, nullptr, 0, p, T_prev, out, (cudaStream_t)stream, &pp);
}

}  // extern "C"

namespace rtgb {

static rt_status transport_one(rt_ctx* ctx, const rt_grid* grid, const rt_opacity* op,
                               const rt_source* sources, int n_sources, const rt_transport_params* p,
                               const double* T_prev, const rt_transport_out* out, cudaStream_t s,
                               const PahPass* pp)
{
    if (!ctx || ctx->magic != kMagic) return fail(RT_ERR_STATE, "rt_transport: bad context");
    if (!grid || !op) return fail(RT_ERR_INVALID_ARG, "rt_transport: NULL grid or opacity");
    if (grid->ctx != ctx || op->ctx != ctx) return fail(RT_ERR_STATE, "rt_transport: handle from another context");
    if (grid->ns != op->ns) return fail(RT_ERR_INVALID_ARG, "rt_transport: grid and opacity species differ");
    if (grid->rho_bad) return fail(RT_ERR_STATE, "rt_transport: the grid's last density update was refused");
    rt_status st = check_params(p);
    if (st != RT_OK) return st;
    st = check_out(out);
    if (st != RT_OK) return st;
    if (p->pid_end < p->pid_begin || p->pid_end > p->n_packets)
        return fail(RT_ERR_INVALID_ARG, "rt_transport: need pid_begin <= pid_end <= n_packets");
    if (p->n_pc_cams > 0 && !out->pc_img)
        return fail(RT_ERR_INVALID_ARG, "rt_transport: photon-counting cameras need out->pc_img");
    if (p->mode == RT_MODE_FROZEN_T && !T_prev)
        return fail(RT_ERR_INVALID_ARG, "rt_transport: frozen-T mode needs T_prev");
    if (p->source_grid_nu || p->source_grid_src) {
        if (!p->source_grid_nu || !p->source_grid_src || p->source_bins == 0 || pp)
            return fail(RT_ERR_INVALID_ARG, "rt_transport: a source grid needs both tables and source_bins > 0");
        for (uint32_t b = 0; b < p->source_bins; ++b)
            if (p->source_grid_nu[b] < 0 || p->source_grid_nu[b] >= op->nf || p->source_grid_src[b] < 0 ||
                p->source_grid_src[b] >= n_sources)
                return fail(RT_ERR_INVALID_ARG, "rt_transport: source grid entry out of range");
    }
    RT_CUDA(cudaSetDevice(ctx->device));
    std::vector<HostModel> hms(1);
    st = make_model(grid, op, sources, n_sources, p->n_packets, p->pid_begin, p->model_id, 0,
                    T_prev, out, hms[0], pp ? pp->xi : 0.0);
    if (st != RT_OK) return st;
    if (p->pid_end == p->pid_begin) return RT_OK;
    const bool acc32 = p->precision == RT_PREC_FP32_ACC32;
    if (acc32 && (grid->refine || pp || p->n_pc_cams || p->defer_events || (out->traj && out->traj_cap)))
        return fail(RT_ERR_INVALID_ARG, "rt_transport: the plain-FP32 form serves uniform grids without "
                                        "trajectories, deferred queue, cameras or PAH sources");
    const int prec = acc32 ? RT_PREC_FP32 : p->precision;     // the transport's arithmetic
    st = pack_grid(const_cast<rt_grid*>(grid), op, p->lucy_mode, p->lucy_tau, prec, s);
    if (st != RT_OK) return st;
    hms[0].md.rho = grid->d_packed;
    hms[0].md.cube_rho = grid->d_cube_packed;
    // FP32 build: this call's deposits go to FP64 scratch in units of xi,
    // seeded with E_abs / xi (zero-started FP32 scratch in the plain-FP32 form)
    const size_t n_acc = (size_t)op->ns * grid->ncell();
    double* acc = nullptr;
    if (prec == RT_PREC_FP32) {
        const size_t bytes = (acc32 ? sizeof(float) : sizeof(double)) * n_acc * (out->esq ? 2 : 1);
        RT_CUDA(cudaMallocAsync((void**)&acc, bytes, s));
        hms[0].md.accE = acc;
        hms[0].md.acc_q = out->esq ? 1 : 0;
        if (acc32) {
            const cudaError_t e = cudaMemsetAsync(acc, 0, bytes, s);
            if (e != cudaSuccess) { cudaFreeAsync(acc, s); return cuda_fail(e, "rt_transport scratch"); }
        } else {
            st = launch_seed(acc, hms[0].md.acc_q, n_acc, hms[0].md.xi, out->E_abs, s);
            if (st != RT_OK) { cudaFreeAsync(acc, s); return st; }
        }
    }
    DeviceModels dm;
    st = stage_models(hms, { p->pid_end - p->pid_begin }, op->nf, true, s, dm);
    if (st != RT_OK) { if (acc) cudaFreeAsync(acc, s); return st; }
    {
        const cudaError_t e = cudaMemsetAsync(dm.work, 0, sizeof(unsigned long long), s);
        if (e != cudaSuccess) {
            cudaFreeAsync(dm.buf, s);
            if (acc) cudaFreeAsync(acc, s);
            return cuda_fail(e, "rt_transport work counter");
        }
    }
    TransportKP kp;
    fill_kp(kp, op, p, dm, 1);
    fill_pc(kp, grid, p, out);
    kp.refined = grid->refine ? 1 : 0;
    kp.acc32 = acc32 ? 1 : 0;
    st = single_model_options(kp, op, p, out, n_sources, hms[0].md);
    if (st != RT_OK) { cudaFreeAsync(dm.buf, s); if (acc) cudaFreeAsync(acc, s); return st; }
    // PAH pass: the emissivity classes' cumulative tables (Eq. 6), FP64 and
    // normalised FP32
    char* ebuf = nullptr;
    if (pp) {
        const int nf = op->nf;
        const size_t n = (size_t)pp->n_eps * nf;
        std::vector<double> c64(n);
        std::vector<float> c32(n);
        for (int k = 0; k < pp->n_eps; ++k) {
            double acc_e = 0.0;
            for (int j = 0; j < nf; ++j) {
                acc_e += pp->eps[(size_t)k * nf + j] * op->dnu[j];
                c64[(size_t)k * nf + j] = acc_e;
            }
            for (int j = 0; j < nf; ++j) c32[(size_t)k * nf + j] = (float)(c64[(size_t)k * nf + j] / acc_e);
            c32[(size_t)k * nf + nf - 1] = 1.0f;
        }
        const size_t o32 = align_up(sizeof(double) * n, 256);
        cudaError_t e = cudaMallocAsync((void**)&ebuf, o32 + sizeof(float) * n, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(ebuf, c64.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(ebuf + o32, c32.data(), sizeof(float) * n, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            cudaFreeAsync(dm.buf, s);
            if (acc) cudaFreeAsync(acc, s);
            if (ebuf) cudaFreeAsync(ebuf, s);
            return cuda_fail(e, "rt_pah_reemit emissivity tables");
        }
        kp.pah_src = pp->rec;
        kp.eps_cdf64 = (const double*)ebuf;
        kp.eps_cdf32 = (const float*)(ebuf + o32);
        kp.eps_class = pp->eps_class;
        kp.n_eps = pp->n_eps;
        kp.smem_cdf = 0;
    }
    // the separate source grid's tables (Eq. 1)
    char* gbuf = nullptr;
    if (p->source_grid_nu) {
        const size_t n = p->source_bins;
        cudaError_t e = cudaMallocAsync((void**)&gbuf, 2 * sizeof(int32_t) * n, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(gbuf, p->source_grid_nu, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(gbuf + sizeof(int32_t) * n, p->source_grid_src, sizeof(int32_t) * n,
                                cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            cudaFreeAsync(dm.buf, s);
            if (acc) cudaFreeAsync(acc, s);
            if (ebuf) cudaFreeAsync(ebuf, s);
            if (gbuf) cudaFreeAsync(gbuf, s);
            return cuda_fail(e, "rt_transport source grid");
        }
        kp.sg_nu = (const int*)gbuf;
        kp.sg_src = (const int*)(gbuf + sizeof(int32_t) * n);
    }
    // deferred packets: a queue in device memory, drained by a second launch
    char* qbuf = nullptr;
    if (p->defer_events > 0) {
        const uint64_t cap = std::min<uint64_t>(p->pid_end - p->pid_begin, kDeferCap);
        const size_t qbytes = sizeof(DeferRec) * cap + 256;
        cudaError_t e = cudaMallocAsync((void**)&qbuf, qbytes, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(qbuf + sizeof(DeferRec) * cap, 0, 256, s);
        if (e != cudaSuccess) {
            cudaFreeAsync(dm.buf, s);
            if (acc) cudaFreeAsync(acc, s);
            if (ebuf) cudaFreeAsync(ebuf, s);
            if (gbuf) cudaFreeAsync(gbuf, s);
            if (qbuf) cudaFreeAsync(qbuf, s);
            return cuda_fail(e, "rt_transport defer queue");
        }
        kp.defer_events = p->defer_events;
        kp.defer = (DeferRec*)qbuf;
        kp.defer_n = (unsigned long long*)(qbuf + sizeof(DeferRec) * cap);
        kp.defer_cap = cap;
    }
    const int threads = p->threads_per_block ? p->threads_per_block : 256;
    st = launch_transport(ctx, op, kp, op->ns, prec, p->schedule, threads, p->blocks_per_sm, s);
    if (st == RT_OK && qbuf) {
        TransportKP kr = kp;
        kr.resume = 1;
        cudaError_t e = cudaMemsetAsync(dm.work, 0, sizeof(unsigned long long), s);
        st = e == cudaSuccess ? launch_transport(ctx, op, kr, op->ns, prec, p->schedule, threads,
                                                 p->blocks_per_sm, s)
                              : cuda_fail(e, "rt_transport resume");
    }
    if (st == RT_OK && acc)
        st = acc32 ? launch_finalize32(reinterpret_cast<const float*>(acc), hms[0].md.acc_q, n_acc,
                                       hms[0].md.xi, out->E_abs, out->esq, s)
                   : launch_finalize(acc, hms[0].md.acc_q, n_acc, hms[0].md.xi, out->E_abs, out->esq, s);
    cudaFreeAsync(dm.buf, s);
    if (acc) cudaFreeAsync(acc, s);
    if (ebuf) cudaFreeAsync(ebuf, s);
    if (gbuf) cudaFreeAsync(gbuf, s);
    if (qbuf) cudaFreeAsync(qbuf, s);
    return st;
}

}  // namespace rtgb

extern "C" {

rt_status rt_batch_create(rt_ctx* ctx, const rt_opacity* op, int n_models, const rt_model* models,
                          const rt_transport_params* p, rt_batch** out)
{
    if (!ctx || ctx->magic != kMagic) return fail(RT_ERR_STATE, "rt_batch_create: bad context");
    if (!op || !models || !out) return fail(RT_ERR_INVALID_ARG, "rt_batch_create: NULL pointer");
    if (n_models < 1 || n_models > 4096) return fail(RT_ERR_INVALID_ARG, "rt_batch_create: n_models must be 1..4096");
    rt_status st = check_params(p);
    if (st != RT_OK) return st;
    if (p->n_pc_cams != 0)
        return fail(RT_ERR_INVALID_ARG, "rt_batch_create: photon-counting cameras are served by rt_transport only");
    if (p->precision == RT_PREC_FP32_ACC32)
        return fail(RT_ERR_INVALID_ARG, "rt_batch_create: the plain-FP32 form is served by rt_transport only");
    if (p->source_grid_nu || p->source_grid_src)
        return fail(RT_ERR_INVALID_ARG, "rt_batch_create: the separate source grid is served by rt_transport only");
    RT_CUDA(cudaSetDevice(ctx->device));
    std::vector<HostModel> hms(n_models);
    std::vector<uint64_t> nwork(n_models);
    for (int m = 0; m < n_models; ++m) {
        const rt_model& M = models[m];
        if (!M.grid || M.grid->ctx != ctx || M.grid->ns != op->ns || M.grid->rho_bad)
            return fail(RT_ERR_INVALID_ARG, "rt_batch_create: grid missing, foreign, with other species or refused density");
        if (M.n_packets == 0) return fail(RT_ERR_INVALID_ARG, "rt_batch_create: n_packets must be > 0");
        if (p->mode == RT_MODE_FROZEN_T && !M.T_prev)
            return fail(RT_ERR_INVALID_ARG, "rt_batch_create: frozen-T mode needs T_prev for every model");
        st = check_out(&M.out);
        if (st != RT_OK) return st;
        st = pack_grid(const_cast<rt_grid*>(M.grid), op, p->lucy_mode, p->lucy_tau, p->precision, 0);
        if (st != RT_OK) return st;
        st = make_model(M.grid, op, M.sources, M.n_sources, M.n_packets, 0, p->model_id + (uint32_t)m, m,
                        M.T_prev, &M.out, hms[m]);
        if (st != RT_OK) return st;
        hms[m].md.rho = M.grid->d_packed;
        hms[m].md.cube_rho = M.grid->d_cube_packed;
        nwork[m] = M.n_packets;
    }
    RT_CUDA(cudaDeviceSynchronize());
    rt_batch* b = new rt_batch();
    b->ctx = ctx; b->op = op; b->p = *p; b->n_models = n_models; b->ns = op->ns;
    b->acc = nullptr;
    b->acc_bytes = 0;
    if (p->precision == RT_PREC_FP32) {
        size_t tot = 0;
        for (int m = 0; m < n_models; ++m) {
            const size_t n = (size_t)op->ns * models[m].grid->ncell();
            tot += n * (models[m].out.esq ? 2 : 1);
        }
        b->acc_bytes = tot * sizeof(double);
        cudaError_t e = cudaMalloc((void**)&b->acc, b->acc_bytes);
        if (e != cudaSuccess) { delete b; return cuda_fail(e, "rt_batch_create scratch"); }
        size_t off = 0;
        for (int m = 0; m < n_models; ++m) {
            const size_t n = (size_t)op->ns * models[m].grid->ncell();
            hms[m].md.accE = b->acc + off;
            hms[m].md.acc_q = models[m].out.esq ? 1 : 0;
            off += n * (models[m].out.esq ? 2 : 1);
        }
    }
    for (int m = 0; m < n_models; ++m) {
        b->host.push_back(hms[m].md);
        b->n_acc.push_back((size_t)op->ns * models[m].grid->ncell());
    }
    st = stage_models(hms, nwork, op->nf, false, 0, b->dm);
    if (st != RT_OK) { cudaFree(b->acc); delete b; return st; }
    fill_kp(b->kp, op, p, b->dm, n_models);
    for (int m = 0; m < n_models; ++m)
        if (models[m].grid->refine) b->kp.refined = 1;   // the two-level traversal for every model
    for (int m = 0; m < n_models; ++m)
        if (models[m].out.traj && models[m].out.traj_cap) b->kp.want_traj = 1;
    if (n_models <= kParamModels) {
        // the staged descriptors also travel in the launch parameters
        for (int m = 0; m < n_models; ++m) b->kp.mp[m] = hms[m].md;
        b->kp.param_models = n_models;
    }
    *out = b;
    return RT_OK;
}

rt_status rt_batch_run(rt_batch* b, rt_stream stream)
{
    if (!b) return fail(RT_ERR_INVALID_ARG, "rt_batch_run: NULL batch");
    cudaStream_t s = (cudaStream_t)stream;
    RT_CUDA(cudaMemsetAsync(b->dm.work, 0, sizeof(unsigned long long), s));
    if (b->acc) {
        for (int m = 0; m < b->n_models; ++m) {
            const ModelDev& md = b->host[m];
            const rt_status st = launch_seed(md.accE, md.acc_q, b->n_acc[m], md.xi, md.E_abs, s);
            if (st != RT_OK) return st;
        }
    }
    const int threads = b->p.threads_per_block ? b->p.threads_per_block : 256;
    rt_status st = launch_transport(b->ctx, b->op, b->kp, b->ns, b->p.precision, b->p.schedule,
                                    threads, b->p.blocks_per_sm, s);
    if (st != RT_OK || !b->acc) return st;
    for (int m = 0; m < b->n_models; ++m) {
        const ModelDev& md = b->host[m];
        st = launch_finalize(md.accE, md.acc_q, b->n_acc[m], md.xi, md.E_abs, md.esq, s);
        if (st != RT_OK) return st;
    }
    return RT_OK;
}

void rt_batch_free(rt_batch* b)
{
    if (!b) return;
    cudaSetDevice(b->ctx->device);
    cudaFree(b->dm.buf);
    cudaFree(b->acc);
    delete b;
}

rt_status rt_transport_batched(rt_ctx* ctx, const rt_opacity* op, int n_models,
                               const rt_model* models, const rt_transport_params* p, rt_stream stream)
{
    rt_batch* b = nullptr;
    rt_status st = rt_batch_create(ctx, op, n_models, models, p, &b);
    if (st != RT_OK) return st;
    st = rt_batch_run(b, stream);
    cudaStream_t s = (cudaStream_t)stream;
    if (st == RT_OK) {
        cudaFreeAsync(b->dm.buf, s);
        b->dm.buf = nullptr;
    }
    rt_batch_free(b);
    return st;
}

rt_status rt_temperatures(rt_ctx* ctx, const rt_grid* grid, const rt_opacity* op,
                          const double* E_abs, double* T, rt_stream stream)
{
    if (!ctx || ctx->magic != kMagic) return fail(RT_ERR_STATE, "rt_temperatures: bad context");
    if (!grid || !op || !E_abs || !T) return fail(RT_ERR_INVALID_ARG, "rt_temperatures: NULL pointer");
    if (grid->ctx != ctx || op->ctx != ctx) return fail(RT_ERR_STATE, "rt_temperatures: handle from another context");
    if (grid->ns != op->ns) return fail(RT_ERR_INVALID_ARG, "rt_temperatures: grid and opacity species differ");
    if (grid->rho_bad) return fail(RT_ERR_STATE, "rt_temperatures: the grid's last density update was refused");
    RT_CUDA(cudaSetDevice(ctx->device));
    return launch_temperatures(ctx, grid, op, E_abs, T, (cudaStream_t)stream);
}

rt_status rt_temperature_guess(rt_ctx* ctx, const rt_grid* grid, const rt_source* src, int nsrc,
                               double* T, rt_stream stream)
{
    if (!ctx || ctx->magic != kMagic) return fail(RT_ERR_STATE, "rt_temperature_guess: bad context");
    if (!grid || !src || !T || nsrc < 1 || nsrc > 64)
        return fail(RT_ERR_INVALID_ARG, "rt_temperature_guess: bad arguments");
    RT_CUDA(cudaSetDevice(ctx->device));
    std::vector<double> pos(3 * nsrc), L(nsrc);
    for (int i = 0; i < nsrc; ++i) {
        for (int a = 0; a < 3; ++a) pos[3 * i + a] = src[i].pos[a];
        L[i] = src[i].L;
    }
    return launch_temperature_guess(ctx, grid, pos.data(), L.data(), nsrc, T, (cudaStream_t)stream);
}

static rt_status check_rt_args(rt_ctx* ctx, const rt_grid* grid, const rt_opacity* op,
                               const double* T, const rt_event* ev, uint64_t nev,
                               const rt_source* src, int nsrc, const rt_camera* cams, int ncam,
                               const int* fidx, int nfi)
{
    if (!ctx || ctx->magic != kMagic) return fail(RT_ERR_STATE, "rt_raytrace: bad context");
    if (!grid || !op || !T || !cams || !fidx) return fail(RT_ERR_INVALID_ARG, "rt_raytrace: NULL pointer");
    if (grid->ctx != ctx || op->ctx != ctx) return fail(RT_ERR_STATE, "rt_raytrace: handle from another context");
    if (grid->ns != op->ns) return fail(RT_ERR_INVALID_ARG, "rt_raytrace: grid and opacity species differ");
    if (grid->rho_bad) return fail(RT_ERR_STATE, "rt_raytrace: the grid's last density update was refused");
    if (nev > 0 && !ev) return fail(RT_ERR_INVALID_ARG, "rt_raytrace: events NULL with n_events > 0");
    if (nsrc < 0 || nsrc > 64 || (nsrc > 0 && !src)) return fail(RT_ERR_INVALID_ARG, "rt_raytrace: bad sources");
    if (ncam < 1 || ncam > 1024) return fail(RT_ERR_INVALID_ARG, "rt_raytrace: n_cams must be 1..1024");
    if (nfi < 1 || nfi > kMaxImgFreq) return fail(RT_ERR_INVALID_ARG, "rt_raytrace: n_f must be 1..16");
    for (int f = 0; f < nfi; ++f)
        if (fidx[f] < 0 || fidx[f] >= op->nf) return fail(RT_ERR_INVALID_ARG, "rt_raytrace: freq_idx out of range");
    for (int c = 0; c < ncam; ++c) {
        if (cams[c].npix != cams[0].npix || cams[c].npix < 1 || cams[c].npix > 16384)
            return fail(RT_ERR_INVALID_ARG, "rt_raytrace: all cameras need the same npix in 1..16384");
        if (!(cams[c].D > 0.0) || !isfin(cams[c].D) || !isfin(cams[c].theta) || !isfin(cams[c].phi))
            return fail(RT_ERR_INVALID_ARG, "rt_raytrace: bad camera");
    }
    return RT_OK;
}

rt_status rt_raytrace(rt_ctx* ctx, const rt_grid* grid, const rt_opacity* op, const double* T,
                      const rt_event* ev, uint64_t nev, const uint64_t* nev_dev, double xi_ev,
                      const rt_source* src, int nsrc,
                      const rt_camera* cams, int ncam, const int* fidx, int nfi, float* images,
                      double* sed, uint64_t* ray_steps, rt_stream stream)
{
    rt_status st = check_rt_args(ctx, grid, op, T, ev, nev, src, nsrc, cams, ncam, fidx, nfi);
    if (st != RT_OK) return st;
    if (!images || !sed) return fail(RT_ERR_INVALID_ARG, "rt_raytrace: NULL output");
    RT_CUDA(cudaSetDevice(ctx->device));
    return raytrace_impl(ctx, grid, op, T, ev, nev, nev_dev, xi_ev, src, nsrc, cams, ncam, fidx, nfi,
                         images, sed, nullptr, nullptr, nullptr, nullptr, (unsigned long long*)ray_steps,
                         false, (cudaStream_t)stream);
}

rt_status rt_visibilities(rt_ctx* ctx, const rt_grid* grid, const rt_camera* cams, int ncam,
                          const float* images, int nf, const double* uv, int nuv, double* vis,
                          rt_stream stream)
{
    if (!ctx || ctx->magic != kMagic) return fail(RT_ERR_STATE, "rt_visibilities: bad context");
    if (!grid || !cams || !images || !uv || !vis) return fail(RT_ERR_INVALID_ARG, "rt_visibilities: NULL pointer");
    if (grid->ctx != ctx) return fail(RT_ERR_STATE, "rt_visibilities: grid from another context");
    if (ncam < 1 || ncam > 1024) return fail(RT_ERR_INVALID_ARG, "rt_visibilities: n_cams must be 1..1024");
    if (nf < 1 || nf > kMaxImgFreq) return fail(RT_ERR_INVALID_ARG, "rt_visibilities: n_f must be 1..16");
    if (nuv < 1 || nuv > 65535) return fail(RT_ERR_INVALID_ARG, "rt_visibilities: n_uv must be 1..65535");
    for (int c = 0; c < ncam; ++c) {
        if (cams[c].npix != cams[0].npix || cams[c].npix < 1 || cams[c].npix > 8192)
            return fail(RT_ERR_INVALID_ARG, "rt_visibilities: all cameras need the same npix in 1..8192");
        if (!(cams[c].D > 0.0) || !isfin(cams[c].D)) return fail(RT_ERR_INVALID_ARG, "rt_visibilities: bad camera");
    }
    for (int k = 0; k < 2 * nuv; ++k)
        if (!isfin(uv[k])) return fail(RT_ERR_INVALID_ARG, "rt_visibilities: non-finite uv");
    RT_CUDA(cudaSetDevice(ctx->device));
    return visibilities_impl(ctx, grid, cams, ncam, images, nf, uv, nuv, vis, (cudaStream_t)stream);
}

rt_status rt_raytrace_backward(rt_ctx* ctx, const rt_grid* grid, const rt_opacity* op,
                               const double* T, const rt_event* ev, uint64_t nev,
                               const uint64_t* nev_dev, double xi_ev,
                               const rt_source* src, int nsrc, const rt_camera* cams, int ncam,
                               const int* fidx, int nfi, const float* dimg, const double* dsed,
                               float* drho, double* dscale, uint64_t* ray_steps, rt_stream stream)
{
    rt_status st = check_rt_args(ctx, grid, op, T, ev, nev, src, nsrc, cams, ncam, fidx, nfi);
    if (st != RT_OK) return st;
    if (!drho || !dscale) return fail(RT_ERR_INVALID_ARG, "rt_raytrace_backward: NULL output");
    RT_CUDA(cudaSetDevice(ctx->device));
    return raytrace_impl(ctx, grid, op, T, ev, nev, nev_dev, xi_ev, src, nsrc, cams, ncam, fidx, nfi,
                         nullptr, nullptr, dimg, dsed, drho, dscale, (unsigned long long*)ray_steps, true,
                         (cudaStream_t)stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free transport.  All scratch of one rt_transport call (the work
// counter, the model table with its source CDFs, the packed density copy, the
// per-call FP64 energy scratch and the kext work array) lives in one
// file-scope device array, so the call itself never allocates device memory.
namespace rtgb {

constexpr size_t kNoAllocBytes = 64ull << 20;     // 64 MiB held by every GPU that loads the library
constexpr size_t kNoAllocStaging = 1ull << 20;    // model table, source tables, work counter
constexpr size_t kNoAllocKext = 64ull << 10;      // ns * nf doubles (4 * 1024 * 8 = 32 KiB)

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

static std::mutex g_noalloc_mutex;
static void* g_noalloc_addr[256];

// Device address of the scratch array on `device` (which must be current).
// Host code cannot use the symbol's own address: on the host it names a
// stand-in object, not device memory.
static rt_status noalloc_scratch(int device, unsigned char** out)
{
    if (device < 0 || device >= 256) return fail(RT_ERR_INVALID_ARG, "rt_transport_noalloc: device id out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        g_noalloc_addr[device] = p;
    }
    *out = (unsigned char*)g_noalloc_addr[device];
    return RT_OK;
}

// stage_models into a given device buffer (host image + one H2D copy)
static rt_status stage_models_into(std::vector<HostModel>& hms, uint64_t nwork, int nf,
                                   unsigned char* base, size_t cap, cudaStream_t s, DeviceModels& dm)
{
    HostModel& hm = hms[0];
    const int nsrc = hm.md.nsrc;
    size_t off = 0;
    const size_t o_models = off; off = align_up(off + sizeof(ModelDev), 64);
    const size_t o_prefix = off; off = align_up(off + sizeof(unsigned long long) * 2, 64);
    const size_t o_work = off; off = align_up(off + sizeof(unsigned long long) * 2, 64);
    const size_t o_pos = off; off = align_up(off + sizeof(double) * 3 * nsrc, 64);
    const size_t o_L = off; off = align_up(off + sizeof(double) * nsrc, 64);
    const size_t o_c64 = off; off = align_up(off + sizeof(double) * nsrc * nf, 64);
    const size_t o_c32 = off; off = align_up(off + sizeof(float) * nsrc * nf, 64);
    if (off > cap) return fail(RT_ERR_CAPACITY, "rt_transport_noalloc: source tables exceed the staging area");
    std::vector<unsigned char> h(off, 0);
    ModelDev md = hm.md;
    std::memcpy(&h[o_pos], hm.pos.data(), sizeof(double) * hm.pos.size());
    std::memcpy(&h[o_L], hm.Lcdf.data(), sizeof(double) * hm.Lcdf.size());
    std::memcpy(&h[o_c64], hm.cdf64.data(), sizeof(double) * hm.cdf64.size());
    std::memcpy(&h[o_c32], hm.cdf32.data(), sizeof(float) * hm.cdf32.size());
    md.src_pos = (const double*)(base + o_pos);
    md.src_Lcdf = (const double*)(base + o_L);
    md.src_cdf64 = (const double*)(base + o_c64);
    md.src_cdf32 = (const float*)(base + o_c32);
    std::memcpy(&h[o_models], &md, sizeof(ModelDev));
    hm.md = md;                        // the host copy now matches the device one
    const unsigned long long prefix[2] = { 0ull, (unsigned long long)nwork };
    std::memcpy(&h[o_prefix], prefix, sizeof(prefix));
    RT_CUDA(cudaMemcpyAsync(base, h.data(), off, cudaMemcpyHostToDevice, s));
    dm.buf = base;
    dm.bytes = off;
    dm.models = (ModelDev*)(base + o_models);
    dm.prefix = (unsigned long long*)(base + o_prefix);
    dm.work = (unsigned long long*)(base + o_work);
    dm.total = nwork;
    return RT_OK;
}

}  // namespace rtgb

extern "C" {

rt_status rt_transport_noalloc(rt_ctx* ctx, const rt_grid* grid, const rt_opacity* op,
                               const rt_source* sources, int n_sources,
                               const rt_transport_params* p, const double* T_prev,
                               const rt_transport_out* out, rt_stream stream)
{
    if (!ctx || ctx->magic != kMagic) return fail(RT_ERR_STATE, "rt_transport_noalloc: bad context");
    if (!grid || !op) return fail(RT_ERR_INVALID_ARG, "rt_transport_noalloc: NULL grid or opacity");
    if (grid->ctx != ctx || op->ctx != ctx) return fail(RT_ERR_STATE, "rt_transport_noalloc: handle from another context");
    if (grid->ns != op->ns) return fail(RT_ERR_INVALID_ARG, "rt_transport_noalloc: grid and opacity species differ");
    if (grid->rho_bad) return fail(RT_ERR_STATE, "rt_transport_noalloc: the grid's last density update was refused");
    rt_status st = check_params(p);
    if (st != RT_OK) return st;
    st = check_out(out);
    if (st != RT_OK) return st;
    if (p->pid_end < p->pid_begin || p->pid_end > p->n_packets)
        return fail(RT_ERR_INVALID_ARG, "rt_transport_noalloc: need pid_begin <= pid_end <= n_packets");
    if (p->n_pc_cams != 0)
        return fail(RT_ERR_INVALID_ARG, "rt_transport_noalloc: photon-counting cameras are served by rt_transport only");
    if (p->precision == RT_PREC_FP32_ACC32)
        return fail(RT_ERR_INVALID_ARG, "rt_transport_noalloc: the plain-FP32 form is served by rt_transport only");
    if (p->defer_events != 0)
        return fail(RT_ERR_INVALID_ARG, "rt_transport_noalloc: the deferred-packet queue (defer_events) is served by rt_transport only");
    if (p->source_grid_nu || p->source_grid_src)
        return fail(RT_ERR_INVALID_ARG, "rt_transport_noalloc: the separate source grid is served by rt_transport only");
    if (p->mode == RT_MODE_FROZEN_T && !T_prev)
        return fail(RT_ERR_INVALID_ARG, "rt_transport_noalloc: frozen-T mode needs T_prev");
    // scratch layout: staging | kext | packed density | packed cube density
    // (refined grids) | FP64 energy scratch
    const size_t nc = grid->ncell();
    const int vec = grid->ns == 1 ? 1 : (grid->ns == 2 ? 2 : 4);
    const size_t packed_bytes = align_up(nc * sizeof(float) * vec, 256) +
                                (grid->refine ? align_up(grid->ncube() * sizeof(float) * vec, 256) : 0);
    const size_t n_acc = (size_t)op->ns * nc;
    const size_t acc_bytes = p->precision == RT_PREC_FP32 ? sizeof(double) * n_acc * (out->esq ? 2 : 1) : 0;
    const size_t need = kNoAllocStaging + kNoAllocKext + packed_bytes + acc_bytes;
    if (need > kNoAllocBytes)
        return fail(RT_ERR_CAPACITY, "rt_transport_noalloc: grid too large for the 64 MiB static scratch (" +
                                         std::to_string(need >> 20) + " MiB needed)");
    RT_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* base = nullptr;
    st = noalloc_scratch(ctx->device, &base);
    if (st != RT_OK) return st;
    std::vector<HostModel> hms(1);
    st = make_model(grid, op, sources, n_sources, p->n_packets, p->pid_begin, p->model_id, 0,
                    T_prev, out, hms[0]);
    if (st != RT_OK) return st;
    if (p->pid_end == p->pid_begin) return RT_OK;
    double* kext = (double*)(base + kNoAllocStaging);
    unsigned char* packed = base + kNoAllocStaging + kNoAllocKext;
    double* acc = acc_bytes ? (double*)(packed + packed_bytes) : nullptr;
    unsigned char* cube_packed = packed + align_up(nc * sizeof(float) * vec, 256);
    st = pack_grid_into(grid, op, p->lucy_mode, p->lucy_tau, p->precision, kext, packed,
                        grid->refine ? cube_packed : nullptr, s);
    if (st != RT_OK) return st;
    hms[0].md.rho = packed;
    hms[0].md.cube_rho = grid->refine ? cube_packed : nullptr;
    if (acc) {
        hms[0].md.accE = acc;
        hms[0].md.acc_q = out->esq ? 1 : 0;
        // the array keeps the last call's sums: seeded afresh from E_abs
        st = launch_seed(acc, hms[0].md.acc_q, n_acc, hms[0].md.xi, out->E_abs, s);
        if (st != RT_OK) return st;
    }
    DeviceModels dm;
    st = stage_models_into(hms, p->pid_end - p->pid_begin, op->nf, base, kNoAllocStaging, s, dm);
    if (st != RT_OK) return st;
    RT_CUDA(cudaMemsetAsync(dm.work, 0, sizeof(unsigned long long), s));
    TransportKP kp;
    fill_kp(kp, op, p, dm, 1);
    kp.refined = grid->refine ? 1 : 0;
    st = single_model_options(kp, op, p, out, n_sources, hms[0].md);
    if (st != RT_OK) return st;
    const int threads = p->threads_per_block ? p->threads_per_block : 256;
    st = launch_transport(ctx, op, kp, op->ns, p->precision, p->schedule, threads, p->blocks_per_sm, s);
    if (st == RT_OK && acc)
        st = launch_finalize(acc, hms[0].md.acc_q, n_acc, hms[0].md.xi, out->E_abs, out->esq, s);
    return st;
}

rt_status rt_philox(rt_ctx* ctx, const uint32_t ctr0[4], const uint32_t key[2], uint64_t n,
                    uint32_t* out, rt_stream stream)
{
    if (!ctx || ctx->magic != kMagic) return fail(RT_ERR_STATE, "rt_philox: bad context");
    if (!ctr0 || !key || !out) return fail(RT_ERR_INVALID_ARG, "rt_philox: NULL pointer");
    if ((uint64_t)ctr0[0] + n > 0x100000000ull) return fail(RT_ERR_INVALID_ARG, "rt_philox: counter word 0 would wrap");
    RT_CUDA(cudaSetDevice(ctx->device));
    return launch_philox(ctr0, key, n, out, (cudaStream_t)stream);
}

rt_status rt_source_grid(const rt_opacity* op, const rt_source* sources, int n_sources, uint32_t m,
                         int32_t* nu_idx, int32_t* src_idx, double* nu_star)
{
    if (!op) return fail(RT_ERR_INVALID_ARG, "rt_source_grid: NULL opacity");
    if (!sources || n_sources < 1) return fail(RT_ERR_INVALID_ARG, "rt_source_grid: no source");
    if (m == 0 || !nu_idx || !src_idx) return fail(RT_ERR_INVALID_ARG, "rt_source_grid: need m > 0 and output arrays");
    for (int i = 0; i < n_sources; ++i)
        if (!(sources[i].L >= 0.0) || (!sources[i].L_nu && !(sources[i].T_eff > 0.0)))
            return fail(RT_ERR_INVALID_ARG, "rt_source_grid: a source needs L >= 0 and T_eff > 0 or L_nu");
    return build_source_grid(op, sources, n_sources, m, nu_idx, src_idx, nu_star);
}

rt_status rt_probe_gather(rt_ctx* ctx, const void* buf, size_t bytes, uint64_t n_reads, uint32_t seed,
                          unsigned long long* sink, rt_stream stream)
{
    if (!ctx || ctx->magic != kMagic) return fail(RT_ERR_STATE, "rt_probe_gather: bad context");
    if (!buf || bytes < 32) return fail(RT_ERR_INVALID_ARG, "rt_probe_gather: need a buffer of at least 32 bytes");
    if (reinterpret_cast<uintptr_t>(buf) % 32 != 0) return fail(RT_ERR_INVALID_ARG, "rt_probe_gather: buffer not 32-byte aligned");
    if (bytes / 32 > 0xFFFFFFFFull) return fail(RT_ERR_INVALID_ARG, "rt_probe_gather: buffer above 128 GiB");
    RT_CUDA(cudaSetDevice(ctx->device));
    return launch_gather_probe(ctx->num_sms, buf, bytes, n_reads, seed, sink, (cudaStream_t)stream);
}

rt_status rt_mrw_sample(rt_ctx* ctx, const rt_opacity* op, const float* u, uint64_t n, float* y,
                        rt_stream stream)
{
    if (!ctx || ctx->magic != kMagic) return fail(RT_ERR_STATE, "rt_mrw_sample: bad context");
    if (!op || op->ctx != ctx) return fail(RT_ERR_STATE, "rt_mrw_sample: opacity from another context");
    if (n > 0 && (!u || !y)) return fail(RT_ERR_INVALID_ARG, "rt_mrw_sample: NULL pointer");
    RT_CUDA(cudaSetDevice(ctx->device));
    return launch_mrw_sample(op->d_mrwS, u, n, y, (cudaStream_t)stream);
}

}  // extern "C"
