// Dust temperatures (Heymann & Siebenmorgen 2012, Eq. 4) and the optically
// thin starting guess of the iterative scheme (Sect. 2), plus the Philox
// test hook.
#include <math.h>

#include "rt_internal.cuh"

namespace rtgb {

namespace {

constexpr double kPi = 3.14159265358979323846;

struct TempKP {
    const float* rho; const double* E; double* T;
    size_t nc; int ns; double vol;
    const unsigned char* leaf_fine;     // refined grids: 1 = sub-cube (volume vol_fine)
    double vol_fine;
    const double2* tz; const TwNode* tw; const float* zinv;
    float zinv_z0[kMaxSpecies], zinv_idz[kMaxSpecies];
    int tw_ok[kMaxSpecies];
    double lnT0, dlnT;
    int nf; const double* nu; const double* dnu; const double* kabs;
};

// z(T) = ln(4 pi sum_j kabs_j B_j(T) dnu_j) solved by binary search for the
// bracketing table interval and Newton iterations on its cubic Hermite
// interpolant; targets outside the table fall back to bisection on the
// Planck sum.
__device__ double solve_z(const TempKP& P, int s, double e, double rv)
{
    const double z = log(e / rv);
    const double2* t = P.tz + (size_t)s * kTz64N;
    if (z >= t[0].x && z <= t[kTz64N - 1].x) {
        int lo = 0, hi = kTz64N - 1;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (t[mid].x <= z) lo = mid; else hi = mid;
        }
        const double2 a = t[lo], b = t[hi];
        const double m0 = a.y * P.dlnT, m1 = b.y * P.dlnT;
        double u = (b.x > a.x) ? (z - a.x) / (b.x - a.x) : 0.0;
        for (int it = 0; it < 6; ++it) {
            const double u2 = u * u, u3 = u2 * u;
            const double H = (2 * u3 - 3 * u2 + 1) * a.x + (u3 - 2 * u2 + u) * m0 +
                             (-2 * u3 + 3 * u2) * b.x + (u3 - u2) * m1;
            const double dH = (6 * u2 - 6 * u) * a.x + (3 * u2 - 4 * u + 1) * m0 +
                              (-6 * u2 + 6 * u) * b.x + (3 * u2 - 2 * u) * m1;
            if (!(dH > 0.0)) break;
            u = fmin(1.0, fmax(0.0, u - (H - z) / dH));
        }
        return exp(P.lnT0 + ((double)lo + u) * P.dlnT);
    }
    const double target = e / rv;
    const double h = 6.62607015e-27, kb = 1.380649e-16, c = 2.99792458e10;
    auto em4pi = [&](double Tc) {
        double Ps = 0.0;
        for (int j = 0; j < P.nf; ++j)
            Ps += 4.0 * kPi * P.kabs[s * P.nf + j] * P.dnu[j] * 2.0 * h * P.nu[j] * P.nu[j] * P.nu[j] /
                  (c * c) / expm1(h * P.nu[j] / (kb * Tc));
        return Ps;
    };
    double lo = 0.0, hi = 1.0e5;
    for (int it = 0; it < 64 && em4pi(hi) < target; ++it) hi *= 2.0;
    for (int it = 0; it < 200 && hi - lo > 1e-12 * hi; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (em4pi(mid) < target) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

// One thread per (species, cell): Eq. 4, 4 pi P(T) = E / (rho V).  GB300 has
// little FP64 throughput, so the solve avoids FP64 logarithms, divisions and
// searches.  An FP32 estimate of z = ln(E / (rho V)) (integer exponent split,
// FP32 log2) indexes a uniform-z table that returns the position t on the
// fine ln T grid.  Two Newton steps on the cubic Hermite interpolant of
// W(u) = 4 pi P in linear space (interval j = floor t, u = t - j; W and dW/du
// at the nodes are exact) solve W(u) rho V = E: the step is the relative
// residual 1 - E / (W rho V) (hardware reciprocal estimate) times
// 1 / (d ln W / du) at the node.  From a start within 0.02 of an interval the
// second step leaves an error far below double rounding of ln T.  The
// interpolant's own error, h^4/384 times the fourth derivative of W
// (h = 2.5e-4), is about 1e-17 (d ln W / d ln T)^3 relative in T; nodes where
// that slope exceeds 20 (the Wien side, T of order 1 K and below) take
// solve_z, as do underflowing nodes and targets off the table.
// T = T_j exp(u h) with a five-term series (u h < 2.5e-4).
__global__ void temperatures_kernel(const __grid_constant__ TempKP P)
{
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= P.nc * P.ns) return;
    const int s = (int)(i / P.nc);
    const double vol = (P.leaf_fine && P.leaf_fine[i - (size_t)s * P.nc]) ? P.vol_fine : P.vol;
    const double rv = (double)P.rho[i] * vol;
    const double e = P.E[i];
    if (!(rv > 0.0) || !(e > 0.0)) { P.T[i] = 0.0; return; }
    if (P.tw_ok[s]) {
        const float z = (log2_d(e) - log2_d(rv)) * 0.693147180559945309f;
        const float f = (z - P.zinv_z0[s]) * P.zinv_idz[s];
        if (f >= 0.0f && f <= (float)(kZinvN - 1)) {
            const float* zi = P.zinv + (size_t)s * kZinvN;
            const int k = min((int)f, kZinvN - 2);
            const float t = zi[k] + (f - (float)k) * (zi[k + 1] - zi[k]);
            const int j = min(max((int)t, 0), kTz64N - 2);
            const TwNode a = P.tw[(size_t)s * kTz64N + j];
            const TwNode b = P.tw[(size_t)s * kTz64N + j + 1];
            if (a.W > 0.0 && a.g * P.dlnT > 0.05) {
                double u = f2d(t - (float)j);
#pragma unroll
                for (int it = 0; it < 2; ++it) {
                    const double u2 = u * u, u3 = u2 * u;
                    const double h01 = 3.0 * u2 - 2.0 * u3;
                    const double W = (1.0 - h01) * a.W + (u3 - 2.0 * u2 + u) * a.m + h01 * b.W +
                                     (u3 - u2) * b.m;
                    const double p = W * rv;
                    u -= (p - e) * rcp_approx(p) * a.g;
                }
                if (u > -0.5 && u < 1.5) {
                    const double d = u * P.dlnT;
                    P.T[i] = a.T * (1.0 + d * (1.0 + d * (0.5 + d * (1.0 / 6.0 + d * (1.0 / 24.0)))));
                    return;
                }
            }
        }
    }
    P.T[i] = solve_z(P, s, e, rv);
}

__global__ void guess_kernel(int nx, int ny, int nz, int ns, double bx, double by, double bz,
                             double cell, const double* pos, const double* L, int nsrc, double* T,
                             size_t nc, int refine, const int* cube, const int* leaf_cube)
{
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const double h = 6.62607015e-27, kb = 1.380649e-16, c = 2.99792458e10;
    const double sigma = 2.0 * pow(kPi, 5) * pow(kb, 4) / (15.0 * h * h * h * c * c);
    // centre of cell i: a cube, or a sub-cube of a divided cube (refined grids)
    const size_t qc = refine ? (size_t)leaf_cube[i] : i;
    const int ix = (int)(qc % nx), iy = (int)((qc / nx) % ny), iz = (int)(qc / ((size_t)nx * ny));
    double fx = 0.5, fy = 0.5, fz = 0.5;
    if (refine && (cube[qc] & kCubeDivided)) {
        const int off = (int)i - (cube[qc] & ~kCubeDivided);
        fx = ((off % refine) + 0.5) / refine;
        fy = (((off / refine) % refine) + 0.5) / refine;
        fz = ((off / (refine * refine)) + 0.5) / refine;
    }
    const double x = bx + (ix + fx) * cell, y = by + (iy + fy) * cell, z = bz + (iz + fz) * cell;
    double q = 0.0;
    for (int k = 0; k < nsrc; ++k) {
        const double dx = x - pos[3 * k], dy = y - pos[3 * k + 1], dz = z - pos[3 * k + 2];
        const double r2 = dx * dx + dy * dy + dz * dz;
        q += r2 > 0.0 ? L[k] / (16.0 * kPi * sigma * r2) : INFINITY;
    }
    double t = pow(q, 0.25);
    if (!(t < 2000.0)) t = 2000.0;
    for (int s = 0; s < ns; ++s) T[s * nc + i] = t;
}

__global__ void philox_kernel(uint4 c0, uint2 key, uint64_t n, uint4* out)
{
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint4 c = c0;
    c.x += (uint32_t)i;
    out[i] = philox4x32_10(c, key);
}

// the FP32 transport's MRW path-length draw for given uniforms (test hook)
__global__ void mrw_sample_kernel(const float* S, const float* u, uint64_t n, float* y)
{
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] = mrw_y32(S, u[i]);
}

}  // namespace

rt_status launch_temperatures(rt_ctx* ctx, const rt_grid* g, const rt_opacity* op, const double* E,
                              double* T, cudaStream_t s)
{
    (void)ctx;
    const size_t nc = g->ncell();
    const size_t n = nc * g->ns;
    TempKP kp;
    kp.rho = g->d_rho; kp.E = E; kp.T = T;
    kp.nc = nc; kp.ns = g->ns; kp.vol = g->cell * g->cell * g->cell;
    kp.leaf_fine = g->d_leaf_fine;
    kp.vol_fine = g->refine ? kp.vol / ((double)g->refine * g->refine * g->refine) : kp.vol;
    kp.tz = op->d_tz; kp.tw = op->d_tw; kp.zinv = op->d_zinv;
    for (int q = 0; q < kMaxSpecies; ++q) {
        kp.zinv_z0[q] = q < g->ns ? op->zinv_z0[q] : 0.0f;
        kp.zinv_idz[q] = q < g->ns ? op->zinv_idz[q] : 0.0f;
        kp.tw_ok[q] = q < g->ns ? op->tw_ok[q] : 0;
    }
    kp.lnT0 = op->tz_lnT0; kp.dlnT = op->tz_dlnT;
    kp.nf = op->nf; kp.nu = op->d_nu; kp.dnu = op->d_dnu; kp.kabs = op->d_kabs;
    const int th = 256;
    temperatures_kernel<<<(unsigned)((n + th - 1) / th), th, 0, s>>>(kp);
    count_launches();
    RT_CUDA(cudaGetLastError());
    return RT_OK;
}

rt_status launch_temperature_guess(rt_ctx* ctx, const rt_grid* g, const double* src_pos,
                                   const double* src_L, int nsrc, double* T, cudaStream_t s)
{
    (void)ctx;
    double* buf = nullptr;
    RT_CUDA(cudaMallocAsync(&buf, sizeof(double) * 4 * nsrc, s));
    RT_CUDA(cudaMemcpyAsync(buf, src_pos, sizeof(double) * 3 * nsrc, cudaMemcpyHostToDevice, s));
    RT_CUDA(cudaMemcpyAsync(buf + 3 * nsrc, src_L, sizeof(double) * nsrc, cudaMemcpyHostToDevice, s));
    const size_t nc = g->ncell();
    guess_kernel<<<(unsigned)((nc + 255) / 256), 256, 0, s>>>(
        g->nx, g->ny, g->nz, g->ns, g->box_min[0], g->box_min[1], g->box_min[2], g->cell, buf,
        buf + 3 * nsrc, nsrc, T, nc, g->refine, g->d_cube, g->d_leaf_cube);
    count_launches();
    RT_CUDA(cudaGetLastError());
    RT_CUDA(cudaFreeAsync(buf, s));
    return RT_OK;
}

rt_status launch_philox(const uint32_t ctr0[4], const uint32_t key[2], uint64_t n, uint32_t* out,
                        cudaStream_t s)
{
    if (n == 0) return RT_OK;
    philox_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
        make_uint4(ctr0[0], ctr0[1], ctr0[2], ctr0[3]), make_uint2(key[0], key[1]), n, (uint4*)out);
    count_launches();
    RT_CUDA(cudaGetLastError());
    return RT_OK;
}

rt_status launch_mrw_sample(const float* table, const float* u, uint64_t n, float* y, cudaStream_t s)
{
    if (n == 0) return RT_OK;
    mrw_sample_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(table, u, n, y);
    count_launches();
    RT_CUDA(cudaGetLastError());
    return RT_OK;
}

}  // namespace rtgb
