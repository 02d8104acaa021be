// Dust temperatures (Heymann & Siebenmorgen 2012, Eq. 4) and the optically
// thin starting guess of the iterative scheme (Sect. 2), plus the Philox
// test hook.
#include <math.h>

#include "rt_internal.cuh"

namespace rtgb {

namespace {

constexpr double kPi = 3.14159265358979323846;

// One thread per (species, cell).  The left-hand side of Eq. 4 in log form,
// z(T) = ln(4 pi sum_j kabs_j B_j(T) dnu_j), is tabulated exactly (value and
// slope dz/dlnT, FP64) on a fine uniform ln T grid from 0.1 K to 1e6 K.  A cell
// solves z(T) = ln(E / (rho V)) by binary search for the bracketing table
// interval and Newton iterations on that interval's cubic Hermite interpolant,
// whose error (h^4/384 times the fourth derivative, h = 2.5e-4) is below double
// rounding.  Targets outside the table fall back to bisection on the Planck sum.
__global__ void temperatures_kernel(const float* rho, const double* E, double* T, size_t nc, int ns,
                                    double vol, const double2* tz, double lnT0, double dlnT, int nf,
                                    const double* nu, const double* dnu, const double* kabs)
{
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= nc * ns) return;
    const int s = (int)(i / nc);
    const double rv = (double)rho[i] * vol;
    const double e = E[i];
    if (!(rv > 0.0) || !(e > 0.0)) { T[i] = 0.0; return; }
    const double target = e / rv;
    const double z = log(target);
    const double2* t = tz + (size_t)s * kTz64N;
    if (z >= t[0].x && z <= t[kTz64N - 1].x) {
        int lo = 0, hi = kTz64N - 1;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (t[mid].x <= z) lo = mid; else hi = mid;
        }
        const double2 a = t[lo], b = t[hi];
        const double m0 = a.y * dlnT, m1 = b.y * dlnT;
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
        T[i] = exp(lnT0 + ((double)lo + u) * dlnT);
        return;
    }
    // outside 0.1 K .. 1e6 K: bisection on 4 pi sum_j kabs B dnu = target
    const double h = 6.62607015e-27, kb = 1.380649e-16, c = 2.99792458e10;
    auto em4pi = [&](double Tc) {
        double P = 0.0;
        for (int j = 0; j < nf; ++j)
            P += 4.0 * kPi * kabs[s * nf + j] * dnu[j] * 2.0 * h * nu[j] * nu[j] * nu[j] /
                 (c * c) / expm1(h * nu[j] / (kb * Tc));
        return P;
    };
    double lo = 0.0, hi = 1.0e5;
    for (int it = 0; it < 64 && em4pi(hi) < target; ++it) hi *= 2.0;
    for (int it = 0; it < 200 && hi - lo > 1e-12 * hi; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (em4pi(mid) < target) lo = mid; else hi = mid;
    }
    T[i] = 0.5 * (lo + hi);
}

__global__ void guess_kernel(int nx, int ny, int nz, int ns, double bx, double by, double bz,
                             double cell, const double* pos, const double* L, int nsrc, double* T)
{
    const size_t nc = (size_t)nx * ny * nz;
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const double h = 6.62607015e-27, kb = 1.380649e-16, c = 2.99792458e10;
    const double sigma = 2.0 * pow(kPi, 5) * pow(kb, 4) / (15.0 * h * h * h * c * c);
    const int ix = (int)(i % nx), iy = (int)((i / nx) % ny), iz = (int)(i / ((size_t)nx * ny));
    const double x = bx + (ix + 0.5) * cell, y = by + (iy + 0.5) * cell, z = bz + (iz + 0.5) * cell;
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

}  // namespace

rt_status launch_temperatures(rt_ctx* ctx, const rt_grid* g, const rt_opacity* op, const double* E,
                              double* T, cudaStream_t s)
{
    (void)ctx;
    const size_t nc = g->ncell();
    const size_t n = nc * g->ns;
    const int th = 256;
    temperatures_kernel<<<(unsigned)((n + th - 1) / th), th, 0, s>>>(
        g->d_rho, E, T, nc, g->ns, g->cell * g->cell * g->cell, op->d_tz, op->tz_lnT0, op->tz_dlnT,
        op->nf, op->d_nu, op->d_dnu, op->d_kabs);
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
        buf + 3 * nsrc, nsrc, T);
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

}  // namespace rtgb
