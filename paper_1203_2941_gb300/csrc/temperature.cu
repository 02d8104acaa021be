// Dust temperatures (Heymann & Siebenmorgen 2012, Eq. 4) and the optically
// thin starting guess of the iterative scheme (Sect. 2), plus the Philox
// test hook.
#include <math.h>

#include "rt_internal.cuh"

namespace rtgb {

namespace {

constexpr double kPi = 3.14159265358979323846;

// One thread per (species, cell).  ln T starts from the tabulated inverse of
// ln(4 pi sum_j kabs_j B_j(T) dnu_j) and is polished by Newton steps on
//   F(ln T) = ln(4 pi P(T)) - ln(E / (rho V)),  F' = T P'(T) / P(T),
// which converge to double precision in two or three steps.  A bracketing
// bisection (same rule as the FP64 reference) takes over if P underflows.
__global__ void temperatures_kernel(const float* rho, const double* E, double* T, size_t nc, int ns,
                                    double vol, int nf, const double* nu, const double* dnu,
                                    const double* kabs, const double* tinv64,
                                    const double* y0, const double* inv_dy)
{
    extern __shared__ double sh[];
    double* a = sh;                 // [ns][nf] 4 pi kabs dnu 2 h nu^3 / c^2
    double* x1 = sh + ns * nf;      // [nf] h nu / k
    const double h = 6.62607015e-27, kb = 1.380649e-16, c = 2.99792458e10;
    for (int i = threadIdx.x; i < ns * nf; i += blockDim.x) {
        const int j = i % nf;
        a[i] = 4.0 * kPi * kabs[i] * dnu[j] * 2.0 * h * nu[j] * nu[j] * nu[j] / (c * c);
    }
    for (int j = threadIdx.x; j < nf; j += blockDim.x) x1[j] = h * nu[j] / kb;
    __syncthreads();

    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= nc * ns) return;
    const int s = (int)(i / nc);
    const double rv = (double)rho[i] * vol;
    const double e = E[i];
    if (!(rv > 0.0) || !(e > 0.0)) { T[i] = 0.0; return; }
    const double target = e / rv;
    const double z = log(target);
    const double* as = a + s * nf;
    double lnT;
    if (inv_dy[s] > 0.0) {
        double f = (z - y0[s]) * inv_dy[s];
        f = fmin(fmax(f, 0.0), (double)(kTinv64N - 1));
        const int k = min((int)f, kTinv64N - 2);
        const double w = f - k;
        const double* t = tinv64 + (size_t)s * kTinv64N;
        lnT = t[k] + w * (t[k + 1] - t[k]);
    } else {
        T[i] = 0.0;
        return;
    }
    bool ok = false;
    for (int it = 0; it < 8; ++it) {
        const double Tc = exp(lnT);
        double P = 0.0, dP = 0.0;
        for (int j = 0; j < nf; ++j) {
            const double x = x1[j] / Tc;
            const double em = exp(-x);
            const double om = x < 0.1 ? -expm1(-x) : 1.0 - em;
            const double b = as[j] * em / om;
            P += b;
            dP += b * x / om;          // T dB/dT summed
        }
        if (!(P > 0.0) || !isfinite(P) || !(dP > 0.0)) break;
        const double step = (log(P) - z) / (dP / P);
        lnT -= step;
        if (fabs(step) < 1e-13) { ok = true; break; }
    }
    if (!ok) {
        // bisection on [0, 1e5] (expanded), 1e-12 relative, as in the reference
        double lo = 0.0, hi = 1.0e5;
        auto em4pi = [&](double Tc) {
            double P = 0.0;
            for (int j = 0; j < nf; ++j) P += as[j] / expm1(x1[j] / Tc);
            return P;
        };
        for (int it = 0; it < 64 && em4pi(hi) < target; ++it) hi *= 2.0;
        for (int it = 0; it < 200 && hi - lo > 1e-12 * hi; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (em4pi(mid) < target) lo = mid; else hi = mid;
        }
        T[i] = 0.5 * (lo + hi);
        return;
    }
    T[i] = exp(lnT);
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
    double* tab = nullptr;
    RT_CUDA(cudaMallocAsync(&tab, sizeof(double) * 2 * kMaxSpecies, s));
    double h[2 * kMaxSpecies];
    for (int k = 0; k < kMaxSpecies; ++k) {
        h[k] = k < op->ns ? op->t64_y0[k] : 0.0;
        h[kMaxSpecies + k] = k < op->ns ? op->t64_inv_dy[k] : 0.0;
    }
    RT_CUDA(cudaMemcpyAsync(tab, h, sizeof(h), cudaMemcpyHostToDevice, s));
    const size_t smem = sizeof(double) * (op->ns * op->nf + op->nf);
    RT_CUDA(cudaFuncSetAttribute(temperatures_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    const int th = 256;
    temperatures_kernel<<<(unsigned)((n + th - 1) / th), th, smem, s>>>(
        g->d_rho, E, T, nc, g->ns, g->cell * g->cell * g->cell, op->nf, op->d_nu, op->d_dnu,
        op->d_kabs, op->d_tinv64, tab, tab + kMaxSpecies);
    count_launches();
    RT_CUDA(cudaGetLastError());
    RT_CUDA(cudaFreeAsync(tab, s));
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
