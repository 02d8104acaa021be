// Host-side construction of the per-opacity device tables:
//  * float4 {kext, kabs, ksca, g} per species and frequency,
//  * re-emission alias tables for the Eq. 5 (B) and Eq. 10 (dB/dT) bin laws,
//  * inverse Planck-mean tables (Eq. 4): log2 T on a uniform grid of
//    log2(4 pi sum_j kabs_j B_j(T) dnu_j) for the FP32 transport and ln T on a
//    uniform ln grid for the FP64 temperature solve,
//  * the survival function of the modified random walk (Sect. 3.2).
#include <math.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "rt_internal.cuh"

namespace rtgb {

static const double kH = 6.62607015e-27;   // erg s
static const double kK = 1.380649e-16;     // erg / K
static const double kC = 2.99792458e10;    // cm / s
static const double kPi = 3.14159265358979323846;

double planck_B_host(double nu, double T)
{
    if (T <= 0.0) return 0.0;
    const double x = kH * nu / (kK * T);
    return 2.0 * kH * nu * nu * nu / (kC * kC) / expm1(x);
}

void source_spectrum(const rt_opacity* op, const rt_source& src, std::vector<double>& lnu)
{
    lnu.assign(op->nf, 0.0);
    double tot = 0.0;
    for (int j = 0; j < op->nf; ++j) {
        lnu[j] = src.L_nu ? src.L_nu[j] : planck_B_host(op->nu[j], src.T_eff);
        tot += lnu[j] * op->dnu[j];
    }
    for (int j = 0; j < op->nf; ++j) lnu[j] = tot > 0.0 ? src.L * lnu[j] / tot : 0.0;
}

// ------------------------------------------------------------------------
// Source frequency grid of Eq. 1 (Sect. 2): the sources' combined luminosity
// cut into m bins of equal energy on each source's own continuous spectrum
// (a blackbody of T_eff; a tabulated L_nu is constant over each model
// frequency bin) between the outer edges of the model bins, whose edges are
// the geometric means of neighbouring frequencies (outer edges mirrored in
// ln nu).  Bin b is monochromatic at the frequency where the cumulative
// luminosity reaches (b + 1/2) L/m -- its source first, by the running sum of
// the sources' luminosities -- and belongs to the model bin holding it.
//
// The blackbody's cumulative is tabulated in ln nu on 2^15 intervals by
// Simpson's rule (relative error ~1e-14); a target inside an interval is
// solved by Newton steps on the single-panel Simpson integral from the
// interval's start.
namespace {

struct SourceCum {
    bool tab = false;
    std::vector<double> F;        // cumulative at the nodes (blackbody) or bin ends (tabulated)
    double t0 = 0.0, h = 0.0, a = 0.0;
    const std::vector<double>* e = nullptr;
    const double* lnu = nullptr;

    double g(double t) const      // integrand in ln nu: B_nu nu (unnormalised)
    {
        const double nu = exp(t);
        const double x = a * nu;
        return x > 700.0 ? 0.0 : nu * nu * nu * nu / expm1(x);
    }

    void build(const std::vector<double>& edges, const rt_source& s)
    {
        e = &edges;
        const int nf = (int)edges.size() - 1;
        if (s.L_nu) {
            tab = true;
            lnu = s.L_nu;
            F.assign(nf + 1, 0.0);
            for (int j = 0; j < nf; ++j) F[j + 1] = F[j] + s.L_nu[j] * (edges[j + 1] - edges[j]);
            return;
        }
        a = kH / (kK * s.T_eff);
        const int K = 1 << 15;
        t0 = log(edges[0]);
        h = (log(edges[nf]) - t0) / K;
        F.assign(K + 1, 0.0);
        for (int k = 0; k < K; ++k) {
            const double tl = t0 + k * h;
            F[k + 1] = F[k] + h / 6.0 * (g(tl) + 4.0 * g(tl + 0.5 * h) + g(tl + h));
        }
    }

    // frequency where the cumulative fraction reaches f (0 < f < 1)
    double invert(double f) const
    {
        const double target = f * F.back();
        const size_t k = std::upper_bound(F.begin(), F.end(), target) - F.begin() - 1;
        const size_t kk = std::min(k, F.size() - 2);
        const double rem = target - F[kk];
        if (tab) {
            const double w = F[kk + 1] - F[kk];
            const double lo = (*e)[kk], hi = (*e)[kk + 1];
            return w > 0.0 ? lo + (hi - lo) * (rem / w) : lo;
        }
        const double tl = t0 + kk * h;
        double dt = F[kk + 1] > F[kk] ? h * rem / (F[kk + 1] - F[kk]) : 0.0;
        for (int it = 0; it < 6; ++it) {
            const double S = dt / 6.0 * (g(tl) + 4.0 * g(tl + 0.5 * dt) + g(tl + dt));
            const double gd = g(tl + dt);
            if (!(gd > 0.0)) break;
            dt -= (S - rem) / gd;
            dt = std::min(std::max(dt, 0.0), h);
        }
        return exp(tl + dt);
    }
};

}  // namespace

rt_status build_source_grid(const rt_opacity* op, const rt_source* src, int nsrc, uint32_t m,
                            int32_t* nu_idx, int32_t* src_idx, double* nu_star)
{
    const int nf = op->nf;
    std::vector<double> e(nf + 1);
    for (int j = 1; j < nf; ++j) e[j] = sqrt(op->nu[j - 1] * op->nu[j]);
    e[0] = nf > 1 ? op->nu[0] * op->nu[0] / e[1] : 0.5 * op->nu[0];
    e[nf] = nf > 1 ? op->nu[nf - 1] * op->nu[nf - 1] / e[nf - 1] : 2.0 * op->nu[0];
    std::vector<SourceCum> cum(nsrc);
    double Ltot = 0.0;
    for (int i = 0; i < nsrc; ++i) {
        cum[i].build(e, src[i]);
        Ltot += src[i].L;
    }
    for (uint32_t b = 0; b < m; ++b) {
        const double target = ((double)b + 0.5) / (double)m * Ltot;
        double below = 0.0;
        int si = 0;
        for (; si < nsrc - 1; ++si) {
            if (below + src[si].L >= target) break;
            below += src[si].L;
        }
        const double f = src[si].L > 0.0 ? (target - below) / src[si].L : 0.5;
        const double nus = cum[si].invert(f);
        const int j = (int)(std::upper_bound(e.begin() + 1, e.begin() + nf, nus) - (e.begin() + 1));
        nu_idx[b] = j;
        src_idx[b] = si;
        if (nu_star) nu_star[b] = nus;
    }
    return RT_OK;
}

// ln(4 pi sum_j kabs_j B(nu_j, T) dnu_j) by log-sum-exp (no underflow at low T);
// lnc[j] = ln(kabs_j dnu_j 2 h nu_j^3 / c^2) (or -inf), x1[j] = h nu_j / k.
// *slope (optional) receives d ln(4 pi P) / d ln T = <x / (1 - e^-x)> over the
// emission-weighted bins.
static double ln_emission(const std::vector<double>& lnc, const std::vector<double>& x1, double T,
                          double* slope = nullptr)
{
    const size_t nf = lnc.size();
    double mx = -INFINITY;
    double t[rtgb::kMaxFreq];
    for (size_t j = 0; j < nf; ++j) {
        if (!std::isfinite(lnc[j])) { t[j] = -INFINITY; continue; }
        const double x = x1[j] / T;
        const double lnexpm1 = x > 30.0 ? x + log1p(-exp(-x)) : log(expm1(x));
        t[j] = lnc[j] - lnexpm1;
        mx = std::max(mx, t[j]);
    }
    if (!std::isfinite(mx)) return -INFINITY;
    double acc = 0.0, acc_s = 0.0;
    for (size_t j = 0; j < nf; ++j)
        if (std::isfinite(t[j])) {
            const double w = exp(t[j] - mx);
            acc += w;
            const double x = x1[j] / T;
            acc_s += w * x / (-expm1(-x));
        }
    if (slope) *slope = acc_s / acc;
    return log(4.0 * kPi) + mx + log(acc);
}

// Invert a monotone increasing dense table (lnT_i, z_i) at uniform z targets
// by linear interpolation between the bracketing dense points.
static void invert_dense(const std::vector<double>& lnT, const std::vector<double>& z, double z0,
                         double dz, int n, std::vector<double>& out)
{
    out.resize(n);
    size_t k = 0;
    for (int i = 0; i < n; ++i) {
        const double zt = z0 + i * dz;
        while (k + 2 < z.size() && z[k + 1] < zt) ++k;
        const double a = z[k], b = z[k + 1];
        const double w = b > a ? std::min(1.0, std::max(0.0, (zt - a) / (b - a))) : 0.0;
        out[i] = lnT[k] + w * (lnT[k + 1] - lnT[k]);
    }
}

// Survival probability of the walk from the centre of an absorbing sphere:
// S(y) = 2 sum_n (-1)^(n+1) exp(-n^2 pi^2 y) = 1 - theta_4 written, for small
// y, through its Poisson-summed form 1 - (2/sqrt(pi y)) sum_m exp(-(m+1/2)^2/y).
static double mrw_S(double y)
{
    if (y <= 0.0) return 1.0;
    double s = 0.0;
    if (y < 0.08) {
        for (int m = 0; m < 40; ++m) {
            const double e = exp(-(m + 0.5) * (m + 0.5) / y);
            s += e;
            if (e < 1e-300) break;
        }
        return 1.0 - 2.0 / sqrt(kPi * y) * s;
    }
    for (int n = 1; n < 100; ++n) {
        const double e = exp(-(double)n * n * kPi * kPi * y);
        s += (n % 2) ? e : -e;
        if (e < 1e-20) break;
    }
    return 2.0 * s;
}

rt_status build_opacity_tables(rt_opacity* op)
{
    const int nf = op->nf, ns = op->ns;
    const size_t sf = (size_t)ns * nf;
    std::vector<float4> o32(sf);
    for (int s = 0; s < ns; ++s)
        for (int j = 0; j < nf; ++j) {
            const double ka = op->kabs[s * nf + j], ks = op->ksca[s * nf + j];
            o32[s * nf + j] = make_float4((float)(ka + ks), (float)ka, (float)ks, (float)op->g[s * nf + j]);
        }

    // Re-emission tables for the FP32 transport: for each species and each
    // temperature of a uniform log2 T grid (0.1 K .. 1e6 K), the bin
    // probabilities kabs B(T) dnu (Eq. 5) and kabs dB/dT dnu (Eq. 10), built in
    // log form in FP64 (no underflow at 0.1 K), as alias tables (Walker 1977,
    // in the form of Vose 1991): with n bins, bin j keeps the threshold q_j
    // and the alias a_j such that drawing j0 = floor(u n) and taking j0 when
    // the fraction u n - j0 is below q_j0, else a_j0, yields bin j with its
    // probability.  One 32-bit word per entry: q in 22-bit fixed point above
    // a 10-bit alias (n <= 1024), so a draw is a single table read.
    const double lg_lo = log2(0.1), lg_hi = log2(1.0e6);
    const double dlg = (lg_hi - lg_lo) / (kReT - 1);
    op->re_lg0 = (float)lg_lo;
    op->re_inv_dlg = (float)(1.0 / dlg);
    std::vector<uint32_t> realias((size_t)2 * ns * kReT * nf);
    {
        std::vector<double> lw(nf), pw(nf);
        std::vector<int> small, large;
        for (int mode = 0; mode < 2; ++mode)
            for (int s = 0; s < ns; ++s)
                for (int k = 0; k < kReT; ++k) {
                    const double T = exp2(lg_lo + k * dlg);
                    double mx = -INFINITY;
                    for (int j = 0; j < nf; ++j) {
                        const double ka = op->kabs[s * nf + j];
                        const double x = kH * op->nu[j] / (kK * T);
                        const double l1m = log(-expm1(-x));          // ln(1 - e^-x)
                        double v = ka > 0.0 ? log(ka) + log(op->dnu[j]) + 3.0 * log(op->nu[j]) - x - l1m
                                            : -INFINITY;
                        if (mode == 1 && ka > 0.0) v += log(op->nu[j]) - l1m;   // dB/dT: one more nu / (1 - e^-x)
                        lw[j] = v;
                        mx = std::max(mx, v);
                    }
                    uint32_t* row = &realias[(((size_t)mode * ns + s) * kReT + k) * nf];
                    double acc = 0.0;
                    for (int j = 0; j < nf; ++j) {
                        pw[j] = std::isfinite(mx) && std::isfinite(lw[j]) ? exp(lw[j] - mx) : 0.0;
                        acc += pw[j];
                    }
                    // scaled probabilities n p_j (uniform when the row is empty)
                    for (int j = 0; j < nf; ++j) pw[j] = acc > 0.0 ? pw[j] * nf / acc : 1.0;
                    std::vector<double> q(nf, 1.0);
                    std::vector<int> al(nf);
                    small.clear();
                    large.clear();
                    for (int j = 0; j < nf; ++j) {
                        al[j] = j;
                        (pw[j] < 1.0 ? small : large).push_back(j);
                    }
                    while (!small.empty() && !large.empty()) {
                        const int l = small.back(), g = large.back();
                        small.pop_back();
                        large.pop_back();
                        q[l] = pw[l];
                        al[l] = g;
                        pw[g] = (pw[g] + pw[l]) - 1.0;
                        (pw[g] < 1.0 ? small : large).push_back(g);
                    }
                    for (int j = 0; j < nf; ++j) {
                        const double qq = std::min(std::max(q[j], 0.0), 1.0);
                        const uint32_t fx = (uint32_t)std::min(std::llround(qq * 4194304.0), 4194304LL);
                        row[j] = (fx << 10) | (uint32_t)al[j];
                    }
                }
    }

    // exact tabulation of z = ln(4 pi P(T)) and dz/dlnT on a uniform ln T grid
    // (FP64 temperatures), inverted on a uniform z grid for the FP32 transport
    const double lnTlo = log(0.1), lnThi = log(1.0e6);
    std::vector<double2> tz((size_t)ns * kTz64N);
    op->tz_lnT0 = lnTlo;
    op->tz_dlnT = (lnThi - lnTlo) / (kTz64N - 1);
    std::vector<float> tinv((size_t)ns * kTinvN);
    std::vector<TwNode> tw((size_t)ns * kTz64N);
    std::vector<float> zinv((size_t)ns * kZinvN);
    std::vector<double> lnTd(kTz64N), zd(kTz64N), inv;
    std::vector<double> x1(nf), lnc(nf);
    for (int j = 0; j < nf; ++j) x1[j] = kH * op->nu[j] / kK;
    for (int s = 0; s < ns; ++s) {
        for (int j = 0; j < nf; ++j) {
            const double ka = op->kabs[s * nf + j];
            lnc[j] = ka > 0.0 ? log(ka) + log(op->dnu[j]) + log(2.0 * kH / (kC * kC)) +
                                    3.0 * log(op->nu[j])
                              : -INFINITY;
        }
        bool ok = true;
        for (int i = 0; i < kTz64N; ++i) {
            double sl = 0.0;
            lnTd[i] = lnTlo + i * op->tz_dlnT;
            zd[i] = ln_emission(lnc, x1, exp(lnTd[i]), &sl);
            tz[(size_t)s * kTz64N + i] = make_double2(zd[i], sl);
            if (!std::isfinite(zd[i]) || (i > 0 && !(zd[i] > zd[i - 1]))) ok = false;
            TwNode& n = tw[(size_t)s * kTz64N + i];
            n.W = exp(zd[i]);                            // 0 where 4 pi P underflows
            n.m = n.W * sl * op->tz_dlnT;
            n.T = exp(lnTd[i]);
            n.g = sl > 0.0 ? 1.0 / (sl * op->tz_dlnT) : 0.0;
        }
        op->tw_ok[s] = ok ? 1 : 0;
        if (!ok) {
            for (int i = 0; i < kZinvN; ++i) zinv[(size_t)s * kZinvN + i] = 0.0f;
            op->zinv_z0[s] = 0.0f; op->zinv_idz[s] = 0.0f;
            // a species without absorption: temperatures stay at the table floor
            for (int i = 0; i < kTinvN; ++i) tinv[(size_t)s * kTinvN + i] = (float)(lnTlo / log(2.0));
            op->tinv_y0[s] = 0.0f; op->tinv_inv_dy[s] = 0.0f;
            continue;
        }
        const double zlo = zd[0], zhi = zd[kTz64N - 1];
        const double dy = (zhi - zlo) / log(2.0) / (kTinvN - 1);
        invert_dense(lnTd, zd, zlo, dy * log(2.0), kTinvN, inv);
        for (int i = 0; i < kTinvN; ++i) tinv[(size_t)s * kTinvN + i] = (float)(inv[i] / log(2.0));
        op->tinv_y0[s] = (float)(zlo / log(2.0));
        op->tinv_inv_dy[s] = (float)(1.0 / dy);
        // grid position (lnT - lnT0) / h on a uniform z grid: the FP32 start
        // of the FP64 temperature solve
        const double dzi = (zhi - zlo) / (kZinvN - 1);
        invert_dense(lnTd, zd, zlo, dzi, kZinvN, inv);
        for (int i = 0; i < kZinvN; ++i)
            zinv[(size_t)s * kZinvN + i] = (float)((inv[i] - lnTlo) / op->tz_dlnT);
        op->zinv_z0[s] = (float)zlo;
        op->zinv_idz[s] = (float)(1.0 / dzi);
    }

    std::vector<float> mrw(kMrwN);
    for (int i = 0; i < kMrwN; ++i) mrw[i] = (float)mrw_S(kMrwYmax * i / (kMrwN - 1));

    RT_CUDA(cudaMalloc(&op->d_nu, sizeof(double) * nf));
    RT_CUDA(cudaMalloc(&op->d_dnu, sizeof(double) * nf));
    RT_CUDA(cudaMalloc(&op->d_kabs, sizeof(double) * sf));
    RT_CUDA(cudaMalloc(&op->d_ksca, sizeof(double) * sf));
    RT_CUDA(cudaMalloc(&op->d_g, sizeof(double) * sf));
    RT_CUDA(cudaMalloc(&op->d_opac32, sizeof(float4) * sf));
    RT_CUDA(cudaMalloc(&op->d_realias, sizeof(uint32_t) * realias.size()));
    RT_CUDA(cudaMalloc(&op->d_tinv, sizeof(float) * tinv.size()));
    RT_CUDA(cudaMalloc(&op->d_tz, sizeof(double2) * tz.size()));
    RT_CUDA(cudaMalloc(&op->d_tw, sizeof(TwNode) * tw.size()));
    RT_CUDA(cudaMalloc(&op->d_zinv, sizeof(float) * zinv.size()));
    RT_CUDA(cudaMalloc(&op->d_mrwS, sizeof(float) * kMrwN));
    RT_CUDA(cudaMemcpy(op->d_nu, op->nu.data(), sizeof(double) * nf, cudaMemcpyHostToDevice));
    RT_CUDA(cudaMemcpy(op->d_dnu, op->dnu.data(), sizeof(double) * nf, cudaMemcpyHostToDevice));
    RT_CUDA(cudaMemcpy(op->d_kabs, op->kabs.data(), sizeof(double) * sf, cudaMemcpyHostToDevice));
    RT_CUDA(cudaMemcpy(op->d_ksca, op->ksca.data(), sizeof(double) * sf, cudaMemcpyHostToDevice));
    RT_CUDA(cudaMemcpy(op->d_g, op->g.data(), sizeof(double) * sf, cudaMemcpyHostToDevice));
    RT_CUDA(cudaMemcpy(op->d_opac32, o32.data(), sizeof(float4) * sf, cudaMemcpyHostToDevice));
    RT_CUDA(cudaMemcpy(op->d_realias, realias.data(), sizeof(uint32_t) * realias.size(), cudaMemcpyHostToDevice));
    RT_CUDA(cudaMemcpy(op->d_tinv, tinv.data(), sizeof(float) * tinv.size(), cudaMemcpyHostToDevice));
    RT_CUDA(cudaMemcpy(op->d_tz, tz.data(), sizeof(double2) * tz.size(), cudaMemcpyHostToDevice));
    RT_CUDA(cudaMemcpy(op->d_tw, tw.data(), sizeof(TwNode) * tw.size(), cudaMemcpyHostToDevice));
    RT_CUDA(cudaMemcpy(op->d_zinv, zinv.data(), sizeof(float) * zinv.size(), cudaMemcpyHostToDevice));
    RT_CUDA(cudaMemcpy(op->d_mrwS, mrw.data(), sizeof(float) * kMrwN, cudaMemcpyHostToDevice));
    return RT_OK;
}

}  // namespace rtgb
