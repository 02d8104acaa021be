// Ray tracer for images and SEDs (Heymann & Siebenmorgen 2012, Sect. 4) and
// its adjoint with respect to the cell densities.
//
//   eta_th[c][f]       = sum_s rho_s kabs_s(nu_f) B(nu_f, T_s)      (Eq. 14)
//   eta[cam][c][f]     = eta_th + xi_ev / (V dnu_f) sum_events P_HG(k_in . k_obs)  (Eq. 16)
// (tables hold eta times the cell size, so FP32 stays far from underflow)
//   I(pixel, f)        = sum_k S_k (1 - exp(-dtau_k)) exp(-tau_<k),  S = eta / chi  (Eqs. 12-13)
//   sed[cam][f]        = sum_pix I A_pix / D^2 + sum_src L_nu exp(-tau_src) / (4 pi D^2)  (Eq. 17)
//
// Rays start on the box face nearest the observer (parallel projection,
// Eq. 11) and march front to back through the grid with an incremental DDA;
// a ray carries all requested frequencies, so each cell visit loads the
// density once and the emissivities of all frequencies as contiguous float4s.
// Optical depths are summed with compensation (Kahan) in FP32.
#include <math.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "rt_internal.cuh"

namespace rtgb {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kCamChunk = 16;

// Pixel rays walk the grid in FP32 with double-float face times.  A face
// time of axis a is affine in the face index, t_a(k) = t_a(0) + k/|d_a|, so
// the walk keeps, per axis, the time of the next face as an unevaluated sum
// hi + lo of two floats (about 48 significant bits) and advances it by the
// double-float 1/|d_a| when the ray crosses that face; the chord of a cell is
// the difference of two such times, rounded once to FP32.  Chords are then
// exact to about 1e-12 cell edges however far the ray has marched, which
// keeps even the short chords of rays clipping a cell's corner accurate: a
// plain FP32 walk (one float per face time, or per distance to a face) lets
// the rounding of the direction and of each step accumulate to about 1e-7
// edges within a few dozen cells.  The entry point, cell and first face times
// are computed in FP64 once per ray.
struct DF {
    float hi, lo;
};

__host__ __device__ __forceinline__ DF df_of(double v)
{
    DF r;
    r.hi = (float)v;
    r.lo = (float)(v - (double)r.hi);
    return r;
}

// a + b (two-sum of the high parts, then the low parts; renormalised)
__host__ __device__ __forceinline__ DF df_add(DF a, DF b)
{
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb);
    const float lo = e + (a.lo + b.lo);
    DF r;
    r.hi = s + lo;
    r.lo = lo - (r.hi - s);
    return r;
}

// a - m b for a small non-negative integer m (exact product error by fma)
__host__ __device__ __forceinline__ DF df_sub_mul(DF a, float m, DF b)
{
    const float p = m * b.hi;
    const float pe = fmaf(m, b.hi, -p) + m * b.lo;
    DF nb;
    nb.hi = -p;
    nb.lo = -pe;
    return df_add(a, nb);
}

// a - b rounded to FP32
__host__ __device__ __forceinline__ float df_diff(DF a, DF b) { return (a.hi - b.hi) + (a.lo - b.lo); }

// a <= b
__host__ __device__ __forceinline__ bool df_le(DF a, DF b) { return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo); }

// Per-camera walk constants: 1/|d_a| and 1/(r |d_a|) (sub-cube face spacing)
// as double-floats, |d_a| r in FP32, and the axes marched towards -axis.
struct WalkCam {
    DF td[3], tds[3];
    float adr[3];              // r |d_a|: time to sub-edges along axis a
};

struct CamDev {
    double k[3], ex[3], ey[3]; // observer direction and image axes (FP64: ray set-up)
    double ik[3];              // 1 / k_a (0 when k_a = 0)
    double pix_cell;           // pixel size in cells
    double apix_d2;            // A_pix / D^2
    WalkCam wc;                // double-float face spacings of the FP32 walk
    unsigned negf, negr;       // axes marched towards -axis: forward (along -k), reverse (along +k)
    int npix;
};

struct RayKP {
    const void* rho;           // packed FP32 grid (rho * cell, Lucy sign bit ignored)
    int nx, ny, nz;
    int ns;                    // species (<= NS, the packed width)
    float cell;
    float kext[kMaxSpecies][kMaxImgFreq];   // cm^2/g (packed density is rho * cell)
    float kext_cell[kMaxSpecies][kMaxImgFreq];  // kext * cell
    int nfi, nfp;
    size_t ncell;
    const float* eta;          // [ncam_total][ncell][nfp] eta * cell
    const float* bk;           // [ns][ncell][nfp] kabs_s B(T_s) * cell (backward)
    CamDev cam[kCamChunk];
    int cam0, ncam;            // cameras of this launch: [cam0, cam0 + ncam)
    float* img;                // [ncam_total][nfi][npix][npix]
    const float* dimg;
    const double* dsed;        // [ncam_total][nfi]
    float* grad;               // [ns][ncell]
    unsigned long long* steps; // ray-cell step counter or nullptr
    const int* cube;           // refined grids: [ncube] first cell | kCubeDivided
    int refine;                // r, or 0
};

// add a per-thread step count to the counter, one atomic per warp
__device__ __forceinline__ void count_steps(unsigned long long* ctr, unsigned n)
{
    if (!ctr) return;
    const unsigned mask = __activemask();
    const unsigned tot = __reduce_add_sync(mask, n);
    if ((threadIdx.x & 31) == __ffs(mask) - 1 && tot) atomicAdd(ctr, (unsigned long long)tot);
}

template <int NS> struct PT;
template <> struct PT<1> { using T = float; };
template <> struct PT<2> { using T = float2; };
template <> struct PT<4> { using T = float4; };
__device__ __forceinline__ void unpack(float v, float* r) { r[0] = fabsf(v); }
__device__ __forceinline__ void unpack(float2 v, float* r) { r[0] = fabsf(v.x); r[1] = v.y; }
__device__ __forceinline__ void unpack(float4 v, float* r) { r[0] = fabsf(v.x); r[1] = v.y; r[2] = v.z; r[3] = v.w; }

__device__ __forceinline__ void kahan_add(float& s, float& comp, float v)
{
    const float y = v - comp;
    const float t = s + y;
    comp = (t - s) - y;
    s = t;
}

// (1 - e^-x) / x and its derivative
__device__ __forceinline__ float phi_f(float x)
{
    return x < 1e-4f ? 1.0f - 0.5f * x : -expm1f(-x) / x;
}
__device__ __forceinline__ float dphi_f(float x)
{
    if (x < 1e-2f) return -0.5f + x * (1.0f / 3.0f) - x * x * 0.125f;
    return (expf(-x) * (1.0f + x) - 1.0f) / (x * x);
}

// Two-level traversal of a grid with one level of refinement (Sect. 2):
// cube indices, sub-cube indices (8 bits per axis, -1 in an undivided cube),
// cell number and per-axis next-face times along p + t d (cube units).  A
// step inside a divided cube moves to the next sub-cube; leaving a cube
// enters the next one at the crossing point (its sub-cube along the other
// axes by position, ties as in the transport) and restarts the face times.
template <typename T>
struct RefWalk {
    int i[3];
    int sub, c;
    T tm[3], td[3];
    T ir;                      // 1 / r
};

template <typename T>
__device__ __forceinline__ void rw_times(RefWalk<T>& w, int r, const T* p, const T* d, T tcur)
{
    const T h = w.sub >= 0 ? w.ir : T(1);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const T lo = T(w.i[a]) + (w.sub >= 0 ? T((w.sub >> (8 * a)) & 255) * h : T(0));
        const T xa = p[a] + tcur * d[a];
        T dist;
        if (d[a] > T(0)) dist = lo + h - xa;
        else if (d[a] < T(0)) dist = xa - lo;
        else dist = T(INFINITY);
        w.tm[a] = d[a] != T(0) ? tcur + fmax(dist, T(0)) * w.td[a] : T(INFINITY);
    }
}

template <typename T>
__device__ __forceinline__ void rw_enter(RefWalk<T>& w, const int* cube, int nx, int ny, int r,
                                         const T* p, const T* d, T tcur, int ea)
{
    const int info = cube[(w.i[2] * ny + w.i[1]) * nx + w.i[0]];
    if (!(info & kCubeDivided)) {
        w.sub = -1;
        w.c = info;
    } else {
        int sb[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const T u = (p[a] + tcur * d[a] - T(w.i[a])) * T(r);
            const T f = floor(u);
            int sa = (int)f;
            if (f == u && d[a] < T(0)) sa -= 1;
            sa = min(max(sa, 0), r - 1);
            if (a == ea) sa = d[a] > T(0) ? 0 : r - 1;
            sb[a] = sa;
        }
        w.sub = sb[0] | (sb[1] << 8) | (sb[2] << 16);
        w.c = (info & ~kCubeDivided) + (sb[2] * r + sb[1]) * r + sb[0];
    }
    rw_times(w, r, p, d, tcur);
}

// start at p: the cube by floor (a coordinate on a face goes to the lower
// cube when d points to -axis), clamped into the grid when `clamp` (ray
// entry points on the box surface); false when p is outside
template <typename T>
__device__ __forceinline__ bool rw_start(RefWalk<T>& w, const int* cube, int nx, int ny, int nz, int r,
                                         const T* p, const T* d, bool clamp)
{
    const int n[3] = { nx, ny, nz };
    bool in = true;
    w.ir = T(1) / T(r);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const T f = floor(p[a]);
        int i = (int)f;
        if (f == p[a] && d[a] < T(0)) i -= 1;
        if (clamp) i = min(max(i, 0), n[a] - 1);
        in = in && i >= 0 && i < n[a];
        w.i[a] = i;
        w.td[a] = d[a] != T(0) ? T(1) / fabs(d[a]) : T(INFINITY);
    }
    if (in) rw_enter(w, cube, nx, ny, r, p, d, T(0), -1);
    return in;
}

// chord of the current cell (seg) and the step to the next; false when the
// path leaves the grid
template <typename T>
__device__ __forceinline__ bool rw_step(RefWalk<T>& w, const int* cube, int nx, int ny, int nz, int r,
                                        const T* p, const T* d, T& tcur, T& seg)
{
    const int a = (w.tm[0] <= w.tm[1] && w.tm[0] <= w.tm[2]) ? 0 : (w.tm[1] <= w.tm[2] ? 1 : 2);
    const T tn = a == 0 ? w.tm[0] : (a == 1 ? w.tm[1] : w.tm[2]);
    seg = tn - tcur;
    tcur = tn;
    const T da = a == 0 ? d[0] : (a == 1 ? d[1] : d[2]);
    const int sg = da > T(0) ? 1 : -1;
    if (w.sub >= 0) {
        const int sa = ((w.sub >> (8 * a)) & 255) + sg;
        if (sa >= 0 && sa < r) {
            w.sub = (w.sub & ~(255 << (8 * a))) | (sa << (8 * a));
            w.c += sg * (a == 0 ? 1 : (a == 1 ? r : r * r));
            if (a == 0) w.tm[0] += w.td[0] * w.ir;
            else if (a == 1) w.tm[1] += w.td[1] * w.ir;
            else w.tm[2] += w.td[2] * w.ir;
            return true;
        }
    }
    w.i[0] += a == 0 ? sg : 0;
    w.i[1] += a == 1 ? sg : 0;
    w.i[2] += a == 2 ? sg : 0;
    const int ia = a == 0 ? w.i[0] : (a == 1 ? w.i[1] : w.i[2]);
    const int n_a = a == 0 ? nx : (a == 1 ? ny : nz);
    if (ia < 0 || ia >= n_a) return false;
    rw_enter(w, cube, nx, ny, r, p, d, tcur, a);
    return true;
}

struct DFWalk {
    int i[3];                  // cube indices
    int sub;                   // refined grids: sub-cube indices, 8 bits per axis, or -1
    int c;                     // cell number
    DF tm[3];                  // time of the current cube's exit face per axis; for an axis
                               // with d_a = 0: {inf, cube-local coordinate} (refined grids)
    DF t;                      // time at the current point
};

// Set up from the entry point p (cell units, FP64) and direction d: cube by
// floor (a coordinate on a face goes to the lower cube when marching towards
// -axis), clamped into the grid; on a refined grid the sub-cube by the same
// rule inside the cube.
__host__ __device__ __forceinline__ void dw_start(DFWalk& w, const double* p, const double* d, int nx,
                                                  int ny, int nz, const int* cube, int r)
{
    const int n[3] = { nx, ny, nz };
    double q[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double f = floor(p[a]);
        int i = (int)f;
        if (f == p[a] && d[a] < 0.0) i -= 1;
        i = i < 0 ? 0 : (i > n[a] - 1 ? n[a] - 1 : i);
        w.i[a] = i;
        double qa = p[a] - (double)i;
        qa = qa < 0.0 ? 0.0 : (qa > 1.0 ? 1.0 : qa);
        q[a] = qa;
        if (d[a] > 0.0) w.tm[a] = df_of((1.0 - qa) / d[a]);
        else if (d[a] < 0.0) w.tm[a] = df_of(qa / -d[a]);
        else { w.tm[a].hi = INFINITY; w.tm[a].lo = (float)qa; }
    }
    w.t.hi = 0.0f;
    w.t.lo = 0.0f;
    const int q0 = (w.i[2] * ny + w.i[1]) * nx + w.i[0];
    const int info = cube ? cube[q0] : q0;
    if (!cube || !(info & kCubeDivided)) {
        w.sub = -1;
        w.c = info;
        return;
    }
    int sb[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double u = q[a] * r;
        const double f = floor(u);
        int s = (int)f;
        if (f == u && d[a] < 0.0) s -= 1;
        sb[a] = s < 0 ? 0 : (s > r - 1 ? r - 1 : s);
    }
    w.sub = sb[0] | (sb[1] << 8) | (sb[2] << 16);
    w.c = (info & ~kCubeDivided) + (sb[2] * r + sb[1]) * r + sb[0];
}

// Uniform grid: chord of the current cell (seg) and the step to the next
// (nearest face, ties to the lowest axis); false when the ray leaves the grid.
// `neg` has bit a set when the ray marches towards -axis a.
__host__ __device__ __forceinline__ bool dw_step(DFWalk& w, const WalkCam& wc, unsigned neg, int nx, int ny,
                                                 int nz, float& seg)
{
    const bool a0 = df_le(w.tm[0], w.tm[1]) && df_le(w.tm[0], w.tm[2]);
    const bool a1 = !a0 && df_le(w.tm[1], w.tm[2]);
    const int a = a0 ? 0 : (a1 ? 1 : 2);
    const DF tn = a == 0 ? w.tm[0] : (a == 1 ? w.tm[1] : w.tm[2]);
    const DF step = a == 0 ? wc.td[0] : (a == 1 ? wc.td[1] : wc.td[2]);
    seg = fmaxf(df_diff(tn, w.t), 0.0f);
    w.t = tn;
    const DF nt = df_add(tn, step);
    w.tm[0] = a == 0 ? nt : w.tm[0];
    w.tm[1] = a == 1 ? nt : w.tm[1];
    w.tm[2] = a == 2 ? nt : w.tm[2];
    const int sg = (neg >> a) & 1 ? -1 : 1;
    if (a == 0) { w.i[0] += sg; return (unsigned)w.i[0] < (unsigned)nx; }
    if (a == 1) { w.i[1] += sg; return (unsigned)w.i[1] < (unsigned)ny; }
    w.i[2] += sg;
    return (unsigned)w.i[2] < (unsigned)nz;
}

// Refined grid: the cube-level face times advance as on a uniform grid of
// cubes; inside a divided cube the next sub-face along axis b lies m_b
// sub-cube spacings before the cube's exit face (m_b = sub-faces still
// ahead).  Leaving a cube enters the next one; when it is divided the
// sub-cube along the entry axis is the first one met, along the other axes
// the one holding the crossing point (from its distance to the cube's exit
// face: a point on a sub-face belongs to the sub-cube ahead of it).
__host__ __device__ __forceinline__ bool dw_step_ref(DFWalk& w, const WalkCam& wc, unsigned neg,
                                                     const int* cube, int nx, int ny, int nz, int r,
                                                     float& seg)
{
    DF tf[3];
    if (w.sub < 0) {
        tf[0] = w.tm[0]; tf[1] = w.tm[1]; tf[2] = w.tm[2];
    } else {
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int s = (w.sub >> (8 * b)) & 255;
            const int m = ((neg >> b) & 1) ? s : r - 1 - s;
            tf[b] = (m == 0 || w.tm[b].hi == INFINITY) ? w.tm[b] : df_sub_mul(w.tm[b], (float)m, wc.tds[b]);
        }
    }
    const bool a0 = df_le(tf[0], tf[1]) && df_le(tf[0], tf[2]);
    const bool a1 = !a0 && df_le(tf[1], tf[2]);
    const int a = a0 ? 0 : (a1 ? 1 : 2);
    const DF tn = a == 0 ? tf[0] : (a == 1 ? tf[1] : tf[2]);
    seg = fmaxf(df_diff(tn, w.t), 0.0f);
    w.t = tn;
    const int sg = (neg >> a) & 1 ? -1 : 1;
    if (w.sub >= 0) {
        const int sa = ((w.sub >> (8 * a)) & 255) + sg;
        if (sa >= 0 && sa < r) {
            w.sub = (w.sub & ~(255 << (8 * a))) | (sa << (8 * a));
            w.c += sg * (a == 0 ? 1 : (a == 1 ? r : r * r));
            return true;
        }
    }
    // leave the cube through its face on axis a (selects, not a run-time
    // index: the walk state stays in registers)
    const DF nt = df_add(tn, a == 0 ? wc.td[0] : (a == 1 ? wc.td[1] : wc.td[2]));
    w.tm[0] = a == 0 ? nt : w.tm[0];
    w.tm[1] = a == 1 ? nt : w.tm[1];
    w.tm[2] = a == 2 ? nt : w.tm[2];
    w.i[0] += a == 0 ? sg : 0;
    w.i[1] += a == 1 ? sg : 0;
    w.i[2] += a == 2 ? sg : 0;
    const int ia = a == 0 ? w.i[0] : (a == 1 ? w.i[1] : w.i[2]);
    const int n_a = a == 0 ? nx : (a == 1 ? ny : nz);
    if (ia < 0 || ia >= n_a) return false;
    const int info = cube[(w.i[2] * ny + w.i[1]) * nx + w.i[0]];
    if (!(info & kCubeDivided)) {
        w.sub = -1;
        w.c = info;
        return true;
    }
    int sb[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const bool nb = (neg >> b) & 1;
        int s;
        if (b == a) {
            s = nb ? r - 1 : 0;
        } else if (w.tm[b].hi == INFINITY) {
            // no motion along b: the sub-cube of the constant coordinate
            s = (int)floorf(w.tm[b].lo * (float)r);
        } else {
            // distance to the cube's exit face along b, in sub-cube edges
            const float D = df_diff(w.tm[b], w.t) * wc.adr[b];
            const int m = (int)ceilf(D) - 1;
            s = nb ? m : r - 1 - m;
        }
        sb[b] = s < 0 ? 0 : (s > r - 1 ? r - 1 : s);
    }
    w.sub = sb[0] | (sb[1] << 8) | (sb[2] << 16);
    w.c = (info & ~kCubeDivided) + (sb[2] * r + sb[1]) * r + sb[0];
    return true;
}

// Entry point (cell units, FP64) and march direction of the ray of pixel
// (ix, iy): on the box face nearest the observer, marching along -kobs, or
// on the far face (reverse), marching along +kobs.  False when the pixel's
// line misses the box.
__device__ __forceinline__ bool ray_entry(const CamDev& cm, int ix, int iy, int nx, int ny, int nz,
                                          bool reverse, double* p, double* d)
{
    const double xp = ((double)ix + 0.5 - 0.5 * cm.npix) * cm.pix_cell;
    const double yp = ((double)iy + 0.5 - 0.5 * cm.npix) * cm.pix_cell;
    const int n[3] = { nx, ny, nz };
    double o[3];
    double lo = -INFINITY, hi = INFINITY;
    bool hit = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        o[a] = 0.5 * n[a] + xp * cm.ex[a] + yp * cm.ey[a];
        if (cm.k[a] != 0.0) {
            double s1 = -o[a] * cm.ik[a], s2 = ((double)n[a] - o[a]) * cm.ik[a];
            if (s1 > s2) { const double t = s1; s1 = s2; s2 = t; }
            lo = fmax(lo, s1);
            hi = fmin(hi, s2);
        } else if (o[a] < 0.0 || o[a] > (double)n[a]) {
            hit = false;
        }
    }
    if (!(hit && lo < hi)) return false;
    const double s0 = reverse ? lo : hi;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        p[a] = o[a] + s0 * cm.k[a];
        d[a] = reverse ? cm.k[a] : -cm.k[a];
    }
    return true;
}

// start the walk of pixel (ix, iy); false when its line misses the box
template <bool REF>
__device__ __forceinline__ bool pixel_walk(DFWalk& w, const CamDev& cm, int ix, int iy, int nx, int ny,
                                           int nz, const int* cube, int r, bool reverse)
{
    double p[3], d[3];
    if (!ray_entry(cm, ix, iy, nx, ny, nz, reverse, p, d)) return false;
    dw_start(w, p, d, nx, ny, nz, REF ? cube : nullptr, r);
    return true;
}

template <int NS>
__device__ __forceinline__ void load_rho(const RayKP& P, int c, float* rho)
{
    const typename PT<NS>::T v = __ldg(reinterpret_cast<const typename PT<NS>::T*>(P.rho) + c);
    float r[4];
    unpack(v, r);
#pragma unroll
    for (int s = 0; s < NS; ++s) rho[s] = r[s];
}

template <int NFP>
__device__ __forceinline__ void load_eta(const float* base, float* eta)
{
    const float4* q = reinterpret_cast<const float4*>(base);
#pragma unroll
    for (int v = 0; v < NFP / 4; ++v) {
        const float4 t = __ldg(q + v);
        eta[4 * v] = t.x; eta[4 * v + 1] = t.y; eta[4 * v + 2] = t.z; eta[4 * v + 3] = t.w;
    }
}

// Forward march.  A ray is served by NFP / 4 consecutive threads, each
// carrying four image frequencies (one float4 of the emissivity row): the
// threads repeat the ray's walk (the same arithmetic, so the same chords) and
// share its density loads, which keeps the compensated sums of a thread in
// few registers and the SMs well occupied.
template <int NS, int NFP, bool REF>
__global__ void __launch_bounds__(128) ray_fwd_kernel(const __grid_constant__ RayKP P)
{
    constexpr int G = NFP / 4;
    const int ci = blockIdx.y;
    const CamDev& cm = P.cam[ci];
    const int np = cm.npix;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long pix = t / G;
    const int g = (int)(t - pix * G);
    if (pix >= (long long)np * np) return;
    const int ix = (int)(pix % np), iy = (int)(pix / np);
    const int cam = P.cam0 + ci;
    float I[4], Ic[4], tau[4], tc[4], ke[NS][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        I[q] = 0.f; Ic[q] = 0.f; tau[q] = 0.f; tc[q] = 0.f;
#pragma unroll
        for (int s = 0; s < NS; ++s) ke[s][q] = P.kext[s][4 * g + q];
    }
    unsigned nsteps = 0;
    DFWalk w;
    if (pixel_walk<REF>(w, cm, ix, iy, P.nx, P.ny, P.nz, P.cube, P.refine, false)) {
        const float* eta_cam = P.eta + (size_t)cam * P.ncell * P.nfp + 4 * g;
        const int maxstep = (P.nx + P.ny + P.nz) * (REF ? P.refine : 1) + 4;
        for (int st = 0; st < maxstep; ++st) {
            ++nsteps;
            const int c = REF ? w.c : (w.i[2] * P.ny + w.i[1]) * P.nx + w.i[0];
            float rho[NS];
            load_rho<NS>(P, c, rho);
            const float4 e4 = __ldg(reinterpret_cast<const float4*>(eta_cam + (size_t)c * NFP));
            const float eta[4] = { e4.x, e4.y, e4.z, e4.w };
            float seg;
            const bool inside = REF ? dw_step_ref(w, cm.wc, cm.negf, P.cube, P.nx, P.ny, P.nz, P.refine, seg)
                                    : dw_step(w, cm.wc, cm.negf, P.nx, P.ny, P.nz, seg);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float chi = 0.f;
#pragma unroll
                for (int s = 0; s < NS; ++s) chi += rho[s] * ke[s][q];
                const float dt = chi * seg;
                const float contrib = eta[q] * seg * phi_f(dt) * expf(-tau[q]);
                kahan_add(I[q], Ic[q], contrib);
                kahan_add(tau[q], tc[q], dt);
            }
            if (!inside) break;
        }
    }
    float* out = P.img + ((size_t)cam * P.nfi) * np * np + pix;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (4 * g + q < P.nfi) out[(size_t)(4 * g + q) * np * np] = I[q];
    count_steps(P.steps, g == 0 ? nsteps : 0u);
}

// Adjoint: pass 1 (front to back) gives tau_total and I_total per frequency;
// pass 2 walks back to front from the far face, where the attenuation of the
// observer-side optical depth is exp(-(tau_total - tau_behind_incl)) and the
// sum of contributions farther than the current cell accumulates directly.
template <int NS, int NFP, bool REF>
__global__ void __launch_bounds__(128) ray_bwd_kernel(const __grid_constant__ RayKP P)
{
    const int ci = blockIdx.y;
    const CamDev& cm = P.cam[ci];
    const int np = cm.npix;
    const long long pix = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (pix >= (long long)np * np) return;
    const int ix = (int)(pix % np), iy = (int)(pix / np);
    const int cam = P.cam0 + ci;
    float w[NFP];
    bool any = false;
#pragma unroll
    for (int f = 0; f < NFP; ++f) {
        float v = 0.f;
        if (f < P.nfi) {
            if (P.dimg) v += P.dimg[((size_t)cam * P.nfi + f) * np * np + pix];
            if (P.dsed) v += (float)(P.dsed[(size_t)cam * P.nfi + f] * cm.apix_d2);
        }
        w[f] = v;
        any = any || v != 0.f;
    }
    if (!any) return;
    DFWalk w1;
    if (!pixel_walk<REF>(w1, cm, ix, iy, P.nx, P.ny, P.nz, P.cube, P.refine, false)) return;
    const float* eta_cam = P.eta + (size_t)cam * P.ncell * P.nfp;
    const int maxstep = (P.nx + P.ny + P.nz) * (REF ? P.refine : 1) + 4;
    float tot[NFP], totc[NFP];
    unsigned nsteps = 0;
#pragma unroll
    for (int f = 0; f < NFP; ++f) { tot[f] = 0.f; totc[f] = 0.f; }
    for (int st = 0; st < maxstep; ++st) {
        ++nsteps;
        const int c = REF ? w1.c : (w1.i[2] * P.ny + w1.i[1]) * P.nx + w1.i[0];
        float rho[NS];
        load_rho<NS>(P, c, rho);
        float seg;
        const bool inside = REF ? dw_step_ref(w1, cm.wc, cm.negf, P.cube, P.nx, P.ny, P.nz, P.refine, seg)
                                : dw_step(w1, cm.wc, cm.negf, P.nx, P.ny, P.nz, seg);
#pragma unroll
        for (int f = 0; f < NFP; ++f) {
            float chi = 0.f;
#pragma unroll
            for (int s = 0; s < NS; ++s) chi += rho[s] * P.kext[s][f];
            kahan_add(tot[f], totc[f], chi * seg);
        }
        if (!inside) break;
    }
    DFWalk w2;
    if (!pixel_walk<REF>(w2, cm, ix, iy, P.nx, P.ny, P.nz, P.cube, P.refine, true)) {
        count_steps(P.steps, nsteps);
        return;
    }
    float tb[NFP], tbc[NFP], beh[NFP], behc[NFP];
#pragma unroll
    for (int f = 0; f < NFP; ++f) { tb[f] = 0.f; tbc[f] = 0.f; beh[f] = 0.f; behc[f] = 0.f; }
    for (int st = 0; st < maxstep; ++st) {
        ++nsteps;
        const int c = REF ? w2.c : (w2.i[2] * P.ny + w2.i[1]) * P.nx + w2.i[0];
        float rho[NS], eta[NFP];
        load_rho<NS>(P, c, rho);
        load_eta<NFP>(eta_cam + (size_t)c * NFP, eta);
        float seg;
        const bool inside = REF ? dw_step_ref(w2, cm.wc, cm.negr, P.cube, P.nx, P.ny, P.nz, P.refine, seg)
                                : dw_step(w2, cm.wc, cm.negr, P.nx, P.ny, P.nz, seg);
        float g[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) g[s] = 0.f;
#pragma unroll
        for (int f = 0; f < NFP; ++f) {
            float chi = 0.f;
#pragma unroll
            for (int s = 0; s < NS; ++s) chi += rho[s] * P.kext[s][f];
            const float dt = chi * seg;
            kahan_add(tb[f], tbc[f], dt);
            const float front = fmaxf(tot[f] - tb[f], 0.0f);      // tau between cell and observer
            const float att = expf(-front);
            const float ph = phi_f(dt);
            const float dph = dphi_f(dt);
            const float contrib = eta[f] * seg * ph * att;
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                if (s >= P.ns) break;            // float4 padding of a 3-species grid
                // per-cell-length quantities: bk and eta carry a factor cell,
                // ke = kext_s cell converts d(dtau)/d(rho_s) = kext_s l_phys
                const float bk = P.bk[((size_t)s * P.ncell + c) * NFP + f];
                const float ke = P.kext_cell[s][f];
                g[s] += w[f] * ((bk * ph + eta[f] * dph * ke * seg) * seg * att - ke * seg * beh[f]);
            }
            kahan_add(beh[f], behc[f], contrib);
        }
#pragma unroll
        for (int s = 0; s < NS; ++s)
            if (s < P.ns && g[s] != 0.f) atomicAdd(&P.grad[(size_t)s * P.ncell + c], g[s]);
        if (!inside) break;
    }
    count_steps(P.steps, nsteps);
}

// eta_th * cell (and bk = kabs_s B(T_s) * cell for the adjoint) for every
// camera's table, in FP32: B = a_f / expm1(h nu_f / k T) with a_f = 2 h nu^3/c^2.
// A thread owns one cell: its NFP values are contiguous, so every camera's
// copy (and each species' bk row) is written as whole float4s.
struct EtaKP {
    const void* rho;           // packed FP32 grid: rho_s * cell
    const double* T;           // [ns][nc]
    size_t nc;
    int ns, nfi, ncam;
    float cell;
    float a[kMaxImgFreq], xh[kMaxImgFreq];
    float kabs[kMaxSpecies][kMaxImgFreq];
    float* eta;
    float* bk;
};

template <int NS, int NFP>
__global__ void eta_thermal_kernel(const __grid_constant__ EtaKP P)
{
    const size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (c >= P.nc) return;
    float rho[NS], invT[NS];
    {
        const typename PT<NS>::T v = __ldg(reinterpret_cast<const typename PT<NS>::T*>(P.rho) + c);
        float r[4];
        unpack(v, r);
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            rho[s] = r[s];
            const float T = s < P.ns ? (float)P.T[s * P.nc + c] : 0.0f;
            invT[s] = T > 0.0f ? 1.0f / T : 0.0f;
        }
    }
    float e[NFP];
#pragma unroll
    for (int f = 0; f < NFP; ++f) e[f] = 0.0f;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        float b[NFP];
#pragma unroll
        for (int f = 0; f < NFP; ++f) {
            b[f] = 0.0f;
            if (f < P.nfi && invT[s] > 0.0f) b[f] = P.kabs[s][f] * P.a[f] / expm1f(P.xh[f] * invT[s]);
            e[f] += rho[s] * b[f];                             // rho * cell * kabs * B
        }
        if (P.bk && s < P.ns) {
            float4* q = reinterpret_cast<float4*>(P.bk + ((size_t)s * P.nc + c) * NFP);
#pragma unroll
            for (int v = 0; v < NFP / 4; ++v)
                q[v] = make_float4(b[4 * v] * P.cell, b[4 * v + 1] * P.cell, b[4 * v + 2] * P.cell,
                                   b[4 * v + 3] * P.cell);
        }
    }
    for (int k = 0; k < P.ncam; ++k) {
        float4* q = reinterpret_cast<float4*>(P.eta + ((size_t)k * P.nc + c) * NFP);
#pragma unroll
        for (int v = 0; v < NFP / 4; ++v) q[v] = make_float4(e[4 * v], e[4 * v + 1], e[4 * v + 2], e[4 * v + 3]);
    }
}

struct ScatKP {
    int ncam, nfi, nfp;
    size_t nc;
    const float* kobs;         // [ncam][3]
    const int* f_of_nu;        // [nf] image-frequency slot or -1
    const float2* ag;          // [ns][nf] {xi cell / (V dnu) (1 - g^2) / (4 pi), g}
    int nf, ns;
    const unsigned char* leaf_fine;   // refined grids: sub-cubes have V / r^3
    float fine_scale;                 // r^3
};

__device__ __forceinline__ float vol_factor(const ScatKP& P, uint32_t cell)
{
    return (P.leaf_fine && P.leaf_fine[cell]) ? P.fine_scale : 1.0f;
}

// Henyey-Greenstein weight towards camera k, FP32: the denominator
// 1 + g^2 - 2 g cos = (1 - g)^2 + 2 g (1 - cos) keeps its precision at
// forward-peaked g and cos near 1.
__device__ __forceinline__ float hg_toward(const rt_event& e, const float* ko, float2 ag)
{
    const float cb = e.k[0] * ko[0] + e.k[1] * ko[1] + e.k[2] * ko[2];
    const float g = ag.y;
    const float d = (1.0f - g) * (1.0f - g) + 2.0f * g * (1.0f - cb);
    return ag.x / (d * sqrtf(d));
}

// number of events to use: min(*nev_dev, cap) when the count lives on the device
__device__ __forceinline__ uint64_t event_count(uint64_t cap, const uint64_t* nev_dev)
{
    if (!nev_dev) return cap;
    const uint64_t n = *nev_dev;
    return n < cap ? n : cap;
}

// eta_sca * cell: every stored event adds xi cell / (V dnu) P_HG(k_in . k_obs)
// (grid-stride over the events)
__global__ void eta_scatter_kernel(const rt_event* ev, uint64_t cap, const uint64_t* nev_dev, ScatKP P,
                                   float* eta)
{
    const uint64_t nev = event_count(cap, nev_dev);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nev;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const rt_event e = ev[i];
        if (e.nu >= P.nf || e.species >= P.ns) continue;
        const int f = P.f_of_nu[e.nu];
        if (f < 0 || (size_t)e.cell >= P.nc) continue;
        const float2 ag = P.ag[e.species * P.nf + e.nu];
        const float vf = vol_factor(P, e.cell);
        for (int k = 0; k < P.ncam; ++k)
            atomicAdd(&eta[((size_t)k * P.nc + e.cell) * P.nfp + f], vf * hg_toward(e, P.kobs + 3 * k, ag));
    }
}

// several image frequencies share one event frequency: handled by a second
// pass over the remaining duplicate slots
__global__ void eta_scatter_dup_kernel(const rt_event* ev, uint64_t cap, const uint64_t* nev_dev, ScatKP P,
                                       const int* dup, int ndup, float* eta)
{
    const uint64_t nev = event_count(cap, nev_dev);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nev;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const rt_event e = ev[i];
        if ((size_t)e.cell >= P.nc || e.nu >= P.nf || e.species >= P.ns) continue;
        for (int q = 0; q < ndup; ++q) {
            const int f = dup[2 * q], j = dup[2 * q + 1];
            if ((int)e.nu != j) continue;
            const float2 ag = P.ag[e.species * P.nf + e.nu];
            const float vf = vol_factor(P, e.cell);
            for (int k = 0; k < P.ncam; ++k)
                atomicAdd(&eta[((size_t)k * P.nc + e.cell) * P.nfp + f], vf * hg_toward(e, P.kobs + 3 * k, ag));
        }
    }
}

// sed[cam][f] = A_pix / D^2 * sum_pix I  (one block of 1024 threads per
// (cam, f), float4 loads when the image size allows, FP64 sums)
__global__ void __launch_bounds__(1024) sed_reduce_kernel(const float* img, int nfi, long long npix2,
                                                          const double* apix_d2, double* sed, int vec4)
{
    const int cf = blockIdx.x;
    const float* p = img + (size_t)cf * npix2;
    double acc = 0.0;
    if (vec4) {
        const float4* q = reinterpret_cast<const float4*>(p);
        for (long long i = threadIdx.x; i < npix2 / 4; i += blockDim.x) {
            const float4 v = q[i];
            acc += ((double)v.x + (double)v.y) + ((double)v.z + (double)v.w);
        }
    } else {
        for (long long i = threadIdx.x; i < npix2; i += blockDim.x) acc += (double)p[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) sed[cf] = v * apix_d2[cf / nfi];
    }
}

struct StarKP {
    const float* rho;          // unpacked [ns][nc]
    int nx, ny, nz, ns, nfi;
    size_t nc;
    double cell;
    double kext[kMaxSpecies][kMaxImgFreq];
    const double* pos_cell;    // [nsrc][3]
    const double* lnu;         // [nsrc][nfi]
    const double* kobs;        // [ncam][3]
    const double* inv4piD2;    // [ncam]
    int nsrc, ncam;
    double* sed;               // forward: += L exp(-tau) / (4 pi D^2)
    const double* dsed;        // backward
    float* grad;
    const int* cube;           // refined grids: [ncube] first cell | kCubeDivided
    int refine;                // r, or 0
};

// Direct light of each source along k_obs (FP64).  One warp per (camera,
// source), one lane per image frequency: the lanes walk the same path (an
// incremental DDA: per-axis face distances advanced by fixed steps, ties to
// the lowest axis) and each adds its own frequency's optical depth, so the
// FP64 work per cell visit is a handful of warp instructions.  Forward adds
// L_nu exp(-tau) / (4 pi D^2) to the SED; backward walks the path again and
// adds -sum_f dL/dF_f F_f kext_s,f l (a warp sum) to the density gradient.
__global__ void __launch_bounds__(32) star_kernel(const __grid_constant__ StarKP P, int backward)
{
    const int t = blockIdx.x;
    if (t >= P.ncam * P.nsrc) return;
    const int si = t % P.nsrc, cam = t / P.nsrc;
    const int f = threadIdx.x;
    const bool act = f < P.nfi;
    const int fc = act ? f : 0;
    double ke[kMaxSpecies];
#pragma unroll
    for (int s = 0; s < kMaxSpecies; ++s) ke[s] = act ? P.kext[s][fc] : 0.0;
    const double d[3] = { P.kobs[3 * cam], P.kobs[3 * cam + 1], P.kobs[3 * cam + 2] };
    const int n[3] = { P.nx, P.ny, P.nz };
    double tau = 0.0, coef = 0.0;
    for (int pass = 0; pass < (backward ? 2 : 1); ++pass) {
        if (pass == 1) {
            if (act) {
                const double F = P.lnu[si * P.nfi + fc] * exp(-tau) * P.inv4piD2[cam];
                coef = -P.dsed[cam * P.nfi + fc] * F;
            }
            if (!__any_sync(0xffffffffu, coef != 0.0)) return;
        }
        if (P.refine) {
            // the same walk on a refined grid
            const double* p0 = P.pos_cell + 3 * si;
            RefWalk<double> w;
            bool in = rw_start(w, P.cube, P.nx, P.ny, P.nz, P.refine, p0, d, false);
            double tcur = 0.0, seg;
            const int maxstep = (P.nx + P.ny + P.nz) * P.refine + 4;
            for (int steps = 0; in && steps < maxstep; ++steps) {
                const size_t c = (size_t)w.c;
                in = rw_step(w, P.cube, P.nx, P.ny, P.nz, P.refine, p0, d, tcur, seg);
                const double l = seg * P.cell;
                if (pass == 0) {
                    double chi = 0.0;
                    for (int s = 0; s < P.ns; ++s) chi += (double)__ldg(&P.rho[s * P.nc + c]) * ke[s];
                    tau += chi * l;
                } else {
                    for (int s = 0; s < P.ns; ++s) {
                        double g = coef * ke[s];
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
                        g *= l;
                        if (f == 0 && g != 0.0) atomicAdd(&P.grad[s * P.nc + c], (float)g);
                    }
                }
            }
            continue;
        }
        int i[3];
        double tm[3], td[3];
        bool in = true;
        for (int a = 0; a < 3; ++a) {
            const double x = P.pos_cell[3 * si + a];
            const double fl = floor(x);
            int k = (int)fl;
            if (fl == x && d[a] < 0.0) k -= 1;
            i[a] = k;
            in = in && k >= 0 && k < n[a];
            if (d[a] > 0.0) {
                td[a] = 1.0 / d[a];
                tm[a] = fmax(((double)(k + 1) - x) * td[a], 0.0);
            } else if (d[a] < 0.0) {
                td[a] = -1.0 / d[a];
                tm[a] = fmax((x - (double)k) * td[a], 0.0);
            } else {
                td[a] = INFINITY;
                tm[a] = INFINITY;
            }
        }
        double tcur = 0.0;
        for (int steps = 0; in && steps < P.nx + P.ny + P.nz + 4; ++steps) {
            const int ba = (tm[0] <= tm[1] && tm[0] <= tm[2]) ? 0 : (tm[1] <= tm[2] ? 1 : 2);
            const double tn = ba == 0 ? tm[0] : (ba == 1 ? tm[1] : tm[2]);
            const double l = (tn - tcur) * P.cell;
            const size_t c = ((size_t)i[2] * P.ny + i[1]) * P.nx + i[0];
            if (pass == 0) {
                double chi = 0.0;
                for (int s = 0; s < P.ns; ++s) chi += (double)__ldg(&P.rho[s * P.nc + c]) * ke[s];
                tau += chi * l;
            } else {
                for (int s = 0; s < P.ns; ++s) {
                    double g = coef * ke[s];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
                    g *= l;
                    if (f == 0 && g != 0.0) atomicAdd(&P.grad[s * P.nc + c], (float)g);
                }
            }
            tcur = tn;
            if (ba == 0) { tm[0] += td[0]; i[0] += d[0] > 0.0 ? 1 : -1; in = i[0] >= 0 && i[0] < n[0]; }
            else if (ba == 1) { tm[1] += td[1]; i[1] += d[1] > 0.0 ? 1 : -1; in = i[1] >= 0 && i[1] < n[1]; }
            else { tm[2] += td[2]; i[2] += d[2] > 0.0 ? 1 : -1; in = i[2] >= 0 && i[2] < n[2]; }
        }
    }
    if (!backward && act)
        atomicAdd(&P.sed[cam * P.nfi + fc], P.lnu[si * P.nfi + fc] * exp(-tau) * P.inv4piD2[cam]);
}

// grad_total += grad_call;  dscale += sum rho * grad_call
__global__ void grad_finish_kernel(const float* rho, const float* g, size_t n, float* drho, double* dscale)
{
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float v = g[i];
        drho[i] += v;
        acc += (double)rho[i] * v;
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(dscale, red[0]);
}

template <int NS, int NFP>
void launch_rays(const RayKP& kp, int npix, bool backward, cudaStream_t s)
{
    const int th = 128;
    const long long nthreads = (long long)npix * npix * (backward ? 1 : NFP / 4);
    dim3 grid((unsigned)((nthreads + th - 1) / th), kp.ncam);
    if (backward && kp.refine) ray_bwd_kernel<NS, NFP, true><<<grid, th, 0, s>>>(kp);
    else if (backward) ray_bwd_kernel<NS, NFP, false><<<grid, th, 0, s>>>(kp);
    else if (kp.refine) ray_fwd_kernel<NS, NFP, true><<<grid, th, 0, s>>>(kp);
    else ray_fwd_kernel<NS, NFP, false><<<grid, th, 0, s>>>(kp);
    count_launches();
}

template <int NS>
void launch_rays_nf(const RayKP& kp, int npix, bool backward, cudaStream_t s)
{
    switch (kp.nfp) {
    case 4: launch_rays<NS, 4>(kp, npix, backward, s); break;
    case 8: launch_rays<NS, 8>(kp, npix, backward, s); break;
    case 12: launch_rays<NS, 12>(kp, npix, backward, s); break;
    default: launch_rays<NS, 16>(kp, npix, backward, s); break;
    }
}

template <int NS>
void launch_eta(const EtaKP& ek, int nfp, unsigned blocks, cudaStream_t s)
{
    switch (nfp) {
    case 4: eta_thermal_kernel<NS, 4><<<blocks, 256, 0, s>>>(ek); break;
    case 8: eta_thermal_kernel<NS, 8><<<blocks, 256, 0, s>>>(ek); break;
    case 12: eta_thermal_kernel<NS, 12><<<blocks, 256, 0, s>>>(ek); break;
    default: eta_thermal_kernel<NS, 16><<<blocks, 256, 0, s>>>(ek); break;
    }
}

template <typename T>
rt_status grow(T*& p, size_t& cap, size_t n)
{
    if (cap >= n && p) return RT_OK;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    RT_CUDA(cudaMalloc(&p, sizeof(T) * n));
    cap = n;
    return RT_OK;
}

}  // namespace

rt_status raytrace_impl(rt_ctx* ctx, const rt_grid* g, const rt_opacity* op, const double* T,
                        const rt_event* ev, uint64_t nev, const uint64_t* nev_dev, double xi_ev,
                        const rt_source* src, int nsrc, const rt_camera* cams, int ncam, const int* fidx, int nfi,
                        float* images, double* sed, const float* dimg, const double* dsed,
                        float* drho, double* dscale, unsigned long long* ray_steps, bool backward,
                        cudaStream_t s)
{
    const size_t nc = g->ncell();
    const int ns = g->ns;
    const int nfp = (nfi + 3) / 4 * 4;
    // packed FP32 density (any Lucy flagging: the ray tracer ignores the flag)
    rt_grid* gm = const_cast<rt_grid*>(g);
    if (!gm->d_packed || gm->packed_prec != RT_PREC_FP32 || gm->packed_opac_serial != op->serial) {
        rt_status st = pack_grid(gm, op, RT_LUCY_OFF, 0.0, RT_PREC_FP32, s);
        if (st != RT_OK) return st;
    }
    rt_status st = grow(ctx->d_eta, ctx->eta_cap, (size_t)ncam * nc * nfp);
    if (st != RT_OK) return st;
    if (backward) {
        st = grow(ctx->d_bk, ctx->bk_cap, (size_t)ns * nc * nfp + (size_t)ns * nc);
        if (st != RT_OK) return st;
    }
    // host-side per-call tables
    std::vector<double> nu_f(nfi), kabs_f((size_t)ns * nfi);
    for (int f = 0; f < nfi; ++f) {
        nu_f[f] = op->nu[fidx[f]];
        for (int sp = 0; sp < ns; ++sp) kabs_f[sp * nfi + f] = op->kabs[sp * op->nf + fidx[f]];
    }
    std::vector<float> kobs(3 * ncam);
    std::vector<double> kobs_d(3 * ncam), inv4piD2(ncam), apix_d2(ncam);
    std::vector<CamDev> cd(ncam);
    const double diag = g->cell * sqrt((double)g->nx * g->nx + (double)g->ny * g->ny + (double)g->nz * g->nz);
    for (int c = 0; c < ncam; ++c) {
        const double st_ = sin(cams[c].theta), ct = cos(cams[c].theta);
        const double sp = sin(cams[c].phi), cp = cos(cams[c].phi);
        const double ko[3] = { st_ * cp, st_ * sp, ct };
        const double ex[3] = { -sp, cp, 0.0 };
        const double ey[3] = { -ct * cp, -ct * sp, st_ };
        const double pix = cams[c].pixel > 0.0 ? cams[c].pixel : diag / cams[c].npix;
        cd[c].negf = cd[c].negr = 0u;
        for (int a = 0; a < 3; ++a) {
            kobs[3 * c + a] = (float)ko[a];
            kobs_d[3 * c + a] = ko[a];
            cd[c].k[a] = ko[a];
            cd[c].ex[a] = ex[a];
            cd[c].ey[a] = ey[a];
            cd[c].ik[a] = ko[a] != 0.0 ? 1.0 / ko[a] : 0.0;
            const double ad = fabs(ko[a]);
            const double rr = g->refine ? (double)g->refine : 1.0;
            cd[c].wc.td[a] = ad > 0.0 ? df_of(1.0 / ad) : DF{ INFINITY, 0.0f };
            cd[c].wc.tds[a] = ad > 0.0 ? df_of(1.0 / (ad * rr)) : DF{ INFINITY, 0.0f };
            cd[c].wc.adr[a] = (float)(ad * rr);
            if (ko[a] > 0.0) cd[c].negf |= 1u << a;
            if (ko[a] < 0.0) cd[c].negr |= 1u << a;
        }
        cd[c].pix_cell = pix / g->cell;
        cd[c].apix_d2 = pix * pix / (cams[c].D * cams[c].D);
        cd[c].npix = cams[c].npix;
        inv4piD2[c] = 1.0 / (4.0 * kPi * cams[c].D * cams[c].D);
        apix_d2[c] = cd[c].apix_d2;
    }
    std::vector<int> f_of_nu(op->nf, -1), dup;
    for (int f = 0; f < nfi; ++f) {
        if (f_of_nu[fidx[f]] < 0) f_of_nu[fidx[f]] = f;
        else { dup.push_back(f); dup.push_back(fidx[f]); }
    }
    std::vector<double> lnu((size_t)std::max(nsrc, 1) * nfi), spos((size_t)std::max(nsrc, 1) * 3);
    std::vector<double> spec;
    for (int i = 0; i < nsrc; ++i) {
        source_spectrum(op, src[i], spec);
        for (int f = 0; f < nfi; ++f) lnu[(size_t)i * nfi + f] = spec[fidx[f]];
        for (int a = 0; a < 3; ++a) spos[3 * i + a] = (src[i].pos[a] - g->box_min[a]) / g->cell;
    }
    // one staging allocation for the small tables
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off = (off + bytes + 255) / 256 * 256; return o; };
    const size_t o_nu = take(sizeof(double) * nfi), o_ka = take(sizeof(double) * ns * nfi);
    const size_t o_ko = take(sizeof(float) * 3 * ncam), o_kd = take(sizeof(double) * 3 * ncam);
    const size_t o_i4 = take(sizeof(double) * ncam), o_ap = take(sizeof(double) * ncam);
    const size_t o_fn = take(sizeof(int) * op->nf), o_du = take(sizeof(int) * (dup.size() + 2));
    const size_t o_ln = take(sizeof(double) * lnu.size()), o_sp = take(sizeof(double) * spos.size());
    // scattering emissivity per event (tables hold eta * cell): xi cell / (V dnu)
    // times the Henyey-Greenstein numerator (1 - g^2) / (4 pi); g alongside
    std::vector<float2> ag((size_t)ns * op->nf);
    for (int sp = 0; sp < ns; ++sp)
        for (int j = 0; j < op->nf; ++j) {
            const double gg = op->g[sp * op->nf + j];
            const double amp = xi_ev / (g->cell * g->cell) / op->dnu[j];
            ag[(size_t)sp * op->nf + j] = make_float2((float)(amp * (1.0 - gg * gg) / (4.0 * kPi)), (float)gg);
        }
    const size_t o_ag = take(sizeof(float2) * ag.size());
    std::vector<unsigned char> h(off, 0);
    std::memcpy(&h[o_nu], nu_f.data(), sizeof(double) * nfi);
    std::memcpy(&h[o_ka], kabs_f.data(), sizeof(double) * ns * nfi);
    std::memcpy(&h[o_ko], kobs.data(), sizeof(float) * 3 * ncam);
    std::memcpy(&h[o_kd], kobs_d.data(), sizeof(double) * 3 * ncam);
    std::memcpy(&h[o_i4], inv4piD2.data(), sizeof(double) * ncam);
    std::memcpy(&h[o_ap], apix_d2.data(), sizeof(double) * ncam);
    std::memcpy(&h[o_fn], f_of_nu.data(), sizeof(int) * op->nf);
    if (!dup.empty()) std::memcpy(&h[o_du], dup.data(), sizeof(int) * dup.size());
    std::memcpy(&h[o_ln], lnu.data(), sizeof(double) * lnu.size());
    std::memcpy(&h[o_sp], spos.data(), sizeof(double) * spos.size());
    std::memcpy(&h[o_ag], ag.data(), sizeof(float2) * ag.size());
    char* dbuf = nullptr;
    RT_CUDA(cudaMallocAsync((void**)&dbuf, off, s));
    RT_CUDA(cudaMemcpyAsync(dbuf, h.data(), off, cudaMemcpyHostToDevice, s));

    float* bk = backward ? ctx->d_bk : nullptr;
    float* gcall = backward ? ctx->d_bk + (size_t)ns * nc * nfp : nullptr;
    {
        EtaKP ek;
        std::memset(&ek, 0, sizeof(ek));
        ek.rho = g->d_packed; ek.T = T; ek.nc = nc; ek.ns = ns; ek.nfi = nfi;
        ek.cell = (float)g->cell;
        ek.ncam = ncam; ek.eta = ctx->d_eta; ek.bk = bk;
        const double hP = 6.62607015e-27, kB = 1.380649e-16, cl = 2.99792458e10;
        for (int f = 0; f < nfi; ++f) {
            const double nu = op->nu[fidx[f]];
            ek.a[f] = (float)(2.0 * hP * nu * nu * nu / (cl * cl));
            ek.xh[f] = (float)(hP * nu / kB);
            for (int sp = 0; sp < ns; ++sp) ek.kabs[sp][f] = (float)op->kabs[sp * op->nf + fidx[f]];
        }
        const unsigned blocks = (unsigned)((nc + 255) / 256);
        const int vec = ns == 1 ? 1 : (ns == 2 ? 2 : 4);
        if (vec == 1) launch_eta<1>(ek, nfp, blocks, s);
        else if (vec == 2) launch_eta<2>(ek, nfp, blocks, s);
        else launch_eta<4>(ek, nfp, blocks, s);
        count_launches();
        RT_CUDA(cudaGetLastError());
    }
    if (nev > 0) {
        ScatKP sk;
        sk.ncam = ncam; sk.nfi = nfi; sk.nfp = nfp; sk.nc = nc;
        sk.ag = (const float2*)(dbuf + o_ag);
        sk.kobs = (const float*)(dbuf + o_ko);
        sk.f_of_nu = (const int*)(dbuf + o_fn);
        sk.nf = op->nf; sk.ns = ns;
        sk.leaf_fine = g->d_leaf_fine;
        sk.fine_scale = (float)((double)g->refine * g->refine * g->refine);
        const unsigned blocks = (unsigned)std::min<uint64_t>((nev + 255) / 256, (uint64_t)ctx->num_sms * 8);
        eta_scatter_kernel<<<blocks, 256, 0, s>>>(ev, nev, nev_dev, sk, ctx->d_eta);
        count_launches();
        if (!dup.empty()) {
            eta_scatter_dup_kernel<<<blocks, 256, 0, s>>>(ev, nev, nev_dev, sk, (const int*)(dbuf + o_du),
                                                          (int)dup.size() / 2, ctx->d_eta);
            count_launches();
        }
        RT_CUDA(cudaGetLastError());
    }
    if (backward) RT_CUDA(cudaMemsetAsync(gcall, 0, sizeof(float) * ns * nc, s));

    RayKP kp;
    std::memset(&kp, 0, sizeof(kp));
    kp.rho = g->d_packed;
    kp.nx = g->nx; kp.ny = g->ny; kp.nz = g->nz;
    kp.ns = ns;
    kp.cell = (float)g->cell;
    for (int sp = 0; sp < ns; ++sp)
        for (int f = 0; f < nfi; ++f) {
            const double ke = op->kabs[sp * op->nf + fidx[f]] + op->ksca[sp * op->nf + fidx[f]];
            kp.kext[sp][f] = (float)ke;
            kp.kext_cell[sp][f] = (float)(ke * g->cell);
        }
    kp.nfi = nfi; kp.nfp = nfp; kp.ncell = nc;
    kp.eta = ctx->d_eta; kp.bk = bk;
    kp.img = images; kp.dimg = dimg; kp.dsed = dsed; kp.grad = gcall;
    kp.steps = ray_steps;
    kp.cube = g->d_cube;
    kp.refine = g->refine;
    const int npix = cams[0].npix;
    for (int c0 = 0; c0 < ncam; c0 += kCamChunk) {
        kp.cam0 = c0;
        kp.ncam = std::min(kCamChunk, ncam - c0);
        for (int k = 0; k < kp.ncam; ++k) kp.cam[k] = cd[c0 + k];
        const int vec = ns == 1 ? 1 : (ns == 2 ? 2 : 4);
        if (vec == 1) launch_rays_nf<1>(kp, npix, backward, s);
        else if (vec == 2) launch_rays_nf<2>(kp, npix, backward, s);
        else launch_rays_nf<4>(kp, npix, backward, s);
        RT_CUDA(cudaGetLastError());
    }
    if (!backward) {
        const long long npix2 = (long long)npix * npix;
        const int vec4 = (npix2 % 4 == 0) && (reinterpret_cast<uintptr_t>(images) % 16 == 0);
        sed_reduce_kernel<<<ncam * nfi, 1024, 0, s>>>(images, nfi, npix2, (const double*)(dbuf + o_ap),
                                                      sed, vec4);
        count_launches();
    }
    if (nsrc > 0 && (!backward || dsed)) {
        StarKP sp;
        std::memset(&sp, 0, sizeof(sp));
        sp.rho = g->d_rho; sp.nx = g->nx; sp.ny = g->ny; sp.nz = g->nz; sp.ns = ns; sp.nfi = nfi;
        sp.nc = nc; sp.cell = g->cell;
        for (int q = 0; q < ns; ++q)
            for (int f = 0; f < nfi; ++f)
                sp.kext[q][f] = op->kabs[q * op->nf + fidx[f]] + op->ksca[q * op->nf + fidx[f]];
        sp.pos_cell = (const double*)(dbuf + o_sp);
        sp.lnu = (const double*)(dbuf + o_ln);
        sp.kobs = (const double*)(dbuf + o_kd);
        sp.inv4piD2 = (const double*)(dbuf + o_i4);
        sp.nsrc = nsrc; sp.ncam = ncam;
        sp.sed = sed; sp.dsed = dsed; sp.grad = gcall;
        sp.cube = g->d_cube; sp.refine = g->refine;
        star_kernel<<<ncam * nsrc, 32, 0, s>>>(sp, backward ? 1 : 0);
        count_launches();
        RT_CUDA(cudaGetLastError());
    }
    if (backward) {
        const size_t n = (size_t)ns * nc;
        const unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, (size_t)ctx->num_sms * 8);
        grad_finish_kernel<<<blocks, 256, 0, s>>>(g->d_rho, gcall, n, drho, dscale);
        count_launches();
        RT_CUDA(cudaGetLastError());
    }
    RT_CUDA(cudaFreeAsync(dbuf, s));
    return RT_OK;
}

}  // namespace rtgb

namespace rtgb {
namespace {

// Complex visibilities of one camera's images at KT (u, v) points: one block
// per (camera, tile of KT points).  exp(-2 pi i (u alpha + v beta))
// separates into a column and a row factor per point; the block tabulates
// them once in shared memory (phases as exact fixed-point fractions of a
// cycle, then FP32 sine and cosine of pi times a number in [-1, 1)) and
// serves every image frequency of the camera with them.  A warp takes a row
// at a time, its lanes stride along the row (coalesced) and keep KT complex
// row sums in FP32, so each pixel is read once per tile; the row sums are
// reduced by shuffles, multiplied by the row factors and accumulated with
// compensated FP32 sums, lane k of the warp serving point k; the warps'
// partial sums are added in FP64.
template <int KT>
__global__ void visibility_kernel(const float* images, int npix, const double* alpha0,
                                  const double* dalpha, const double* scale, int nf, const double* uv,
                                  int nuv, double* vis)
{
    extern __shared__ float2 tab[];                    // [KT][npix] columns, [KT][npix] rows
    __shared__ double red[2][KT][32];
    __shared__ unsigned long long ph0[2 * KT], dph[2 * KT];
    const int cam = blockIdx.y, k0 = blockIdx.x * KT;
    // Phase of pixel p along an axis, in cycles: w (a0 + da p) = w a0 + p (w da).
    // Both terms are reduced mod 1 once per point in FP64 and kept as 64-bit
    // fixed-point fractions, so the per-pixel phases are exact integer
    // sums mod 1 (resolution 2^-64 cycle; 2^-32 after the cut to 32 bits)
    // and need no FP64 work.
    if (threadIdx.x < 2 * KT) {
        const int rowf = threadIdx.x >= KT, kk = threadIdx.x - (rowf ? KT : 0);
        const int k = min(k0 + kk, nuv - 1);           // a partial last tile repeats a point
        const double w = uv[2 * k + rowf];
        const double c0 = w * alpha0[cam], d = w * dalpha[cam];
        ph0[threadIdx.x] = __double2ull_rn((c0 - floor(c0)) * 18446744073709551616.0);
        dph[threadIdx.x] = __double2ull_rn((d - floor(d)) * 18446744073709551616.0);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * KT * npix; i += blockDim.x) {
        const int rowf = i >= KT * npix;               // row factors follow the column ones
        const int q = rowf ? i - KT * npix : i;
        const int kk = q / npix, p = q - kk * npix;
        const int slot = rowf * KT + kk;
        const unsigned long long cyc = ph0[slot] + (unsigned long long)p * dph[slot];   // mod 1
        const float x = (float)(int)(unsigned)(cyc >> 32) * 2.3283064365386963e-10f;   // [-1/2, 1/2)
        float sn, cs;
        sincospif(-2.0f * x, &sn, &cs);
        tab[i] = make_float2(cs, sn);
    }
    __syncthreads();
    const float2* col = tab;
    const float2* row = tab + KT * npix;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int f = 0; f < nf; ++f) {
        const int img = cam * nf + f;
        const float* I = images + (size_t)img * npix * npix;
        float re = 0.f, rec = 0.f, im = 0.f, imc = 0.f;   // lane kk < KT: point kk, compensated
        for (int y = warp; y < npix; y += nw) {
            float sr[KT], si[KT];
#pragma unroll
            for (int kk = 0; kk < KT; ++kk) { sr[kk] = 0.f; si[kk] = 0.f; }
            for (int x = lane; x < npix; x += 32) {
                const float q = I[(size_t)y * npix + x];
#pragma unroll
                for (int kk = 0; kk < KT; ++kk) {
                    const float2 c = col[kk * npix + x];
                    sr[kk] += q * c.x;
                    si[kk] += q * c.y;
                }
            }
#pragma unroll
            for (int kk = 0; kk < KT; ++kk) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    sr[kk] += __shfl_xor_sync(0xffffffffu, sr[kk], o);
                    si[kk] += __shfl_xor_sync(0xffffffffu, si[kk], o);
                }
            }
            // every lane holds every sum after the butterfly; lane kk takes
            // point kk and adds the row product with a compensated FP32 sum
            float mr = 0.f, mi = 0.f;
#pragma unroll
            for (int kk = 0; kk < KT; ++kk)
                if (lane == kk) { mr = sr[kk]; mi = si[kk]; }
            if (lane < KT) {
                const float2 r = row[lane * npix + y];
                kahan_add(re, rec, mr * r.x - mi * r.y);
                kahan_add(im, imc, mr * r.y + mi * r.x);
            }
        }
        if (lane < KT) {
            red[0][lane][warp] = (double)re - (double)rec;
            red[1][lane][warp] = (double)im - (double)imc;
        }
        __syncthreads();
        if (threadIdx.x < KT && k0 + (int)threadIdx.x < nuv) {
            const int kk = threadIdx.x;
            double R = 0.0, M = 0.0;
            for (int w = 0; w < nw; ++w) { R += red[0][kk][w]; M += red[1][kk][w]; }
            vis[2 * ((size_t)img * nuv + k0 + kk)] = R * scale[cam];
            vis[2 * ((size_t)img * nuv + k0 + kk) + 1] = M * scale[cam];
        }
        __syncthreads();                               // red is reused by the next image
    }
}

template <int KT>
rt_status launch_vis(const float* images, int npix, const double* d, int ncam, int nf, int nuv,
                     double* vis, cudaStream_t s)
{
    const size_t smem = sizeof(float2) * 2 * KT * (size_t)npix;
    if (smem > 48 * 1024)
        RT_CUDA(cudaFuncSetAttribute(visibility_kernel<KT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((unsigned)((nuv + KT - 1) / KT), (unsigned)ncam);
    visibility_kernel<KT><<<grid, 256, smem, s>>>(images, npix, d, d + ncam, d + 2 * ncam, nf,
                                                  d + 3 * ncam, nuv, vis);
    count_launches();
    RT_CUDA(cudaGetLastError());
    return RT_OK;
}

}  // namespace

rt_status visibilities_impl(rt_ctx* ctx, const rt_grid* g, const rt_camera* cams, int ncam,
                            const float* images, int nf, const double* uv, int nuv, double* vis,
                            cudaStream_t s)
{
    (void)ctx;
    const int npix = cams[0].npix;
    const double diag = g->cell * sqrt((double)g->nx * g->nx + (double)g->ny * g->ny + (double)g->nz * g->nz);
    // per camera: first pixel centre and pixel size in radians, A_pix / D^2; then uv
    std::vector<double> h(3 * (size_t)ncam + 2 * (size_t)nuv);
    for (int c = 0; c < ncam; ++c) {
        const double pix = cams[c].pixel > 0.0 ? cams[c].pixel : diag / cams[c].npix;
        h[c] = (0.5 - 0.5 * npix) * pix / cams[c].D;
        h[ncam + c] = pix / cams[c].D;
        h[2 * ncam + c] = pix * pix / (cams[c].D * cams[c].D);
    }
    std::memcpy(&h[3 * (size_t)ncam], uv, sizeof(double) * 2 * nuv);
    double* d = nullptr;
    RT_CUDA(cudaMallocAsync((void**)&d, sizeof(double) * h.size(), s));
    RT_CUDA(cudaMemcpyAsync(d, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, s));
    // (u, v) points per block: as many as keep the factor tables within
    // 64 KiB of shared memory (one for the largest images)
    rt_status st;
    if (npix <= 512) st = launch_vis<8>(images, npix, d, ncam, nf, nuv, vis, s);
    else if (npix <= 1024) st = launch_vis<4>(images, npix, d, ncam, nf, nuv, vis, s);
    else if (npix <= 2048) st = launch_vis<2>(images, npix, d, ncam, nf, nuv, vis, s);
    else st = launch_vis<1>(images, npix, d, ncam, nf, nuv, vis, s);
    RT_CUDA(cudaFreeAsync(d, s));
    return st;
}

}  // namespace rtgb
