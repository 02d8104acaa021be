// Photon-packet transport (Heymann & Siebenmorgen 2012, Sects. 2 and 3).
//
// One persistent kernel processes all packets of one or many models.  Each
// lane carries one packet at a time; lanes whose packet ended pull new packet
// ids with one warp-aggregated atomic.  A warp advances in phases:
//   refill   lanes without a packet emit a new one (Sect. 2: equal-energy
//            packet, frequency bin from the source CDF, isotropic direction)
//   flight   lanes at a new flight origin either take a modified-random-walk
//            step (Sect. 3.2) or draw tau = -ln(u) and set up the traversal
//   march    all marching lanes cross cells together, one crossing per warp
//            vote (Eq. 2 test against the remaining tau, Lucy deposits in
//            thin cells, Sect. 3.1) until at most `march_min_active` lanes
//            are still marching
//   events   lanes that stopped inside a cell interact (albedo choice, HG
//            scattering Eq. 15, absorption with B&W Eq. 4 + Eq. 10 or frozen-T
//            Eq. 5 re-emission); lanes that left the grid tally the escape.
// Keeping interactions out of the march loop lets the expensive event code
// run for several lanes at once instead of stalling the crossing lanes.
//
// The cell traversal tracks, per flight, the distance to the next x, y and z
// face (incremental DDA); the cell index is integer-exact and the packet
// leaves the grid when an index leaves [0, n).  Positions are in cell units
// relative to the grid corner.  The FP32 kernel reads a packed grid holding
// rho_s * cell (so the optical depth of a chord is sum_s rho_s kext_s * l
// with l in cells) with the Lucy flag in the sign bit of species 0; the FP64
// debug kernel reads rho_s unscaled and follows the same algorithm with every
// quantity in double precision, reproducing the FP64 CPU reference packet by
// packet.
#include <math.h>

#include <algorithm>

#include <type_traits>
#include "rt_internal.cuh"

namespace rtgb {

namespace {

constexpr unsigned FULL = 0xffffffffu;
enum { ST_NEED = 0, ST_FLIGHT = 1, ST_MARCH = 2, ST_INTERACT = 3, ST_ESCAPE = 4, ST_DONE = 5 };
constexpr double kPi = 3.14159265358979323846;
constexpr int kLaneStats = RT_STAT_EMITTED + 1;   // stats counted per thread (the rest are cursors)

template <int NS> struct PackedT;
template <> struct PackedT<1> { using T = float; };
template <> struct PackedT<2> { using T = float2; };
template <> struct PackedT<4> { using T = float4; };

__device__ __forceinline__ void unpack(float v, float* r) { r[0] = v; }
__device__ __forceinline__ void unpack(float2 v, float* r) { r[0] = v.x; r[1] = v.y; }
__device__ __forceinline__ void unpack(float4 v, float* r) { r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w; }

// ------------------------------------------------------------- random numbers
// Per-packet Philox stream: key = (seed_lo, seed_hi ^ model_id), counter =
// (draw/2, 0, pid_lo, pid_hi).  The key's first word is the launch seed and is
// passed in, so a lane keeps five words (six in the FP64 build).
struct Rng {
    uint32_t ky, plo, phi, draw, c_lo, c_hi;
};

__device__ __forceinline__ void rng_init(Rng& r, uint64_t seed, uint32_t model_id, uint64_t pid)
{
    r.ky = (uint32_t)(seed >> 32) ^ model_id;
    r.plo = (uint32_t)pid;
    r.phi = (uint32_t)(pid >> 32);
    r.draw = 0;
    r.c_lo = 0;
    r.c_hi = 0;
}

template <typename R> __device__ __forceinline__ R rng_u(Rng& r, uint32_t kx);

template <> __device__ __forceinline__ float rng_u<float>(Rng& r, uint32_t kx)
{
    const uint32_t d = r.draw++;
    uint32_t hi;
    if ((d & 1u) == 0) {
        const uint4 b = philox4x32_10(make_uint4(d >> 1, 0u, r.plo, r.phi), make_uint2(kx, r.ky));
        hi = b.y;
        r.c_hi = b.w;
    } else {
        hi = r.c_hi;
    }
    return (float)((hi >> 8) + 1u) * 0x1p-24f;
}

template <> __device__ __forceinline__ double rng_u<double>(Rng& r, uint32_t kx)
{
    const uint32_t d = r.draw++;
    uint32_t lo, hi;
    if ((d & 1u) == 0) {
        const uint4 b = philox4x32_10(make_uint4(d >> 1, 0u, r.plo, r.phi), make_uint2(kx, r.ky));
        lo = b.x; hi = b.y;
        r.c_lo = b.z; r.c_hi = b.w;
    } else {
        lo = r.c_lo; hi = r.c_hi;
    }
    const uint64_t w = ((uint64_t)hi << 32) | lo;
    return (double)((w >> 11) + 1u) * 0x1p-53;
}

// ------------------------------------------------------------- math shims
__device__ __forceinline__ float r_log(float x) { return logf(x); }
__device__ __forceinline__ double r_log(double x) { return log(x); }
__device__ __forceinline__ float r_expm1(float x) { return expm1f(x); }
__device__ __forceinline__ double r_expm1(double x) { return expm1(x); }
__device__ __forceinline__ float r_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double r_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ void r_sincos2pi(float z, float* s, float* c) { sincospif(2.0f * z, s, c); }
__device__ __forceinline__ void r_sincos2pi(double z, double* s, double* c) { sincospi(2.0 * z, s, c); }

// Isotropic direction: phi = 2 pi zeta1, cos(theta) = 1 - 2 zeta2, zeta = 1 - u.
template <typename R>
__device__ __forceinline__ void iso_dir(R u1, R u2, R* k)
{
    const R mu = R(1) - R(2) * (R(1) - u2);
    const R st = r_sqrt(fmax(R(0), R(1) - mu * mu));
    R sp, cp;
    r_sincos2pi(R(1) - u1, &sp, &cp);
    k[0] = st * cp;
    k[1] = st * sp;
    k[2] = mu;
}

// Henyey-Greenstein inverse CDF for the cosine of the scattering angle.
template <typename R>
__device__ __forceinline__ R hg_mu(R g, R u)
{
    const R z = R(1) - u;
    R mu;
    if (fabs(g) > R(1e-6)) {
        const R t = (R(1) - g * g) / (R(1) - g + R(2) * g * z);
        mu = (R(1) + g * g - t * t) / (R(2) * g);
    } else {
        mu = R(2) * z - R(1);
    }
    return fmin(R(1), fmax(R(-1), mu));
}

template <typename R>
__device__ __forceinline__ void rotate(R* k, R mu, R u_phi)
{
    const R st = r_sqrt(fmax(R(0), R(1) - mu * mu));
    R sp, cp;
    r_sincos2pi(R(1) - u_phi, &sp, &cp);
    R n0, n1, n2;
    if (fabs(k[2]) > R(0.99999)) {
        n0 = st * cp;
        n1 = st * sp;
        n2 = k[2] > R(0) ? mu : -mu;
    } else {
        const R t = r_sqrt(R(1) - k[2] * k[2]);
        n0 = st * (k[0] * k[2] * cp - k[1] * sp) / t + k[0] * mu;
        n1 = st * (k[1] * k[2] * cp + k[0] * sp) / t + k[1] * mu;
        n2 = -st * cp * t + k[2] * mu;
    }
    const R l = r_sqrt(n0 * n0 + n1 * n1 + n2 * n2);
    k[0] = n0 / l; k[1] = n1 / l; k[2] = n2 / l;
}

// ------------------------------------------------------------- Planck (FP64 debug path)
__device__ __forceinline__ double planck_B(double nu, double T)
{
    if (T <= 0.0) return 0.0;
    const double h = 6.62607015e-27, kb = 1.380649e-16, c = 2.99792458e10;
    const double x = h * nu / (kb * T);
    return 2.0 * h * nu * nu * nu / (c * c) / expm1(x);
}

__device__ __forceinline__ double planck_dBdT(double nu, double T)
{
    if (T <= 0.0) return 0.0;
    const double h = 6.62607015e-27, kb = 1.380649e-16, c = 2.99792458e10;
    const double x = h * nu / (kb * T);
    return 2.0 * h * nu * nu * nu / (c * c) * (x / T) / (expm1(x) * (-expm1(-x)));
}

__device__ double planck_mean64(const TransportKP& P, int s, double T)
{
    double acc = 0.0;
    for (int j = 0; j < P.nf; ++j) acc += P.kabs[s * P.nf + j] * planck_B(P.nu[j], T) * P.dnu[j];
    return acc;
}

// Eq. 4 by bisection to 1e-12 relative (debug path; same stopping rule as the
// FP64 reference so that both return the same root to ~1e-12).
__device__ double solve_T64(const TransportKP& P, int s, double target)
{
    if (!(target > 0.0)) return 0.0;
    double lo = 0.0, hi = 1.0e5;
    while (4.0 * kPi * planck_mean64(P, s, hi) < target && hi < 1e12) hi *= 2.0;
    for (int it = 0; it < 400 && hi - lo > 1e-12 * hi; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (4.0 * kPi * planck_mean64(P, s, mid) < target) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

// MRW survival S(y) (debug path; large-time series, image series for small y)
__device__ double mrw_S64(double y)
{
    if (y <= 0.0) return 1.0;
    double s = 0.0;
    if (y < 0.1) {
        for (int m = 0; m < 60; ++m) {
            const double t = exp(-(m + 0.5) * (m + 0.5) / y);
            s += t;
            if (t < 1e-300) break;
        }
        return 1.0 - 2.0 / sqrt(kPi * y) * s;
    }
    for (int n = 1; n < 200; ++n) {
        const double t = exp(-(double)n * n * kPi * kPi * y);
        s += (n & 1) ? t : -t;
        if (t < 1e-22) break;
    }
    return 2.0 * s;
}

__device__ double mrw_y64(double u)
{
    if (u >= 1.0) return 0.0;
    double lo = 0.0, hi = fmax(log(2.0 / u) / (kPi * kPi), 1e-3);
    for (int it = 0; it < 64 && mrw_S64(hi) > u; ++it) hi *= 2.0;
    for (int it = 0; it < 200 && hi - lo > 1e-15 * hi; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mrw_S64(mid) > u) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

// ------------------------------------------------------------- per-lane packet state
// Registers decide occupancy for this latency-bound kernel, so the state is
// kept lean: the cell is one linear index, and per flight each axis keeps its
// signed linear stride and the number of steps left before the grid boundary
// (indices are recovered from the linear index at a flight start).
template <typename R, int NS>
struct Lane {
    int st, m;                 // state, model index
    Rng rng;
    uint32_t seq, nev;         // trajectory record number, events of this packet
    R x[3], k[3];              // flight origin (cell units) and direction
    int c;                     // linear cell index
    int rem[3], dc[3];         // per axis: steps left inside the grid, signed stride
    int j;                     // frequency index
    R tau, tcur;
    R tm[3], td[3];
    R rho[NS];                 // current cell (FP32: rho*cell; FP64: rho)
    bool lucy;
    R chi;                     // extinction per cell length at frequency j
    R kex[NS], kab[NS];        // kext, kabs at frequency j (FP64: times cell)
    typename PackedT<NS>::T pf;  // prefetched packed density of the next cell
    int cn, nax;               // next cell's linear index, axis of the next face
    bool outn;                 // the next face is the grid boundary
    const void* grid;          // packed cells of the packet's model
    uint32_t ncross, nlucy;    // crossings and Lucy deposits of the current packet
    int sub;                   // refined grids: sub-cube indices (8 bits per axis)
                               // or -1 for an undivided cube (rem then holds the
                               // cube's indices)
    int cinfo;                 // refined grids: the next cube's first cell | divided
                               // flag when the next crossing leaves the cube, else -1
};

// a[s] for a register array and a run-time index, without local memory
template <typename R, int NS>
__device__ __forceinline__ R sel(const R (&a)[NS], int s)
{
    R v = a[0];
#pragma unroll
    for (int q = 1; q < NS; ++q) v = (s == q) ? a[q] : v;
    return v;
}

__device__ __forceinline__ int sel3(const int (&a)[3], int i)
{
    return i == 0 ? a[0] : (i == 1 ? a[1] : a[2]);
}

__device__ __forceinline__ unsigned char* smem_raw()
{
    extern __shared__ __align__(16) unsigned char smem_bytes[];
    return smem_bytes;
}

// position of the n-th (from 0) set bit of m (n below the number of set bits)
__device__ __forceinline__ int nth_bit(unsigned m, unsigned n)
{
    for (unsigned i = 0; i < n; ++i) m &= m - 1u;
    return __ffs(m) - 1;
}

// FEAT bits: 1 = modified random walk compiled in, 2 = trajectory logging
// compiled in, 4 = model descriptors read from the launch parameters (constant
// bank) instead of global memory, 8 = a single model (its index and grid
// pointer are constants, not lane registers), 16 = the deferred-packet queue
// compiled in, 32 = PAH re-emission sources compiled in, 64 = one level of
// sub-cube refinement (two-level traversal), 128 = photon-counting cameras,
// 256 = FP32 per-cell accumulators (the plain-FP32 form), 512 = per-warp
// packet compaction (RT_SCHED_COMPACT); production launches leave unused
// paths out of the hot code.
template <typename R, int NS, int FEAT>
struct Kernel {
    using PT = typename PackedT<NS>::T;
    static constexpr bool DBG = sizeof(R) == 8;
    static constexpr bool HAS_MRW = (FEAT & 1) != 0;
    static constexpr bool HAS_TRAJ = (FEAT & 2) != 0;
    static constexpr bool PARAM = (FEAT & 4) != 0;
    static constexpr bool SINGLE = (FEAT & 8) != 0;
    static constexpr bool HAS_DEFER = (FEAT & 16) != 0;
    static constexpr bool HAS_PAH = (FEAT & 32) != 0;
    static constexpr bool HAS_REF = (FEAT & 64) != 0;
    static constexpr bool HAS_PC = (FEAT & 128) != 0;
    static constexpr bool ACC32 = (FEAT & 256) != 0;
    static constexpr bool COMPACT = (FEAT & 512) != 0;
    using Acc = typename std::conditional<ACC32, float, double>::type;

    // the call's per-cell scratch: {sum, sum of squares} of deposits in units of xi
    __device__ __forceinline__ Acc* acc_at(size_t idx) const
    {
        return reinterpret_cast<Acc*>(md->accE) + (idx << md->acc_q);
    }
    __device__ __forceinline__ Acc to_acc(float v) const
    {
        if constexpr (ACC32) return v;
        else return f2d(v);
    }

    const TransportKP& P;
    const ModelDev* md;        // model of the lane's current packet

    __device__ explicit Kernel(const TransportKP& p) : P(p), md(PARAM ? &p.mp[0] : p.models) {}

    __device__ __forceinline__ const ModelDev* model(int m) const
    {
        if constexpr (PARAM) return &P.mp[m];
        else return &P.models[m];
    }

    // descriptor of the lane's model, before a call that uses md
    __device__ __forceinline__ void bind(const Lane<R, NS>& L)
    {
        if constexpr (!SINGLE) md = model(L.m);
    }

    __device__ __forceinline__ const PT* cells(const Lane<R, NS>& L) const
    {
        if constexpr (SINGLE) return reinterpret_cast<const PT*>(P.rho0);
        else return reinterpret_cast<const PT*>(L.grid);
    }

    // shared-memory tables (offsets set by the host launcher)
    __device__ __forceinline__ const float4* s_op() const { return reinterpret_cast<const float4*>(smem_raw() + P.so_op); }
    __device__ __forceinline__ const float* s_mrw() const { return reinterpret_cast<const float*>(smem_raw() + P.so_mrw); }
    __device__ __forceinline__ const float* s_cdf() const { return reinterpret_cast<const float*>(smem_raw() + P.so_cdf); }
    __device__ __forceinline__ double* s_sed() const { return reinterpret_cast<double*>(smem_raw() + P.so_sed); }
    __device__ __forceinline__ unsigned* s_cnt() const { return reinterpret_cast<unsigned*>(smem_raw() + P.so_cnt); }
    __device__ __forceinline__ unsigned long long* s_ctr() const { return reinterpret_cast<unsigned long long*>(smem_raw() + P.so_ctr); }

    __device__ __forceinline__ R U(Lane<R, NS>& L) const { return rng_u<R>(L.rng, (uint32_t)P.seed); }

    // Event counters of the lane's current model: per thread in shared memory
    // (plain adds, no atomics), handed to the model's stats when the lane
    // moves to another model and at the end of the kernel.
    __device__ __forceinline__ unsigned long long& slot(int stat) const
    {
        return s_ctr()[stat * blockDim.x + threadIdx.x];
    }

    __device__ __forceinline__ void count(int stat, unsigned v) const { slot(stat) += v; }

    __device__ __forceinline__ void flush_lane(int m) const
    {
        unsigned long long* st = P.models[m].stats;
#pragma unroll
        for (int i = 0; i < kLaneStats; ++i) {
            unsigned long long& c = slot(i);
            if (c) atomicAdd(&st[i], c);
            c = 0;
        }
    }

    // the packet ends: its crossings and Lucy deposits go to the counters
    __device__ __forceinline__ void end_packet(Lane<R, NS>& L)
    {
        count(RT_STAT_CROSSINGS, L.ncross);
        count(RT_STAT_LUCY, L.nlucy);
        L.ncross = 0;
        L.nlucy = 0;
        L.st = ST_NEED;
    }

    __device__ __forceinline__ void load_cell(Lane<R, NS>& L)
    {
        use_cell(L, __ldg(cells(L) + L.c));
    }

    // Next cell of the traversal (nearest face, ties to the lowest axis); its
    // density load is issued now and consumed one crossing later.
    __device__ __forceinline__ void prefetch_next(Lane<R, NS>& L)
    {
        const int a = (L.tm[0] <= L.tm[1] && L.tm[0] <= L.tm[2]) ? 0 : (L.tm[1] <= L.tm[2] ? 1 : 2);
        L.nax = a;
        L.outn = sel3(L.rem, a) == 0;
        L.cn = L.c + sel3(L.dc, a);
        if (!L.outn) L.pf = __ldg(cells(L) + L.cn);
    }

    __device__ __forceinline__ void use_cell(Lane<R, NS>& L, const PT v)
    {
        float r[4];
        unpack(v, r);
        L.lucy = signbit(r[0]);
        r[0] = fabsf(r[0]);
        R chi = R(0);
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            L.rho[s] = (R)r[s];
            chi += L.rho[s] * L.kex[s];
        }
        L.chi = chi;
    }

    // kext, kabs of every species at the lane's frequency
    __device__ __forceinline__ void load_freq(Lane<R, NS>& L)
    {
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            if constexpr (DBG) {
                const double ka = s < P.ns ? P.kabs[s * P.nf + L.j] : 0.0;
                const double ks = s < P.ns ? P.ksca[s * P.nf + L.j] : 0.0;
                L.kex[s] = (ka + ks) * md->cell;
                L.kab[s] = ka * md->cell;
            } else {
                const float4 o = s_op()[s * P.nf + L.j];
                L.kex[s] = o.x;
                L.kab[s] = o.y;
            }
        }
        R chi = R(0);
#pragma unroll
        for (int s = 0; s < NS; ++s) chi += L.rho[s] * L.kex[s];
        L.chi = chi;
    }

    __device__ __forceinline__ void traj(Lane<R, NS>& L, uint32_t type, const R* x)
    {
        if constexpr (!HAS_TRAJ) return;
        const uint32_t q = L.seq++;
        if (md->traj == nullptr) return;
        const unsigned long long slot = atomicAdd(&md->stats[RT_STAT_N_TRAJ], 1ull);
        if (slot >= md->traj_cap) {
            atomicAdd(&md->stats[RT_STAT_TRAJ_DROPPED], 1ull);
            return;
        }
        rt_traj t;
        t.pid = ((uint64_t)L.rng.phi << 32) | L.rng.plo;
        t.seq = q; t.type = type; t.cell = (uint32_t)L.c; t.nu = (uint32_t)L.j;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            t.x[a] = md->box_min[a] + (double)x[a] * md->cell;
            t.k[a] = (double)L.k[a];
        }
        md->traj[slot] = t;
    }

    // smallest j with cdf[j] >= u * cdf[n-1] (binary search, cdf non-decreasing)
    template <typename C>
    __device__ __forceinline__ int search_cdf(const C* cdf, int n, C target)
    {
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (cdf[mid] >= target) hi = mid; else lo = mid + 1;
        }
        return lo;
    }

    // Set the packet aside at the start of a flight (defer_events): its state
    // goes to the queue, its crossings so far to the counters, and the lane
    // is free.  false: the queue is full and the packet carries on.
    __device__ __forceinline__ bool defer(Lane<R, NS>& L)
    {
        const unsigned long long slot = atomicAdd(P.defer_n, 1ull);
        if (slot >= P.defer_cap) return false;
        DeferRec r;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            r.x[a] = (double)L.x[a];
            r.k[a] = (double)L.k[a];
        }
        r.pid = ((uint64_t)L.rng.phi << 32) | L.rng.plo;
        r.cell = (uint32_t)L.c; r.j = (uint32_t)L.j; r.m = (uint32_t)L.m;
        r.nev = L.nev; r.seq = L.seq;
        r.draw = L.rng.draw; r.c_lo = L.rng.c_lo; r.c_hi = L.rng.c_hi;
        P.defer[slot] = r;
        atomicAdd(&md->stats[RT_STAT_DEFERRED], 1ull);
        end_packet(L);
        return true;
    }

    // Resume pass: queue record w becomes the lane's packet, at the start of
    // the flight it was set aside at (same Philox position, so the rest of
    // its trajectory is the one it would have had)
    __device__ __forceinline__ void resume(Lane<R, NS>& L, uint64_t w)
    {
        const DeferRec r = P.defer[w];
        if constexpr (!SINGLE) {
            const int m = (int)r.m;
            if (m != L.m) {
                if (L.m >= 0) flush_lane(L.m);
                L.m = m;
            }
            md = model(m);
            L.grid = md->rho;
        } else {
            L.m = 0;
        }
        rng_init(L.rng, P.seed, md->model_id, r.pid);
        L.rng.draw = r.draw; L.rng.c_lo = r.c_lo; L.rng.c_hi = r.c_hi;
        L.seq = r.seq;
        L.nev = r.nev;
        L.ncross = 0;
        L.nlucy = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            L.x[a] = (R)r.x[a];
            L.k[a] = (R)r.k[a];
        }
        L.c = (int)r.cell;
        if constexpr (HAS_REF) set_from_cell(L, L.c);
        L.j = (int)r.j;
#pragma unroll
        for (int s = 0; s < NS; ++s) L.rho[s] = R(0);
        load_freq(L);
        load_cell(L);
        L.st = ST_FLIGHT;
    }

    // ------------------------------------------------ refined grids (Sect. 2)
    // Cells are numbered cube by cube; a divided cube's r^3 sub-cubes follow
    // one another in z, y, x order.  Positions and path lengths stay in cube
    // edges; a sub-cube's edge is 1/r.

    // 1 / r in the build's precision
    __device__ __forceinline__ R inv_r() const
    {
        if constexpr (DBG) return md->inv_refine;
        else return md->inv_refine32;
    }

    // cube indices of cube number q
    __device__ __forceinline__ void cube_idx(int q, int* id) const
    {
        const int nxy = md->nx * md->ny;
        id[2] = q / nxy;
        const int rr = q - id[2] * nxy;
        id[1] = rr / md->nx;
        id[0] = rr - id[1] * md->nx;
    }

    // cube and sub-cube of cell c (a uniform grid of a batch that holds
    // refined grids has no tables: its cells are its cubes)
    __device__ __forceinline__ void set_from_cell(Lane<R, NS>& L, int c) const
    {
        const int q = md->refine ? md->leaf_cube[c] : c;
        const int info = md->refine ? md->cube[q] : q;
        cube_idx(q, L.rem);
        if (info & kCubeDivided) {
            const int r = md->refine;
            const int off = c - (info & ~kCubeDivided);
            const int s0 = off % r, s1 = (off / r) % r, s2 = off / (r * r);
            L.sub = s0 | (s1 << 8) | (s2 << 16);
        } else {
            L.sub = -1;
        }
    }

    // Enter cube q at position xc (cube units): its cell, descending into
    // the sub-cube that holds xc when the cube is divided (a coordinate on a
    // sub-face belongs to the lower sub-cube when moving towards -axis).
    // Axis `ea` (0..2, or -1) is the one the packet entered through.
    __device__ __forceinline__ void enter_cube(Lane<R, NS>& L, int q, const int* id, const R* xc,
                                               int ea) const
    {
        const int info = md->refine ? md->cube[q] : q;
#pragma unroll
        for (int a = 0; a < 3; ++a) L.rem[a] = id[a];
        if (!(info & kCubeDivided)) {
            L.sub = -1;
            L.c = info;
            return;
        }
        descend(L, info, xc, ea);
    }

    // The sub-cube of the divided cube L.rem (first cell | flag `info`) that
    // holds xc, entered through axis ea (or -1), as in enter_cube
    __device__ __forceinline__ void descend(Lane<R, NS>& L, int info, const R* xc, int ea) const
    {
        const int r = md->refine;
        int sb[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const R u = (xc[a] - (R)L.rem[a]) * (R)r;
            const R f = floor(u);
            int sa = (int)f;
            if (f == u && L.k[a] < R(0)) sa -= 1;
            sa = min(max(sa, 0), r - 1);
            if (a == ea) sa = L.k[a] > R(0) ? 0 : r - 1;
            sb[a] = sa;
        }
        L.sub = sb[0] | (sb[1] << 8) | (sb[2] << 16);
        L.c = (info & ~kCubeDivided) + (sb[2] * r + sb[1]) * r + sb[0];
    }

    // packed densities of a refined grid's undivided cubes
    __device__ __forceinline__ const PT* cube_cells() const
    {
        return reinterpret_cast<const PT*>(md->cube_rho);
    }

    // lower corner (cube units) and edge of the lane's cell
    __device__ __forceinline__ R cell_box(const Lane<R, NS>& L, R* lo) const
    {
        if (L.sub < 0) {
#pragma unroll
            for (int a = 0; a < 3; ++a) lo[a] = (R)L.rem[a];
            return R(1);
        }
        const R h = inv_r();
#pragma unroll
        for (int a = 0; a < 3; ++a) lo[a] = (R)L.rem[a] + (R)((L.sub >> (8 * a)) & 255) * h;
        return h;
    }

    // Next-face times of every axis from the current point x + tcur k
    // (td holds 1/|k| per axis).
    __device__ __forceinline__ void face_times(Lane<R, NS>& L) const
    {
        R lo[3];
        const R h = cell_box(L, lo);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const R xa = L.x[a] + L.tcur * L.k[a];
            R d;
            if (L.k[a] > R(0)) d = lo[a] + h - xa;
            else if (L.k[a] < R(0)) d = xa - lo[a];
            else d = R(INFINITY);
            L.tm[a] = L.k[a] != R(0) ? L.tcur + fmax(d, R(0)) * L.td[a] : R(INFINITY);
        }
    }

    // The next crossing of a refined grid's traversal, found one crossing
    // ahead as on the uniform grid (nearest face, ties to the lowest axis):
    // inside a divided cube, the next sub-cube, whose density is requested
    // now (cinfo = -1); else the next cube, whose first cell (cinfo) and
    // packed density (undivided) are requested now side by side, or
    // cinfo = kLeaveGrid when the face is the grid's.  A uniform grid in a
    // batch of refined ones has no cube tables: its cubes are its cells.
    // Written with selects and one load of a selected address, so that
    // lanes stepping inside a cube and between cubes stay converged.
    static constexpr int kLeaveGrid = -2;

    __device__ __forceinline__ void prefetch_ref(Lane<R, NS>& L)
    {
        const int a = (L.tm[0] <= L.tm[1] && L.tm[0] <= L.tm[2]) ? 0 : (L.tm[1] <= L.tm[2] ? 1 : 2);
        L.nax = a;
        const R ka = a == 0 ? L.k[0] : (a == 1 ? L.k[1] : L.k[2]);
        const int sg = ka > R(0) ? 1 : -1;
        const int r = md->refine;
        const int sa = ((L.sub >> (8 * a)) & 255) + sg;
        const bool inside = L.sub >= 0 && sa >= 0 && sa < r;
        const int ia = (a == 0 ? L.rem[0] : (a == 1 ? L.rem[1] : L.rem[2])) + sg;
        const int n_a = a == 0 ? md->nx : (a == 1 ? md->ny : md->nz);
        const bool leave = !inside && (ia < 0 || ia >= n_a);
        const int i0 = a == 0 ? ia : L.rem[0], i1 = a == 1 ? ia : L.rem[1], i2 = a == 2 ? ia : L.rem[2];
        const int q = (i2 * md->ny + i1) * md->nx + i0;
        const PT* src = inside ? cells(L) + (L.c + sg * (a == 0 ? 1 : (a == 1 ? r : r * r)))
                               : (r ? cube_cells() : cells(L)) + q;
        if (!leave) L.pf = __ldg(src);
        int info = q;
        if (r && !inside && !leave) info = __ldg(md->cube + q);
        L.cinfo = inside ? -1 : (leave ? kLeaveGrid : info);
    }

    // Crossing of a refined grid's traversal through the face on axis a
    // (the one prefetch_ref found).  Steps that stay on one level take the
    // face spacing (td, or td / r in sub-cubes: a product, no division per
    // step) and the prefetched density: to the next sub-cube of the cube,
    // from an undivided cube to the next undivided one, and (FP32 build)
    // from a divided cube into the next divided one, whose sub-cubes continue
    // the same fine grid (the sub-cube index along a wraps, the others carry
    // over; its density is the one load not issued a crossing ahead).  A
    // change of level restarts the face times from the point; the descent
    // from an undivided into a divided cube takes the sub-cube that holds
    // the entry point.  The FP64 build takes the oracle's order of
    // operations, for trajectories equal to rounding: every cube step out of
    // or into a divided cube descends at the point and restarts the face
    // times.  Leaving the grid escapes.
    __device__ __forceinline__ void step_ref(Lane<R, NS>& L, int a)
    {
        if (L.cinfo == kLeaveGrid) {
            L.st = ST_ESCAPE;              // c keeps the last cell inside
            return;
        }
        const R ka = a == 0 ? L.k[0] : (a == 1 ? L.k[1] : L.k[2]);
        const bool pos = ka > R(0);
        const int sg = pos ? 1 : -1;
        const int r = md->refine;
        const bool inside = L.cinfo < 0;
        const bool fine = L.sub >= 0;
        const bool divided = !inside && (L.cinfo & kCubeDivided) != 0;
        const R h = fine ? inv_r() : R(1);
        // one-level update, for every lane (selects, not a run-time index)
        L.tm[0] = a == 0 ? L.tm[0] + L.td[0] * h : L.tm[0];
        L.tm[1] = a == 1 ? L.tm[1] + L.td[1] * h : L.tm[1];
        L.tm[2] = a == 2 ? L.tm[2] + L.td[2] * h : L.tm[2];
        const int dr = inside ? 0 : sg;
        L.rem[0] += a == 0 ? dr : 0;
        L.rem[1] += a == 1 ? dr : 0;
        L.rem[2] += a == 2 ? dr : 0;
        const int sh = 8 * a;
        const int sa = inside ? ((L.sub >> sh) & 255) + sg : (pos ? 0 : r - 1);
        const int sub = (L.sub & ~(255 << sh)) | (sa << sh);
        L.sub = (inside || divided) ? sub : -1;
        const int off = (((sub >> 16) & 255) * r + ((sub >> 8) & 255)) * r + (sub & 255);
        L.c = inside ? L.c + sg * (a == 0 ? 1 : (a == 1 ? r : r * r))
                     : (divided ? (L.cinfo & ~kCubeDivided) + off : L.cinfo);
        PT v = L.pf;
        if (fine && divided) v = __ldg(cells(L) + L.c);
        use_cell(L, v);
        const bool restart = DBG ? (!inside && (fine || divided)) : (fine != (inside || divided));
        if (restart) {
            if (divided) {
                R xc[3];
#pragma unroll
                for (int b = 0; b < 3; ++b) xc[b] = L.x[b] + L.tcur * L.k[b];
                descend(L, L.cinfo, xc, a);
                load_cell(L);
            }
            face_times(L);
        }
        prefetch_ref(L);
    }

    __device__ __forceinline__ void emit(Lane<R, NS>& L, uint64_t w)
    {
        if constexpr (HAS_DEFER) {
            if (P.resume) {
                resume(L, w);
                return;
            }
        }
        int lo = 0;
        if constexpr (!SINGLE) {
            // model lookup: largest m with prefix[m] <= w
            int hi = P.n_models - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (P.prefix[mid] <= w) lo = mid; else hi = mid - 1;
            }
            if (lo != L.m) {
                if (L.m >= 0) flush_lane(L.m);
                L.m = lo;
            }
            md = model(lo);
            L.grid = md->rho;
        } else {
            L.m = 0;
        }
        rng_init(L.rng, P.seed, md->model_id, md->pid_begin + (w - P.prefix[lo]));
        L.seq = 0;
        L.nev = 0;
        L.ncross = 0;
        L.nlucy = 0;
        if constexpr (HAS_PAH) {
            if (P.pah_src) {
                emit_pah(L, md->pid_begin + (w - P.prefix[lo]));
                return;
            }
        }
        int si = 0;
        R ub;
        bool binned = false;
        if (P.source_bins && P.sg_nu) {
            // the separate source grid of Eq. 1: source bin b's source and model bin
            const uint64_t pid = ((uint64_t)L.rng.phi << 32) | L.rng.plo;
            const uint64_t b = (pid * P.source_bins) / md->n_emit;
            si = P.sg_src[b];
            L.j = P.sg_nu[b];
            ub = R(0);
            binned = true;
        } else if (P.source_bins) {
            // Eq. 1: equal-energy source bins, packet pid from bin floor(pid m / N)
            // at the point (b + 1/2) / m of the cumulative luminosity: its source,
            // then (by the fraction of that source below the point) its bin
            const uint64_t pid = ((uint64_t)L.rng.phi << 32) | L.rng.plo;
            const uint64_t b = (pid * P.source_bins) / md->n_emit;
            const double target = ((double)b + 0.5) / (double)P.source_bins * md->src_Lcdf[md->nsrc - 1];
            si = search_cdf(md->src_Lcdf, md->nsrc, target);
            const double below = si > 0 ? md->src_Lcdf[si - 1] : 0.0;
            ub = (R)((target - below) / (md->src_Lcdf[si] - below));
        } else {
            if (md->nsrc > 1) {
                const double u = (double)U(L);
                si = search_cdf(md->src_Lcdf, md->nsrc, u * md->src_Lcdf[md->nsrc - 1]);
            }
            ub = U(L);
        }
        if (!binned) {
            if constexpr (DBG) {
                const double* cdf = md->src_cdf64 + (size_t)si * P.nf;
                L.j = search_cdf(cdf, P.nf, ub * cdf[P.nf - 1]);
            } else {
                L.j = search_cdf((P.smem_cdf ? s_cdf() : md->src_cdf32) + (size_t)si * P.nf, P.nf, ub);
            }
        }
        const R u1 = U(L), u2 = U(L);
        iso_dir(u1, u2, L.k);
        int idx[3];
        const int n[3] = { md->nx, md->ny, md->nz };
        bool in = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            L.x[a] = (R)md->src_pos[si * 3 + a];
            const R f = floor(L.x[a]);
            int i = (int)f;
            if (f == L.x[a] && L.k[a] < R(0)) i -= 1;
            idx[a] = i;
            in = in && (i >= 0 && i < n[a]);
        }
        L.c = in ? (idx[2] * n[1] + idx[1]) * n[0] + idx[0] : 0;
        if constexpr (HAS_REF) {
            if (in) enter_cube(L, L.c, idx, L.x, -1);
        }
        count(RT_STAT_EMITTED, 1);
        traj(L, RT_TRAJ_EMIT, L.x);
        if (!in) {
            L.tcur = R(0);
            L.st = ST_ESCAPE;
            return;
        }
#pragma unroll
        for (int s = 0; s < NS; ++s) L.rho[s] = R(0);
        load_freq(L);
        load_cell(L);
        L.st = ST_FLIGHT;
    }

    // PAH re-emission (Sect. 2.1): the stored absorption's cell is the
    // source; the bin follows Eq. 6 with the cell's emissivity class, the
    // point is uniform in the cell (one draw per axis), the direction
    // isotropic.  A record outside the grid, or a cell whose class is out of
    // range, is counted as stuck and emits nothing.
    __device__ __forceinline__ void emit_pah(Lane<R, NS>& L, uint64_t pid)
    {
        const int c = (int)P.pah_src[pid].cell;
        const R ub = U(L);
        const R ux = U(L), uy = U(L), uz = U(L);
        const R u1 = U(L), u2 = U(L);
        const bool in = (unsigned)c < (unsigned)md->ncell;
        const int n = !in ? -1 : (P.eps_class ? P.eps_class[c] : 0);
        count(RT_STAT_EMITTED, 1);
        if ((unsigned)n >= (unsigned)P.n_eps) {
            count(RT_STAT_STUCK, 1);
            end_packet(L);
            return;
        }
        if constexpr (DBG) {
            const double* cdf = P.eps_cdf64 + (size_t)n * P.nf;
            L.j = search_cdf(cdf, P.nf, ub * cdf[P.nf - 1]);
        } else {
            L.j = search_cdf(P.eps_cdf32 + (size_t)n * P.nf, P.nf, ub);
        }
        if constexpr (HAS_REF) {
            set_from_cell(L, c);
            R lo[3];
            const R h = cell_box(L, lo);
            L.x[0] = lo[0] + ux * h;
            L.x[1] = lo[1] + uy * h;
            L.x[2] = lo[2] + uz * h;
        } else {
            const int ix = c % md->nx, iy = (c / md->nx) % md->ny, iz = c / (md->nx * md->ny);
            L.x[0] = (R)ix + ux;
            L.x[1] = (R)iy + uy;
            L.x[2] = (R)iz + uz;
        }
        iso_dir(u1, u2, L.k);
        L.c = c;
        traj(L, RT_TRAJ_EMIT, L.x);
#pragma unroll
        for (int s = 0; s < NS; ++s) L.rho[s] = R(0);
        load_freq(L);
        load_cell(L);
        L.st = ST_FLIGHT;
    }

    // Energy deposited along a path of l cells in a Lucy cell (Sect. 3.1).
    // FP64 build: straight into E_abs.  FP32 build: into the call's FP64
    // scratch in units of xi, converted with integer work and added by L2
    // atomics, so the crossing loop issues no FP64 arithmetic.
    __device__ __forceinline__ void deposit_lucy(Lane<R, NS>& L, R l)
    {
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const size_t idx = (size_t)s * md->ncell + L.c;
            R ta = L.kab[s] * L.rho[s] * l;
            if (P.lucy_form == RT_LUCY_EXPM1) ta = -r_expm1(-ta);
            if constexpr (DBG) {
                const double e = ta * md->xi;
                if (e != 0.0) {
                    atomicAdd(&md->E_abs[idx], e);
                    if (md->esq) atomicAdd(&md->esq[idx], e * e);
                }
            } else {
                if (ta > 0.0f) {
                    Acc* e = acc_at(idx);
                    atomicAdd(e, to_acc(ta));
                    if (md->acc_q) atomicAdd(e + 1, to_acc(ta * ta));
                }
            }
        }
        L.nlucy++;
    }

    // Accumulated absorbed power (erg/s) of species s in the lane's cell,
    // including this call's FP32-build scratch; `old` is the value an atomic
    // add just returned (then the packet's own xi is added).  The FP64
    // scratch starts each call at E_abs / xi (seed_kernel), so it alone holds
    // the accumulated energy and an absorption reads nothing beyond its
    // atomic; the FP32 scratch of the plain-FP32 form starts at zero.
    __device__ __forceinline__ double energy(const Lane<R, NS>& L, int s, double old, bool have_old)
    {
        const size_t i = (size_t)s * md->ncell + L.c;
        if constexpr (DBG) {
            return have_old ? old + md->xi : __ldcg(&md->E_abs[i]);
        } else if constexpr (ACC32) {
            const double acc = have_old ? old + 1.0 : (double)__ldcg(acc_at(i));
            return __ldcg(&md->E_abs[i]) + acc * md->xi;
        } else {
            return (have_old ? old + 1.0 : __ldcg(acc_at(i))) * md->xi;
        }
    }

    // Temperature of species s in cell c from the accumulated energy (Eq. 4),
    // FP64 build
    __device__ __forceinline__ double temperature64(const Lane<R, NS>& L, int s, double E)
    {
        double rv = sel(L.rho, s) * md->vol;
        if constexpr (HAS_REF) {
            if (L.sub >= 0) rv /= (double)md->refine * md->refine * md->refine;   // sub-cube volume
        }
        return rv > 0.0 ? solve_T64(P, s, E / rv) : 0.0;
    }

    // FP32 build: log2 of the temperature that sets the re-emission spectrum,
    // Eq. 4 at the updated energy (B&W; FP32 inverse table of 4 pi P) or the
    // previous iteration's value (frozen T); -inf when there is none
    __device__ __forceinline__ float emission_log2T(const Lane<R, NS>& L, int s, double E)
    {
        if (P.mode == RT_MODE_BW) {
            const float rs = sel(L.rho, s);
            if (!(E > 0.0) || !(rs > 0.0f)) return -INFINITY;
            float y = log2_d(E) - __log2f(rs) - (float)md->log2_4piV;
            if constexpr (HAS_REF) {
                if (L.sub >= 0) y += 3.0f * __log2f((float)md->refine);       // sub-cube volume
            }
            float f = (y - P.tinv_y0[s]) * P.tinv_inv_dy[s];
            f = fminf(fmaxf(f, 0.0f), (float)(kTinvN - 1));
            const int i = min((int)f, kTinvN - 2);
            const float w = f - (float)i;
            const float* t = P.tinv + (size_t)s * kTinvN;
            return t[i] + w * (t[i + 1] - t[i]);
        }
        const double T = md->T_prev[(size_t)s * md->ncell + L.c];
        return T > 0.0 ? log2_d(T) : -INFINITY;
    }

    // Re-emission frequency bin: Eq. 10 (B&W, dB/dT weights) or Eq. 5 (frozen
    // T).  FP64 build: the exact cumulative sum over bins.  FP32 build: the
    // bin law tabulated on a uniform log2 T grid as alias tables; between the
    // two bracketing rows the upper one is taken with probability equal to
    // the interpolation weight (a draw from the linearly interpolated
    // spectrum), then one alias-table read gives the bin.
    __device__ __forceinline__ int reemit(Lane<R, NS>& L, int s, double E, R u)
    {
        if constexpr (DBG) {
            const double T = P.mode == RT_MODE_BW ? temperature64(L, s, E)
                                                  : md->T_prev[(size_t)s * md->ncell + L.c];
            const bool bw = P.mode == RT_MODE_BW;
            const int nf = P.nf;
            double tot = 0.0;
            for (int l = 0; l < nf; ++l) {
                const double b = bw ? planck_dBdT(P.nu[l], T) : planck_B(P.nu[l], T);
                tot += P.kabs[s * nf + l] * b * P.dnu[l];
            }
            const double target = u * tot;
            double acc = 0.0;
            for (int l = 0; l < nf; ++l) {
                const double b = bw ? planck_dBdT(P.nu[l], T) : planck_B(P.nu[l], T);
                acc += P.kabs[s * nf + l] * b * P.dnu[l];
                if (acc >= target) return l;
            }
            return nf - 1;
        } else {
            const float lg = emission_log2T(L, s, E);
            const float u_row = U(L);
            if (!(lg > -1.0e30f)) return 0;
            float f = (lg - P.re_lg0) * P.re_inv_dlg;
            f = fminf(fmaxf(f, 0.0f), (float)(kReT - 1));
            int k = min((int)f, kReT - 2);
            if (u_row < f - (float)k) ++k;
            // alias table of the row: one read
            const uint32_t* row = P.realias + ((size_t)s * kReT + k) * P.nf;
            const float x = u * (float)P.nf;
            const int j0 = min((int)x, P.nf - 1);
            const uint32_t w = __ldg(row + j0);
            return x - (float)j0 < (float)(w >> 10) * 0x1p-22f ? j0 : (int)(w & 1023u);
        }
    }

    // after the re-emission bin is known: isotropic direction, new flight
    __device__ __forceinline__ void finish_absorb(Lane<R, NS>& L)
    {
        { const R u1 = U(L), u2 = U(L); iso_dir(u1, u2, L.k); }
        load_freq(L);
        traj(L, RT_TRAJ_ABSORB, L.x);
        L.st = ST_FLIGHT;
    }

    __device__ __forceinline__ int pick_species(const Lane<R, NS>& L, bool sca, R u)
    {
        R w[NS];
        R tot = R(0);
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            R ks;
            if constexpr (DBG) ks = s >= P.ns ? 0.0 : (sca ? P.ksca[s * P.nf + L.j] : P.kabs[s * P.nf + L.j]);
            else ks = sca ? s_op()[s * P.nf + L.j].z : s_op()[s * P.nf + L.j].y;
            w[s] = L.rho[s] * ks;
            tot += w[s];
        }
        const R target = u * tot;
        R acc = R(0);
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            acc += w[s];
            if (acc >= target) return s;
        }
        return P.ns - 1;
    }

    // A slot of a per-model append cursor for each calling lane: the lanes of
    // a warp appending to the same model's list share one atomic (a hot
    // address otherwise serialises in L2), each taking base + its rank.
    __device__ __forceinline__ unsigned long long claim_slot(unsigned long long* cursor, unsigned key) const
    {
        const unsigned grp = __match_any_sync(__activemask(), key);
        const int leader = __ffs(grp) - 1;
        const unsigned lane = threadIdx.x & 31;
        unsigned long long base = 0;
        if ((int)lane == leader) base = atomicAdd(cursor, (unsigned long long)__popc(grp));
        base = __shfl_sync(grp, base, leader);
        return base + __popc(grp & ((1u << lane) - 1u));
    }

    __device__ __forceinline__ void store_pah(Lane<R, NS>& L, const R* x)
    {
        const unsigned long long slot = claim_slot(&md->stats[RT_STAT_N_PAH], (unsigned)L.m);
        if (md->pah && slot < md->pah_cap) {
            rt_pah_event e;
            e.cell = (uint32_t)L.c; e.nu = (uint16_t)L.j; e.model = (uint16_t)md->model_index;
            md->pah[slot] = e;
        } else {
            atomicAdd(&md->stats[RT_STAT_PAH_DROPPED], 1ull);
        }
        count(RT_STAT_PAH, 1);
        traj(L, RT_TRAJ_PAH, x);
        end_packet(L);
    }

    __device__ __forceinline__ bool is_pah(int s) const { return (P.pah_mask >> s) & 1; }

    // A new flight from L.x along L.k: MRW step or tau draw + traversal set-up
    __device__ __forceinline__ void flight(Lane<R, NS>& L)
    {
        if constexpr (HAS_DEFER) {
            if (P.defer_events && !P.resume && L.nev >= P.defer_events && defer(L)) return;
        }
        if constexpr (HAS_REF) {
            flight_ref(L);
            return;
        }
        const int nx = md->nx, ny = md->ny, nz = md->nz;
        const int iz = L.c / (nx * ny);
        const int r = L.c - iz * nx * ny;
        const int iy = r / nx;
        const int ix = r - iy * nx;
        const int id[3] = { ix, iy, iz };
        if constexpr (HAS_MRW) {
            if (P.mrw && P.mode != RT_MODE_NOREEMIT && L.chi > (R)P.mrw_tau_cell) {
                R R0 = R(1e30);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const R d1 = L.x[a] - (R)id[a], d2 = (R)(id[a] + 1) - L.x[a];
                    R0 = fmin(R0, fmin(d1, d2));
                }
                R0 = fmax(R0, R(0));
                if (R0 * L.chi >= (R)P.mrw_gamma) {
                    mrw_step(L, R0);
                    return;
                }
            }
        }
        L.tau = -r_log(U(L));
        const int n[3] = { nx, ny, nz };
        const int stride[3] = { 1, nx, nx * ny };
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const R ka = L.k[a];
            if (ka > R(0)) {
                L.td[a] = R(1) / ka;
                L.tm[a] = fmax(((R)(id[a] + 1) - L.x[a]) * L.td[a], R(0));
                L.rem[a] = n[a] - 1 - id[a];
                L.dc[a] = stride[a];
            } else if (ka < R(0)) {
                L.td[a] = R(-1) / ka;
                L.tm[a] = fmax((L.x[a] - (R)id[a]) * L.td[a], R(0));
                L.rem[a] = id[a];
                L.dc[a] = -stride[a];
            } else {
                L.td[a] = R(INFINITY);
                L.tm[a] = R(INFINITY);
                L.rem[a] = 1;
                L.dc[a] = 0;
            }
        }
        L.tcur = R(0);
        prefetch_next(L);
        L.st = ST_MARCH;
    }

    // Flight of a refined grid's packet: the MRW sphere and threshold use the
    // cell's own box (a sub-cube's in divided cubes), then the two-level
    // traversal starts from the cell's faces.
    __device__ __forceinline__ void flight_ref(Lane<R, NS>& L)
    {
        R lo[3];
        const R h = cell_box(L, lo);
        if constexpr (HAS_MRW) {
            if (P.mrw && P.mode != RT_MODE_NOREEMIT && L.chi * h > (R)P.mrw_tau_cell) {
                R R0 = R(1e30);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const R d1 = L.x[a] - lo[a], d2 = lo[a] + h - L.x[a];
                    R0 = fmin(R0, fmin(d1, d2));
                }
                R0 = fmax(R0, R(0));
                if (R0 * L.chi >= (R)P.mrw_gamma) {
                    mrw_step(L, R0);
                    return;
                }
            }
        }
        L.tau = -r_log(U(L));
#pragma unroll
        for (int a = 0; a < 3; ++a) L.td[a] = L.k[a] != R(0) ? R(1) / fabs(L.k[a]) : R(INFINITY);
        L.tcur = R(0);
        face_times(L);
        prefetch_ref(L);
        L.st = ST_MARCH;
    }

    // One crossing step of a refined grid's traversal (exit face and next
    // cell found one crossing earlier by prefetch_ref)
    __device__ __forceinline__ void march_ref(Lane<R, NS>& L)
    {
        const int a = L.nax;
        const R tn = a == 0 ? L.tm[0] : (a == 1 ? L.tm[1] : L.tm[2]);
        const R seg = tn - L.tcur;
        const R dtau = L.chi * seg;
        if (dtau <= L.tau) {
            if (L.lucy) deposit_lucy(L, seg);
            L.tau -= dtau;
            L.tcur = tn;
            L.ncross++;
            step_ref(L, a);
        } else {
            const R d = L.tau / L.chi;
            if (L.lucy) deposit_lucy(L, d);
            L.tcur += d;
#pragma unroll
            for (int a2 = 0; a2 < 3; ++a2) L.x[a2] += L.tcur * L.k[a2];
            L.st = ST_INTERACT;
        }
    }

    __device__ __forceinline__ void mrw_step(Lane<R, NS>& L, R R0)
    {
        if (++L.nev > P.max_events) {
            count(RT_STAT_STUCK, 1);
            traj(L, RT_TRAJ_STUCK, L.x);
            end_packet(L);
            return;
        }
        const R u = U(L);
        R y;
        if constexpr (DBG) y = mrw_y64(u);
        else y = mrw_y32(s_mrw(), u);
        const R l = R(3) * L.chi * R0 * R0 * y;          // path length in cells
        R nh[3];
        { const R u1 = U(L), u2 = U(L); iso_dir(u1, u2, nh); }
#pragma unroll
        for (int a = 0; a < 3; ++a) L.x[a] += R0 * nh[a];
        { const R u3 = U(L), u4 = U(L); iso_dir(u3, u4, L.k); }
        R ca = R(0);
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const size_t idx = (size_t)s * md->ncell + L.c;
            const R ta = L.kab[s] * L.rho[s] * l;
            ca += L.kab[s] * L.rho[s];
            if constexpr (DBG) {
                const double e = ta * md->xi;
                if (e != 0.0) {
                    atomicAdd(&md->E_abs[idx], e);
                    if (md->esq) atomicAdd(&md->esq[idx], e * e);
                }
            } else if (ta > 0.0f) {
                Acc* e = acc_at(idx);
                atomicAdd(e, to_acc(ta));
                if (md->acc_q) atomicAdd(e + 1, to_acc(ta * ta));
            }
        }
        count(RT_STAT_MRW, 1);
        if (U(L) < -r_expm1(-ca * l)) {
            int s = 0;
            if (NS > 1) s = pick_species(L, false, U(L));
            if (is_pah(s)) { store_pah(L, L.x); return; }
            const double E = energy(L, s, 0.0, false);
            L.j = reemit(L, s, E, U(L));
            load_freq(L);
        }
        traj(L, RT_TRAJ_MRW, L.x);
        L.st = ST_FLIGHT;
    }

    // One cell traversal step of a marching lane.  The exit face and the
    // next cell were found (and the next density requested) one step earlier;
    // updates are branch-free so lanes stepping along different axes stay
    // converged.
    __device__ __forceinline__ void march(Lane<R, NS>& L)
    {
        if constexpr (HAS_REF) {
            march_ref(L);
            return;
        }
        const int a = L.nax;
        const R tn = a == 0 ? L.tm[0] : (a == 1 ? L.tm[1] : L.tm[2]);
        const R seg = tn - L.tcur;
        const R dtau = L.chi * seg;
        if (dtau <= L.tau) {
            if (L.lucy) deposit_lucy(L, seg);
            L.tau -= dtau;
            L.tcur = tn;
            L.ncross++;
            if (L.outn) {
                L.st = ST_ESCAPE;          // c keeps the last cell inside
            } else {
                L.tm[0] = a == 0 ? L.tm[0] + L.td[0] : L.tm[0];
                L.tm[1] = a == 1 ? L.tm[1] + L.td[1] : L.tm[1];
                L.tm[2] = a == 2 ? L.tm[2] + L.td[2] : L.tm[2];
                L.rem[0] -= a == 0;
                L.rem[1] -= a == 1;
                L.rem[2] -= a == 2;
                L.c = L.cn;
                use_cell(L, L.pf);
                prefetch_next(L);
            }
        } else {
            const R d = L.tau / L.chi;
            if (L.lucy) deposit_lucy(L, d);
            L.tcur += d;
#pragma unroll
            for (int a2 = 0; a2 < 3; ++a2) L.x[a2] += L.tcur * L.k[a2];
            L.st = ST_INTERACT;
        }
    }

    __device__ __forceinline__ void interact(Lane<R, NS>& L)
    {
        if (++L.nev > P.max_events) {
            count(RT_STAT_STUCK, 1);
            traj(L, RT_TRAJ_STUCK, L.x);
            end_packet(L);
            return;
        }
        count(RT_STAT_INTERACTIONS, 1);
        R cs = R(0);
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            R ks;
            if constexpr (DBG) ks = s < P.ns ? P.ksca[s * P.nf + L.j] * md->cell : 0.0;
            else ks = s_op()[s * P.nf + L.j].z;
            cs += L.rho[s] * ks;
        }
        const R albedo = cs / L.chi;
        if (U(L) < albedo) {
            int s = 0;
            if (NS > 1) s = pick_species(L, true, U(L));
            R g;
            if constexpr (DBG) g = P.g[s * P.nf + L.j];
            else g = s_op()[s * P.nf + L.j].w;
            const R mu = hg_mu(g, U(L));
            const R uphi = U(L);
            if (P.record_events && ((P.ev_mask[L.j >> 5] >> (L.j & 31)) & 1u)) {
                const unsigned long long slot = claim_slot(&md->stats[RT_STAT_N_EVENTS], (unsigned)L.m);
                if (md->events && slot < md->event_cap) {
                    rt_event e;
                    e.cell = (uint32_t)L.c; e.nu = (uint16_t)L.j; e.species = (uint8_t)s;
                    e.model = (uint8_t)md->model_index;
                    e.k[0] = (float)L.k[0]; e.k[1] = (float)L.k[1]; e.k[2] = (float)L.k[2];
                    md->events[slot] = e;
                } else {
                    atomicAdd(&md->stats[RT_STAT_EVENTS_DROPPED], 1ull);
                }
            }
            rotate(L.k, mu, uphi);
            count(RT_STAT_SCATTERS, 1);
            traj(L, RT_TRAJ_SCATTER, L.x);
            L.st = ST_FLIGHT;
            return;
        }
        count(RT_STAT_ABSORPTIONS, 1);
        int s = 0;
        if (NS > 1) s = pick_species(L, false, U(L));
        if (is_pah(s)) { store_pah(L, L.x); return; }
        const size_t idx = (size_t)s * md->ncell + L.c;
        double E = 0.0;
        if constexpr (DBG) {
            if (!L.lucy) {
                const double old = atomicAdd(&md->E_abs[idx], md->xi);
                if (md->esq) atomicAdd(&md->esq[idx], md->xi * md->xi);
                if (P.mode == RT_MODE_BW) E = energy(L, s, old, true);
            } else if (P.mode == RT_MODE_BW) {
                E = energy(L, s, 0.0, false);
            }
            atomicAdd(&md->count[idx], 1u);
        } else {
            // Lanes absorbing in the same cell and species combine into one
            // atomic: the group leader adds the group size, and lane r of the
            // group sees the old value plus r (as if the lanes absorbed one
            // after another in lane order).  Optically thick cells next to a
            // source receive most absorptions; per-lane atomics on them
            // serialise in L2.
            const unsigned grp = __match_any_sync(__activemask(), (unsigned long long)idx * 2u + (L.lucy ? 1u : 0u));
            const int leader = __ffs(grp) - 1;
            const unsigned rank = __popc(grp & ((1u << (threadIdx.x & 31)) - 1u));
            const unsigned n = __popc(grp);
            const bool lead = (int)(threadIdx.x & 31) == leader;
            double old = 0.0;
            if (!L.lucy) {
                Acc* e = acc_at(idx);
                if (lead) {
                    if (P.mode == RT_MODE_BW) old = (double)atomicAdd(e, (Acc)n);
                    else atomicAdd(e, (Acc)n);
                    if (md->acc_q) atomicAdd(e + 1, (Acc)n);
                }
                if (P.mode == RT_MODE_BW) {
                    old = __shfl_sync(grp, old, leader) + (double)rank;
                    E = energy(L, s, old, true);
                }
            } else if (P.mode == RT_MODE_BW) {
                E = energy(L, s, 0.0, false);
            }
            if (lead) atomicAdd(&md->count[idx], n);
        }
        if (P.mode == RT_MODE_NOREEMIT) {
            traj(L, RT_TRAJ_ABSORB_END, L.x);
            end_packet(L);
            return;
        }
        const R u = U(L);
        L.j = reemit(L, s, E, u);
        finish_absorb(L);
    }

    // Photon counting (Sect. 4): the escaping packet's power goes to the
    // pixel of its exit point projected on each camera whose acceptance cone
    // holds its direction; the projection runs in FP64 in cell units.
    __device__ __forceinline__ void photon_count(const Lane<R, NS>& L) const
    {
        double xe[3], k[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            k[a] = (double)L.k[a];
            xe[a] = (double)L.x[a] + (double)L.tcur * k[a] - P.pc_ctr[a];
        }
        for (int c = 0; c < P.n_pc; ++c) {
            const PcDev& q = P.pc[c];
            const double kd = k[0] * q.kobs[0] + k[1] * q.kobs[1] + k[2] * q.kobs[2];
            if (!(kd >= q.cos_accept)) continue;
            const double xp = xe[0] * q.ex[0] + xe[1] * q.ex[1] + xe[2] * q.ex[2];
            const double yp = xe[0] * q.ey[0] + xe[1] * q.ey[1] + xe[2] * q.ey[2];
            const double fx = floor(xp * q.pix_per_cell + q.half_npix);
            const double fy = floor(yp * q.pix_per_cell + q.half_npix);
            if (fx >= 0.0 && fx < q.npix && fy >= 0.0 && fy < q.npix)
                atomicAdd(&P.pc_img[q.off + ((unsigned long long)L.j * q.npix + (int)fy) * q.npix + (int)fx],
                          md->xi);
        }
    }

    __device__ __forceinline__ void escape(Lane<R, NS>& L)
    {
        int b = (int)floor((L.k[2] + R(1)) * R(5));
        b = min(max(b, 0), kSedBins - 1);
        if (P.smem_sed && !DBG) {
            atomicAdd(&s_sed()[b * P.nf + L.j], md->xi);
            atomicAdd(&s_cnt()[b * P.nf + L.j], 1u);
        } else if constexpr (DBG) {
            atomicAdd(&md->sed_esc[b * P.nf + L.j], md->xi);
            atomicAdd(&md->sed_cnt[b * P.nf + L.j], 1ull);
        } else {
            // the lanes of a warp escaping into the same model's bin add once
            const unsigned key = ((unsigned)L.m << 16) | (unsigned)(b * P.nf + L.j);
            const unsigned grp = __match_any_sync(__activemask(), key);
            if ((int)(threadIdx.x & 31) == __ffs(grp) - 1) {
                const unsigned n = __popc(grp);
                atomicAdd(&md->sed_esc[b * P.nf + L.j], md->xi * (double)n);
                atomicAdd(&md->sed_cnt[b * P.nf + L.j], (unsigned long long)n);
            }
        }
        count(RT_STAT_ESCAPED, 1);
        if constexpr (HAS_PC) {
            if (P.n_pc) photon_count(L);
        }
        if constexpr (HAS_TRAJ) {
            if (md->traj) {
                R xe[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) xe[a] = L.x[a] + L.tcur * L.k[a];
                traj(L, RT_TRAJ_ESCAPE, xe);
            }
        }
        end_packet(L);
    }

    // ------------------------------------------------ per-warp compaction
    // A packet parks in a stash record of six uint4 (96 bytes): Philox
    // position, event count, cell, frequency bin, state, remaining optical
    // depth, flight origin and time, direction, next-face times and spacings,
    // steps left per axis.  Its crossing and Lucy counters go to the parking
    // lane's tallies first.  Unparking restores the registers exactly (the
    // rest -- densities of the cell, opacities of the bin, strides, the
    // prefetched next cell -- is reloaded), so a packet's trajectory does not
    // depend on the lanes it visits.
    __device__ __forceinline__ void park(Lane<R, NS>& L, uint4* rec)
    {
        count(RT_STAT_CROSSINGS, L.ncross);
        count(RT_STAT_LUCY, L.nlucy);
        L.ncross = 0;
        L.nlucy = 0;
        rec[0] = make_uint4(L.rng.plo, L.rng.phi, L.rng.draw, L.rng.c_hi);
        rec[1] = make_uint4(L.nev, (unsigned)L.c, (unsigned)L.j | ((unsigned)L.st << 24), __float_as_uint(L.tau));
        rec[2] = make_uint4(__float_as_uint(L.x[0]), __float_as_uint(L.x[1]), __float_as_uint(L.x[2]),
                            __float_as_uint(L.tcur));
        rec[3] = make_uint4(__float_as_uint(L.k[0]), __float_as_uint(L.k[1]), __float_as_uint(L.k[2]),
                            (unsigned)L.rem[0]);
        rec[4] = make_uint4(__float_as_uint(L.tm[0]), __float_as_uint(L.tm[1]), __float_as_uint(L.tm[2]),
                            (unsigned)L.rem[1]);
        rec[5] = make_uint4(__float_as_uint(L.td[0]), __float_as_uint(L.td[1]), __float_as_uint(L.td[2]),
                            (unsigned)L.rem[2]);
    }

    __device__ __forceinline__ void unpark(Lane<R, NS>& L, const uint4* rec)
    {
        L.rng.ky = (uint32_t)(P.seed >> 32) ^ md->model_id;
        { const uint4 r = rec[0]; L.rng.plo = r.x; L.rng.phi = r.y; L.rng.draw = r.z; L.rng.c_hi = r.w; }
        L.rng.c_lo = 0;
        {
            const uint4 r = rec[1];
            L.nev = r.x;
            L.c = (int)r.y;
            L.j = (int)(r.z & 0xffffffu);
            L.st = (int)(r.z >> 24);
            L.tau = __uint_as_float(r.w);
        }
        {
            const uint4 r = rec[2];
            L.x[0] = __uint_as_float(r.x); L.x[1] = __uint_as_float(r.y); L.x[2] = __uint_as_float(r.z);
            L.tcur = __uint_as_float(r.w);
        }
        {
            const uint4 r = rec[3];
            L.k[0] = __uint_as_float(r.x); L.k[1] = __uint_as_float(r.y); L.k[2] = __uint_as_float(r.z);
            L.rem[0] = (int)r.w;
        }
        {
            const uint4 r = rec[4];
            L.tm[0] = __uint_as_float(r.x); L.tm[1] = __uint_as_float(r.y); L.tm[2] = __uint_as_float(r.z);
            L.rem[1] = (int)r.w;
        }
        {
            const uint4 r = rec[5];
            L.td[0] = __uint_as_float(r.x); L.td[1] = __uint_as_float(r.y); L.td[2] = __uint_as_float(r.z);
            L.rem[2] = (int)r.w;
        }
        L.m = 0;
        L.seq = 0;
        L.ncross = 0;
        L.nlucy = 0;
        load_freq(L);
        load_cell(L);
        if (L.st == ST_MARCH) {
            const int stride[3] = { 1, md->nx, md->nx * md->ny };
#pragma unroll
            for (int a = 0; a < 3; ++a)
                L.dc[a] = L.k[a] > R(0) ? stride[a] : (L.k[a] < R(0) ? -stride[a] : 0);
            prefetch_next(L);
        }
    }

    // End of the persistent loop (all lanes converged): counters of warps
    // whose lanes share one model are summed with shuffles first.
    __device__ __forceinline__ void flush_warp(int m) const
    {
        const int m0 = __shfl_sync(FULL, m, 0);
        if (__all_sync(FULL, m == m0)) {
            if (m0 < 0) return;
            unsigned long long* st = P.models[m0].stats;
#pragma unroll
            for (int i = 0; i < kLaneStats; ++i) {
                unsigned long long v = slot(i);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
                if ((threadIdx.x & 31) == 0 && v) atomicAdd(&st[i], v);
            }
        } else if (m >= 0) {
            flush_lane(m);
        }
    }

    // block SED tallies to global memory (thread-strided, after a barrier)
    __device__ __forceinline__ void flush_sed(int t, int nt) const
    {
        if (P.smem_sed && !DBG) {
            const ModelDev& m0 = P.models[0];
            const double* sed = s_sed();
            const unsigned* cnt = s_cnt();
            for (int i = t; i < kSedBins * P.nf; i += nt)
                if (cnt[i]) {
                    atomicAdd(&m0.sed_esc[i], sed[i]);
                    atomicAdd(&m0.sed_cnt[i], (unsigned long long)cnt[i]);
                }
        }
    }
};

// Packets claimed per warp in chunks from the global work counter (one
// atomic per chunk; 256 down to 32 ids as the work runs out), the warp's
// unclaimed range kept in shared memory: lanes in state NEED emit the next
// ids; lanes that find none become DONE once every id has been claimed.
template <typename R, int NS, int FEAT>
__device__ __forceinline__ void refill(Kernel<R, NS, FEAT>& K, Lane<R, NS>& L, const TransportKP& P,
                                       unsigned long long* claim, unsigned long long total_work, int lane)
{
    const unsigned need = __ballot_sync(FULL, L.st == ST_NEED);
    if (!need) return;
    unsigned long long w_next = claim[0], w_end = claim[1];
    if (w_next == w_end && w_end < total_work) {
        unsigned long long base = 0;
        const unsigned long long n_warps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
        unsigned long long chunk = (total_work - w_end) / (4ull * n_warps);
        chunk = chunk < 32ull ? 32ull : (chunk > 256ull ? 256ull : chunk);
        if (lane == 0) base = atomicAdd(P.work_ctr, chunk);
        base = __shfl_sync(FULL, base, 0);
        if (base >= total_work) {
            w_next = w_end = total_work;
        } else {
            w_next = base;
            w_end = base + chunk < total_work ? base + chunk : total_work;
        }
    }
    const unsigned avail = (unsigned)(w_end - w_next);
    const unsigned rank = __popc(need & ((1u << lane) - 1u));
    if (L.st == ST_NEED) {
        if (rank < avail) K.emit(L, w_next + rank);
        else if (w_end >= total_work) L.st = ST_DONE;
    }
    w_next += __popc(need) < avail ? __popc(need) : avail;
    __syncwarp();
    if (lane == 0) { claim[0] = w_next; claim[1] = w_end; }
    __syncwarp();
}

// Per-warp packet compaction (RT_SCHED_COMPACT; the load balancing of Sect.
// 3.4 done inside a warp).  Each warp owns a stash of kStash packet records
// in shared memory, besides the 32 packets its lanes hold, and alternates two
// phases so that its lanes run the same code:
//   event phase  lanes still marching park their packets and take pending
//                ones (stopped at an interaction or escape, or between MRW
//                steps); lanes without a packet take pending ones, then new
//                packets; every lane serves its interaction, escape or
//                emission and starts its next flight
//   march phase  all lanes cross cells together; once at most compact_swap
//                lanes still march, the stopped lanes park their packets and
//                take parked marching ones (one batch per trade); the phase
//                ends when no parked marching packet is left and at most
//                march_min_active (at most kStash / 2) lanes still march.
// A trade parks into a free slot before it reads the other packet, so no
// lane holds two packets at once; the bound on the lanes left marching
// keeps the stash within kStash records (at most kStash / 2 parked between
// phases, plus those being traded).  The stash slots of parked marching and
// pending packets are warp-uniform bit masks.
constexpr int kStash = 16;

template <typename R, int NS, int FEAT>
__device__ __forceinline__ void compact_loop(Kernel<R, NS, FEAT>& K, Lane<R, NS>& L, const TransportKP& P,
                                             unsigned char* sm, unsigned long long total_work, int lane)
{
    unsigned long long* claim = reinterpret_cast<unsigned long long*>(sm + P.so_claim) + 2 * (threadIdx.x >> 5);
    if (lane == 0) { claim[0] = 0; claim[1] = 0; }
    uint4* stash = reinterpret_cast<uint4*>(sm + P.so_stash) + (size_t)(threadIdx.x >> 5) * (kStash * 6);
    __syncwarp();
    const unsigned lt = (1u << lane) - 1u;
    const unsigned all = (1u << kStash) - 1u;
    const int t_end = P.march_min_active < kStash / 2 ? P.march_min_active : kStash / 2;
    const int t_swap = P.compact_swap > t_end ? P.compact_swap : t_end;
    unsigned mm = 0u, em = 0u;                  // slots of parked marching / pending packets
    for (;;) {
        // event phase: marching lanes park, then take pending packets
        {
            const unsigned mar = __ballot_sync(FULL, L.st == ST_MARCH);
            if (mar) {
                const unsigned fr = ~(mm | em) & all;
                const unsigned ne = __popc(em);
                int put = -1, get = -1;
                if (L.st == ST_MARCH) {
                    const unsigned r = __popc(mar & lt);
                    put = nth_bit(fr, r);
                    if (r < ne) get = nth_bit(em, r);
                    K.park(L, stash + put * 6);
                    if (get >= 0) K.unpark(L, stash + get * 6);
                    else L.st = ST_NEED;
                }
                mm |= __reduce_or_sync(FULL, put >= 0 ? 1u << put : 0u);
                em &= ~__reduce_or_sync(FULL, get >= 0 ? 1u << get : 0u);
                __syncwarp();
            }
        }
        // lanes without a packet take pending packets, then new ones
        {
            const unsigned fre = __ballot_sync(FULL, L.st == ST_NEED || L.st == ST_DONE);
            if (fre && em) {
                int get = -1;
                if (L.st == ST_NEED || L.st == ST_DONE) {
                    const unsigned r = __popc(fre & lt);
                    if (r < (unsigned)__popc(em)) get = nth_bit(em, r);
                }
                if (get >= 0) K.unpark(L, stash + get * 6);
                em &= ~__reduce_or_sync(FULL, get >= 0 ? 1u << get : 0u);
                __syncwarp();
            }
        }
        refill(K, L, P, claim, total_work, lane);
        // no new packet left: lanes without one take parked marching packets
        {
            const unsigned dn = __ballot_sync(FULL, L.st == ST_DONE);
            if (dn && mm) {
                int get = -1;
                if (L.st == ST_DONE) {
                    const unsigned r = __popc(dn & lt);
                    if (r < (unsigned)__popc(mm)) get = nth_bit(mm, r);
                }
                if (get >= 0) K.unpark(L, stash + get * 6);
                mm &= ~__reduce_or_sync(FULL, get >= 0 ? 1u << get : 0u);
                __syncwarp();
            }
        }
        if (__all_sync(FULL, L.st == ST_DONE) && mm == 0u && em == 0u) break;
        if (L.st == ST_INTERACT) K.interact(L);
        else if (L.st == ST_ESCAPE) K.escape(L);
        if (L.st == ST_FLIGHT) K.flight(L);
        if (L.st == ST_FLIGHT) K.flight(L);     // a second modified-random-walk step
        // march phase
        for (;;) {
            if (L.st == ST_MARCH) K.march(L);
            const unsigned mar = __ballot_sync(FULL, L.st == ST_MARCH);
            const int nm = __popc(mar);
            if (nm > t_swap) continue;
            if (mm) {
                const unsigned fr = ~(mm | em) & all;
                int put = -1, get = -1;
                if (L.st != ST_MARCH) {
                    const unsigned r = __popc(~mar & lt);
                    if (r < (unsigned)__popc(mm)) {
                        get = nth_bit(mm, r);
                        if (L.st != ST_NEED && L.st != ST_DONE) {
                            put = nth_bit(fr, r);
                            K.park(L, stash + put * 6);
                        }
                        K.unpark(L, stash + get * 6);
                    }
                }
                mm &= ~__reduce_or_sync(FULL, get >= 0 ? 1u << get : 0u);
                em |= __reduce_or_sync(FULL, put >= 0 ? 1u << put : 0u);
                __syncwarp();
                continue;
            }
            if (nm > t_end) continue;
            break;
        }
    }
}

// Occupancy target of the FP32 kernel: 4 blocks of 256 threads per SM (64
// registers); four-species variants carry four-wide density and opacity
// state and run at 3 blocks (80 registers), where they spill far less.
#ifndef RT_TRANSPORT_MIN_BLOCKS
#define RT_TRANSPORT_MIN_BLOCKS 4
#endif
template <typename R, int NS, int FEAT>
__global__ void __launch_bounds__(256, sizeof(R) == 8 ? 1 : (NS == 4 ? 3 : RT_TRANSPORT_MIN_BLOCKS))
    transport_kernel(const __grid_constant__ TransportKP P, int serial)
{
    unsigned char* sm = smem_raw();
    {
        float4* s_op = reinterpret_cast<float4*>(sm + P.so_op);
        // species beyond the opacity's (padding of a 3-species float4 grid) get zeros
        for (int i = threadIdx.x; i < NS * P.nf; i += blockDim.x)
            s_op[i] = i < P.ns * P.nf ? P.opac32[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        if ((FEAT & 1) && P.mrw) {
            float* s_mrw = reinterpret_cast<float*>(sm + P.so_mrw);
            for (int i = threadIdx.x; i < kMrwN; i += blockDim.x) s_mrw[i] = P.mrwS[i];
        }
        float* s_cdf = reinterpret_cast<float*>(sm + P.so_cdf);
        for (int i = threadIdx.x; i < P.smem_cdf; i += blockDim.x) s_cdf[i] = P.models[0].src_cdf32[i];
        if (P.smem_sed) {
            double* s_sed = reinterpret_cast<double*>(sm + P.so_sed);
            unsigned* s_cnt = reinterpret_cast<unsigned*>(sm + P.so_cnt);
            for (int i = threadIdx.x; i < kSedBins * P.nf; i += blockDim.x) { s_sed[i] = 0.0; s_cnt[i] = 0u; }
        }
        unsigned long long* s_ctr = reinterpret_cast<unsigned long long*>(sm + P.so_ctr);
        for (int i = threadIdx.x; i < kLaneStats * (int)blockDim.x; i += blockDim.x) s_ctr[i] = 0ull;
    }
    __syncthreads();

    Kernel<R, NS, FEAT> K(P);
    // packets of this launch: emission ids, or the queue filled by the main pass
    unsigned long long total_work = P.total_work;
    if ((FEAT & 16) && P.resume) {
        const unsigned long long q = *P.defer_n;
        total_work = q < P.defer_cap ? q : P.defer_cap;
    }
    Lane<R, NS> L;
    L.st = ST_NEED;
    L.m = -1;
    const int lane = threadIdx.x & 31;

    if (serial) {
        // one thread, packets in id order: the order-dependent B&W temperatures
        // evolve exactly as in a sequential run
        if (blockIdx.x != 0 || threadIdx.x != 0) return;
        for (unsigned long long w = 0; w < total_work; ++w) {
            K.emit(L, w);
            while (L.st != ST_NEED) {
                if (L.st == ST_FLIGHT) K.flight(L);
                else if (L.st == ST_MARCH) K.march(L);
                else if (L.st == ST_INTERACT) K.interact(L);
                else if (L.st == ST_ESCAPE) K.escape(L);
            }
        }
        if (L.m >= 0) K.flush_lane(L.m);
        K.flush_sed(0, 1);
        return;
    }

    const int min_active = P.march_min_active;
    if constexpr ((FEAT & 512) != 0) {
        compact_loop<R, NS, FEAT>(K, L, P, sm, total_work, lane);
        K.flush_warp(0);
        if (P.smem_sed) {
            __syncthreads();
            K.flush_sed(threadIdx.x, blockDim.x);
        }
        return;
    }
    // Packet ids are claimed per warp in chunks (one global atomic per chunk);
    // the chunk shrinks from 256 to 32 ids as the work runs out, which keeps
    // the tail balanced.  The warp's unclaimed range [claim[0], claim[1]) is
    // kept in shared memory, off the registers of the crossing loop; once a
    // range ends at total_work every id has been claimed.
    unsigned long long* claim = reinterpret_cast<unsigned long long*>(sm + P.so_claim) + 2 * (threadIdx.x >> 5);
    if (lane == 0) { claim[0] = 0; claim[1] = 0; }
    __syncwarp();
    for (;;) {
        const unsigned need = __ballot_sync(FULL, L.st == ST_NEED);
        if (need) {
            unsigned long long w_next = claim[0], w_end = claim[1];
            if (w_next == w_end && w_end < total_work) {
                unsigned long long base = 0;
                const unsigned long long n_warps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
                unsigned long long chunk = (total_work - w_end) / (4ull * n_warps);
                chunk = chunk < 32ull ? 32ull : (chunk > 256ull ? 256ull : chunk);
                if (lane == 0) base = atomicAdd(P.work_ctr, chunk);
                base = __shfl_sync(FULL, base, 0);
                if (base >= total_work) {
                    w_next = w_end = total_work;
                } else {
                    w_next = base;
                    w_end = base + chunk < total_work ? base + chunk : total_work;
                }
            }
            const unsigned avail = (unsigned)(w_end - w_next);
            const unsigned rank = __popc(need & ((1u << lane) - 1u));
            if (L.st == ST_NEED) {
                if (rank < avail) K.emit(L, w_next + rank);
                else if (w_end >= total_work) L.st = ST_DONE;
            }
            w_next += __popc(need) < avail ? __popc(need) : avail;
            __syncwarp();
            if (lane == 0) { claim[0] = w_next; claim[1] = w_end; }
            __syncwarp();
        }
        if (__all_sync(FULL, L.st == ST_DONE)) break;
        if (L.st == ST_FLIGHT) {
            K.bind(L);
            K.flight(L);
        }
        int nm;
        do {
            if (L.st == ST_MARCH) {
                K.bind(L);
                K.march(L);
            }
            nm = __popc(__ballot_sync(FULL, L.st == ST_MARCH));
        } while (nm > min_active);
        if (L.st == ST_INTERACT) {
            K.bind(L);
            K.interact(L);
        } else if (L.st == ST_ESCAPE) {
            K.bind(L);
            K.escape(L);
        }
    }
    K.flush_warp(Kernel<R, NS, FEAT>::SINGLE ? 0 : L.m);
    if (P.smem_sed) {
        __syncthreads();
        K.flush_sed(threadIdx.x, blockDim.x);
    }
}

// ------------------------------------------------------------- grid packing
template <typename PT, int NS>
__global__ void pack_kernel(const float* rho, size_t nc, double kext_max, PT* out,
                            int prec, double cube, const unsigned char* leaf_fine, double inv_r,
                            int lucy_mode, double lucy_tau, const double* kext, int nf)
{
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= nc) return;
    // the Lucy criterion is on the cell's own edge (a sub-cube's in refined
    // cubes); the packed density stays rho * cube edge (paths in cube units)
    const double cell = (leaf_fine && leaf_fine[i]) ? cube * inv_r : cube;
    float r[4] = { 0.f, 0.f, 0.f, 0.f };
    double dust = 0.0;
    for (int s = 0; s < NS; ++s) {
        r[s] = rho[s * nc + i];
        dust += r[s];
    }
    bool lucy = false;
    if (dust > 0.0) {
        if (lucy_mode == RT_LUCY_ALL) {
            lucy = true;
        } else if (lucy_mode == RT_LUCY_THIN) {
            double mx = 0.0;
            if constexpr (NS == 1) {
                // one species: rounding is monotonic, so the largest of
                // fl(fl(rho kext_j) cell) over j is the one at the largest kext
                mx = ((double)r[0] * kext_max) * cell;
            } else {
                for (int j = 0; j < nf; ++j) {
                    double chi = 0.0;
                    for (int s = 0; s < NS; ++s) chi += (double)r[s] * kext[s * nf + j];
                    mx = fmax(mx, chi * cell);
                }
            }
            lucy = mx < lucy_tau;
        }
    }
    float v[4];
    for (int s = 0; s < 4; ++s) v[s] = prec == RT_PREC_FP32 ? (float)((double)r[s] * cube) : r[s];
    v[0] = lucy ? -fabsf(v[0]) : fabsf(v[0]);
    if constexpr (NS == 1) out[i] = v[0];
    else if constexpr (NS == 2) out[i] = make_float2(v[0], v[1]);
    else out[i] = make_float4(v[0], v[1], v[2], v[3]);
}

// Packed density of every undivided cube of a refined grid, copied from its
// one cell after the packing (zero for divided cubes, whose sub-cubes are
// read instead): the traversal reads a cube's first cell and density side by
// side, one crossing ahead
template <typename PT>
__global__ void cube_pack_kernel(const int* cube, size_t ncube, const PT* packed, PT* out)
{
    const size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (q >= ncube) return;
    const int info = cube[q];
    out[q] = (info & kCubeDivided) ? PT{} : packed[info];
}

// The FP64 scratch of one model (FP32 build) before a transport: the sum
// starts at E_abs / xi (taken as E_abs * (1 / xi), the same product the
// finalize compares with), so that B&W temperatures read the accumulated
// energy from the scratch alone; the sum of squares (acc_q = 1, interleaved)
// at 0.  xi <= 0 (no luminosity) deposits nothing: the sum starts at 0.
__global__ void seed_kernel(double* acc, int acc_q, size_t n, double inv_xi, const double* E_abs)
{
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    acc[i << acc_q] = inv_xi > 0.0 ? E_abs[i] * inv_xi : 0.0;
    if (acc_q) acc[2 * i + 1] = 0.0;
}

// After a transport (FP32 build), for one model: E_abs = acc * xi where the
// FP64 scratch (seeded with E_abs / xi) received deposits, E_abs += acc * xi
// from the zero-started FP32 scratch of the plain-FP32 form, and
// esq += acc_sq * xi^2; with acc_q = 1 the scratch interleaves the two sums
// per cell.
template <typename A>
__global__ void finalize_kernel(const A* acc, int acc_q, size_t n, double xi, double inv_xi,
                                double* E_abs, double* esq)
{
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double a = (double)acc[i << acc_q];
    if constexpr (sizeof(A) == 8) {
        if (!(inv_xi > 0.0)) return;
        if (a != E_abs[i] * inv_xi) E_abs[i] = a * xi;
    } else {
        if (a != 0.0) E_abs[i] += a * xi;
    }
    if (acc_q && esq) {
        const double q = (double)acc[2 * i + 1];
        if (q != 0.0) esq[i] += q * xi * xi;
    }
}

__global__ void kext_kernel(const double* kabs, const double* ksca, double* kext, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) kext[i] = kabs[i] + ksca[i];
}

template <typename R, int NS, int FEAT>
rt_status launch_one(rt_ctx* ctx, const TransportKP& kp, int schedule, int threads,
                     int blocks_per_sm, cudaStream_t s)
{
    TransportKP k = kp;
    const size_t nsed = kp.smem_sed ? (size_t)kSedBins * kp.nf : 0;
    size_t off = 0;
    auto place = [&](size_t bytes, size_t align) {
        off = (off + align - 1) / align * align;
        const int o = (int)off;
        off += bytes;
        return o;
    };
    k.so_claim = place(16 * (threads / 32 + 1), 16);
    k.so_ctr = place(sizeof(unsigned long long) * kLaneStats * (schedule == RT_SCHED_SERIAL ? 32 : threads), 16);
    k.so_sed = place(sizeof(double) * nsed, 16);
    k.so_op = place(sizeof(float4) * NS * kp.nf, 16);
    k.so_cnt = place(sizeof(unsigned) * nsed, 16);
    k.so_mrw = place((FEAT & 1) && kp.mrw ? sizeof(float) * kMrwN : 0, 16);
    k.so_cdf = place(sizeof(float) * kp.smem_cdf, 16);
    k.so_stash = place((FEAT & 512) ? sizeof(uint4) * 6 * kStash * (threads / 32) : 0, 16);
    const size_t smem = (off + 15) / 16 * 16;
    auto fn = transport_kernel<R, NS, FEAT>;
    RT_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (schedule == RT_SCHED_SERIAL) {
        fn<<<1, 32, smem, s>>>(k, 1);
        count_launches();
    } else {
        int nb = blocks_per_sm;
        if (nb <= 0) {
            RT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem));
            nb = std::max(nb, 1);
        }
        fn<<<ctx->num_sms * nb, threads, smem, s>>>(k, 0);
        count_launches();
    }
    RT_CUDA(cudaGetLastError());
    return RT_OK;
}

// FP32: instantiate only the feature set a launch needs; FP64 debug: all.
// The generic variants (every optional path, photon counting included) are
// FEAT 147 (uniform grid), 179 (+ PAH sources), 211 (+ refinement) and 243
// (both); single-model launches with cameras take 140/141.
template <typename R, int NS>
rt_status launch_feat(rt_ctx* ctx, const TransportKP& kp, int schedule, int threads,
                      int blocks_per_sm, cudaStream_t s)
{
    // refined grids: single-model FP32 launches without trajectories, the
    // deferred queue or cameras take the lean variants
    if (kp.refined) {
        if (kp.pah_src) return launch_one<R, NS, 243>(ctx, kp, schedule, threads, blocks_per_sm, s);
        if constexpr (sizeof(R) == 4) {
            if (kp.single && kp.param_models && !kp.want_traj && !kp.defer_events && !kp.n_pc) {
                if (kp.mrw) return launch_one<R, NS, 77>(ctx, kp, schedule, threads, blocks_per_sm, s);
                return launch_one<R, NS, 76>(ctx, kp, schedule, threads, blocks_per_sm, s);
            }
        }
        return launch_one<R, NS, 211>(ctx, kp, schedule, threads, blocks_per_sm, s);
    }
    if constexpr (sizeof(R) == 8) {
        if (kp.pah_src) return launch_one<R, NS, 179>(ctx, kp, schedule, threads, blocks_per_sm, s);
        return launch_one<R, NS, 147>(ctx, kp, schedule, threads, blocks_per_sm, s);
    } else {
        // PAH re-emission pass: the single-model variant, or the generic one
        if (kp.pah_src) {
            if (!kp.mrw && !kp.want_traj && !kp.defer_events && kp.single && !kp.n_pc)
                return launch_one<R, NS, 44>(ctx, kp, schedule, threads, blocks_per_sm, s);
            return launch_one<R, NS, 179>(ctx, kp, schedule, threads, blocks_per_sm, s);
        }
        if (kp.n_pc) {
            // cameras: the single-model variants with photon counting compiled in
            if (kp.single && kp.param_models && !kp.want_traj && !kp.defer_events) {
                if (kp.mrw) return launch_one<R, NS, 141>(ctx, kp, schedule, threads, blocks_per_sm, s);
                return launch_one<R, NS, 140>(ctx, kp, schedule, threads, blocks_per_sm, s);
            }
            return launch_one<R, NS, 147>(ctx, kp, schedule, threads, blocks_per_sm, s);
        }
        if (kp.acc32) {
            // the plain-FP32 form: single-model uniform-grid launches only
            if (!kp.single || !kp.param_models || kp.want_traj || kp.defer_events)
                return fail(RT_ERR_STATE, "transport: no plain-FP32 variant for this feature set");
            if (kp.mrw) return launch_one<R, NS, 269>(ctx, kp, schedule, threads, blocks_per_sm, s);
            return launch_one<R, NS, 268>(ctx, kp, schedule, threads, blocks_per_sm, s);
        }
        // trajectory logging runs the generic variants; otherwise descriptors
        // come from the parameters when they fit, and one model is constant
        const int feat = (kp.mrw ? 1 : 0) |
                         (kp.want_traj ? 2 : ((kp.param_models ? 4 : 0) | (kp.single ? 8 : 0))) |
                         (kp.defer_events ? 16 : 0);
        if (schedule == RT_SCHED_COMPACT && (feat == 12 || feat == 13)) {
            if (feat == 13) return launch_one<R, NS, 525>(ctx, kp, schedule, threads, blocks_per_sm, s);
            return launch_one<R, NS, 524>(ctx, kp, schedule, threads, blocks_per_sm, s);
        }
        switch (feat) {
        case 0: return launch_one<R, NS, 0>(ctx, kp, schedule, threads, blocks_per_sm, s);
        case 1: return launch_one<R, NS, 1>(ctx, kp, schedule, threads, blocks_per_sm, s);
        case 2: return launch_one<R, NS, 2>(ctx, kp, schedule, threads, blocks_per_sm, s);
        case 3: return launch_one<R, NS, 3>(ctx, kp, schedule, threads, blocks_per_sm, s);
        case 4: return launch_one<R, NS, 4>(ctx, kp, schedule, threads, blocks_per_sm, s);
        case 5: return launch_one<R, NS, 5>(ctx, kp, schedule, threads, blocks_per_sm, s);
        case 12: return launch_one<R, NS, 12>(ctx, kp, schedule, threads, blocks_per_sm, s);
        case 13: return launch_one<R, NS, 13>(ctx, kp, schedule, threads, blocks_per_sm, s);
        case 18: return launch_one<R, NS, 18>(ctx, kp, schedule, threads, blocks_per_sm, s);
        case 19: return launch_one<R, NS, 19>(ctx, kp, schedule, threads, blocks_per_sm, s);
        case 28: return launch_one<R, NS, 28>(ctx, kp, schedule, threads, blocks_per_sm, s);
        case 29: return launch_one<R, NS, 29>(ctx, kp, schedule, threads, blocks_per_sm, s);
        default: return fail(RT_ERR_STATE, "transport: no kernel variant for this feature set");
        }
    }
}

}  // namespace

#ifndef RT_TRANSPORT_NS
// This translation unit: grid packing, finalize and the dispatcher.  The
// transport kernel variants are compiled in transport_ns1/2/4.cu (which
// define RT_TRANSPORT_NS and include this file), one per packed species
// width, so the three compile in parallel.
// largest kabs + ksca of species 0 over the frequency grid (the one-species
// Lucy criterion), summed as the kext kernel sums it
static double kext_max(const rt_opacity* op)
{
    double mx = 0.0;
    for (int j = 0; j < op->nf; ++j) mx = std::max(mx, op->kabs[j] + op->ksca[j]);
    return mx;
}

// cube_pack_kernel over a refined grid's cubes (packed: its packed cells)
static rt_status pack_cubes(const rt_grid* g, const void* packed, void* dst, cudaStream_t s)
{
    const int vec = g->ns == 1 ? 1 : (g->ns == 2 ? 2 : 4);
    const size_t nq = g->ncube();
    const unsigned blocks = (unsigned)((nq + 255) / 256);
    if (vec == 1)
        cube_pack_kernel<float><<<blocks, 256, 0, s>>>(g->d_cube, nq, (const float*)packed, (float*)dst);
    else if (vec == 2)
        cube_pack_kernel<float2><<<blocks, 256, 0, s>>>(g->d_cube, nq, (const float2*)packed, (float2*)dst);
    else
        cube_pack_kernel<float4><<<blocks, 256, 0, s>>>(g->d_cube, nq, (const float4*)packed, (float4*)dst);
    count_launches();
    RT_CUDA(cudaGetLastError());
    return RT_OK;
}

rt_status pack_grid(rt_grid* g, const rt_opacity* op, int lucy_mode, double lucy_tau, int prec,
                    cudaStream_t s)
{
    const int vec = g->ns == 1 ? 1 : (g->ns == 2 ? 2 : 4);
    if (g->d_packed && g->packed_opac_serial == op->serial && g->packed_lucy_mode == lucy_mode &&
        g->packed_lucy_tau == lucy_tau && g->packed_prec == prec)
        return RT_OK;
    const size_t nc = g->ncell();
    if (!g->d_packed) RT_CUDA(cudaMalloc(&g->d_packed, nc * sizeof(float) * vec));
    double* kext = nullptr;
    const int n = op->ns * op->nf;
    RT_CUDA(cudaMallocAsync(&kext, sizeof(double) * n, s));
    kext_kernel<<<(n + 255) / 256, 256, 0, s>>>(op->d_kabs, op->d_ksca, kext, n);
    count_launches(2);   // this one and the packing kernel below
    const int th = 256;
    const unsigned blocks = (unsigned)((nc + th - 1) / th);
    if (vec == 1)
        pack_kernel<float, 1><<<blocks, th, 0, s>>>(g->d_rho, nc, kext_max(op), (float*)g->d_packed, prec,
                                                     g->cell, g->d_leaf_fine, g->refine ? 1.0 / g->refine : 1.0,
                                                     lucy_mode, lucy_tau, kext, op->nf);
    else if (vec == 2)
        pack_kernel<float2, 2><<<blocks, th, 0, s>>>(g->d_rho, nc, kext_max(op), (float2*)g->d_packed,
                                                      prec, g->cell, g->d_leaf_fine, g->refine ? 1.0 / g->refine : 1.0,
                                                     lucy_mode, lucy_tau, kext, op->nf);
    else if (g->ns == 3)
        pack_kernel<float4, 3><<<blocks, th, 0, s>>>(g->d_rho, nc, kext_max(op), (float4*)g->d_packed,
                                                      prec, g->cell, g->d_leaf_fine, g->refine ? 1.0 / g->refine : 1.0,
                                                     lucy_mode, lucy_tau, kext, op->nf);
    else
        pack_kernel<float4, 4><<<blocks, th, 0, s>>>(g->d_rho, nc, kext_max(op), (float4*)g->d_packed,
                                                      prec, g->cell, g->d_leaf_fine, g->refine ? 1.0 / g->refine : 1.0,
                                                     lucy_mode, lucy_tau, kext, op->nf);
    RT_CUDA(cudaGetLastError());
    RT_CUDA(cudaFreeAsync(kext, s));
    if (g->refine) {
        if (!g->d_cube_packed) RT_CUDA(cudaMalloc(&g->d_cube_packed, g->ncube() * sizeof(float) * vec));
        const rt_status st = pack_cubes(g, g->d_packed, g->d_cube_packed, s);
        if (st != RT_OK) return st;
    }
    g->packed_vec = vec;
    g->packed_opac_serial = op->serial;
    g->packed_lucy_mode = lucy_mode;
    g->packed_lucy_tau = lucy_tau;
    g->packed_prec = prec;
    return RT_OK;
}

// 1 / xi for the seed and finalize kernels (0 when xi <= 0: nothing deposited)
static double inv_of(double xi) { return xi > 0.0 ? 1.0 / xi : 0.0; }

rt_status launch_finalize(const double* acc, int acc_q, size_t n, double xi, double* E_abs,
                          double* esq, cudaStream_t s)
{
    if (n == 0) return RT_OK;
    finalize_kernel<double><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(acc, acc_q, n, xi, inv_of(xi),
                                                                       E_abs, esq);
    count_launches();
    RT_CUDA(cudaGetLastError());
    return RT_OK;
}

rt_status launch_seed(double* acc, int acc_q, size_t n, double xi, const double* E_abs,
                      cudaStream_t s)
{
    if (n == 0) return RT_OK;
    seed_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(acc, acc_q, n, inv_of(xi), E_abs);
    count_launches();
    RT_CUDA(cudaGetLastError());
    return RT_OK;
}

rt_status launch_finalize32(const float* acc, int acc_q, size_t n, double xi, double* E_abs,
                            double* esq, cudaStream_t s)
{
    if (n == 0) return RT_OK;
    finalize_kernel<float><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(acc, acc_q, n, xi, inv_of(xi),
                                                                      E_abs, esq);
    count_launches();
    RT_CUDA(cudaGetLastError());
    return RT_OK;
}

// Pack the grid into `dst` (ncell cells of 1, 2 or 4 floats) with the Lucy
// flags of (lucy_mode, lucy_tau), and a refined grid's cube densities into
// `cube_dst` (ncube entries of the same width); `kext` receives ns * nf
// doubles of work space.  Allocates nothing.
rt_status pack_grid_into(const rt_grid* g, const rt_opacity* op, int lucy_mode, double lucy_tau,
                         int prec, double* kext, void* dst, void* cube_dst, cudaStream_t s)
{
    const int vec = g->ns == 1 ? 1 : (g->ns == 2 ? 2 : 4);
    const size_t nc = g->ncell();
    const int n = op->ns * op->nf;
    kext_kernel<<<(n + 255) / 256, 256, 0, s>>>(op->d_kabs, op->d_ksca, kext, n);
    const unsigned blocks = (unsigned)((nc + 255) / 256);
    if (vec == 1)
        pack_kernel<float, 1><<<blocks, 256, 0, s>>>(g->d_rho, nc, kext_max(op), (float*)dst, prec,
                                                      g->cell, g->d_leaf_fine, g->refine ? 1.0 / g->refine : 1.0,
                                                     lucy_mode, lucy_tau, kext, op->nf);
    else if (vec == 2)
        pack_kernel<float2, 2><<<blocks, 256, 0, s>>>(g->d_rho, nc, kext_max(op), (float2*)dst, prec,
                                                       g->cell, g->d_leaf_fine, g->refine ? 1.0 / g->refine : 1.0,
                                                     lucy_mode, lucy_tau, kext, op->nf);
    else if (g->ns == 3)
        pack_kernel<float4, 3><<<blocks, 256, 0, s>>>(g->d_rho, nc, kext_max(op), (float4*)dst, prec,
                                                       g->cell, g->d_leaf_fine, g->refine ? 1.0 / g->refine : 1.0,
                                                     lucy_mode, lucy_tau, kext, op->nf);
    else
        pack_kernel<float4, 4><<<blocks, 256, 0, s>>>(g->d_rho, nc, kext_max(op), (float4*)dst, prec,
                                                       g->cell, g->d_leaf_fine, g->refine ? 1.0 / g->refine : 1.0,
                                                     lucy_mode, lucy_tau, kext, op->nf);
    count_launches(2);
    RT_CUDA(cudaGetLastError());
    if (g->refine) return pack_cubes(g, dst, cube_dst, s);
    return RT_OK;
}

rt_status launch_transport(rt_ctx* ctx, const rt_opacity* op, const TransportKP& kp, int ns,
                           int prec, int schedule, int threads, int blocks_per_sm, cudaStream_t s)
{
    (void)op;
    const int vec = ns == 1 ? 1 : (ns == 2 ? 2 : 4);
    if (vec == 1) return launch_transport_ns<1>(ctx, kp, prec, schedule, threads, blocks_per_sm, s);
    if (vec == 2) return launch_transport_ns<2>(ctx, kp, prec, schedule, threads, blocks_per_sm, s);
    return launch_transport_ns<4>(ctx, kp, prec, schedule, threads, blocks_per_sm, s);
}
#else
template <>
rt_status launch_transport_ns<RT_TRANSPORT_NS>(rt_ctx* ctx, const TransportKP& kp, int prec, int schedule,
                                                int threads, int blocks_per_sm, cudaStream_t s)
{
    if (prec == RT_PREC_FP64)
        return launch_feat<double, RT_TRANSPORT_NS>(ctx, kp, schedule, threads, blocks_per_sm, s);
    return launch_feat<float, RT_TRANSPORT_NS>(ctx, kp, schedule, threads, blocks_per_sm, s);
}
#endif

}  // namespace rtgb
