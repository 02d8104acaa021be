// Memory-level probe for the roofline of the gather-bound kernels: random
// 32-byte sector reads from a device buffer, the access pattern of the
// transport's per-crossing density loads (one word of one sector, at an
// unpredictable cell) and of the ray march's emissivity rows.  Timed by the
// caller with CUDA events, it gives the sector rate that the memory level
// holding the buffer serves: L2 for a buffer well inside the L2, HBM for one
// far larger than it.
#include "rt_internal.cuh"

namespace rtgb {
namespace {

// Each thread walks its own linear-congruential sequence of sector indices
// (independent of the data read, so every read can be in flight at once) and
// folds the words it reads into a checksum that is written only if it takes
// an impossible value, which keeps the reads live.
__global__ void __launch_bounds__(256) gather_probe_kernel(const unsigned* buf, uint64_t n_sectors,
                                                           uint64_t per_thread, uint32_t seed,
                                                           unsigned long long* sink)
{
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    uint32_t h = (uint32_t)tid * 0x9E3779B9u ^ seed;
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    unsigned acc = 0u;
    // four reads per iteration, each at its own sector: independent loads in
    // flight per thread (the transport has one per lane plus the prefetch)
    uint64_t k = 0;
    for (; k + 4 <= per_thread; k += 4) {
        unsigned v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            h = h * 1664525u + 1013904223u;
            const uint64_t sct = ((uint64_t)h * n_sectors) >> 32;
            v[q] = __ldg(buf + 8 * sct + (h >> 29));
        }
        acc += (v[0] ^ v[1]) + (v[2] ^ v[3]);
    }
    for (; k < per_thread; ++k) {
        h = h * 1664525u + 1013904223u;
        const uint64_t sct = ((uint64_t)h * n_sectors) >> 32;
        acc += __ldg(buf + 8 * sct + (h >> 29));
    }
    if (acc == 0x9E3779B9u && sink) atomicAdd(sink, 1ull);
}

}  // namespace

rt_status launch_gather_probe(int num_sms, const void* buf, size_t bytes, uint64_t n_reads, uint32_t seed,
                              unsigned long long* sink, cudaStream_t s)
{
    const uint64_t n_sectors = bytes / 32;
    const unsigned blocks = (unsigned)num_sms * 8u;
    const uint64_t threads = (uint64_t)blocks * 256u;
    const uint64_t per = (n_reads + threads - 1) / threads;
    if (per == 0 || n_sectors == 0) return RT_OK;
    gather_probe_kernel<<<blocks, 256, 0, s>>>((const unsigned*)buf, n_sectors, per, seed, sink);
    count_launches();
    RT_CUDA(cudaGetLastError());
    return RT_OK;
}

}  // namespace rtgb
