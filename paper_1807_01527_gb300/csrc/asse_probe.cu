// Measurement aid (no counterpart in the paper): the rate at which the GPU
// serves independent random 4-byte reads from a buffer the size of a pool,
// one 32-byte sector each.  The ingest's pool traffic is of this kind (r
// random words per pair new to the slice), so this rate, timed by the caller
// around asse_probe_random_reads, is the random-access roofline the ingest is
// compared with beside the streaming HBM bandwidth.
#include <cuda_runtime.h>

#include <cstdint>

#include "asse_internal.h"

namespace asse {

namespace {

// XOR of everything read, so the loads cannot be dropped.
__device__ unsigned long long g_probe_sink;

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_UNROLL = 8;  // independent loads in flight per thread

__global__ void __launch_bounds__(PROBE_THREADS) random_read_kernel(const uint32_t *__restrict__ buf,
                                                                    uint64_t n_words, uint64_t rounds)
{
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t x = (tid + 1) * 0x9E3779B97F4A7C15ull;
    uint32_t acc = 0;
    for (uint64_t i = 0; i < rounds; i++) {
        uint32_t v[PROBE_UNROLL];
#pragma unroll
        for (int j = 0; j < PROBE_UNROLL; j++) {
            // xorshift64 step, then a word index in [0, n_words) by multiply-high
            x ^= x << 13;
            x ^= x >> 7;
            x ^= x << 17;
            v[j] = __ldcg(buf + __umul64hi(x, n_words));
        }
#pragma unroll
        for (int j = 0; j < PROBE_UNROLL; j++)
            acc ^= v[j];
    }
    for (int off = 16; off > 0; off >>= 1)
        acc ^= __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0)
        atomicXor(&g_probe_sink, (unsigned long long)acc);
}

}  // namespace

cudaError_t launch_random_reads(const uint32_t *buf, uint64_t n_words, uint64_t n_reads, int sms, cudaStream_t s,
                                uint64_t *launches, uint64_t *issued)
{
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, random_read_kernel, PROBE_THREADS, 0);
    if (e != cudaSuccess)
        return e;
    const uint64_t threads = (uint64_t)sms * (occ > 0 ? occ : 1) * PROBE_THREADS;
    const uint64_t rounds = (n_reads + threads * PROBE_UNROLL - 1) / (threads * PROBE_UNROLL);
    *issued = rounds * threads * PROBE_UNROLL;
    *launches += 1;
    random_read_kernel<<<(unsigned)(threads / PROBE_THREADS), PROBE_THREADS, 0, s>>>(buf, n_words, rounds);
    return cudaGetLastError();
}

}  // namespace asse
