// Measurement aid (no counterpart in the paper): the rate at which the GPU
// serves independent random 4-byte reads from a buffer the size of a pool,
// one 32-byte sector each.  The ingest's pool traffic is of this kind (r
// random words per pair new to the slice), so this rate, timed by the caller
// around asse_probe_random_reads, is the random-access roofline the ingest is
// compared with beside the streaming HBM bandwidth.
//
// Also a self-test of the bounded device waits (asse_probe_bounded_wait): the
// mbarrier try-wait loop with a clock bound, run on a barrier that may never
// complete, so the give-up path and its ASSE_ETIMEOUT status can be exercised
// without hanging the GPU.
#include <cuda_runtime.h>

#include <cstdint>

#include "asse_internal.h"
#include "asse_ptx.cuh"

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

// Result of the bounded-wait self-test: [0] 1 if the wait completed, 2 if it
// gave up; [1] the cycles it took.
__device__ unsigned long long g_wait_result[2];

// One thread: an mbarrier expecting one arrival, which this thread makes
// first only when `complete` is set; then the same try-wait loop with a
// clock bound that the staging and tensor-core kernels use, here with the
// caller's bound.
__global__ void bounded_wait_kernel(long long limit, int complete)
{
    __shared__ __align__(8) uint64_t bar;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (complete)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&bar)) : "memory");
    const long long t0 = clock64();
    bool done = false;
    for (;;) {
        if (mbar_try_wait(&bar, 0)) {
            done = true;
            break;
        }
        if (clock64() - t0 > limit)
            break;
    }
    g_wait_result[0] = done ? 1ull : 2ull;
    g_wait_result[1] = (unsigned long long)(clock64() - t0);
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

extern "C" int asse_probe_bounded_wait(void *stream, uint64_t limit_cycles, int complete, uint64_t *cycles_waited)
{
    using namespace asse;
    if (limit_cycles < 1 || limit_cycles > (1ull << 36))
        return ASSE_EINVAL;
    const cudaStream_t s = (cudaStream_t)stream;
    unsigned long long res[2] = {0, 0};
    if (cudaMemcpyToSymbolAsync(g_wait_result, res, sizeof res, 0, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return ASSE_ECUDA;
    bounded_wait_kernel<<<1, 1, 0, s>>>((long long)limit_cycles, complete);
    if (cudaGetLastError() != cudaSuccess)
        return ASSE_ECUDA;
    if (cudaMemcpyFromSymbolAsync(res, g_wait_result, sizeof res, 0, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess || res[0] == 0)
        return ASSE_ECUDA;
    if (cycles_waited)
        *cycles_waited = res[1];
    return res[0] == 2 ? ASSE_ETIMEOUT : ASSE_OK;
}
