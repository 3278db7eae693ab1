// K1: Algorithm 3 (Scan IP pair, Sec. 4.1) over a batch of (aip, bip) pairs.
//
// One thread takes two pairs per 128-bit streaming load (evict-first, so the
// pair stream does not push the pool out of L2), computes f(aip), the frame,
// the r column indices, BH(bip) and the ACT of that AT in registers, issues
// the r word loads together, then sets the r fields.  A field that already
// holds the slice's value costs one (usually cached) load and no atomic.
#include <cuda_runtime.h>

#include <cstdint>

#include "asse_device.cuh"

namespace asse {

namespace {

template <int WB>
__device__ __forceinline__ void prep_pair(const Params &P, uint32_t c0, uint32_t aip, uint32_t bip, uint64_t &LL,
                                          uint32_t &z, uint32_t &q, uint32_t &sh, uint32_t &val)
{
    constexpr uint32_t F = 32 / WB;
    const uint32_t f = mangle(P.A, aip);
    z = f & (P.nf - 1);
    LL = lbs_twice(P, f);
    const uint32_t h = bip_hash(P, bip);
    q = h / F;
    sh = (h - q * F) * WB;
    val = P.ace ? P.k : act_of(P, c0, act_block(P, h));
}

// SetAT on one packed field; old is a possibly stale read of the word.
// Within a slice every writer of a field writes the same value, so the bits
// outside that value are only ever cleared and the bits inside it only ever
// set.  Clearing what the read still shows and setting what it lacks
// therefore always ends at the value, in any interleaving.
__device__ __forceinline__ void set_field(uint32_t *addr, uint32_t old, uint32_t sh, uint32_t val, uint32_t fm)
{
    const uint32_t f = (old >> sh) & fm;
    if (f != val) {
        const uint32_t clr = (f & ~val) << sh;
        const uint32_t set = (val & ~f) << sh;
        if (clr)
            atomicAnd(addr, ~clr);
        if (set)
            atomicOr(addr, set);
    }
}

__device__ __forceinline__ uint32_t *field_word(const Params &P, uint32_t *pool, int i, uint32_t z, uint64_t LL,
                                                uint32_t q)
{
    return pool + (((uint64_t)i << P.E_log2) + ((z << P.c) | column(P, LL, i))) * P.Wd + q;
}

template <int WB, int R>
__global__ void __launch_bounds__(256) ingest_kernel(Params P, uint32_t *pool, const uint4 *__restrict__ pairs,
                                                     uint64_t nvec, const uint2 *__restrict__ tail, uint32_t c0)
{
    constexpr uint32_t FM = (1u << WB) - 1;
    constexpr int RM = R ? R : 8;
    const int r = R ? R : (int)P.r;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (uint64_t v = tid; v < nvec; v += stride) {
        const uint4 pr = __ldcs(pairs + v);
        uint64_t LL0, LL1;
        uint32_t z0, z1, q0, q1, sh0, sh1, val0, val1;
        prep_pair<WB>(P, c0, pr.x, pr.y, LL0, z0, q0, sh0, val0);
        prep_pair<WB>(P, c0, pr.z, pr.w, LL1, z1, q1, sh1, val1);
        uint32_t *a0[RM], *a1[RM];
        uint32_t o0[RM], o1[RM];
#pragma unroll
        for (int i = 0; i < RM; i++) {
            if (i < r) {
                a0[i] = field_word(P, pool, i, z0, LL0, q0);
                a1[i] = field_word(P, pool, i, z1, LL1, q1);
            }
        }
#pragma unroll
        for (int i = 0; i < RM; i++) {
            if (i < r) {
                o0[i] = *a0[i];
                o1[i] = *a1[i];
            }
        }
#pragma unroll
        for (int i = 0; i < RM; i++) {
            if (i < r) {
                set_field(a0[i], o0[i], sh0, val0, FM);
                set_field(a1[i], o1[i], sh1, val1, FM);
            }
        }
    }
    if (tail != nullptr && tid == 0) {
        const uint2 pr = *tail;
        uint64_t LL;
        uint32_t z, q, sh, val;
        prep_pair<WB>(P, c0, pr.x, pr.y, LL, z, q, sh, val);
        for (int i = 0; i < r; i++) {
            uint32_t *a = field_word(P, pool, i, z, LL, q);
            set_field(a, *a, sh, val, FM);
        }
    }
}

}  // namespace

cudaError_t launch_ingest(const Params &P, uint32_t w, uint32_t *pool, const uint32_t *pairs, uint64_t n, uint32_t c0,
                          int sms, cudaStream_t s, uint64_t *launches)
{
    if (n == 0)
        return cudaSuccess;
    const uint64_t nvec = n / 2;
    const uint2 *tail = (n & 1) ? reinterpret_cast<const uint2 *>(pairs + 2 * (n - 1)) : nullptr;
    const uint4 *p4 = reinterpret_cast<const uint4 *>(pairs);
    *launches += 1;
    return dispatch_w(w, [&](auto wb) {
        constexpr int WB = decltype(wb)::value;
        auto kern = P.r == 4 ? ingest_kernel<WB, 4> : ingest_kernel<WB, 0>;
        static int per_sm[2] = {0, 0};
        int &occ = per_sm[P.r == 4 ? 0 : 1];
        if (occ == 0)
            occ = resident_blocks(kern, 256, 0);
        const uint64_t want = (nvec + 255) / 256;
        const uint64_t full = (uint64_t)sms * occ;
        const unsigned grid = (unsigned)(want < 1 ? 1 : (want < full ? want : full));
        kern<<<grid, 256, 0, s>>>(P, pool, p4, nvec, tail, c0);
        return cudaGetLastError();
    });
}

}  // namespace asse
