// Feature rows of every ATV of a pool (asse_features, include/asse_learn.h).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/asse_learn.h"
#include "asse_features.cuh"

namespace asse {

namespace {

using bf16 = __nv_bfloat16;
constexpr int FEAT = ASSE_FEAT;

constexpr int FEAT_WARPS = 8;

// M: words per lane, the smallest of 4, 8, 16 that holds the ATV.
// ctl non-null: C0 of the open slice comes from the device slice state (a
// captured graph replays the launch slice after slice).
template <int WB, int M>
__global__ void __launch_bounds__(FEAT_WARPS * 32) features_kernel(Params P, const uint32_t *pool, uint32_t c0,
                                                                   const SliceCtl *ctl, uint32_t kp,
                                                                   const unsigned long long *aat, bf16 *x,
                                                                   uint32_t total_atv)
{
    extern __shared__ uint32_t fsm[];
    if (ctl)
        c0 = ctl->c0;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint16_t *hist = reinterpret_cast<uint16_t *>(fsm + warp * HIST_WORDS);
    // load features of every (row, frame), then UP and mean P of every frame,
    // once per block (FP64, then stored as FP32)
    RangeDesc *desc = reinterpret_cast<RangeDesc *>(fsm + FEAT_WARPS * HIST_WORDS);  // [Wd]
    uint32_t *actw = reinterpret_cast<uint32_t *>(desc + P.Wd);                       // [Wd]
    float *ltab = reinterpret_cast<float *>(actw + P.Wd);                             // [(r + 2) nf]
    feature_tables<WB>(P, c0, kp, desc, actw);
    const double denom = (double)P.g * (double)(P.cmask + 1);
    for (uint32_t frame = threadIdx.x; frame < P.nf; frame += blockDim.x) {
        double up = 1.0, sum = 0.0;
        for (uint32_t i = 0; i < P.r; i++) {
            const double pi = (double)aat[(size_t)i * P.nf + frame] / denom;
            up *= pi;
            sum += pi;
            ltab[i * P.nf + frame] = (float)pi;
        }
        ltab[P.r * P.nf + frame] = (float)up;
        ltab[(P.r + 1) * P.nf + frame] = (float)(sum / P.r);
    }
    for (uint32_t i = lane; i < HIST_WORDS; i += 32)
        fsm[warp * HIST_WORDS + i] = 0;
    __syncthreads();
    // all of an ATV's words are loaded at once (one memory latency per ATV)
    for (uint32_t atv = blockIdx.x * FEAT_WARPS + warp; atv < total_atv; atv += gridDim.x * FEAT_WARPS) {
        uint32_t wreg[M];
        load_atv_words<WB, M>(P, pool + (size_t)atv * P.Wd, lane, wreg);
        const uint32_t row = atv >> P.E_log2, frame = (atv & ((1u << P.E_log2) - 1)) >> P.c;
        atv_features<WB, M>(P, wreg, desc, actw, kp, ltab[row * P.nf + frame], ltab[P.r * P.nf + frame],
                            ltab[(P.r + 1) * P.nf + frame], hist, x + (size_t)atv * FEAT, lane, nullptr);
    }
}

// BF16 bits of v (round to nearest even).
__device__ __forceinline__ uint32_t bf16_bits(float v)
{
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v));
}

// Feature rows of a pool with slice counts (ASSE_COUNTER_AT_HIST): the
// active ATs of age a are the count of the slice a slices back, phase c0 - a
// (mod 2k), so a row needs the k' counts of its ATV (2 bytes each, 64
// contiguous bytes per warp and phase) instead of its words.  A thread builds
// the row of one ATV in registers and writes it as ten 16-byte stores (VEC,
// x 16-byte aligned) or 80 2-byte stores; the L2 merges the rows' sectors
// (staging a warp's rows in shared memory for fully coalesced stores took
// longer: 0.205 against 0.153 ms for the long pool, fewer resident warps).
// The values are the ones the word kernel computes: count / g and the three
// loads, rounded to BF16.
template <bool VEC>
__global__ void __launch_bounds__(256) hist_features_kernel(Params P, uint32_t c0, const SliceCtl *ctl, uint32_t kp,
                                                            const unsigned long long *aat, bf16 *x,
                                                            uint32_t total_atv)
{
    extern __shared__ uint32_t fsm[];
    if (ctl)
        c0 = ctl->c0;
    float *ltab = reinterpret_cast<float *>(fsm);  // [(r + 2) nf]
    const double denom = (double)P.g * (double)(P.cmask + 1);
    for (uint32_t frame = threadIdx.x; frame < P.nf; frame += blockDim.x) {
        double up = 1.0, sum = 0.0;
        for (uint32_t i = 0; i < P.r; i++) {
            const double pi = (double)aat[(size_t)i * P.nf + frame] / denom;
            up *= pi;
            sum += pi;
            ltab[i * P.nf + frame] = (float)pi;
        }
        ltab[P.r * P.nf + frame] = (float)up;
        ltab[(P.r + 1) * P.nf + frame] = (float)(sum / P.r);
    }
    __syncthreads();
    const float inv_g = 1.0f / (float)P.g;
    for (uint32_t atv = blockIdx.x * blockDim.x + threadIdx.x; atv < total_atv; atv += gridDim.x * blockDim.x) {
        uint32_t pk[FEAT / 2];  // element e in bits 16 (e & 1) of pk[e / 2]
#pragma unroll
        for (int j = 0; j < FEAT / 2; j++)
            pk[j] = 0;
        uint32_t cnt = 0, ph = c0;
#pragma unroll
        for (int a = 0; a < 64; a++) {
            if ((uint32_t)a < kp) {
                const uint32_t c = P.hist[(uint64_t)ph * total_atv + atv];
                cnt += c;
                pk[(1 + a) >> 1] |= bf16_bits((float)c * inv_g) << (16 * ((1 + a) & 1));
                ph = ph == 0 ? P.k2 - 1 : ph - 1;
            }
        }
        const uint32_t row = atv >> P.E_log2, frame = (atv & ((1u << P.E_log2) - 1)) >> P.c;
        pk[0] |= bf16_bits((float)cnt * inv_g);
        pk[32] |= bf16_bits(ltab[row * P.nf + frame]) << 16;                                   // 65: P
        pk[33] = bf16_bits(ltab[P.r * P.nf + frame]) | (bf16_bits(ltab[(P.r + 1) * P.nf + frame]) << 16);  // 66, 67
        bf16 *dst = x + (size_t)atv * FEAT;
        if constexpr (VEC) {
            uint4 *d4 = reinterpret_cast<uint4 *>(dst);
#pragma unroll
            for (int j = 0; j < FEAT / 8; j++)
                d4[j] = make_uint4(pk[4 * j], pk[4 * j + 1], pk[4 * j + 2], pk[4 * j + 3]);
        } else {
            uint16_t *d = reinterpret_cast<uint16_t *>(dst);
#pragma unroll
            for (int e = 0; e < FEAT; e++)
                d[e] = (uint16_t)(pk[e >> 1] >> (16 * (e & 1)));
        }
    }
}

}  // namespace

}  // namespace asse

using namespace asse;

namespace asse {

cudaError_t launch_features(const FeatureView &v, uint16_t *x_dev)
{
    const uint32_t total = v.P.r << v.P.E_log2;
    if (v.P.hist != nullptr && v.kp <= 64) {
        // slice counts: the rows from the counts, not from the words
        const size_t smem = (size_t)(v.P.r + 2) * v.P.nf * sizeof(float);
        const bool vec = ((uintptr_t)x_dev & 15) == 0;
        auto kern = vec ? hist_features_kernel<true> : hist_features_kernel<false>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        const uint64_t want = (total + 255) / 256;
        const uint64_t full = (uint64_t)v.sms * resident_blocks(kern, 256, smem);
        kern<<<(unsigned)(want < full ? want : full), 256, smem, v.stream>>>(
            v.P, v.c0, v.ctl, v.kp, v.aat, reinterpret_cast<bf16 *>(x_dev), total);
        *v.launches += 1;
        return cudaGetLastError();
    }
    cudaError_t e = dispatch_w(v.w, [&](auto wb) {
        constexpr int WB = decltype(wb)::value;
        const size_t smem = ((size_t)FEAT_WARPS * HIST_WORDS + (size_t)(v.P.r + 2) * v.P.nf) * sizeof(uint32_t) +
                            (size_t)v.P.Wd * (sizeof(RangeDesc) + sizeof(uint32_t));
        constexpr uint32_t F = 32 / WB;
        const uint32_t per_lane = ((v.P.g + F - 1) / F + 31) / 32;
        auto kern = per_lane <= 4 ? features_kernel<WB, 4> : (per_lane <= 8 ? features_kernel<WB, 8>
                                                                           : features_kernel<WB, 16>);
        cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e2 != cudaSuccess)
            return e2;
        const unsigned grid = (unsigned)v.sms * 4;
        kern<<<grid, FEAT_WARPS * 32, smem, v.stream>>>(v.P, v.pool, v.c0, v.ctl, v.kp, v.aat,
                                                       reinterpret_cast<bf16 *>(x_dev), total);
        return cudaGetLastError();
    });
    *v.launches += 1;
    return e;
}

}  // namespace asse

extern "C" {

int asse_features(asse_pool *pool, uint16_t *x_dev)
{
    if (!pool || !x_dev)
        return pool ? pool_fail(pool, ASSE_EINVAL, "x_dev is NULL") : ASSE_EINVAL;
    FeatureView v;
    if (int rc = pool_feature_view(pool, &v))
        return rc;
    if (v.kp > 64)
        return pool_fail(pool, ASSE_EINVAL, "features need k' <= 64");
    const cudaError_t e = launch_features(v, x_dev);
    if (e != cudaSuccess)
        return pool_fail(pool, ASSE_ECUDA, std::string("features launch: ") + cudaGetErrorString(e));
    return ASSE_OK;
}

}  // extern "C"
