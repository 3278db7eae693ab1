// Feature rows of ATV states for the learned estimator (include/asse_learn.h):
// the per-warp device function shared by the pool's feature kernel
// (asse_features.cu) and the synthetic training states (asse_learn.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/asse_learn.h"
#include "asse_device.cuh"
#include "asse_swar.cuh"

namespace asse {

// Feature row of one ATV from its packed words, computed by one warp: active
// ATs per age (Algorithm 1 for the latest kp slices) and their total, then
// the three load features.  A word's active fields come from the SWAR range
// test with the window's per-position ranges (desc); only those fields are
// visited, their age taken from the ACT of their block (actw: the ACTs of a
// word's fields packed like the word).  Each lane counts ages in its own
// column of hist ([64][32] 16-bit counters, zero on entry and left zero), so
// the histogram needs no atomics; the lanes then add up one age row each,
// reading the row rotated by the age so that no two lanes hit one bank.
constexpr uint32_t HIST_WORDS = 64 * 32 / 2;  // [64][32] 16-bit counters (a lane counts at most g/32 <= 128)

constexpr int FEAT_MAXM = 16;  // words per lane: an ATV has at most 512 words

// The words q = lane + 32 m (m < M) of one ATV, 0 past the used ones.
template <int WB, int M = FEAT_MAXM>
__device__ __forceinline__ void load_atv_words(const Params &P, const uint32_t *words, uint32_t lane, uint32_t *w)
{
    constexpr uint32_t F = 32 / WB;
    const uint32_t nw = (P.g + F - 1) / F;
#pragma unroll
    for (int m = 0; m < M; m++) {
        const uint32_t q = lane + 32u * m;
        w[m] = q < nw ? words[q] : 0u;
    }
}

// Per-position tables of the window ending at the slice whose block 0 has ACT
// c0: desc[q] the count ranges of word q, actw[q] the ACT of each of its
// fields (AT counters; unused for aging counters).  All threads of the block.
template <int WB>
__device__ void feature_tables(const Params &P, uint32_t c0, uint32_t kp, RangeDesc *desc, uint32_t *actw)
{
    constexpr uint32_t F = 32 / WB;
    for (uint32_t q = threadIdx.x; q < P.Wd; q += blockDim.x) {
        desc[q] = count_desc<WB>(P, q, c0, kp);
        uint32_t a = 0;
        for (uint32_t j = 0; j < F; j++) {
            const uint32_t h = q * F + j;
            if (h < P.g)
                a |= act_of(P, c0, pos_block(P, h)) << (j * WB);
        }
        actw[q] = a;
    }
}

template <int WB, int M = FEAT_MAXM>
__device__ void atv_features(const Params &P, const uint32_t *wreg, const RangeDesc *desc, const uint32_t *actw,
                             uint32_t kp, float lp, float lup, float lmean, uint16_t *hist, __nv_bfloat16 *row,
                             uint32_t lane, uint32_t *cnt_out)
{
    constexpr uint32_t F = 32 / WB;
    constexpr uint32_t FM = (1u << WB) - 1;
    uint32_t cnt = 0;
    const uint32_t nw = (P.g + F - 1) / F;
#pragma unroll
    for (int m = 0; m < M; m++) {
        const uint32_t q = lane + 32u * m;
        if (32u * m >= nw)
            break;
        if (q >= nw)
            continue;
        const uint32_t w = wreg[m];
        uint32_t am = field_bits<WB>(w, desc[q]);
        if (am == 0)
            continue;
        cnt += __popc(am);
        const uint32_t acts = actw[q];
        do {
            const uint32_t j = __ffs(am) - 1;
            am &= am - 1;
            const uint32_t v = (w >> (j * WB)) & FM;
            uint32_t age;
            if (P.ace) {
                age = P.k - v;  // a counter visited age slices ago holds k - age
            } else {
                age = ((acts >> (j * WB)) & FM) + P.k2 - v;  // (ACT of the AT's block - v) mod 2k
                age = age >= P.k2 ? age - P.k2 : age;
            }
            hist[age * 32 + lane] += 1;
        } while (am);
    }
    cnt = __reduce_add_sync(FULL_MASK, cnt);
    __syncwarp();
    uint32_t bins[2] = {0, 0};
#pragma unroll
    for (uint32_t t = 0; t < 2; t++) {
        const uint32_t e = lane + 32 * t;
        if (e < kp) {
            uint16_t *hr = hist + e * 32;
            uint32_t acc = 0;
            for (uint32_t j = 0; j < 32; j++) {
                const uint32_t c = (j + e) & 31;
                acc += hr[c];
                hr[c] = 0;
            }
            bins[t] = acc;
        }
    }
    const float inv_g = 1.0f / (float)P.g;
#pragma unroll
    for (uint32_t m = 0; m < (ASSE_FEAT + 31) / 32; m++) {
        const uint32_t e = lane + 32 * m;
        // age e - 1 is held by lane (e - 1) mod 32, in bins[(e - 1) / 32]
        const uint32_t src = (e + 31) & 31;
        const uint32_t b0 = __shfl_sync(FULL_MASK, bins[0], src);
        const uint32_t b1 = __shfl_sync(FULL_MASK, bins[1], src);
        if (e >= ASSE_FEAT)
            continue;
        float v = 0.0f;
        if (e == 0)
            v = (float)cnt * inv_g;
        else if (e <= 64)
            v = (float)(e - 1 < 32 ? b0 : b1) * inv_g;
        else if (e == 65)
            v = lp;
        else if (e == 66)
            v = lup;
        else if (e == 67)
            v = lmean;
        row[e] = __float2bfloat16_rn(v);
    }
    if (cnt_out)
        *cnt_out = cnt;
    __syncwarp();
}

}  // namespace asse
