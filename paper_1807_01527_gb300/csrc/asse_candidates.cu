// Feature rows of candidate super points, the input of a learned replacement
// of Eq. 4 (include/asse_learn.h): for a host, the ATs active in all r ATVs
// of RRH(host) (Algorithm 5's NAT) binned by the age of their oldest
// timestamp, its frame's row loads and its ATVs' active counts.  The same
// per-warp device function serves the rows of a pool's hosts and the rows of
// the synthetic candidate states the model is trained on.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>

#include "../../include/asse_learn.h"
#include "asse_device.cuh"
#include "asse_features.cuh"
#include "asse_synth.cuh"

namespace asse {

namespace {

using bf16 = __nv_bfloat16;
constexpr int FEAT = ASSE_FEAT;
constexpr int CAND_WARPS = 8;
constexpr uint32_t MAX_ROWS = 8;

// The feature row of one host, computed by one warp from the words of its r
// ATVs (atv[i]: the Wd words of row i's ATV), the window's per-position count
// ranges (desc) and packed ACTs (actw), and its frame's row loads.  Bins:
// an AT active in every row adds one to the bin of its largest age over the
// rows.  Each lane counts in its own column of hist ([64][32] 16-bit, zero
// on entry and left zero).  *nat_out (lane 0) receives NAT.
template <int WB>
__device__ void candidate_row(const Params &P, const uint32_t *const *atv, const RangeDesc *desc, const uint32_t *actw,
                              uint32_t kp, const double *loads, uint16_t *hist, bf16 *row, uint32_t lane,
                              uint32_t *nat_out)
{
    constexpr uint32_t F = 32 / WB;
    constexpr uint32_t FM = (1u << WB) - 1;
    const uint32_t nw = (P.g + F - 1) / F;
    uint32_t cnt[MAX_ROWS];
#pragma unroll
    for (uint32_t i = 0; i < MAX_ROWS; i++)
        cnt[i] = 0;
    uint32_t nat = 0;
    for (uint32_t q = lane; q < nw; q += 32) {
        uint32_t w[MAX_ROWS];
        uint32_t all = ~0u;
#pragma unroll
        for (uint32_t i = 0; i < MAX_ROWS; i++) {
            if (i < P.r) {
                w[i] = atv[i][q];
                const uint32_t am = field_bits<WB>(w[i], desc[q]);  // fields past g never count
                cnt[i] += __popc(am);
                all &= am;
            } else {
                w[i] = 0;
            }
        }
        nat += __popc(all);
        const uint32_t acts = actw[q];
        while (all) {
            const uint32_t j = __ffs(all) - 1;
            all &= all - 1;
            uint32_t oldest = 0;
#pragma unroll
            for (uint32_t i = 0; i < MAX_ROWS; i++) {
                if (i < P.r) {
                    const uint32_t v = (w[i] >> (j * WB)) & FM;
                    uint32_t age;
                    if (P.ace) {
                        age = P.k - v;
                    } else {
                        age = ((acts >> (j * WB)) & FM) + P.k2 - v;  // (ACT - v) mod 2k
                        age = age >= P.k2 ? age - P.k2 : age;
                    }
                    oldest = age > oldest ? age : oldest;
                }
            }
            hist[oldest * 32 + lane] += 1;
        }
    }
    nat = __reduce_add_sync(FULL_MASK, nat);
#pragma unroll
    for (uint32_t i = 0; i < MAX_ROWS; i++)
        cnt[i] = __reduce_add_sync(FULL_MASK, cnt[i]);
    __syncwarp();
    uint32_t bins[2] = {0, 0};
#pragma unroll
    for (uint32_t t = 0; t < 2; t++) {
        const uint32_t e = lane + 32 * t;
        if (e < kp) {
            uint16_t *hr = hist + e * 32;
            uint32_t acc = 0;
            for (uint32_t j = 0; j < 32; j++) {
                const uint32_t c = (j + e) & 31;  // rotated: no two lanes in one bank
                acc += hr[c];
                hr[c] = 0;
            }
            bins[t] = acc;
        }
    }
    double up = 1.0, lmin = loads[0], lmax = loads[0];
    for (uint32_t i = 0; i < P.r; i++) {
        up *= loads[i];
        lmin = fmin(lmin, loads[i]);
        lmax = fmax(lmax, loads[i]);
    }
    const float inv_g = 1.0f / (float)P.g;
#pragma unroll
    for (uint32_t m = 0; m < (FEAT + 31) / 32; m++) {
        const uint32_t e = lane + 32 * m;
        const uint32_t src = (e + 31) & 31;  // age e - 1 is held by lane (e - 1) mod 32
        const uint32_t b0 = __shfl_sync(FULL_MASK, bins[0], src);
        const uint32_t b1 = __shfl_sync(FULL_MASK, bins[1], src);
        if (e >= FEAT)
            continue;
        float v = 0.0f;
        if (e == 0)
            v = (float)nat * inv_g;
        else if (e <= 64)
            v = (float)(e - 1 < 32 ? b0 : b1) * inv_g;
        else if (e == 65)
            v = (float)up;
        else if (e == 66)
            v = (float)lmin;
        else if (e == 67)
            v = (float)lmax;
        else if (e >= 68 && e < 68 + P.r) {
#pragma unroll
            for (uint32_t i = 0; i < MAX_ROWS; i++)
                if (e == 68 + i)
                    v = (float)cnt[i] * inv_g;
        }
        row[e] = __float2bfloat16_rn(v);
    }
    if (nat_out && lane == 0)
        *nat_out = nat;
    __syncwarp();
}

// The rows of n hosts of a pool: one warp per host, its ATVs addressed by
// RRH(host) (Sec. 4.1), its loads from the last scan's row-frame loads.
template <int WB>
__global__ void __launch_bounds__(CAND_WARPS * 32) candidate_features_kernel(Params P, const uint32_t *pool, uint32_t c0,
                                                                             uint32_t kp,
                                                                             const unsigned long long *aat,
                                                                             const uint32_t *aips, uint64_t n, bf16 *x)
{
    extern __shared__ uint32_t csm[];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint16_t *hist = reinterpret_cast<uint16_t *>(csm + warp * HIST_WORDS);
    RangeDesc *desc = reinterpret_cast<RangeDesc *>(csm + CAND_WARPS * HIST_WORDS);  // [Wd]
    uint32_t *actw = reinterpret_cast<uint32_t *>(desc + P.Wd);                       // [Wd]
    feature_tables<WB>(P, c0, kp, desc, actw);
    for (uint32_t i = lane; i < HIST_WORDS; i += 32)
        csm[warp * HIST_WORDS + i] = 0;
    __syncthreads();
    const double denom = (double)P.g * (double)(P.cmask + 1);
    for (uint64_t h = (uint64_t)blockIdx.x * CAND_WARPS + warp; h < n; h += (uint64_t)gridDim.x * CAND_WARPS) {
        const uint32_t f = mangle(P.A, aips[h]);
        const uint32_t z = f & (P.nf - 1);
        const uint64_t LL = lbs_twice(P, f);
        const uint32_t *atv[MAX_ROWS];
        double loads[MAX_ROWS];
#pragma unroll
        for (uint32_t i = 0; i < MAX_ROWS; i++) {
            const uint32_t ii = i < P.r ? i : 0;
            const uint32_t e = (ii << P.E_log2) | (z << P.c) | column(P, LL, (int)ii);
            atv[i] = pool + (size_t)e * P.Wd;
            loads[i] = (double)aat[(size_t)ii * P.nf + z] / denom;
        }
        candidate_row<WB>(P, atv, desc, actw, kp, loads, hist, x + h * FEAT, lane, nullptr);
    }
}

struct CandArgs {
    uint64_t seed;
    uint32_t n_max_log2;
    float bg_max;
};

// Synthetic candidate states, one block per state: a host of cardinality n
// (log-uniform in [1, 2^n_max_log2]) spread over the k slices with random
// shares, whose bips set the same AT in all r ATVs, and in each row its own
// background: every AT of row i set in each slice with probability p_i
// (drawn in [0, bg_max] per state and row).  The r ATVs are packed as
// ingest would leave them at the end of slice k - 1, and the feature row
// comes from candidate_row with the loads P_i = 1 - (1 - p_i)^k (the
// background activity of the window).  Labels: ln n, and Eq. 4's estimate
// from the state's NAT and UP = product of the P_i.
template <int WB>
__global__ void __launch_bounds__(256) synth_candidates_kernel(Params P, CandArgs S, uint64_t first, uint64_t n,
                                                               bf16 *x, float *log_n, float *eq4)
{
    constexpr uint32_t F = 32 / WB;
    extern __shared__ uint32_t ssm[];
    int16_t *last = reinterpret_cast<int16_t *>(ssm);                              // [r][g]
    uint32_t *words = ssm + (P.r * P.g + 1) / 2;                                   // [r][Wd]
    uint16_t *hist = reinterpret_cast<uint16_t *>(words + P.r * P.Wd);             // [64][32] 16-bit, left zero
    RangeDesc *desc = reinterpret_cast<RangeDesc *>(words + P.r * P.Wd + HIST_WORDS);  // [Wd]
    uint32_t *actw = reinterpret_cast<uint32_t *>(desc + P.Wd);                        // [Wd]
    __shared__ uint32_t end[65];
    __shared__ uint32_t card;
    __shared__ float pb[MAX_ROWS];
    __shared__ uint32_t nat_s;
    const uint32_t tid = threadIdx.x;
    for (uint32_t i = tid; i < HIST_WORDS; i += blockDim.x)
        reinterpret_cast<uint32_t *>(hist)[i] = 0;
    // packed as of the end of slice k - 1 (block 0's ACT (k-1) mod 2k)
    feature_tables<WB>(P, (P.k - 1) % P.k2, P.k, desc, actw);
    __syncthreads();
    for (uint64_t si = blockIdx.x; si < n; si += gridDim.x) {
        const uint64_t key = splitmix(S.seed ^ splitmix(first + si + 0x3C6EF372FE94F82Bull));
        if (tid == 0) {
            const double lnmax = (double)S.n_max_log2 * 0.6931471805599453;
            const double c = floor(exp(unit(key, 1) * lnmax));
            card = (uint32_t)(c < 1.0 ? 1.0 : c);
            for (uint32_t i = 0; i < P.r; i++)
                pb[i] = (float)(unit(key, 4 + i) * (double)S.bg_max);
            double tot = 0.0, w[64];
            for (uint32_t s = 0; s < P.k; s++) {
                w[s] = -log(unit(key, 16 + s) + 1e-300);
                tot += w[s];
            }
            double cum = 0.0;
            end[0] = 0;
            for (uint32_t s = 0; s < P.k; s++) {
                cum += w[s];
                end[s + 1] = s + 1 == P.k ? card : (uint32_t)floor((double)card * cum / tot);
            }
        }
        for (uint32_t e = tid; e < P.r * P.g; e += blockDim.x)
            last[e] = -1;
        __syncthreads();
        const uint32_t base = (uint32_t)(key >> 32);
        for (uint32_t s = 0; s < P.k; s++) {
            for (uint32_t e = tid; e < P.r * P.g; e += blockDim.x) {
                const uint32_t i = e / P.g, h = e - i * P.g;
                if (unit(key ^ (0xB5ull + 0x100ull * (i + 1)), ((uint64_t)s << 32) | h) < (double)pb[i])
                    last[e] = (int16_t)s;
            }
            __syncthreads();
            for (uint32_t j = end[s] + tid; j < end[s + 1]; j += blockDim.x) {
                const uint32_t h = bip_hash(P, mix32(base + j));
                for (uint32_t i = 0; i < P.r; i++)
                    last[i * P.g + h] = (int16_t)s;
            }
            __syncthreads();
        }
        // pack: an AT last set in slice s holds that slice's ACT (C0 = s)
        for (uint32_t e = tid; e < P.r * P.Wd; e += blockDim.x) {
            const uint32_t i = e / P.Wd, q = e - i * P.Wd;
            uint32_t wd = 0;
            for (uint32_t j = 0; j < F; j++) {
                const uint32_t pos = q * F + j;
                if (pos < P.g) {
                    const uint32_t h = pos_at(P, pos);  // the AT stored there
                    const int s = last[i * P.g + h];
                    const uint32_t v = s < 0 ? P.k2 : act_of(P, (uint32_t)s, act_block(P, h));
                    wd |= v << (j * WB);
                }
            }
            words[e] = wd;
        }
        __syncthreads();
        if (tid < 32) {
            const uint32_t *atv[MAX_ROWS];
            double loads[MAX_ROWS];
#pragma unroll
            for (uint32_t i = 0; i < MAX_ROWS; i++) {
                const uint32_t ii = i < P.r ? i : 0;
                atv[i] = words + ii * P.Wd;
                loads[i] = (double)(1.0f - powf(1.0f - pb[ii], (float)P.k));
            }
            candidate_row<WB>(P, atv, desc, actw, P.k, loads, hist, x + si * FEAT, tid, &nat_s);
            if (tid == 0) {
                log_n[si] = (float)log((double)card);
                double up = 1.0;
                for (uint32_t i = 0; i < P.r; i++)
                    up *= loads[i];
                const double g = (double)P.g;
                double est;
                if (nat_s >= P.g || up >= 1.0) {
                    est = INFINITY;
                } else {
                    const double ratio = (g - (double)nat_s) / (g * (1.0 - up));
                    est = ratio >= 1.0 ? 0.0 : -g * log(ratio);
                }
                eq4[si] = (float)est;
            }
        }
        __syncthreads();
    }
}

}  // namespace

}  // namespace asse

using namespace asse;

extern "C" {

int asse_candidate_features(asse_pool *pool, const uint32_t *aips_dev, uint64_t n, uint16_t *x_dev)
{
    if (!pool || (n > 0 && (!aips_dev || !x_dev)))
        return pool ? pool_fail(pool, ASSE_EINVAL, "NULL argument") : ASSE_EINVAL;
    FeatureView v;
    if (int rc = pool_feature_view(pool, &v))
        return rc;
    if (v.kp > 64)
        return pool_fail(pool, ASSE_EINVAL, "features need k' <= 64");
    if (n == 0)
        return ASSE_OK;
    cudaError_t e = dispatch_w(v.w, [&](auto wb) {
        constexpr int WB = decltype(wb)::value;
        const size_t smem =
            (size_t)CAND_WARPS * HIST_WORDS * sizeof(uint32_t) + (size_t)v.P.Wd * (sizeof(RangeDesc) + sizeof(uint32_t));
        cudaError_t e2 = cudaFuncSetAttribute(candidate_features_kernel<WB>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e2 != cudaSuccess)
            return e2;
        const uint64_t want = (n + CAND_WARPS - 1) / CAND_WARPS;
        const uint64_t full = (uint64_t)v.sms * 4;
        candidate_features_kernel<WB><<<(unsigned)(want < full ? want : full), CAND_WARPS * 32, smem, v.stream>>>(
            v.P, v.pool, v.c0, v.kp, v.aat, aips_dev, n, reinterpret_cast<bf16 *>(x_dev));
        return cudaGetLastError();
    });
    *v.launches += 1;
    if (e != cudaSuccess)
        return pool_fail(pool, ASSE_ECUDA, std::string("candidate features launch: ") + cudaGetErrorString(e));
    return ASSE_OK;
}

int asse_synth_candidates(const asse_synth_cfg *cfg, uint64_t first, uint64_t n, uint16_t *x_dev, float *log_n_dev,
                          float *eq4_dev, void *stream)
{
    if (!cfg || (n > 0 && (!x_dev || !log_n_dev || !eq4_dev)))
        return ASSE_EINVAL;
    if (cfg->k < 1 || cfg->k > 64 || cfg->g < 2 * cfg->k || cfg->g > 4096 || cfg->r < 1 || cfg->r > MAX_ROWS ||
        cfg->n_max_log2 > 24 || (cfg->bh_a & 1) == 0 || !(cfg->bg_max >= 0.0f && cfg->bg_max <= 1.0f))
        return ASSE_EINVAL;
    if (n == 0)
        return ASSE_OK;
    Params P{};
    P.k = cfg->k;
    P.k2 = 2 * cfg->k;
    P.g = cfg->g;
    P.r = cfg->r;
    P.blk = cfg->g / (2 * cfg->k);
    P.blk_magic = ((1ull << 32) + P.blk - 1) / P.blk;
    P.paired = 1;  // the storage order of a timestamp pool's ACT blocks
    P.bh_a = cfg->bh_a;
    P.bh_b = cfg->bh_b;
    const uint32_t w = packed_width(ASSE_COUNTER_AT, cfg->k);
    const uint32_t Fw = 32 / w;
    P.Wd = ((cfg->g + Fw - 1) / Fw + 7) / 8 * 8;
    const CandArgs S{cfg->seed, cfg->n_max_log2, cfg->bg_max};
    const size_t smem = ((size_t)(P.r * P.g + 1) / 2 + (size_t)P.r * P.Wd + HIST_WORDS) * sizeof(uint32_t) +
                        (size_t)P.Wd * (sizeof(RangeDesc) + sizeof(uint32_t));
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid = (unsigned)(n < (uint64_t)sms * 8 ? n : (uint64_t)sms * 8);
    cudaError_t e = dispatch_w(w, [&](auto wb) {
        constexpr int WB = decltype(wb)::value;
        cudaError_t e2 = cudaFuncSetAttribute(synth_candidates_kernel<WB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem);
        if (e2 != cudaSuccess)
            return e2;
        synth_candidates_kernel<WB><<<grid, 256, smem, (cudaStream_t)stream>>>(
            P, S, first, n, reinterpret_cast<bf16 *>(x_dev), log_n_dev, eq4_dev);
        return cudaGetLastError();
    });
    return e == cudaSuccess ? ASSE_OK : ASSE_ECUDA;
}

}  // extern "C"
