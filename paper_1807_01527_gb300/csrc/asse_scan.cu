// K2: the per-slice scan of the whole pool, with the refresh fused in, and
// the standalone refresh kernels.
//
// scan_kernel streams the pool in tiles of TA whole ATVs (at most 1024 words,
// one 128-bit load per thread, the next tile prefetched while this one is
// processed).  Per ATV it forms |ATV|^{k'} (Algorithm 1 on every field,
// Sec. 3) by shared-memory sums, adds it to the row-frame load |AAT(k',i,j)|
// (Sec. 4.3) through a warp-segmented reduction, and for super ATVs (count
// >= ceil(g - g e^{-theta/g}), Sec. 4.2) records the column index and the
// g-bit active mask that the restore intersects.  With FUSE, each thread then
// applies Algorithm 2 for the next slice to its words of the two refreshed ACT
// blocks (or the per-slice decrement of aging counters) and writes back the
// words that changed, so the refresh costs no extra read of the pool.
#include <cuda_runtime.h>

#include <cstdint>

#include "asse_device.cuh"

namespace asse {

namespace {

constexpr uint32_t NO_SLOT = 0xffffffffu;
constexpr int SCAN_THREADS = 256;

// Algorithm 2 on every field of a word whose new ACT is 0 or k.
template <int WB>
__device__ __forceinline__ uint32_t refresh_word(const Params &P, uint32_t word, uint32_t q, uint32_t c0n)
{
    constexpr uint32_t F = 32 / WB;
    constexpr uint32_t FM = (1u << WB) - 1;
    uint32_t out = word;
#pragma unroll
    for (uint32_t j = 0; j < F; j++) {
        const uint32_t h = q * F + j;
        if (h < P.g) {
            const uint32_t a = act_of(P, c0n, act_block(P, h));
            const uint32_t v = (word >> (j * WB)) & FM;
            out = (out & ~(FM << (j * WB))) | (preserve(P, v, a) << (j * WB));
        }
    }
    return out;
}

// Aging counters: every non-zero field loses one.
template <int WB>
__device__ __forceinline__ uint32_t decay_word(uint32_t word)
{
    constexpr uint32_t F = 32 / WB;
    constexpr uint32_t FM = (1u << WB) - 1;
    uint32_t dec = 0;
#pragma unroll
    for (uint32_t j = 0; j < F; j++)
        dec |= (uint32_t)(((word >> (j * WB)) & FM) != 0) << (j * WB);
    return word - dec;  // no borrow crosses a field: each decremented field is >= 1
}

__device__ __forceinline__ bool in_refresh(const Refresh &R, uint32_t q)
{
    return (R.n_ranges > 0 && q >= R.q_lo[0] && q <= R.q_hi[0]) ||
           (R.n_ranges > 1 && q >= R.q_lo[1] && q <= R.q_hi[1]);
}

template <int WB, bool FUSE>
__global__ void __launch_bounds__(SCAN_THREADS) scan_kernel(Params P, uint32_t *pool, uint32_t c0, uint32_t kp,
                                                            Refresh R, ScanOut o, uint32_t total_atv, uint32_t TA)
{
    constexpr uint32_t F = 32 / WB;
    extern __shared__ uint32_t sm[];
    uint32_t *cnt_s = sm;           // [TA] active counts
    uint32_t *slot_s = sm + TA;     // [TA] SA slot of super ATVs
    uint32_t *mask_s = sm + 2 * TA; // [TA][mw] active masks of super ATVs
    __shared__ int any_super;
    const uint32_t tid = threadIdx.x;
    const uint32_t vpa = P.Wd / 4;            // 128-bit vectors per ATV
    const uint32_t nv = TA * vpa;             // vectors per tile, <= SCAN_THREADS
    const uint32_t a_loc = tid / vpa;         // this thread's ATV within the tile
    const uint32_t q0 = (tid - a_loc * vpa) * 4;
    const uint32_t ntiles = (total_atv + TA - 1) / TA;
    const uint32_t cols = P.cmask + 1;
    const uint32_t mw = P.mw;

    auto load = [&](uint32_t tile) {
        const uint32_t atv = tile * TA + a_loc;
        if (tile < ntiles && tid < nv && atv < total_atv)
            return reinterpret_cast<const uint4 *>(pool + (size_t)atv * P.Wd)[q0 / 4];
        return make_uint4(0, 0, 0, 0);
    };

    uint4 next = load(blockIdx.x);
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint32_t atv0 = tile * TA;
        const uint32_t atv = atv0 + a_loc;
        const bool mine = tid < nv && atv < total_atv;
        const uint4 w = next;
        next = load(tile + gridDim.x);
        if (tid < TA)
            cnt_s[tid] = 0;
        if (tid == 0)
            any_super = 0;
        __syncthreads();
        uint32_t am[4] = {0, 0, 0, 0};
        if (mine) {
            uint32_t c = 0;
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const uint32_t q = q0 + e;
                if (q * F < P.g) {
                    am[e] = active_fields<WB>(P, u4get(w, e), q, c0, kp);
                    c += __popc(am[e]);
                }
            }
            if (c)
                atomicAdd(&cnt_s[a_loc], c);
        }
        __syncthreads();
        {
            // one thread per ATV of the tile: count, row-frame load, super test
            const uint32_t a = atv0 + tid;
            const bool fin = tid < TA && a < total_atv;
            const unsigned act = __ballot_sync(FULL_MASK, fin);
            if (fin) {
                const uint32_t c = cnt_s[tid];
                o.cnt[a] = (uint16_t)c;
                const uint32_t sg = a >> P.c;  // row * 2^u + frame
                const unsigned grp = __match_any_sync(act, sg);
                const uint32_t sum = __reduce_add_sync(grp, c);
                if ((uint32_t)(__ffs(grp) - 1) == (tid & 31) && sum)
                    atomicAdd(&o.aat[sg], (unsigned long long)sum);
                uint32_t slot = NO_SLOT;
                if (c >= P.T) {
                    slot = atomicAdd(&o.sa_n[sg], 1u);
                    o.sa_x[(size_t)sg * cols + slot] = a & P.cmask;
                    any_super = 1;
                }
                slot_s[tid] = slot;
            }
        }
        __syncthreads();
        if (any_super) {
            for (uint32_t i = tid; i < TA * mw; i += SCAN_THREADS)
                if (slot_s[i / mw] != NO_SLOT)
                    mask_s[i] = 0;
            __syncthreads();
            if (mine && slot_s[a_loc] != NO_SLOT) {
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    if (am[e]) {
                        const uint32_t pos = (q0 + e) * F, off = pos & 31;
                        uint32_t *m = mask_s + a_loc * mw + (pos >> 5);
                        atomicOr(m, am[e] << off);
                        if (off + F > 32 && (am[e] >> (32 - off)))
                            atomicOr(m + 1, am[e] >> (32 - off));
                    }
                }
            }
            __syncthreads();
            for (uint32_t i = tid; i < TA * mw; i += SCAN_THREADS) {
                const uint32_t al = i / mw;
                const uint32_t slot = slot_s[al];
                if (slot != NO_SLOT) {
                    const uint32_t sg = (atv0 + al) >> P.c;
                    o.sa_mask[((size_t)sg * cols + slot) * mw + (i - al * mw)] = mask_s[i];
                }
            }
        }
        if (FUSE && mine) {
            uint32_t *wp = pool + (size_t)atv * P.Wd;
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const uint32_t q = q0 + e;
                if (q * F < P.g) {
                    const uint32_t word = u4get(w, e);
                    uint32_t nw = word;
                    if (P.ace)
                        nw = decay_word<WB>(word);
                    else if (in_refresh(R, q))
                        nw = refresh_word<WB>(P, word, q, R.c0n);
                    if (nw != word)
                        wp[q] = nw;
                }
            }
        }
        __syncthreads();
    }
}

// A3 alone: one thread per (ATV, word of the two refreshed blocks).
template <int WB>
__global__ void __launch_bounds__(256) refresh_kernel(Params P, uint32_t *pool, Refresh R, uint32_t total_atv)
{
    const uint32_t nw0 = R.n_ranges > 0 ? R.q_hi[0] - R.q_lo[0] + 1 : 0;
    const uint32_t nw1 = R.n_ranges > 1 ? R.q_hi[1] - R.q_lo[1] + 1 : 0;
    const uint64_t nw = nw0 + nw1;
    const uint64_t total = (uint64_t)total_atv * nw;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += stride) {
        const uint64_t atv = idx / nw;
        const uint32_t kq = (uint32_t)(idx - atv * nw);
        const uint32_t q = kq < nw0 ? R.q_lo[0] + kq : R.q_lo[1] + (kq - nw0);
        uint32_t *wp = pool + atv * P.Wd + q;
        const uint32_t word = *wp;
        const uint32_t nwd = refresh_word<WB>(P, word, q, R.c0n);
        if (nwd != word)
            *wp = nwd;
    }
}

// Aging counters alone: the full-pool decrement of every slice.
template <int WB>
__global__ void __launch_bounds__(256) ace_decay_kernel(uint4 *pool, uint64_t nvec)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvec; v += stride) {
        const uint4 a = pool[v];
        const uint4 b = make_uint4(decay_word<WB>(a.x), decay_word<WB>(a.y), decay_word<WB>(a.z),
                                   decay_word<WB>(a.w));
        if (a.x != b.x || a.y != b.y || a.z != b.z || a.w != b.w)
            pool[v] = b;
    }
}

}  // namespace

uint32_t scan_tile_atvs(uint32_t Wd)
{
    const uint32_t ta = (SCAN_THREADS * 4) / Wd;
    return ta < 1 ? 1 : ta;
}

cudaError_t launch_scan(const Params &P, uint32_t w, uint32_t *pool, uint32_t c0, uint32_t kp, const Refresh *fuse,
                        const ScanOut &o, int sms, cudaStream_t s, uint64_t *launches)
{
    const uint32_t total = P.r << P.E_log2;
    const uint32_t TA = scan_tile_atvs(P.Wd);
    const size_t smem = (size_t)(2 * TA + TA * P.mw) * sizeof(uint32_t);
    const uint32_t ntiles = (total + TA - 1) / TA;
    const Refresh R = fuse ? *fuse : Refresh{};
    *launches += 1;
    return dispatch_w(w, [&](auto wb) {
        constexpr int WB = decltype(wb)::value;
        auto kern = fuse ? scan_kernel<WB, true> : scan_kernel<WB, false>;
        const int occ = resident_blocks(kern, SCAN_THREADS, smem);
        const uint64_t full = (uint64_t)sms * occ;
        const unsigned grid = (unsigned)(ntiles < full ? ntiles : full);
        kern<<<grid, SCAN_THREADS, smem, s>>>(P, pool, c0, kp, R, o, total, TA);
        return cudaGetLastError();
    });
}

cudaError_t launch_refresh(const Params &P, uint32_t w, uint32_t *pool, const Refresh &R, int sms, cudaStream_t s,
                           uint64_t *launches)
{
    const uint32_t total = P.r << P.E_log2;
    if (P.ace) {
        const uint64_t nvec = (uint64_t)total * P.Wd / 4;
        *launches += 1;
        return dispatch_w(w, [&](auto wb) {
            constexpr int WB = decltype(wb)::value;
            const uint64_t full = (uint64_t)sms * resident_blocks(ace_decay_kernel<WB>, 256, 0);
            const uint64_t want = (nvec + 255) / 256;
            ace_decay_kernel<WB><<<(unsigned)(want < full ? want : full), 256, 0, s>>>(
                reinterpret_cast<uint4 *>(pool), nvec);
            return cudaGetLastError();
        });
    }
    if (R.n_ranges == 0)
        return cudaSuccess;
    *launches += 1;
    return dispatch_w(w, [&](auto wb) {
        constexpr int WB = decltype(wb)::value;
        const unsigned grid = (unsigned)sms * resident_blocks(refresh_kernel<WB>, 256, 0);
        refresh_kernel<WB><<<grid, 256, 0, s>>>(P, pool, R, total);
        return cudaGetLastError();
    });
}

}  // namespace asse
