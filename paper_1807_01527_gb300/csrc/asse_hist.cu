// The close of a pool with slice counts (ASSE_COUNTER_AT_HIST).
//
// The ingest keeps, for every ATV, how many of its ATs each slice phase
// (t mod 2k) set last, and the sum of those counts over the window of the
// latest k slices (asse_ingest.cu).  An AT is active in the window of the
// latest k' slices iff it was set in one of them (Sec. 3), so |ATV|^{k'} is
// the window sum for k' = k (one 2-byte read per ATV), or the sum of the
// counts of the k' latest phases (2 bytes per ATV and phase, coalesced across
// the ATVs: the counts are phase-major), instead of the whole ATV.  The
// row-frame loads and the super-ATV lists follow as in the full scan; only a
// super ATV's words are read, to build its g-bit active mask for Algorithm 5.
// In the close of a slice the same kernel then runs the refresh of the two
// checked blocks (Algorithm 2), takes the phase leaving the window out of the
// sums and zeroes the counts of the opening slice's phase; the stepwise scan
// leaves all three to the refresh kernel of asse_advance.
#include <cuda_runtime.h>

#include <cstdint>

#include "asse_device.cuh"
#include "asse_swar.cuh"

namespace asse {

namespace {

constexpr int HIST_THREADS = 256;
constexpr int HIST_WARPS = HIST_THREADS / 32;
// ATVs of a thread whose refreshed words are loaded together (measured on the
// long pool's close: 2 -> 0.075 ms, 4 -> 0.082, 8 -> 0.082, one word at a
// time -> 0.080; more registers cost resident warps)
constexpr int RG = 2;

// V consecutive 16-bit counts from p (V = 8: one 16-byte load).
template <int V>
__device__ __forceinline__ void load_counts(const uint16_t *p, uint32_t (&c)[V])
{
    if constexpr (V == 8) {
        const uint4 h = *reinterpret_cast<const uint4 *>(p);
        c[0] = h.x & 0xffffu;
        c[1] = h.x >> 16;
        c[2] = h.y & 0xffffu;
        c[3] = h.y >> 16;
        c[4] = h.z & 0xffffu;
        c[5] = h.z >> 16;
        c[6] = h.w & 0xffffu;
        c[7] = h.w >> 16;
    } else {
        c[0] = p[0];
    }
}

template <int V>
__device__ __forceinline__ void store_counts(uint16_t *p, const uint32_t (&c)[V])
{
    if constexpr (V == 8)
        *reinterpret_cast<uint4 *>(p) =
            make_uint4(c[0] | (c[1] << 16), c[2] | (c[3] << 16), c[4] | (c[5] << 16), c[6] | (c[7] << 16));
    else
        p[0] = (uint16_t)c[0];
}

// V ATVs per thread (8: one 16-byte load per phase, the ATVs of one thread
// in one row-frame; 1 for pools with fewer than 8 columns).  SUM: the
// window is the full k slices, whose counts the ATV's running sum holds (one
// read instead of k).  FUSE: the close of a slice, which also runs Algorithm
// 2 on the two checked blocks of each of the thread's ATVs (after the warp
// has built the masks of its super ATVs from the unrefreshed words), takes
// the phase that is about to leave the window out of the running sums and
// zeroes the counts of the opening slice's phase (not a phase of the window
// being counted).
template <int WB, bool FUSE, int V, bool SUM>
__global__ void __launch_bounds__(HIST_THREADS) hist_scan_kernel(Params P, uint32_t *pool, uint32_t kp,
                                                                 const SliceCtl *ctl, ScanOut o, uint32_t total_atv)
{
    constexpr uint32_t F = 32 / WB;
    extern __shared__ __align__(16) uint8_t hsm[];
    RangeDesc *desc = reinterpret_cast<RangeDesc *>(hsm);                  // [Wd] count ranges
    RangeDesc *rdesc = desc + P.Wd;                                        // [Wd] refresh ranges (FUSE)
    uint32_t *maskbuf = reinterpret_cast<uint32_t *>(rdesc + (FUSE ? P.Wd : 0));  // [warps][mw]
    const uint32_t c0 = ctl->c0;
    const Refresh R = ctl->R;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t q = threadIdx.x; q < P.Wd; q += blockDim.x) {
        desc[q] = count_desc<WB>(P, q, c0, kp);
        if (FUSE)
            rdesc[q] = refresh_desc<WB>(P, q, R.c0n);
    }
    __syncthreads();
    uint32_t *my_mask = maskbuf + warp * P.mw;
    // the refreshed words as up to four slots when the (at most two) ranges
    // hold at most four words together
    const uint32_t n0 = R.n_ranges > 0 ? R.q_hi[0] - R.q_lo[0] + 1 : 0;
    const uint32_t n1 = R.n_ranges > 1 ? R.q_hi[1] - R.q_lo[1] + 1 : 0;
    const bool short_ranges = n0 + n1 <= 4;
    uint32_t rq[4];
#pragma unroll
    for (uint32_t j = 0; j < 4; j++)
        rq[j] = j < n0 ? R.q_lo[0] + j : R.q_lo[1] + (j - n0);
    const uint32_t rmask = (1u << (short_ranges ? n0 + n1 : 0u)) - 1u;
    const uint32_t cols = P.cmask + 1;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x * V;
    for (uint64_t base = ((uint64_t)blockIdx.x * blockDim.x + warp * 32u) * V; base < total_atv; base += stride) {
        const uint64_t a0 = base + (uint64_t)lane * V;
        const bool mine = a0 < total_atv;
        uint32_t c[V];
#pragma unroll
        for (int v = 0; v < V; v++)
            c[v] = 0;
        if (mine) {
            if constexpr (SUM) {
                load_counts<V>(P.hsum + a0, c);
            } else {
                // phases c0, c0-1, ..., c0-k'+1 (mod 2k): the slices of the window
                uint32_t ph = c0;
                for (uint32_t a = 0; a < kp; a++) {
                    uint32_t h[V];
                    load_counts<V>(P.hist + (uint64_t)ph * total_atv + a0, h);
#pragma unroll
                    for (int v = 0; v < V; v++)
                        c[v] += h[v];
                    ph = ph == 0 ? P.k2 - 1 : ph - 1;
                }
            }
            store_counts<V>(o.cnt + a0, c);
        }
        // the V ATVs of a thread share a row-frame (2^c is a multiple of V)
        const uint32_t sg = mine ? (uint32_t)(a0 >> P.c) : 0xffffffffu;  // row * 2^u + frame
        const unsigned grp = __match_any_sync(FULL_MASK, sg);
        {
            uint32_t sum = 0;
#pragma unroll
            for (int v = 0; v < V; v++)
                sum += c[v];
            const uint32_t s = __reduce_add_sync(grp, mine ? sum : 0u);
            if (mine && (uint32_t)(__ffs(grp) - 1) == lane && s)
                atomicAdd(&o.aat[sg], (unsigned long long)s);
        }
#pragma unroll 1
        for (int v = 0; v < V; v++) {
            uint32_t cv = 0;
#pragma unroll
            for (int vv = 0; vv < V; vv++)
                if (vv == v)
                    cv = c[vv];
            const bool sup = mine && cv >= P.T;
            uint32_t slot = 0;
            if (sup) {
                slot = atomicAdd(&o.sa_n[sg], 1u);
                o.sa_x[(size_t)sg * cols + slot] = (uint32_t)(a0 + v) & P.cmask;
            }
            unsigned sbits = __ballot_sync(FULL_MASK, sup);
            while (sbits) {
                // the g-bit active mask of one super ATV from its words
                const uint32_t hl = __ffs(sbits) - 1;
                sbits &= sbits - 1;
                const uint32_t slot_a = __shfl_sync(FULL_MASK, slot, hl);
                const uint64_t atv_a = base + (uint64_t)hl * V + v;
                const uint32_t sg_a = (uint32_t)(atv_a >> P.c);
                for (uint32_t k = lane; k < P.mw; k += 32)
                    my_mask[k] = 0;
                __syncwarp();
                for (uint32_t q = lane; q < P.Wd; q += 32) {
                    const uint32_t word = pool[atv_a * P.Wd + q];
                    const uint32_t am = field_bits<WB>(word, desc[q]);
                    if (am) {
                        const uint32_t pos = q * F, off = pos & 31;
                        atomicOr(&my_mask[pos >> 5], am << off);
                        if (off + F > 32 && (am >> (32 - off)))
                            atomicOr(&my_mask[(pos >> 5) + 1], am >> (32 - off));
                    }
                }
                __syncwarp();
                uint32_t *dst = o.sa_mask + ((size_t)sg_a * cols + slot_a) * P.mw;
                for (uint32_t k = lane; k < P.mw; k += 32)
                    dst[k] = my_mask[k];
                __syncwarp();
            }
        }
        if (FUSE && mine) {
            // Algorithm 2 for the next slice on the words of the two checked
            // blocks of each ATV, and the counts of the opening phase zeroed.
            // At most four words (two blocks of up to eight byte-wide fields,
            // every pair but the one with the long last block): the words of
            // RG ATVs are loaded before any is written back, so the thread
            // has them in flight together.
            if (short_ranges) {
                constexpr int G = V < RG ? V : RG;
#pragma unroll 1
                for (int v0 = 0; v0 < V; v0 += G) {
                    uint32_t wv[G][4];
#pragma unroll
                    for (int v = 0; v < G; v++) {
                        const uint32_t *atw = pool + (a0 + v0 + v) * P.Wd;
#pragma unroll
                        for (int j = 0; j < 4; j++)
                            wv[v][j] = (rmask >> j) & 1 ? atw[rq[j]] : 0u;
                    }
#pragma unroll
                    for (int v = 0; v < G; v++) {
                        uint32_t *atw = pool + (a0 + v0 + v) * P.Wd;
#pragma unroll
                        for (int j = 0; j < 4; j++) {
                            if ((rmask >> j) & 1) {
                                const uint32_t nw = refresh_swar<WB>(P, wv[v][j], rdesc[rq[j]]);
                                if (nw != wv[v][j])
                                    atw[rq[j]] = nw;
                            }
                        }
                    }
                }
            } else {
#pragma unroll 1
                for (int v = 0; v < V; v++) {
                    uint32_t *atw = pool + (a0 + v) * P.Wd;
                    for (uint32_t rr = 0; rr < R.n_ranges; rr++)
                        for (uint32_t q = R.q_lo[rr]; q <= R.q_hi[rr]; q++) {
                            const uint32_t w = atw[q];
                            const uint32_t nw = refresh_swar<WB>(P, w, rdesc[q]);
                            if (nw != w)
                                atw[q] = nw;
                        }
                }
            }
            // the window after this slice loses phase c0 - k + 1 (mod 2k)
            const uint32_t leave = c0 + P.k + 1 >= P.k2 ? c0 + P.k + 1 - P.k2 : c0 + P.k + 1;
            uint32_t lc[V], sv[V];
            load_counts<V>(P.hist + (uint64_t)leave * total_atv + a0, lc);
            if constexpr (SUM) {
#pragma unroll
                for (int v = 0; v < V; v++)
                    sv[v] = c[v] - lc[v];
            } else {
                load_counts<V>(P.hsum + a0, sv);
#pragma unroll
                for (int v = 0; v < V; v++)
                    sv[v] -= lc[v];
            }
            store_counts<V>(P.hsum + a0, sv);
            const uint32_t zero[V] = {};
            store_counts<V>(P.hist + (uint64_t)R.c0n * total_atv + a0, zero);
        }
    }
}

// The slice counts of a pool counted from its words (after asse_load): every
// AT set d < k slices ago, d = (ACT - value) mod 2k, adds one to the count of
// phase t - d and to the ATV's window sum.  Counts of older phases stay zero
// (no window reads them).
template <int WB>
__global__ void __launch_bounds__(HIST_THREADS) hist_rebuild_kernel(Params P, const uint32_t *pool, const SliceCtl *ctl,
                                                                    uint32_t total_atv)
{
    constexpr uint32_t F = 32 / WB;
    constexpr uint32_t FM = (1u << WB) - 1;
    const uint32_t c0 = ctl->c0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t atv = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; atv < total_atv; atv += stride) {
        for (uint32_t q = 0; q < P.Wd; q++) {
            const uint32_t word = pool[atv * P.Wd + q];
            for (uint32_t j = 0; j < F; j++) {
                const uint32_t h = q * F + j;
                const uint32_t v = (word >> (j * WB)) & FM;
                if (h >= P.g || v >= P.k2)
                    continue;
                uint32_t age = act_of(P, c0, pos_block(P, h)) + P.k2 - v;
                age = age >= P.k2 ? age - P.k2 : age;
                if (age < P.k) {
                    const uint32_t ph = c0 >= age ? c0 - age : c0 + P.k2 - age;
                    hist_add(P.hist, (uint64_t)ph * total_atv + atv, 1);
                    hist_add(P.hsum, atv, 1);
                }
            }
        }
    }
}

}  // namespace

cudaError_t launch_hist_scan(const Params &P, uint32_t w, uint32_t *pool, uint32_t kp, bool fuse, const SliceCtl *ctl,
                             const ScanOut &o, int sms, cudaStream_t s, uint64_t *launches)
{
    const uint32_t total = P.r << P.E_log2;
    const size_t smem = (size_t)P.Wd * sizeof(RangeDesc) * (fuse ? 2 : 1) + (size_t)HIST_WARPS * P.mw * sizeof(uint32_t);
    // 8 ATVs a thread when a row-frame holds a multiple of 8 of them
    const bool v8 = (P.cmask + 1) % 8 == 0;
    *launches += 1;
    return dispatch_w(w, [&](auto wb) {
        constexpr int WB = decltype(wb)::value;
        // a window of all k slices reads the running sums
        const bool sum = kp == P.k;
        auto kern = fuse ? (sum ? (v8 ? hist_scan_kernel<WB, true, 8, true> : hist_scan_kernel<WB, true, 1, true>)
                                : (v8 ? hist_scan_kernel<WB, true, 8, false> : hist_scan_kernel<WB, true, 1, false>))
                         : (sum ? (v8 ? hist_scan_kernel<WB, false, 8, true> : hist_scan_kernel<WB, false, 1, true>)
                                : (v8 ? hist_scan_kernel<WB, false, 8, false> : hist_scan_kernel<WB, false, 1, false>));
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        const uint32_t per = v8 ? 8 : 1;
        const uint64_t want = (total / per + HIST_THREADS - 1) / HIST_THREADS;
        const uint64_t full = (uint64_t)sms * resident_blocks(kern, HIST_THREADS, smem);
        kern<<<(unsigned)(want < full ? (want < 1 ? 1 : want) : full), HIST_THREADS, smem, s>>>(P, pool, kp, ctl, o,
                                                                                           total);
        return cudaGetLastError();
    });
}

cudaError_t launch_hist_rebuild(const Params &P, uint32_t w, const uint32_t *pool, const SliceCtl *ctl, int sms,
                                cudaStream_t s, uint64_t *launches)
{
    const uint32_t total = P.r << P.E_log2;
    cudaError_t e = cudaMemsetAsync(P.hist, 0, (size_t)P.k2 * total * sizeof(uint16_t), s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(P.hsum, 0, (size_t)total * sizeof(uint16_t), s);
    if (e != cudaSuccess)
        return e;
    *launches += 1;
    return dispatch_w(w, [&](auto wb) {
        constexpr int WB = decltype(wb)::value;
        const uint64_t want = (total + HIST_THREADS - 1) / HIST_THREADS;
        const uint64_t full = (uint64_t)sms * resident_blocks(hist_rebuild_kernel<WB>, HIST_THREADS, 0);
        hist_rebuild_kernel<WB><<<(unsigned)(want < full ? want : full), HIST_THREADS, 0, s>>>(P, pool, ctl, total);
        return cudaGetLastError();
    });
}

}  // namespace asse
