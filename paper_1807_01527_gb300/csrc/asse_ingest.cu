// K1: Algorithm 3 (Scan IP pair, Sec. 4.1) over a batch of (aip, bip) pairs.
//
// One thread takes two pairs per 128-bit streaming load (evict-first, so the
// pair stream does not push the pool out of L2), issued one round ahead.  It
// first computes BH(bip) and looks the key (aip, BH(bip)) up in a
// direct-mapped table of recently seen keys in shared memory: a pair whose
// key this block already handled in this launch sets exactly the same r
// fields to the same values, so it is skipped (SetAT is idempotent within a
// slice; a key pushed out of the table only means a repeat is processed
// again).  Unseen keys go to a per-warp queue.  A pool larger than the L2
// cache also has a key table in device memory shared by every block and
// every ingest of the slice: every 32 queued keys, each lane claims one there
// (one L2 access), and only keys new to the slice go on, through a second
// per-warp queue, to Algorithm 3: each lane takes one, computes f(aip), the
// frame, the r column indices and the ACT of the AT in registers, issues the
// r word loads together, then sets the r fields; a field that already holds
// the slice's value costs one load and no atomic.  Across the 152 blocks a
// hot key reaches the pool once instead of once per block, which spares r
// DRAM sectors per repeat; with the pool in L2 a pool word costs what a claim
// costs, so such pools have no key table.  The shared-memory table is 64 KB:
// the rest of the SM's 256 KB of L1 / shared memory stays L1 cache, which
// serves the pool words of keys the table missed (a 128 KB table ran 13 %
// slower, a 192 KB one 2x slower).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "asse_device.cuh"

namespace asse {

namespace {

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

// f(aip), its frame and LBS twice over (the column windows are shifts of it).
__device__ __forceinline__ void prep_host(const Params &P, uint32_t aip, uint64_t &LL, uint32_t &z)
{
    const uint32_t f = mangle(P.A, aip);
    z = f & (P.nf - 1);
    LL = lbs_twice(P, f);
}

__device__ __forceinline__ uint32_t *field_word(const Params &P, uint32_t *pool, int i, uint32_t z, uint64_t LL,
                                                uint32_t q)
{
    const uint32_t atv = ((uint32_t)i << P.E_log2) | (z << P.c) | column(P, LL, i);
    return pool + (uint64_t)atv * P.Wd + q;
}

constexpr int INGEST_THREADS = 1024;
constexpr int INGEST_WARPS = INGEST_THREADS / 32;
constexpr int INGEST_BLOCKS_PER_SM = 1;
constexpr uint32_t SEEN_LOG2 = 13;  // 8,192 keys = 64 KB of shared memory per block
constexpr uint32_t QCAP = 96;       // per-warp queue of keys new to the block (below 32 between rounds, + 64)
constexpr uint32_t Q2CAP = 64;      // per-warp queue of keys new to the slice (below 32 between rounds, + 32)
constexpr unsigned long long NO_KEY = ~0ull;  // BH values are < 2^16, so never a real key

__device__ __forceinline__ uint32_t seen_slot(uint32_t aip, uint32_t h)
{
    return (aip * 0x9E3779B1u ^ h * 0x85EBCA77u) >> (32 - SEEN_LOG2);
}

// True if (aip, h) was recorded in the table of seen keys; records it
// otherwise.  CL = 1: the block's own table.  CL > 1: the CTAs of a
// thread-block cluster share one table of CL x 8,192 keys, each CTA holding
// the keys whose hash picks it, reached by the others through distributed
// shared memory; a key repeated across the cluster's SMs is then set once.
// Plain loads and stores: two CTAs that both miss a key set it twice, which
// only repeats an idempotent SetAT.
template <int CL>
__device__ __forceinline__ bool seen_before(unsigned long long *seen, uint32_t aip, uint32_t h)
{
    const unsigned long long key = ((unsigned long long)aip << 32) | h;
    if constexpr (CL == 1) {
        const uint32_t s = seen_slot(aip, h);
        if (seen[s] == key)
            return true;
        seen[s] = key;
        return false;
    } else {
        constexpr uint32_t CL_LOG2 = CL == 2 ? 1 : (CL == 4 ? 2 : 3);
        const uint32_t s_all = (aip * 0x9E3779B1u ^ h * 0x85EBCA77u) >> (32 - SEEN_LOG2 - CL_LOG2);
        const uint32_t owner = s_all >> SEEN_LOG2, s = s_all & ((1u << SEEN_LOG2) - 1);
        namespace cg = cooperative_groups;
        cg::cluster_group cluster = cg::this_cluster();
        unsigned long long *t = owner == cluster.block_rank() ? seen : cluster.map_shared_rank(seen, owner);
        if (t[s] == key)
            return true;
        t[s] = key;
        return false;
    }
}

// L2 accesses to the key table carry the evict-last priority: the pool words
// and the pair stream that pass through L2 during an ingest would otherwise
// push the table out between two claims of the same key (measured on the
// 1.07 GB pool: 0.362 against 0.378 ms; the evict-first priority on the pool
// words instead made it slower, 0.45 ms, as their compare-and-swap follows
// the read).
__device__ __forceinline__ uint64_t l2_evict_last_policy()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ unsigned long long ld_l2_hint(const unsigned long long *a, uint64_t pol)
{
    unsigned long long v;
    asm volatile("ld.global.cg.L2::cache_hint.b64 %0, [%1], %2;" : "=l"(v) : "l"(a), "l"(pol) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long exch_l2_hint(unsigned long long *a, unsigned long long x, uint64_t pol)
{
    unsigned long long v;
    asm volatile("atom.global.exch.L2::cache_hint.b64 %0, [%1], %2, %3;" : "=l"(v) : "l"(a), "l"(x), "l"(pol)
                 : "memory");
    return v;
}

// True if this lane is the first of the slice to claim key (aip, h) in the
// key table shared by all blocks.  A key that another block (or an earlier
// ingest of the same slice) claimed has had, or will have by the end of this
// launch, its r fields set to the same values, so it is skipped.  A key
// pushed out of the table by another only costs a repeat.  The plain read
// first spares the exchange for the keys already claimed, most of them.
__device__ __forceinline__ bool claim_key(const Params &P, uint32_t gen, uint32_t aip, uint32_t h, bool ok)
{
    if (!ok)
        return false;
    const unsigned long long x = key_mix(aip, h);
    const uint32_t tb = 48 - P.klg;
    const unsigned long long want = ((unsigned long long)gen << 32) | (x & ((1ull << tb) - 1));
    unsigned long long *slot = P.keys + (x >> tb);
    const uint64_t pol = l2_evict_last_policy();
    if (ld_l2_hint(slot, pol) == want)
        return false;
    return exch_l2_hint(slot, want, pol) != want;
}

// Slice counts (ASSE_COUNTER_AT_HIST) after this lane changed a field of ATV
// atv from f to the slice's value val: the count of the open slice's phase
// gains one and, if f was set less than k slices ago, the count of f's slice
// loses one (a count older than that is outside every window and is zeroed
// before its phase comes round again); otherwise the ATV's sum over the
// window gains one.
__device__ __forceinline__ void hist_moved(const Params &P, uint32_t f, uint32_t val, uint32_t c0, uint32_t atv)
{
    const uint64_t n_atv = (uint64_t)P.r << P.E_log2;
    hist_add(P.hist, (uint64_t)c0 * n_atv + atv, 1);
    bool in_window = false;
    if (f != P.k2) {
        uint32_t age = val + P.k2 - f;  // (ACT now - ACT then) mod 2k: slices since f was set
        age = age >= P.k2 ? age - P.k2 : age;
        if (age < P.k) {
            const uint32_t ph = c0 >= age ? c0 - age : c0 + P.k2 - age;
            hist_add(P.hist, (uint64_t)ph * n_atv + atv, -1);
            in_window = true;
        }
    }
    // the ATV's window sum gains the AT unless it moved within the window
    if (!in_window)
        hist_add(P.hsum, atv, 1);
}

// SetAT with slice counts: the field is set with a compare-and-swap, which
// tells its old value; old is the word as last seen (a read, or a failed
// compare-and-swap), retried until this lane changes the field or finds it
// already holding val.
__device__ __forceinline__ void set_field_hist(const Params &P, uint32_t *addr, uint32_t old, uint32_t sh, uint32_t val,
                                               uint32_t fm, uint32_t c0, uint32_t atv)
{
    uint32_t f;
    for (;;) {
        f = (old >> sh) & fm;
        if (f == val)
            return;  // already the slice's value: nothing changes
        const uint32_t nw = (old & ~(fm << sh)) | (val << sh);
        const uint32_t prev = atomicCAS(addr, old, nw);
        if (prev == old)
            break;
        old = prev;
    }
    hist_moved(P, f, val, c0, atv);
}

// Algorithm 3 for one key (aip, h = BH(bip)) of this lane, if ok: f(aip), the
// r column windows, the ACT of AT h, the r word loads together, then the
// field sets (with the slice counts when HIST).
template <int WB, int R, bool HIST = false>
__device__ __forceinline__ void set_key(const Params &P, uint32_t *pool, uint32_t c0, int r, uint32_t aip, uint32_t h,
                                        bool ok)
{
    constexpr uint32_t F = 32 / WB;
    constexpr uint32_t FM = (1u << WB) - 1;
    constexpr int RM = R ? R : 8;
    if (!ok)
        return;
    uint64_t LL;
    uint32_t z;
    prep_host(P, aip, LL, z);
    const uint32_t val = P.ace ? P.k : act_of(P, c0, act_block(P, h));
    const uint32_t pos = at_pos(P, h);  // where AT h is stored in its ATV
    const uint32_t q = pos / F;
    const uint32_t sh = (pos - q * F) * WB;
    uint32_t *a[RM];
    uint32_t o[RM];
#pragma unroll
    for (int i = 0; i < RM; i++)
        if (i < r)
            a[i] = field_word(P, pool, i, z, LL, q);
#pragma unroll
    for (int i = 0; i < RM; i++)
        if (i < r)
            o[i] = *a[i];
    if constexpr (HIST) {
        // the r compare-and-swaps issued together; one that lost a race with
        // another lane's change of the same word retries on what it returned
        uint32_t prev[RM];
#pragma unroll
        for (int i = 0; i < RM; i++)
            if (i < r)
                prev[i] = ((o[i] >> sh) & FM) != val ? atomicCAS(a[i], o[i], (o[i] & ~(FM << sh)) | (val << sh)) : o[i];
#pragma unroll
        for (int i = 0; i < RM; i++) {
            if (i < r) {
                const uint32_t f = (o[i] >> sh) & FM;
                if (f == val)
                    continue;
                const uint32_t atv = (uint32_t)((a[i] - pool) / P.Wd);
                if (prev[i] == o[i])
                    hist_moved(P, f, val, c0, atv);
                else
                    set_field_hist(P, a[i], prev[i], sh, val, FM, c0, atv);
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < RM; i++)
            if (i < r)
                set_field(a[i], o[i], sh, val, FM);
    }
}

// Keys new to the block (one per lane, if ok) are claimed in the key table;
// the ones new to the slice join the warp's second queue, and every 32 of
// those run Algorithm 3 with all lanes busy.  Without a key table, Algorithm
// 3 runs on them directly.
template <int WB, int R, bool HIST>
__device__ __forceinline__ void claim_and_set(const Params &P, uint32_t *pool, uint32_t c0, uint32_t gen, int r,
                                              uint2 e, bool ok, uint2 *q2, uint32_t &q2n, unsigned lt)
{
    bool run = ok;
    if (P.keys != nullptr) {
        const bool fresh = claim_key(P, gen, e.x, e.y, ok);
        const unsigned m = __ballot_sync(FULL_MASK, fresh);
        if (fresh)
            q2[q2n + __popc(m & lt)] = e;
        q2n += __popc(m);
        run = q2n >= 32;
        if (run) {
            __syncwarp();
            q2n -= 32;
            e = q2[q2n + threadIdx.x % 32];
            __syncwarp();
        }
    }
    set_key<WB, R, HIST>(P, pool, c0, r, e.x, e.y, run);
}

template <int WB, int R, bool HIST, int CL>
__global__ void __launch_bounds__(INGEST_THREADS, INGEST_BLOCKS_PER_SM)
    ingest_kernel(Params P, uint32_t *pool, const uint32_t *__restrict__ pairs_raw, uint64_t n_arg,
                  const unsigned long long *n_dev, const SliceCtl *ctl)
{
    const uint32_t c0 = ctl->c0;
    const uint32_t gen = (uint32_t)ctl->t;
    const uint64_t n = n_dev ? *n_dev : n_arg;
    const uint64_t nvec = n / 2;
    const uint4 *__restrict__ pairs = reinterpret_cast<const uint4 *>(pairs_raw);
    const uint2 *__restrict__ tail = (n & 1) ? reinterpret_cast<const uint2 *>(pairs_raw + 2 * (n - 1)) : nullptr;
    extern __shared__ unsigned long long seen[];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // the second queue only exists with a key table (its 16 KB otherwise stay L1 cache)
    uint2 *queue = reinterpret_cast<uint2 *>(seen + (1u << SEEN_LOG2)) + warp * (QCAP + (P.keys ? Q2CAP : 0));
    uint2 *q2 = queue + QCAP;
    for (uint32_t i = threadIdx.x; i < (1u << SEEN_LOG2); i += blockDim.x)
        seen[i] = NO_KEY;
    // every table of the cluster is empty before any CTA reaches into another's
    if constexpr (CL > 1)
        cooperative_groups::this_cluster().sync();
    else
        __syncthreads();
    const int r = R ? R : (int)P.r;
    // Warp-uniform loop: the 32 lanes of a warp take 32 consecutive vectors.
    // Keys the block's table has not seen go to the warp's queue; whenever it
    // holds 32 of them, every lane claims one in the slice's key table.
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t base0 = (uint64_t)blockIdx.x * blockDim.x + warp * 32u;
    const unsigned lt = (1u << lane) - 1u;
    uint32_t qn = 0, q2n = 0;
    // the next round's pairs are loaded before this round's are processed,
    // so the stream's DRAM latency overlaps the pool accesses
    uint4 pr = base0 + lane < nvec ? __ldcs(pairs + base0 + lane) : make_uint4(0, 0, 0, 0);
    for (uint64_t vb = base0; vb < nvec; vb += stride) {
        const uint64_t v = vb + lane;
        const uint4 cur = pr;
        if (v + stride < nvec)
            pr = __ldcs(pairs + v + stride);
        bool do0 = false, do1 = false;
        uint32_t h0 = 0, h1 = 0;
        if (v < nvec) {
            h0 = bip_hash(P, cur.y);
            h1 = bip_hash(P, cur.w);
            do0 = !seen_before<CL>(seen, cur.x, h0);
            do1 = !seen_before<CL>(seen, cur.z, h1);
        }
        const unsigned m0 = __ballot_sync(FULL_MASK, do0), m1 = __ballot_sync(FULL_MASK, do1);
        if (do0)
            queue[qn + __popc(m0 & lt)] = make_uint2(cur.x, h0);
        qn += __popc(m0);
        if (do1)
            queue[qn + __popc(m1 & lt)] = make_uint2(cur.z, h1);
        qn += __popc(m1);
        while (qn >= 32) {
            __syncwarp();
            qn -= 32;
            const uint2 e = queue[qn + lane];
            __syncwarp();
            claim_and_set<WB, R, HIST>(P, pool, c0, gen, r, e, true, q2, q2n, lt);
        }
    }
    __syncwarp();
    if (qn > 0) {
        const bool ok = lane < qn;
        claim_and_set<WB, R, HIST>(P, pool, c0, gen, r, ok ? queue[lane] : make_uint2(0, 0), ok, q2, q2n, lt);
    }
    __syncwarp();
    if (q2n > 0) {
        const bool ok = lane < q2n;
        const uint2 f = ok ? q2[lane] : make_uint2(0, 0);
        set_key<WB, R, HIST>(P, pool, c0, r, f.x, f.y, ok);
    }
    if (tail != nullptr && blockIdx.x == 0 && threadIdx.x == 0) {
        const uint2 pr1 = *tail;
        set_key<WB, R, HIST>(P, pool, c0, r, pr1.x, bip_hash(P, pr1.y), true);
    }
    // no CTA leaves while another may still read its table
    if constexpr (CL > 1)
        cooperative_groups::this_cluster().sync();
}

}  // namespace

cudaError_t launch_ingest(const Params &P, uint32_t w, uint32_t *pool, const uint32_t *pairs, uint64_t n,
                          const unsigned long long *n_dev, const SliceCtl *ctl, int sms, cudaStream_t s,
                          uint64_t *launches)
{
    if (n == 0 && n_dev == nullptr)
        return cudaSuccess;
    const uint64_t nvec = n / 2;
    *launches += 1;
    const size_t smem = (sizeof(unsigned long long) << SEEN_LOG2) +
                        (size_t)INGEST_WARPS * (QCAP + (P.keys ? Q2CAP : 0)) * sizeof(uint2);
    return dispatch_w(w, [&](auto wb) {
        constexpr int WB = decltype(wb)::value;
        auto pick = [&](auto cl) {
            constexpr int CL = decltype(cl)::value;
            return P.hist ? (P.r == 4 ? ingest_kernel<WB, 4, true, CL> : ingest_kernel<WB, 0, true, CL>)
                          : (P.r == 4 ? ingest_kernel<WB, 4, false, CL> : ingest_kernel<WB, 0, false, CL>);
        };
        auto kern = P.cl == 8   ? pick(std::integral_constant<int, 8>())
                    : P.cl == 4 ? pick(std::integral_constant<int, 4>())
                    : P.cl == 2 ? pick(std::integral_constant<int, 2>())
                                : pick(std::integral_constant<int, 1>());
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        const uint64_t want = (nvec + INGEST_THREADS - 1) / INGEST_THREADS;
        cudaLaunchConfig_t lc{};
        cudaLaunchAttribute attr[1];
        lc.blockDim = dim3(INGEST_THREADS);
        lc.dynamicSmemBytes = smem;
        lc.stream = s;
        uint64_t full;
        if (P.cl > 1) {
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = P.cl;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            lc.attrs = attr;
            lc.numAttrs = 1;
            // as many whole clusters as are resident at once
            lc.gridDim = dim3(P.cl);
            int nc = 0;
            e = cudaOccupancyMaxActiveClusters(&nc, kern, &lc);
            if (e != cudaSuccess || nc < 1)
                return e != cudaSuccess ? e : cudaErrorInvalidConfiguration;
            full = (uint64_t)nc * P.cl;
        } else {
            full = (uint64_t)sms * resident_blocks(kern, INGEST_THREADS, smem);
        }
        // with the count only known on the device, the full resident grid
        uint64_t grid = n_dev ? full : (want < 1 ? 1 : (want < full ? want : full));
        grid = (grid + P.cl - 1) / P.cl * P.cl;
        lc.gridDim = dim3((unsigned)grid);
        return cudaLaunchKernelEx(&lc, kern, P, pool, pairs, n, n_dev, ctl);
    });
}

namespace {

__global__ void advance_ctl_kernel(Params P, SliceCtl *ctl)
{
    open_next_slice(P, ctl);
}

__global__ void reset_kernel(unsigned long long *aat, uint32_t *sa_n, uint32_t nseg, Status *status)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nseg; i += gridDim.x * blockDim.x) {
        aat[i] = 0;
        sa_n[i] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        *status = Status{};
}

}  // namespace

cudaError_t launch_advance_ctl(const Params &P, SliceCtl *ctl, cudaStream_t s, uint64_t *launches)
{
    *launches += 1;
    advance_ctl_kernel<<<1, 256, 0, s>>>(P, ctl);
    return cudaGetLastError();
}

// Zero the scan outputs that are accumulated with atomics, and the status.
cudaError_t launch_reset(unsigned long long *aat, uint32_t *sa_n, uint32_t nseg, Status *status, cudaStream_t s,
                         uint64_t *launches)
{
    *launches += 1;
    reset_kernel<<<(nseg + 255) / 256 < 1 ? 1 : (nseg + 255) / 256, 256, 0, s>>>(aat, sa_n, nseg, status);
    return cudaGetLastError();
}

}  // namespace asse
