// K2: the per-slice scan of the whole pool, with the refresh fused in, and
// the standalone refresh kernels.
//
// scan_kernel is a persistent kernel (one CTA per SM).  Every warp streams
// tiles of whole ATVs from global memory into shared memory with bulk async
// copies (cp.async.bulk, completion on an mbarrier, two buffers per warp so the
// next tile is in flight while this one is processed).  Inside a tile one lane
// owns one ATV, or a share of a wide ATV, in one of two layouts: a 1/2, 1/4,
// 1/8 segment at a shared-memory stride of an odd number of 16-byte units, or
// (interleaved) every lpa-th 16-byte chunk of an ATV stored back to back, when
// the ATV length in chunks makes the lanes of a quarter warp hit distinct
// banks; either way the lanes' 128-bit reads never conflict, and a tile of
// whole, unpadded ATVs moves with one bulk copy.
//
// Activity test (Algorithm 1 on every field of a word at once): the active
// values of a block form the cyclic window act-k'+1 .. act (mod 2k), i.e. at
// most two plain ranges.  The even and the odd fields of a word are tested
// separately, each field then having w free bits above it; with a guard bit
// just above each field, (v | guard) - lo keeps the guard iff v >= lo and
// (hi | guard) - v keeps it iff v <= hi, with no borrow between fields.  The
// per-position constants carry each field's own range, so words that straddle
// two ACT blocks and the fields past g (empty ranges) need no special case.
// The refresh (Algorithm 2: values 0..k at new ACT 0; value 0 and k..2k-1 at
// new ACT k) uses the same range machinery to find the fields to clear.
//
// Per ATV the lanes form |ATV|^{k'} (Sec. 3), the row-frame loads |AAT(k',i,j)|
// (Sec. 4.3) and, for a super ATV (Sec. 4.2), its column and g-bit active
// mask.  With FUSE the refreshed words (AT) are written back at once, or for
// aging counters every word is decremented in shared memory and each segment
// is stored back with a bulk copy.
#include <cuda_runtime.h>

#include <cstdint>

#include "asse_device.cuh"
#include "asse_ptx.cuh"
#include "asse_swar.cuh"

namespace asse {

namespace {

// Threads of a scan CTA: 20 warps for the interleaved layout (4 KB tiles of
// wide ATVs, at most 102 registers a thread), 16 for the segment layouts,
// whose code needs more registers.
constexpr int scan_threads(bool ilv) { return ilv ? 640 : 512; }

// ---------------------------------------------------------------- scan kernel

// NW: the most windows this instantiation counts (1, or MAX_WINDOWS for the
// multi-window close, which runs W.n <= NW of them).  BG: byte-wide fields
// with values below 128, tested four at a time with the in-field guard bit
// (one 16-byte range entry per word instead of two).
// ILV: the interleaved tile layout (G.ilv), fixed at compile time so that
// the per-word index arithmetic of the inner loop has no layout branch.
template <int WB, bool FUSE, int NW, bool BG, bool ILV>
__global__ void __launch_bounds__(scan_threads(ILV), 1) scan_kernel(Params P, uint32_t *pool, const ScanWindows W,
                                                               const SliceCtl *ctl, uint32_t total_atv, ScanGeom G)
{
    static_assert(!BG || WB == 8, "the in-field guard needs byte-wide fields");
    const uint32_t c0 = ctl->c0;
    const Refresh R = ctl->R;
    extern __shared__ __align__(128) uint8_t smem[];
    // The count ranges of word q sit in two 16-byte halves at index q + (the
    // segment of q): the lanes of one warp read positions one segment apart,
    // and the skew puts those reads in distinct bank groups.
    // Window m's table starts at m * n_cd.
    const uint32_t nw = NW == 1 ? 1u : W.n;
    const uint32_t n_cd = P.Wd + G.lpa;
    const uint32_t nchunk = P.Wd / 4;
    // index of word q's range entry in window m's table: skewed by segment
    // (segments), or chunk-major per word of the chunk (interleaved), so that
    // the lanes' reads of one step fall in distinct banks
    auto didx = [&](uint32_t m, uint32_t q) {
        return m * n_cd + (ILV ? (q & 3u) * nchunk + (q >> 2) : q + q / G.wseg);
    };
    uint4 *cd_lo = reinterpret_cast<uint4 *>(smem);                          // [nw][Wd + lpa]
    uint4 *cd_hi = cd_lo + nw * n_cd;                                        // [nw][Wd + lpa]
    RangeDesc *rdesc = reinterpret_cast<RangeDesc *>(cd_hi + nw * n_cd);     // [Wd]
    uint64_t *mbar = reinterpret_cast<uint64_t *>(rdesc + P.Wd);             // [warps][2]
    uint32_t *maskbuf = reinterpret_cast<uint32_t *>(mbar + 2 * G.warps);    // [warps][mw]
    uint32_t *tiles = reinterpret_cast<uint32_t *>(smem + G.tile_offset);    // [warps][2][tile_words]

    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t e = threadIdx.x; e < nw * P.Wd; e += blockDim.x) {
        const uint32_t m = e / P.Wd, q = e - m * P.Wd;
        const uint32_t x = didx(m, q);
        if constexpr (BG) {
            cd_lo[x] = count_desc_bytes(P, q, c0, W.kp[m]);
            if (FUSE && m == 0) {
                const uint4 r = refresh_desc_bytes(P, q, R.c0n);
                rdesc[q] = RangeDesc{r.x, r.y, r.z, r.w, 0, 0, 0, 0};
            }
        } else {
            const RangeDesc d = count_desc<WB>(P, q, c0, W.kp[m]);
            cd_lo[x] = make_uint4(d.lo1e, d.hih1e, d.lo1o, d.hih1o);
            cd_hi[x] = make_uint4(d.lo2e, d.hih2e, d.lo2o, d.hih2o);
            if (FUSE && m == 0)
                rdesc[q] = refresh_desc<WB>(P, q, R.c0n);
        }
    }
    if (warp < G.warps && lane == 0) {
        mbar_init(&mbar[2 * warp], 1);
        mbar_init(&mbar[2 * warp + 1], 1);
    }
    fence_async_smem();
    __syncthreads();
    if (warp >= G.warps)
        return;

    const uint32_t a = lane / G.lpa, part = lane - a * G.lpa;  // this lane's ATV in the tile and share
    const uint32_t q_first = ILV ? 4 * part : part * G.wseg;  // its first word
    const uint32_t q_step = ILV ? 4 * G.lpa : 4;               // words between its chunks, in the ATV and in smem
    const uint32_t lane_off = ILV ? a * P.Wd + 4 * part : lane * G.seg_stride;  // its first word in the tile
    // word q of the tile's ATV a_ in shared memory
    auto tile_word = [&](const uint32_t *tb, uint32_t a_, uint32_t q) {
        if (ILV)
            return tb[a_ * P.Wd + q];
        const uint32_t pq = q / G.wseg;  // the segment holding word q
        return tb[(a_ * G.lpa + pq) * G.seg_stride + (q - pq * G.wseg)];
    };
    const uint32_t cols = P.cmask + 1;
    const uint32_t ntiles = (total_atv + G.apt - 1) / G.apt;
    uint32_t *my_mask = maskbuf + warp * P.mw;
    // buffer b of this warp, its mbarrier and phase parity (bit b of par);
    // computed, not indexed arrays, so that nothing lives in local memory
    auto tile_buf = [&](int b) { return tiles + (2 * warp + b) * G.tile_words; };
    auto bar = [&](int b) { return &mbar[2 * warp + b]; };
    uint32_t par = 0;

    // Segments of an odd number of 16-byte units need no padding: the tile
    // is then one contiguous stretch of the pool, fetched with one copy.
    const bool whole = ILV || G.seg_stride == G.wseg;
    auto issue = [&](uint32_t tile, int b) {
        const uint32_t atv0 = tile * G.apt;
        const uint32_t n_atv = min(G.apt, total_atv - atv0);
        if (whole) {
            if (lane == 0) {
                mbar_expect_tx(bar(b), n_atv * P.Wd * 4u);
                bulk_load(tile_buf(b), pool + (size_t)atv0 * P.Wd, n_atv * P.Wd * 4u, bar(b));
            }
            return;
        }
        if (lane == 0)
            mbar_expect_tx(bar(b), n_atv * P.Wd * 4u);
        __syncwarp();
        if (a < n_atv)
            bulk_load(tile_buf(b) + lane * G.seg_stride, pool + (size_t)(atv0 + a) * P.Wd + q_first, G.wseg * 4u,
                      bar(b));
    };
    // tiles are dealt round-robin over all warps of the grid: every tile
    // costs the same, and at any moment the warps stream one contiguous
    // stretch of the pool
    const uint32_t n_warps = gridDim.x * G.warps;
    uint32_t tile = blockIdx.x * G.warps + warp;
    int b = 0;
    if (tile < ntiles)
        issue(tile, 0);
    uint32_t next = tile < ntiles ? tile + n_warps : ntiles;
    if (next < ntiles)
        issue(next, 1);
    while (tile < ntiles) {
        if (!__all_sync(FULL_MASK, mbar_wait(bar(b), (par >> b) & 1u))) {
            // the copy did not land: flag it, give the other copy in flight a
            // bounded chance to finish, and leave
            if (lane == 0)
                for (uint32_t m = 0; m < nw; m++)
                    atomicExch(&W.o[m].status->error, 1u);
            if (next < ntiles)
                mbar_wait(bar(b ^ 1), (par >> (b ^ 1)) & 1u);
            return;
        }
        par ^= 1u << b;
        const uint32_t atv0 = tile * G.apt;
        const uint32_t n_atv = min(G.apt, total_atv - atv0);
        const bool mine = a < n_atv;
        uint32_t *row = tile_buf(b) + lane_off;
        uint32_t cnt[NW];
#pragma unroll
        for (int m = 0; m < NW; m++)
            cnt[m] = 0;
        if (mine) {
#pragma unroll 2
            for (uint32_t i = 0; i < G.wseg / 4; i++) {
                const uint4 x = *reinterpret_cast<const uint4 *>(row + i * q_step);
                const uint32_t q = q_first + i * q_step;
#pragma unroll
                for (int m = 0; m < NW; m++) {
                    if (m < (int)nw) {
                        // the range entries of words q .. q+3: consecutive (skewed by the
                        // segment), or a chunk apart (q is a multiple of 4)
                        const uint32_t xq = m * n_cd + (ILV ? (q >> 2) : q + part), dx = ILV ? nchunk : 1u;
                        if constexpr (BG) {
                            // per-byte counts (at most 64 words per lane: no carry between bytes)
                            cnt[m] += (in_ranges_bytes(x.x, cd_lo[xq]) >> 7) +
                                      (in_ranges_bytes(x.y, cd_lo[xq + dx]) >> 7) +
                                      (in_ranges_bytes(x.z, cd_lo[xq + 2 * dx]) >> 7) +
                                      (in_ranges_bytes(x.w, cd_lo[xq + 3 * dx]) >> 7);
                        } else {
                            cnt[m] += count_word<WB>(x.x, load_desc(cd_lo, cd_hi, xq)) +
                                      count_word<WB>(x.y, load_desc(cd_lo, cd_hi, xq + dx)) +
                                      count_word<WB>(x.z, load_desc(cd_lo, cd_hi, xq + 2 * dx)) +
                                      count_word<WB>(x.w, load_desc(cd_lo, cd_hi, xq + 3 * dx));
                        }
                    }
                }
            }
        }
        if constexpr (BG) {
#pragma unroll
            for (int m = 0; m < NW; m++)
                cnt[m] = (cnt[m] * BYTE_ONES) >> 24;  // the four byte counts added
        }
        const uint32_t atv = atv0 + a;
        const bool head = mine && part == 0;
        const uint32_t sg = head ? atv >> P.c : 0xffffffffu;  // row * 2^u + frame
        const unsigned grp = __match_any_sync(FULL_MASK, sg);
#pragma unroll 1
        for (uint32_t m = 0; m < nw; m++) {
            const ScanOut &o = W.o[m];
            uint32_t c = NW == 1 ? cnt[0] : 0u;
            if (NW > 1) {
#pragma unroll
                for (int mm = 0; mm < NW; mm++)
                    if ((uint32_t)mm == m)
                        c = cnt[mm];
            }
            for (uint32_t off = 1; off < G.lpa; off <<= 1)
                c += __shfl_xor_sync(FULL_MASK, c, off);

            // one lane per ATV: count, row-frame load, super test
            if (head)
                o.cnt[atv] = (uint16_t)c;
            {
                const uint32_t s = __reduce_add_sync(grp, head ? c : 0u);
                if (head && (uint32_t)(__ffs(grp) - 1) == lane && s)
                    atomicAdd(&o.aat[sg], (unsigned long long)s);
            }
            const bool sup = head && c >= P.T;
            uint32_t slot = 0;
            if (sup) {
                slot = atomicAdd(&o.sa_n[sg], 1u);
                o.sa_x[(size_t)sg * cols + slot] = atv & P.cmask;
            }
            unsigned sbits = __ballot_sync(FULL_MASK, sup);
            while (sbits) {
                // the g-bit active mask of one super ATV, for Algorithm 5;
                // all 32 lanes share its words (segment by segment in the tile)
                const uint32_t hl = __ffs(sbits) - 1;
                sbits &= sbits - 1;
                const uint32_t slot_a = __shfl_sync(FULL_MASK, slot, hl);
                const uint32_t a_s = hl / G.lpa;
                const uint32_t sg_a = (atv0 + a_s) >> P.c;
                for (uint32_t k = lane; k < P.mw; k += 32)
                    my_mask[k] = 0;
                __syncwarp();
                {
                    constexpr uint32_t F = 32 / WB;
                    for (uint32_t q = lane; q < P.Wd; q += 32) {
                        const uint32_t word = tile_word(tile_buf(b), a_s, q);
                        const uint32_t am = BG ? field_bits_bytes(word, cd_lo[didx(m, q)])
                                               : field_bits<WB>(word, load_desc(cd_lo, cd_hi, didx(m, q)));
                        if (am) {
                            const uint32_t pos = q * F, off = pos & 31;
                            atomicOr(&my_mask[pos >> 5], am << off);
                            if (off + F > 32 && (am >> (32 - off)))
                                atomicOr(&my_mask[(pos >> 5) + 1], am >> (32 - off));
                        }
                    }
                }
                __syncwarp();
                uint32_t *dst = o.sa_mask + ((size_t)sg_a * cols + slot_a) * P.mw;
                for (uint32_t k = lane; k < P.mw; k += 32)
                    dst[k] = my_mask[k];
                __syncwarp();
            }
        }

        if (FUSE && !P.ace) {
            // Algorithm 2 for the next slice on the words of the two refreshed blocks
            for (uint32_t rr = 0; rr < R.n_ranges; rr++) {
                // segments: the lane's own words of the range; interleaved: the
                // words of its chunks
                const uint32_t lo = ILV ? R.q_lo[rr] : max(R.q_lo[rr], q_first);
                const uint32_t hi = ILV ? R.q_hi[rr] + 1 : min(R.q_hi[rr] + 1, q_first + G.wseg);
                if (mine) {
                    for (uint32_t q = lo; q < hi; q++) {
                        if (ILV && ((q >> 2) & (G.lpa - 1)) != part)
                            continue;
                        const uint32_t w = tile_word(tile_buf(b), a, q);
                        const RangeDesc &rd = rdesc[q];
                        const uint32_t nw = BG ? refresh_bytes(P.k2, w, make_uint4(rd.lo1e, rd.hih1e, rd.lo1o, rd.hih1o))
                                               : refresh_swar<WB>(P, w, rd);
                        if (nw != w)
                            pool[(size_t)atv * P.Wd + q] = nw;
                    }
                }
            }
        }
        if (FUSE && P.ace) {
            // every aging counter loses one: decrement in place, store the segment back
            if (mine && !ILV) {
                for (uint32_t i = 0; i < G.wseg; i++)
                    row[i] = BG ? decay_bytes(row[i]) : decay_swar<WB>(row[i]);
                fence_async_smem();
                if (!whole)
                    bulk_store(pool + (size_t)atv * P.Wd + q_first, row, G.wseg * 4u);
            }
            if (ILV) {
                uint32_t *tb = tile_buf(b);
                for (uint32_t i = lane; i < n_atv * P.Wd; i += 32)
                    tb[i] = BG ? decay_bytes(tb[i]) : decay_swar<WB>(tb[i]);
                fence_async_smem();
            }
            if (whole) {
                __syncwarp();
                if (lane == 0)
                    bulk_store(pool + (size_t)atv0 * P.Wd, tile_buf(b), n_atv * P.Wd * 4u);
            }
        }
        // this buffer is free again: fetch the tile after next into it
        __syncwarp();
        tile = next;
        next = tile < ntiles ? tile + n_warps : ntiles;
        if (next < ntiles) {
            if (FUSE && P.ace)
                bulk_store_drain();  // this buffer's write-back has read its source
            fence_async_smem();
            __syncwarp();
            issue(next, b);
        }
        b ^= 1;
    }
    if (FUSE && P.ace)
        bulk_store_drain();
}

// ---------------------------------------------------------------- A3 alone

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
            const uint32_t a = act_of(P, c0n, pos_block(P, h));
            const uint32_t v = (word >> (j * WB)) & FM;
            out = (out & ~(FM << (j * WB))) | (preserve(P, v, a) << (j * WB));
        }
    }
    return out;
}

// One thread per (ATV, word of the two refreshed blocks).
template <int WB>
__global__ void __launch_bounds__(256) refresh_kernel(Params P, uint32_t *pool, const SliceCtl *ctl, uint32_t total_atv)
{
    const Refresh R = ctl->R;
    const uint32_t nw0 = R.n_ranges > 0 ? R.q_hi[0] - R.q_lo[0] + 1 : 0;
    const uint32_t nw1 = R.n_ranges > 1 ? R.q_hi[1] - R.q_lo[1] + 1 : 0;
    const uint64_t nw = nw0 + nw1;
    const uint64_t total = (uint64_t)total_atv * nw;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    if (P.hist) {
        // the window sums lose the phase that leaves the window (c0 - k + 1
        // mod 2k), and the slice counts of the opening slice's phase start
        // again from zero: every AT they counted (set 2k slices ago) has been
        // cleared by now
        const uint32_t c0 = ctl->c0;
        const uint32_t leave = c0 + P.k + 1 >= P.k2 ? c0 + P.k + 1 - P.k2 : c0 + P.k + 1;
        const uint16_t *hl = P.hist + (uint64_t)leave * total_atv;
        uint16_t *hz = P.hist + (uint64_t)R.c0n * total_atv;
        for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total_atv; i += stride) {
            P.hsum[i] = (uint16_t)(P.hsum[i] - hl[i]);
            hz[i] = 0;
        }
    }
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
        const uint4 b = make_uint4(decay_swar<WB>(a.x), decay_swar<WB>(a.y), decay_swar<WB>(a.z),
                                   decay_swar<WB>(a.w));
        if (a.x != b.x || a.y != b.y || a.z != b.z || a.w != b.w)
            pool[v] = b;
    }
}

}  // namespace

// Tile geometry of the scan for ATVs of Wd words: lanes per ATV (so a lane
// holds at most 48 words where Wd allows), the shared-memory stride of a lane's segment (an odd
// number of 16-byte units) and how many warps fit the shared memory.
ScanGeom scan_geometry(uint32_t Wd, uint32_t mw, uint32_t nw, size_t smem_limit)
{
    ScanGeom G{};
    G.lpa = 1;
    while (Wd / G.lpa > 48 && Wd % (8 * G.lpa) == 0 && G.lpa < 8)
        G.lpa *= 2;
    G.wseg = Wd / G.lpa;
    uint32_t units = G.wseg / 4;
    // Interleaved chunks where a segment would need padding and the ATV
    // length S = Wd/4 chunks keeps the chunks the 8 lanes of a quarter warp
    // read at once in distinct 16-byte bank groups: the quarter holds 8/lpa
    // ATVs whose lanes read chunks a*S + p (+ i*lpa), distinct mod 8 when S is
    // lpa times an odd number modulo 8 (any S with lpa = 8).
    const uint32_t S = Wd / 4;
    const bool ilv_ok = Wd % (4 * G.lpa) == 0 &&
                        (G.lpa == 8 || (G.lpa == 4 && S % 8 == 4) || (G.lpa == 2 && S % 4 == 2) ||
                         (G.lpa == 1 && S % 2 == 1));
    G.ilv = (units & 1) == 0 && ilv_ok ? 1u : 0u;
    if ((units & 1) == 0 && !G.ilv)
        units += 1;
    G.seg_stride = G.ilv ? G.wseg : units * 4;
    G.apt = 32 / G.lpa;
    G.tile_words = 32 * G.seg_stride;
    const size_t fixed = (size_t)nw * (Wd + G.lpa) * 2 * sizeof(uint4) + (size_t)Wd * sizeof(RangeDesc);
    auto head = [&](uint32_t warps) {
        const size_t h = fixed + 2 * warps * sizeof(uint64_t) + (size_t)warps * mw * 4;
        return (h + 127) / 128 * 128;
    };
    G.warps = scan_threads(G.ilv) / 32;
    while (G.warps > 1 && head(G.warps) + (size_t)G.warps * 2 * G.tile_words * 4 > smem_limit)
        G.warps--;
    G.tile_offset = (uint32_t)head(G.warps);
    G.smem = G.tile_offset + G.warps * 2 * G.tile_words * 4;
    return G;
}

namespace {

template <int NW>
cudaError_t launch_scan_nw(const Params &P, uint32_t w, uint32_t *pool, const ScanWindows &W, bool fuse,
                           const SliceCtl *ctl, int sms, cudaStream_t s)
{
    const uint32_t total = P.r << P.E_log2;
    const ScanGeom G = scan_geometry(P.Wd, P.mw, W.n, 200 * 1024);
    const uint32_t ntiles = (total + G.apt - 1) / G.apt;
    const bool bg = byte_guard(w, P.ace ? ASSE_COUNTER_ACE : ASSE_COUNTER_AT, P.k);
    return dispatch_w(w, [&](auto wb) {
        constexpr int WB = decltype(wb)::value;
        auto pick = [&](auto ilv) {
            constexpr bool ILV = decltype(ilv)::value;
            auto k = scan_kernel<WB, true, NW, false, ILV>;
            if constexpr (NW == 1) {
                if (!fuse)
                    k = scan_kernel<WB, false, 1, false, ILV>;
            }
            if constexpr (WB == 8) {
                if (bg) {
                    k = scan_kernel<8, true, NW, true, ILV>;
                    if constexpr (NW == 1) {
                        if (!fuse)
                            k = scan_kernel<8, false, 1, true, ILV>;
                    }
                }
            }
            return k;
        };
        auto kern = G.ilv ? pick(std::true_type()) : pick(std::false_type());
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G.smem);
        if (e != cudaSuccess)
            return e;
        const uint64_t want = (ntiles + G.warps - 1) / G.warps;
        const unsigned grid = (unsigned)(want < (uint64_t)sms ? (want < 1 ? 1 : want) : (uint64_t)sms);
        kern<<<grid, scan_threads(G.ilv), G.smem, s>>>(P, pool, W, ctl, total, G);
        return cudaGetLastError();
    });
}

}  // namespace

cudaError_t launch_scan(const Params &P, uint32_t w, uint32_t *pool, uint32_t kp, bool fuse, const SliceCtl *ctl,
                        const ScanOut &o, int sms, cudaStream_t s, uint64_t *launches)
{
    ScanWindows W{};
    W.n = 1;
    W.kp[0] = kp;
    W.o[0] = o;
    *launches += 1;
    return launch_scan_nw<1>(P, w, pool, W, fuse, ctl, sms, s);
}

cudaError_t launch_scan_windows(const Params &P, uint32_t w, uint32_t *pool, const ScanWindows &W,
                                const SliceCtl *ctl, int sms, cudaStream_t s, uint64_t *launches)
{
    if (W.n < 1 || W.n > (uint32_t)MAX_WINDOWS)
        return cudaErrorInvalidValue;
    *launches += 1;
    return launch_scan_nw<MAX_WINDOWS>(P, w, pool, W, true, ctl, sms, s);
}

cudaError_t launch_refresh(const Params &P, uint32_t w, uint32_t *pool, const SliceCtl *ctl, int sms, cudaStream_t s,
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
    *launches += 1;
    return dispatch_w(w, [&](auto wb) {
        constexpr int WB = decltype(wb)::value;
        const unsigned grid = (unsigned)sms * resident_blocks(refresh_kernel<WB>, 256, 0);
        refresh_kernel<WB><<<grid, 256, 0, s>>>(P, pool, ctl, total);
        return cudaGetLastError();
    });
}

}  // namespace asse
