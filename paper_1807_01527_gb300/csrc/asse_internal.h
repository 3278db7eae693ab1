// Internal declarations shared by the host API (asse_api.cu) and the kernel
// files (asse_ingest.cu, asse_scan.cu, asse_restore.cu, asse_probe.cu).  Not
// part of the ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/asse.h"
#include "../../include/asse_learn.h"

namespace asse {

// Launch-time constants of one pool, passed by value to every kernel.
struct Params {
    uint32_t k, k2, g, r, c, u, W, E_log2;
    uint32_t Wd;        // 32-bit words per ATV
    uint32_t A;         // mangling multiplier
    uint32_t cmask;     // 2^c - 1
    uint32_t T;         // super-ATV count threshold
    uint32_t theta;
    uint32_t ace;       // 1: aging counters
    uint32_t nf;        // frames 2^u
    uint32_t mw;        // 32-bit words of one active mask, ceil(g/32)
    uint32_t blk;       // ATs per ACT block: floor(g/2k)
    uint32_t F;         // fields per 32-bit word: floor(32/w)
    uint64_t blk_magic; // ceil(2^32 / blk)
    uint64_t Ainv;      // A^-1 mod p (may exceed 2^32)
    uint64_t bh_a, bh_b;
    uint32_t xshift[8]; // 2W - c - s*i: shift of the doubled LBS giving x_i
    // Table of the (aip, BH(bip)) keys set in the open slice, shared by every
    // ingest block: 2^klg 64-bit entries, each a tag of the key and the low
    // 32 bits of the slice (all ones = empty).  Null for a pool that fits in
    // the L2 cache.
    unsigned long long *keys;
    uint32_t klg;
    // ASSE_COUNTER_AT_HIST: per ATV, the ATs last set in each slice phase
    // t mod 2k, phase-major ([2k][r * E] 16-bit counts); null otherwise.
    uint16_t *hist;
    // ASSE_COUNTER_AT_HIST: per ATV ([r * E] 16-bit), the ATs set in the
    // latest k slices, i.e. the sum of the k latest phase counts, kept by the
    // ingest and the refresh so the close of a full window reads one count
    // per ATV; null otherwise.
    uint16_t *hsum;
    // CTAs of a thread-block cluster sharing the ingest's table of seen keys (1, 2, 4, 8)
    uint32_t cl;
    // 1: the 2k ACT blocks of an ATV are stored in pairs (block_slot below);
    // 0: AT h at position h (aging counters, the aligned variant)
    uint32_t paired;
};

// Storage order of the ACT blocks of a timestamp ATV with 2k blocks: block b
// and block b + k, which Algorithm 2 checks in the same slice (their ACTs
// differ by k), sit side by side: 0, k, 1, k + 1, ..., k - 1, 2k - 1.  Every
// block but the last holds blk ATs and the last (2k - 1) also comes last, so
// slot s starts at position s * blk.  A refresh then touches one stretch of
// each ATV instead of two stretches k blocks apart.
__host__ __device__ inline uint32_t block_slot(uint32_t k, uint32_t b)
{
    return b < k ? 2 * b : 2 * (b - k) + 1;
}

__host__ __device__ inline uint32_t slot_block(uint32_t k, uint32_t s)
{
    return (s & 1) ? k + (s >> 1) : s >> 1;
}

// Add delta to the 16-bit count hist[i] (a 32-bit atomic on the word that
// holds it; a count stays in 0..g, so its neighbour never sees a carry).
#ifdef __CUDACC__
__device__ __forceinline__ void hist_add(uint16_t *hist, uint64_t i, int delta)
{
    uint32_t *w = reinterpret_cast<uint32_t *>(hist + (i & ~1ull));
    atomicAdd(w, (uint32_t)delta << (16 * (uint32_t)(i & 1)));
}
#endif

// Bits of one counter field in the packed words: the counter's own width,
// ceil(log2(2k+1)) for timestamps (values 0..2k, Sec. 3) or ceil(log2(k+1))
// for aging counters (values 0..k), except that 7 becomes 8.  A word holds
// floor(32/7) = floor(32/8) = 4 fields either way, so the byte-wide fields
// cost no memory, and their top bit, never set by a 7-bit value, lets one
// SWAR step test all four fields of a word (asse_swar.cuh).
inline uint32_t packed_width(uint32_t counter, uint32_t k)
{
    uint32_t v = counter == ASSE_COUNTER_ACE ? k + 1 : 2 * k + 1, b = 0;
    while ((1u << b) < v)
        b++;
    if (b == 0)
        b = 1;
    return b == 7 ? 8 : b;
}

// Byte-wide fields whose values stay below 128 (packed_width turned 7 into
// 8): the scan tests them with the in-field guard bit.
inline bool byte_guard(uint32_t w, uint32_t counter, uint32_t k)
{
    return w == 8 && (counter == ASSE_COUNTER_ACE ? k : 2 * k) < 128;
}

// Key table size for a pool of n_atv ATVs: 4 entries per ATV, 2^17 .. 2^22,
// or none (0): with ASSE_KEYS_OFF, or with ASSE_KEYS_AUTO when the pool's
// bytes fit in an L2 cache of l2_bytes.  (At least 2^17 entries keeps a tag
// below 2^31, so no entry is all ones.)
inline uint32_t key_table_log2(unsigned long long n_atv, unsigned long long pool_bytes,
                               unsigned long long l2_bytes, uint32_t mode)
{
    if (mode == ASSE_KEYS_OFF || (mode == ASSE_KEYS_AUTO && pool_bytes <= l2_bytes))
        return 0;
    uint32_t lg = 17;
    while (lg < 22 && (1ull << lg) < 4 * n_atv)
        lg++;
    return lg;
}

// A bijection of the 48-bit value aip * 2^16 + h (h < 4096): two odd
// multiplications modulo 2^48, each followed by an xor-shift.  Its top klg
// bits pick the ingest's key table slot and the other 48 - klg bits are the
// tag, so (slot, tag) identifies the key exactly.
__host__ __device__ __forceinline__ unsigned long long key_mix(uint32_t aip, uint32_t h)
{
    constexpr unsigned long long M48 = (1ull << 48) - 1;
    unsigned long long x = ((unsigned long long)aip << 16) | h;
    x = (x * 0x9E3779B97F4Bull) & M48;
    x ^= x >> 23;
    x = (x * 0xC2B2AE3D27D5ull) & M48;
    x ^= x >> 21;
    return x;
}

// Device-resident status of one close, reset by every scan.
struct Status {
    unsigned long long n_csip;    // candidates restored (Algorithm 4)
    unsigned long long n_report;  // candidates with estimate >= theta
    unsigned long long needed;    // tuples the overflowing join level needed
    unsigned int overflow;        // a frame exceeded the restore capacity
    unsigned int error;           // a device-side wait gave up (bounded mbarrier wait)
    unsigned int pad[4];
};

// A partial or complete column tuple of the restore join.
struct Tuple {
    uint32_t L;       // bits of LBS known so far
    uint32_t known;   // positions of LBS covered so far
    uint16_t slot[8]; // index in SA(i, frame) of each row's column
};

// Word ranges of one refresh: fields [h_lo[b], h_hi[b]) of ACT block b get
// Algorithm 2 with new ACT act[b]; words [q_lo[b], q_hi[b]] hold them.
struct Refresh {
    uint32_t c0n;      // ACT of block 0 in the new slice
    uint32_t q_lo[2], q_hi[2];
    uint32_t n_ranges; // 0, 1 or 2 distinct word ranges
};

// Tile geometry of the scan kernel (asse_scan.cu).
struct ScanGeom {
    uint32_t lpa;         // lanes per ATV
    uint32_t apt;         // ATVs per warp tile (32 / lpa)
    uint32_t wseg;        // words per lane segment (Wd / lpa)
    uint32_t seg_stride;  // shared-memory words per lane segment (odd number of 16-byte units)
    uint32_t tile_words;  // 32 * seg_stride
    uint32_t warps;       // warps per CTA that stream tiles
    uint32_t tile_offset; // byte offset of the tile buffers in dynamic shared memory
    uint32_t smem;        // dynamic shared memory bytes
    uint32_t ilv;         // 1: interleaved chunks (lane p of an ATV owns its 16-byte chunks p, p + lpa, ...;
                          //    the tile is apt whole ATVs back to back, one bulk copy); 0: lane segments
};
// nw windows: the count ranges of every window are kept in shared memory
ScanGeom scan_geometry(uint32_t Wd, uint32_t mw, uint32_t nw, size_t smem_limit);

// Slice-dependent launch arguments, kept in device memory so that a captured
// CUDA graph replays unchanged from slice to slice: the open slice, the ACT
// of its block 0, and the words Algorithm 2 checks when the next slice opens.
struct SliceCtl {
    unsigned long long t;
    uint32_t c0;
    uint32_t pad;
    Refresh R;
};

// Words holding the ACT blocks whose ACT becomes 0 or k when slice t_new
// opens.  Blocks are contiguous runs of ATs: the first 2k-1 of blk ATs, the
// last the rest of g; paired: stored in the order of block_slot, which puts
// the two blocks side by side (one range).  blk == g is the aligned variant:
// the ATV is one block with ACT C0, which reaches 0 or k once every k slices
// (no range in between).
__host__ __device__ inline Refresh refresh_for(uint32_t k, uint32_t g, uint32_t blk, uint32_t F,
                                               unsigned long long t_new, bool paired)
{
    const uint32_t k2 = 2 * k;
    const uint32_t nblk = blk >= g ? 1 : k2;
    Refresh R{};
    R.c0n = (uint32_t)(t_new % k2);
    const uint32_t b[2] = {(k2 - R.c0n) % k2, (k + k2 - R.c0n) % k2};
    uint32_t lo[2] = {0, 0}, hi[2] = {0, 0}, n = 0;
    for (int i = 0; i < 2; i++) {
        if (b[i] >= nblk)
            continue;
        const uint32_t sl = paired ? block_slot(k, b[i]) : b[i];
        const uint32_t flo = sl * blk, fhi = sl == nblk - 1 ? g : (sl + 1) * blk;
        lo[n] = flo / F;
        hi[n] = (fhi - 1) / F;
        n++;
    }
    if (n < 2) {
        R.q_lo[0] = lo[0];
        R.q_hi[0] = hi[0];
        R.n_ranges = n;
        return R;
    }
    if (lo[1] < lo[0]) {
        const uint32_t a = lo[0], c = hi[0];
        lo[0] = lo[1];
        hi[0] = hi[1];
        lo[1] = a;
        hi[1] = c;
    }
    if (lo[1] <= hi[0] + 1) {
        R.q_lo[0] = lo[0];
        R.q_hi[0] = hi[1] > hi[0] ? hi[1] : hi[0];
        R.n_ranges = 1;
    } else {
        R.q_lo[0] = lo[0];
        R.q_hi[0] = hi[0];
        R.q_lo[1] = lo[1];
        R.q_hi[1] = hi[1];
        R.n_ranges = 2;
    }
    return R;
}

__host__ __device__ inline SliceCtl slice_ctl(const Params &P, unsigned long long t)
{
    SliceCtl c{};
    c.t = t;
    c.c0 = (uint32_t)(t % P.k2);
    c.R = refresh_for(P.k, P.g, P.blk, P.F, t + 1, P.paired != 0);
    return c;
}

#ifdef __CUDACC__
// Open the slice after ctl->t; every thread of one block calls this.  The
// ingest's key table tags its entries with the low 32 bits of the slice, so
// when those wrap to 0 the block empties the table: entries of the previous
// 2^32 slices would otherwise match again.
__device__ inline void open_next_slice(const Params &P, SliceCtl *ctl)
{
    const unsigned long long tn = ctl->t + 1;
    __syncthreads();
    if (threadIdx.x == 0)
        *ctl = slice_ctl(P, tn);
    if ((uint32_t)tn == 0 && P.keys != nullptr)
        for (uint32_t i = threadIdx.x; i < (1u << P.klg); i += blockDim.x)
            P.keys[i] = ~0ull;
}
#endif

struct ScanOut {
    uint16_t *cnt;
    unsigned long long *aat;
    uint32_t *sa_n, *sa_x, *sa_mask;
    Status *status;
};

// Kernel launchers (asse_ingest.cu, asse_scan.cu, asse_restore.cu).  Each returns the cudaError_t of its
// launch and adds the number of kernels it launched to *launches.
// n pairs, or (n_dev != null) as many as *n_dev says at run time.
cudaError_t launch_ingest(const Params &P, uint32_t w, uint32_t *pool, const uint32_t *pairs, uint64_t n,
                          const unsigned long long *n_dev, const SliceCtl *ctl, int sms, cudaStream_t s,
                          uint64_t *launches);
// Open the next slice on the device: ctl = slice_ctl(ctl->t + 1).
cudaError_t launch_advance_ctl(const Params &P, SliceCtl *ctl, cudaStream_t s, uint64_t *launches);
cudaError_t launch_reset(unsigned long long *aat, uint32_t *sa_n, uint32_t nseg, Status *status, cudaStream_t s,
                         uint64_t *launches);
cudaError_t launch_scan(const Params &P, uint32_t w, uint32_t *pool, uint32_t kp, bool fuse, const SliceCtl *ctl,
                        const ScanOut &o, int sms, cudaStream_t s, uint64_t *launches);
// Several windows k' (Sec. 3: the same ATs answer every k' <= k) counted in
// one pass over the pool, each into its own outputs; fused refresh.
constexpr int MAX_WINDOWS = ASSE_MAX_WINDOWS;
struct ScanWindows {
    uint32_t n;
    uint32_t kp[MAX_WINDOWS];
    ScanOut o[MAX_WINDOWS];
};
cudaError_t launch_scan_windows(const Params &P, uint32_t w, uint32_t *pool, const ScanWindows &W,
                                const SliceCtl *ctl, int sms, cudaStream_t s, uint64_t *launches);
cudaError_t launch_refresh(const Params &P, uint32_t w, uint32_t *pool, const SliceCtl *ctl, int sms, cudaStream_t s,
                           uint64_t *launches);
// advance (may be null): the restore also opens the next slice, as
// launch_advance_ctl would (the fused close saves that launch).
cudaError_t launch_restore(const Params &P, const ScanOut &o, Tuple *scratch, uint32_t cap, asse_superpoint *csip,
                           asse_superpoint *report, uint64_t out_cap, cudaStream_t s, uint64_t *launches,
                           SliceCtl *advance = nullptr);
cudaError_t launch_estimate(const Params &P, uint32_t w, const uint32_t *pool, uint32_t c0, uint32_t kp,
                            const unsigned long long *aat, const uint32_t *aips, uint64_t n, asse_superpoint *out,
                            int sms, cudaStream_t s, uint64_t *launches);

// ASSE_COUNTER_AT_HIST (asse_hist.cu): the scan of a pool with slice counts
// (|ATV|^{k'} from the counts of the k' latest phases, row-frame loads,
// super ATVs and their masks from their words), and the rebuild of the
// counts from the pool's words (asse_load).
// fuse: the close of a slice (refresh of the checked blocks and zeroing of
// the opening phase's counts in the same pass).
cudaError_t launch_hist_scan(const Params &P, uint32_t w, uint32_t *pool, uint32_t kp, bool fuse, const SliceCtl *ctl,
                             const ScanOut &o, int sms, cudaStream_t s, uint64_t *launches);
cudaError_t launch_hist_rebuild(const Params &P, uint32_t w, const uint32_t *pool, const SliceCtl *ctl, int sms,
                                cudaStream_t s, uint64_t *launches);

// At least n_reads random 4-byte reads of buf[0, n_words) on stream s, with
// every SM busy (asse_probe.cu); *issued receives the number launched.
cudaError_t launch_random_reads(const uint32_t *buf, uint64_t n_words, uint64_t n_reads, int sms, cudaStream_t s,
                                uint64_t *launches, uint64_t *issued);

// What asse_restore_static (asse_static.cu) needs from a pool: the launch
// constants, the last scan's outputs and the stream.  Returns ASSE_ESTATE if
// the pool has no scan to restore from.
struct RestoreView {
    Params P;
    ScanOut o;
    cudaStream_t stream;
    uint64_t *launches;
};
int pool_restore_view(asse_pool *p, RestoreView *v);

// What asse_features (asse_learn.cu) needs: the live pool state of the open
// slice and the last scan's window and loads.  ESTATE unless the pool was
// scanned and neither refreshed nor ingested into since.
struct FeatureView {
    Params P;
    uint32_t w;
    const uint32_t *pool;
    uint32_t c0, kp;
    const SliceCtl *ctl;  // non-null: the kernel reads c0 from the device slice state (graph replays)
    const unsigned long long *aat;
    const uint16_t *cnt;  // |ATV|^{k'} of every ATV, from the same scan
    cudaStream_t stream;
    uint64_t *launches;
    int sms;
};
int pool_feature_view(asse_pool *p, FeatureView *v);
// The view of a close enqueued by pool_enqueue_scan: no host bookkeeping
// checks, C0 from the device slice state.
FeatureView pool_feature_view_device(asse_pool *p, uint32_t kp);
// Enqueue the feature rows of every ATV (asse_features.cu).
cudaError_t launch_features(const FeatureView &v, uint16_t *x_dev);
// Enqueue on v.stream the learned estimate of every ATV of the view: feature
// rows into x_dev, the model, and est_dev = exp(model) inside the training
// range, else Eq. 2 (asse_estimate_learned's rule); *nfb_dev counts the
// fallbacks.  The model's parameters are only read (asse_learn.cu).
int mlp_enqueue_learned(asse_mlp *m, const FeatureView &v, float max_log_n, uint16_t *x_dev, float *est_dev,
                        uint32_t *nfb_dev, std::string *why);
int pool_fail(asse_pool *p, int code, const std::string &msg);

// Pieces of asse_close_slice / asse_ingest for the server (asse_serve.cu),
// which captures them into CUDA graphs: enqueue the device work of a close
// (no host bookkeeping), do the host bookkeeping of one close, and enqueue an
// ingest whose pair count is read from device memory.
int pool_enqueue_close(asse_pool *p, uint32_t kp, bool timed = false);
// The same close in three parts, for a close with learned inference between
// the scan and the refresh (the refresh changes the state the features read):
// the scan alone, then (after the caller's work) the restore, the refresh and
// the opening of the next slice.
int pool_enqueue_scan(asse_pool *p, uint32_t kp);
int pool_enqueue_restore_refresh(asse_pool *p);
void pool_after_close(asse_pool *p, uint32_t kp);
int pool_enqueue_ingest(asse_pool *p, const uint32_t *pairs_dev, const unsigned long long *n_dev);
struct PoolBuffers {
    Status *status;
    asse_superpoint *report;
    uint64_t out_cap;
    cudaStream_t stream;
    uint32_t cap;
};
PoolBuffers pool_buffers(asse_pool *p);
uint64_t pool_device_bytes(const asse_config *cfg);

}  // namespace asse
