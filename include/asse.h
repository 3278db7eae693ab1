/*
 * asse.h -- C ABI of the GB300 (sm_103a) ASSE library: sliding-window
 * super-point detection and cardinality estimation with asynchronous
 * timestamps (Xu, arXiv 1807.01527).
 *
 * One pool (an "ATV cube": r rows x 2^(c+u) ATVs x g ATs, Sec. 4) lives in
 * device memory owned by the library.  A slice is processed as
 *
 *     asse_ingest(...)       any number of batches of (aip, bip) pairs
 *     asse_close_slice(...)  scan + refresh + restore + estimate, then the
 *                            next slice opens
 *     asse_report(...)       read the super points of the window just closed
 *
 * or, step by step, asse_scan -> asse_restore -> [asse_estimate] ->
 * asse_advance (identical results; close_slice fuses the refresh into the
 * scan).
 *
 * Conventions for every entry point:
 *  - Return value: ASSE_OK (0) or one of the ASSE_E* codes; no exception or
 *    device trap ever crosses the ABI.  asse_last_error() returns a message
 *    for the last failing call on a pool.
 *  - Pointers are plain host or device addresses; `where` says which
 *    (ASSE_HOST / ASSE_DEVICE).  The caller owns every buffer it passes.
 *  - All work is enqueued on the pool's CUDA stream (a cudaStream_t passed as
 *    void*; NULL = the legacy default stream) and is asynchronous unless the
 *    entry point says it synchronises.
 *  - A pool is not thread-safe; distinct pools may be used from distinct
 *    threads and streams.
 */
#ifndef ASSE_H
#define ASSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define ASSE_API __attribute__((visibility("default")))
#else
#define ASSE_API
#endif

/* Status codes. */
#define ASSE_OK 0
#define ASSE_EINVAL 1    /* invalid argument or parameter combination */
#define ASSE_ENOMEM 2    /* device or host allocation failed */
#define ASSE_ECAPACITY 3 /* an output or the restore scratch is too small */
#define ASSE_ECUDA 4     /* a CUDA runtime call or kernel launch failed */
#define ASSE_ESTATE 5    /* call out of order (e.g. restore before scan) */
/* 6 is ASSE_EAGAIN of asse_serve.h. */
#define ASSE_ETIMEOUT 7  /* a bounded device-side wait gave up: a bulk copy or a
                          * tensor-core pipeline stage did not complete within
                          * about 2 s of SM clock.  The kernel returned instead
                          * of hanging and the CUDA context stays usable, but the
                          * outputs of that work are invalid (reload the pool
                          * from a snapshot or recreate it). */

/* Buffer locations. */
#define ASSE_HOST 0
#define ASSE_DEVICE 1

/* Counter kinds. */
#define ASSE_COUNTER_AT 0  /* asynchronous timestamp, log2(2k+1) bits (Sec. 3) */
#define ASSE_COUNTER_ACE 1 /* aging counter, log2(k+1) bits, decremented every slice (Sec. 2.3) */
/* Asynchronous timestamps with one ACT for the whole ATV (all 2k blocks of
 * Sec. 3 aligned): the same counters and Algorithms 1-3, but preserveAT reaches
 * every AT at once, at the slices where C0 = t mod 2k is 0 or k, instead of two
 * of 2k blocks every slice.  Results equal the staggered pool's; the refresh
 * work comes in bursts of the whole pool every k slices. */
#define ASSE_COUNTER_AT_ALIGNED 2
/* Asynchronous timestamps (exactly ASSE_COUNTER_AT's counters, layout and
 * results) plus, for every ATV, how many of its ATs each of the last 2k
 * slices set (2k 16-bit counts, one per slice phase t mod 2k), kept by the
 * ingest: a field that changes is set with a compare-and-swap, which returns
 * its old value, and the counts of the old and the new slice are moved.  The
 * close then counts |ATV|^{k'} from the k' latest counts instead of reading
 * every AT (Sec. 3: the window's active ATs are those set in its slices), and
 * reads AT words only for the super ATVs and the two blocks preserveAT
 * checks.  A count is zeroed when its phase comes round again (every AT it
 * counted has been cleared by then, Algorithm 2), so ATs cleared by the
 * refresh need no update.  A running sum of the k latest counts per ATV
 * (kept by the ingest and the refresh) answers the full window k' = k with
 * one read.  Costs 4k + 2 bytes per ATV. */
#define ASSE_COUNTER_AT_HIST 3

/* Flags of asse_superpoint. */
#define ASSE_SP_SATURATED 1u /* NAT == g: Eq. 4 is +infinity */
#define ASSE_SP_REPORTED 2u  /* estimate >= theta */
#define ASSE_SP_LEARNED 4u   /* est is the learned candidate estimate (asse_report_learned), not Eq. 4 */

/* Pool parameters (Sec. 3 and Sec. 4.1).
 *  k       window size in slices (1..127); AT values are 0..2k, 2k inactive.
 *  theta   super-point threshold on the cardinality (Sec. 2.1).
 *  g       ATs per ATV, 2k <= g <= 4096 and g <= 512 * floor(32/w) (an ATV
 *          fits in 512 words).  The 2k ACT blocks are contiguous runs of
 *          AT indices: the first 2k-1 hold floor(g/2k) ATs each, the last
 *          the rest (their storage order: asse_pool_info.paired).
 *  r       rows, 2..8.
 *  c       column-index bits (ATVs per row and frame = 2^c), 1..16.
 *  u       frame bits (frames = 2^u), 0..8; c + u <= 24.
 *  s       offset between consecutive rows' column windows on LBS(f, 32-u):
 *          1 <= s <= c, s*(r-1) < 32-u, and c + s*(r-1) >= 32-u
 *          (completeness, Sec. 4.1).
 *  A       mangling multiplier of f(aip) = A*aip mod (2^32+15), 2 <= A < 2^32.
 *  bh_a    BH multiplier (must be odd), bh_b BH offset:
 *          BH(bip) = (hi32(bh_a*bip + bh_b mod 2^64) * g) >> 32.
 *  counter ASSE_COUNTER_AT, ASSE_COUNTER_ACE, ASSE_COUNTER_AT_ALIGNED or
 *          ASSE_COUNTER_AT_HIST.
 *  restore_cap  column tuples held per frame at any join level of the
 *          restore; 0 selects 4096.  The candidate lists hold up to
 *          restore_cap * 2^u entries.
 *  max_batch    device staging capacity in pairs for ASSE_HOST ingest
 *          (copied in chunks of this size); 0 selects 4 Mi.
 *  key_table    ASSE_KEYS_AUTO, ASSE_KEYS_ON or ASSE_KEYS_OFF: whether the
 *          ingest keeps a device table of the (aip, BH(bip)) keys already set
 *          in the open slice (4 entries of 8 bytes per ATV, 1 to 32 MiB), so
 *          that a key repeated across the SMs reaches the pool once.  AUTO
 *          keeps one when the pool is larger than the device's L2 cache (the
 *          repeats then cost DRAM sectors); with the pool in L2 a pool word
 *          costs what a table entry costs.  Results are the same either way.
 *  cluster CTAs of a thread-block cluster that share one table of the keys
 *          their ingest has seen (each CTA's shared-memory table holds the
 *          keys that hash to it, reached by the others through distributed
 *          shared memory), so that a key repeated across those SMs is set
 *          once: ASSE_CLUSTER_AUTO (0, no sharing), or 1 (no sharing), 2, 4
 *          or 8.  Results are the same either way; on a GB300 the remote
 *          lookup of every pair costs more than the repeats it removes, so
 *          AUTO does not share.
 */
typedef struct asse_config {
    uint32_t k, theta, g, r, c, u, s, A;
    uint64_t bh_a, bh_b;
    uint32_t counter;
    uint32_t restore_cap;
    uint64_t max_batch;
    uint32_t key_table;
    uint32_t cluster;
} asse_config;

/* Value of asse_config.cluster that lets the library choose. */
#define ASSE_CLUSTER_AUTO 0

/* Values of asse_config.key_table. */
#define ASSE_KEYS_AUTO 0
#define ASSE_KEYS_ON 1
#define ASSE_KEYS_OFF 2

/* One candidate or reported super point (Sec. 4.2-4.3). */
typedef struct asse_superpoint {
    uint32_t aip;   /* restored host address */
    uint32_t nat;   /* NAT(aip), Algorithm 5 */
    float est;      /* Eq. 4 estimate, stored FP32: evaluated in FP32 where an error bound keeps
                     * it within 8e-6 relative of the FP64 value, else in FP64; +inf if saturated */
    uint32_t flags; /* ASSE_SP_* */
} asse_superpoint;

/* Derived layout of a pool, for callers that read the packed state. */
typedef struct asse_pool_info {
    uint32_t w;          /* bits per packed counter field: ceil(log2(2k+1)) (AT) or ceil(log2(k+1))
                          * (ACE), except 8 where that is 7 (four byte-wide fields per word, as many
                          * as 7-bit fields would give; the top bit of each byte stays 0) */
    uint32_t fields;     /* counters per 32-bit word: floor(32/w); the counter at position p of an
                          * ATV is field p % fields, bits [j*w, j*w+w), of its word p / fields */
    uint32_t words;      /* 32-bit words per ATV, ceil(g/fields) rounded up to a multiple of 8 */
    uint32_t E;          /* ATVs per row: 2^(c+u); ATV index in a row = (frame << c) | column */
    uint32_t threshold;  /* super-ATV count threshold ceil(g - g*exp(-theta/g)) (Sec. 4.2) */
    uint32_t block;      /* ATs per ACT block: floor(g/2k) (g for ASSE_COUNTER_AT_ALIGNED); block b
                          * holds ATs [b*block, (b+1)*block) and the last of the 2k blocks the rest of g */
    uint32_t k;          /* slices per window (cfg k) */
    uint32_t paired;     /* 1 (ASSE_COUNTER_AT, ASSE_COUNTER_AT_HIST): the 2k blocks are stored in the
                          * order 0, k, 1, k+1, ..., k-1, 2k-1, so the two blocks one refresh
                          * (Algorithm 2) checks are adjacent: AT h of block b sits at position
                          * h - b*block + s*block, s = 2b (b < k) or 2(b-k)+1; 0: AT h at position h */
    uint64_t slice;      /* index of the open slice (0 after create) */
    uint64_t pool_words; /* r * E * words */
    const uint32_t *pool;/* device address of the packed pool, [r][E][words] */
} asse_pool_info;

typedef struct asse_pool asse_pool;

/* Create a pool: validate cfg, allocate the device state, InitAT every
 * counter (Sec. 3: value 2k; ACE: 0), open slice 0.  stream is the
 * cudaStream_t all later work of this pool is enqueued on.  Synchronises.
 * Errors: EINVAL (cfg), ENOMEM, ECUDA.  *out is NULL on error. */
ASSE_API int asse_create(const asse_config *cfg, void *stream, asse_pool **out);

/* Free every device and host resource of the pool (NULL is ignored).
 * Synchronises the pool's stream first. */
ASSE_API void asse_destroy(asse_pool *pool);

/* Change the stream later work is enqueued on. */
ASSE_API int asse_set_stream(asse_pool *pool, void *stream);

/* Algorithm 3 (Scan IP pair, Sec. 4.1) on n pairs of the open slice.
 * pairs: n (aip, bip) uint32 pairs, interleaved (aip0, bip0, aip1, ...).
 *   ASSE_DEVICE: a device address, 16-byte aligned, that must stay valid
 *   until the stream reaches this work; nothing is copied.
 *   ASSE_HOST: host memory (pinned memory gives full copy-engine bandwidth),
 *   copied in max_batch chunks into device staging, the copy of chunk i+1
 *   overlapping the ingest of chunk i.  The call returns once the last chunk
 *   is copied: the host buffer may then be reused, and the ingest of the last
 *   chunk (and a close queued after it) run on while the caller prepares its
 *   next batch.
 * Order and repetition of pairs within a slice do not change the result.
 * Errors: EINVAL (NULL with n > 0, misalignment), ECUDA. */
ASSE_API int asse_ingest(asse_pool *pool, const uint32_t *pairs, uint64_t n, int where);

/* Close the open slice for the window of the latest kp slices (1 <= kp <= k):
 * the per-ATV active counts |ATV|^{k'} (Algorithm 1, Sec. 3), the row-frame
 * loads |AAT(k',i,j)| (Sec. 4.3), the super ATVs SA(i,j) (Sec. 4.2), with
 * preserveAT (Algorithm 2) for the next slice fused into the same pass; then
 * the restore (Algorithm 4) and, for every candidate, NAT (Algorithm 5) and
 * Eq. 4; then slice t+1 opens.  Asynchronous.  A restore that needs more
 * than restore_cap tuples is reported by asse_report / asse_candidates.
 * Errors: EINVAL (kp), ECUDA. */
ASSE_API int asse_close_slice(asse_pool *pool, uint32_t kp);

#define ASSE_MAX_WINDOWS 4

/* asse_close_slice for several windows at once: the same ATs answer every
 * window k' <= k (Sec. 3, Algorithm 1), so one pass over the pool counts
 * |ATV|^{k'} for each kps[i] (1 <= kps[i] <= k, 1 <= n_windows <=
 * ASSE_MAX_WINDOWS), with the refresh fused as in asse_close_slice; then the
 * restore, NAT and Eq. 4 of each window; then slice t+1 opens.  The first
 * call with a given number of windows allocates the extra windows' outputs
 * (the size of asse_close_slice's outputs each).  Results of window i are read
 * with asse_report, asse_candidates, asse_counts and asse_loads after
 * asse_select_window(pool, i); window 0 is selected on return.  Asynchronous.
 * Errors: EINVAL (kps, n_windows), ENOMEM, ECUDA. */
ASSE_API int asse_close_slice_multi(asse_pool *pool, const uint32_t *kps, uint32_t n_windows);

/* Make the readers (asse_report, asse_candidates, asse_counts, asse_loads)
 * return window `window` of the last close.  Errors: EINVAL (window >= the
 * number of windows of the last close; a plain close or scan has one). */
ASSE_API int asse_select_window(asse_pool *pool, uint32_t window);

/* Stepwise close, part 1: the scan of asse_close_slice without the refresh.
 * The pool state is unchanged.  Asynchronous.  Errors: EINVAL, ECUDA. */
ASSE_API int asse_scan(asse_pool *pool, uint32_t kp);

/* Stepwise close, part 2: Algorithm 4, Algorithm 5 and Eq. 4 on the super
 * ATVs of the last scan.  Asynchronous.  Errors: ESTATE (no scan), ECUDA. */
ASSE_API int asse_restore(asse_pool *pool);

/* Size of the fixed restore scratch of asse_restore_static, in column tuples. */
#define ASSE_STATIC_RESTORE_TUPLES 131072u

/* No counterpart in the paper: the restore of asse_restore, for callers that
 * cannot allocate device memory while they run it.  A slice-closing loop with
 * a latency budget cannot call cudaMalloc or cudaFree, since those may
 * synchronise the device and stall the streams that feed it, and some hosts
 * give all device memory to another allocator at start-up so that nothing may
 * be allocated later.  This call allocates nothing and calls no allocating
 * routine: the join's partial column tuples live in one array of
 * ASSE_STATIC_RESTORE_TUPLES tuples (3 MiB) compiled into the library, which
 * every GPU that loads the library holds until the process exits.
 *
 * It restores the window selected by asse_select_window (window 0 after a
 * scan or a single-window close) from the outputs of the last scan or close.
 *
 *  tuples_per_frame  tuples kept per frame and join level (the role of
 *                    restore_cap); tuples_per_frame * 2 * 2^u must not exceed
 *                    ASSE_STATIC_RESTORE_TUPLES, else ASSE_EINVAL.
 *  candidates, reported  device arrays of cap records each: every restored
 *                    candidate, and those whose estimate is >= theta, in
 *                    unspecified order (as asse_candidates / asse_report).
 *  counters          device array of 4 uint64_t, zeroed by this call and then
 *                    filled by the kernel: [0] candidates, [1] reported,
 *                    [2] tuples an overflowing frame needed, [3] non-zero if
 *                    a frame overflowed tuples_per_frame (the lists are then
 *                    incomplete).  Counts above cap mean the lists were cut.
 * Asynchronous on the pool's stream.  The first call on a device (with that
 * device current) looks up the scratch array's device address and caches it;
 * make that first call before any stream capture.  Every call shares the one
 * array: two calls whose kernels overlap on a GPU (different streams or
 * pools) race on it and must be ordered by the caller.
 * Errors: EINVAL (NULL or oversized arguments), ESTATE (no scan), ECUDA. */
ASSE_API int asse_restore_static(asse_pool *pool, uint32_t tuples_per_frame, asse_superpoint *candidates,
                                 asse_superpoint *reported, uint64_t cap, uint64_t *counters);

/* Stepwise close, part 3: preserveAT (Algorithm 2) on the two ACT blocks of
 * every ATV whose ACT becomes 0 or k in the next slice (AT pool), or the
 * per-slice decrement of every aging counter (ACE pool); then the next
 * slice opens.  Asynchronous.  Errors: ECUDA. */
ASSE_API int asse_advance(asse_pool *pool);

/* Sec. 4.3 for arbitrary hosts: NAT (Algorithm 5) and Eq. 4 of each of the
 * n addresses in aips, for the window and loads of the last scan.  Must run
 * after asse_scan and before asse_advance (the refresh changes the state).
 * aips and out live at `where` (both host or both device); out[i].flags has
 * ASSE_SP_REPORTED when est >= theta.  Host buffers synchronise.
 * Errors: ESTATE, EINVAL, ECUDA. */
ASSE_API int asse_estimate(asse_pool *pool, const uint32_t *aips, uint64_t n, asse_superpoint *out, int where);

/* Read the super points reported by the last close/restore: the candidates
 * whose Eq. 4 estimate is >= theta, in unspecified order.  Copies
 * min(count, cap) entries to out (host or device), stores the count in
 * *n_out, and waits for them.  After asse_close_slice, a host read of up to
 * 4,096 entries waits only for that close (work queued on the stream after
 * it, such as the next batch's ingest, keeps running); otherwise the call
 * synchronises the stream.  Returns ECAPACITY if cap < count, or
 * if the restore overflowed restore_cap (then *n_out is the number of
 * column tuples the overflowing join level needed, a lower bound on the
 * capacity to configure, and out is not written).  Errors: ESTATE,
 * ETIMEOUT (a bounded wait of the scan gave up; the lists are invalid), ECUDA. */
ASSE_API int asse_report(asse_pool *pool, asse_superpoint *out, uint64_t cap, uint64_t *n_out, int where);

/* As asse_report, but every restored candidate (CSIP, Algorithm 4), reported
 * or not. */
ASSE_API int asse_candidates(asse_pool *pool, asse_superpoint *out, uint64_t cap, uint64_t *n_out, int where);

/* Per-ATV active counts of the last scan, r*E uint16 ([row][ATV]), copied to
 * out at `where`.  Host copies synchronise.  Errors: ESTATE, ECUDA. */
ASSE_API int asse_counts(asse_pool *pool, uint16_t *out, int where);

/* Row-frame loads |AAT(k',i,j)| of the last scan, r*2^u uint64 ([row][frame]),
 * copied to host memory.  Synchronises.  Errors: ESTATE, ECUDA. */
ASSE_API int asse_loads(asse_pool *pool, uint64_t *out);

/* Layout of the packed pool and the open slice index. */
ASSE_API int asse_info(const asse_pool *pool, asse_pool_info *out);

/* Copy the packed pool (pool_words uint32) to out at `where`.  Host copies
 * synchronise.  Errors: ECUDA. */
ASSE_API int asse_read_pool(asse_pool *pool, uint32_t *out, int where);

/* Checkpoint: write a self-describing image of the pool (header with cfg and
 * slice index, then the packed words) to host memory dst of cap bytes.
 * *n_out receives the image size; with dst == NULL only the size is
 * returned.  Synchronises.  Errors: ECAPACITY (cap too small), ECUDA. */
ASSE_API int asse_snapshot(asse_pool *pool, void *dst, uint64_t cap, uint64_t *n_out);

/* Restore a pool from an image written by asse_snapshot of a pool with the
 * same cfg (checked).  Synchronises.  Errors: EINVAL (mismatch), ECUDA. */
ASSE_API int asse_load(asse_pool *pool, const void *src, uint64_t n);

/* Measurement aid, no counterpart in the paper: enqueue on the pool's stream
 * at least n_reads (<= 2^34) independent random 4-byte reads of the pool's
 * own packed words (one 32-byte sector each, spread over every SM), and
 * store the number actually issued in *n_issued (may be NULL).  The pool is
 * not changed.  Timed by the caller with events around the call, this gives
 * the random-sector read rate of a buffer of the pool's size, in L2 or in
 * HBM as the pool is: the random-access roofline of the ingest, whose pool
 * traffic is r random words per pair new to the slice.  Does not
 * synchronise.  Errors: EINVAL, ECUDA. */
ASSE_API int asse_probe_random_reads(asse_pool *pool, uint64_t n_reads, uint64_t *n_issued);

/* Self-test of the device-side waits, no counterpart in the paper: the
 * kernels that stage data with bulk copies or drive the tensor cores wait on
 * mbarriers with a bound, and report ASSE_ETIMEOUT instead of hanging when a
 * wait gives up.  This call runs that wait once in a one-thread kernel on
 * `stream` (a cudaStream_t as void*, NULL = legacy default stream), on an
 * mbarrier that the kernel completes first if `complete` != 0 and that
 * nothing completes otherwise, with a bound of limit_cycles SM clock cycles
 * (1 .. 2^36).  *cycles_waited (may be NULL) receives the cycles the wait
 * took.  The result travels through one fixed device variable, so calls
 * that overlap on a device race on it.  Synchronises the stream.
 * Returns ASSE_OK if the wait completed, ASSE_ETIMEOUT if it gave up.
 * Errors: EINVAL (limit out of range), ECUDA. */
ASSE_API int asse_probe_bounded_wait(void *stream, uint64_t limit_cycles, int complete, uint64_t *cycles_waited);

/* Measurement aid, no counterpart in the paper: with on != 0, every later
 * asse_close_slice records CUDA events on the pool's stream before and after
 * its scan kernel and after its restore kernel (the work of the close that
 * runs on the device), for asse_close_timing.  on = 0 stops recording.
 * Errors: ECUDA (event creation). */
ASSE_API int asse_set_timing(asse_pool *pool, int on);

/* Device time of the last asse_close_slice recorded with timing on, in
 * milliseconds: ms[0] the scan (Algorithm 1 counts, loads, super ATVs and the
 * fused Algorithm 2 refresh), ms[1] the restore (Algorithms 4-5, Eq. 4 and
 * the opening of the next slice).  Waits for that close.  Errors: EINVAL
 * (NULL), ESTATE (no timed close since timing was turned on), ECUDA. */
ASSE_API int asse_close_timing(asse_pool *pool, float *ms);

/* Number of kernels this pool has launched since creation. */
ASSE_API uint64_t asse_launches(const asse_pool *pool);

/* Message of the last failing call on pool ("" if none). */
ASSE_API const char *asse_last_error(const asse_pool *pool);

/* Name of a status code. */
ASSE_API const char *asse_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* ASSE_H */
