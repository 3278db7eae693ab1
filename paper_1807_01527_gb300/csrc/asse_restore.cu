// K3: restore (Algorithm 4, Sec. 4.2) and cardinality estimation (Algorithm
// 5 and Eq. 4, Sec. 4.3), plus the estimate of caller-given hosts.
//
// restore_kernel runs one CTA per frame.  Instead of enumerating the whole
// product SA(0,j) x ... x SA(r-1,j) and testing each tuple, it joins the rows
// one at a time: a partial tuple carries the LBS bits its columns fixed and
// the positions they cover, and a column of the next row is kept only if it
// agrees on every position already covered.  Since the column windows are
// contiguous runs of positions, agreeing with all earlier rows is the same
// as the paper's check of each row against the next, so the surviving tuples
// are exactly Algorithm 4's.  Complete tuples give LBS, f = LBS.frame and
// aip = f^-1(f); NAT is the popcount of the AND of the r active masks the
// scan kept, and Eq. 4 is evaluated in FP64.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "asse_device.cuh"

namespace asse {

namespace {

// Eq. 4 with explicit rounding (no contraction): n = -g ln((g-NAT)/(g(1-UP))),
// +inf when NAT = g or UP = 1, 0 when the ratio is 1 or more.
__device__ __forceinline__ void eq4(uint32_t g, uint32_t theta, uint32_t nat, double up, float &est, uint32_t &flags)
{
    flags = 0;
    if (nat >= g || up >= 1.0) {
        est = INFINITY;
        flags = ASSE_SP_SATURATED | ASSE_SP_REPORTED;
        return;
    }
    const double num = (double)(g - nat);
    const double den = __dmul_rn((double)g, __dsub_rn(1.0, up));
    const double ratio = __ddiv_rn(num, den);
    double e = 0.0;
    if (ratio < 1.0)
        e = __dmul_rn(-(double)g, log(ratio));
    est = (float)e;
    if (e >= (double)theta)
        flags |= ASSE_SP_REPORTED;
}

// Eq. 4 for the candidates of one frame, in FP32 where that is provably
// within 8e-6 relative of the FP64 value above, else by eq4: FP64 on this GPU
// runs at a small fraction of the FP32 rate, and the restore's FP64 chains
// were a third of its time.  ln((g-NAT)/(g(1-UP))) = a - b with
// a = ln(1 - NAT/g) and b = ln(1 - UP).  For NAT < g/2, a = log1pf(-NAT/g):
// the rounding of NAT/g is amplified at most 1.5x, so a is within 5e-7
// relative; above, a = logf(g-NAT) - logf(g) of exact integers, within 2e-6
// absolute (1 ulp of logs below ln 4096) while |a| >= ln 2, so within 3e-6
// relative.  b = log1pf(-UP) with UP < 1/2 is within 5e-7.  When
// |a - b| >= max(|a|, |b|) / 2 the difference is within 2 x 3.5e-6, and the
// product by g and the FP32 result add 1e-7.  The FP64 path takes every
// ratio near or above 1 and every estimate within 0.1 % of theta, so the
// report decision is FP64's.
__device__ __forceinline__ void eq4_fast(uint32_t g, uint32_t theta, uint32_t nat, double up, float b_up,
                                         float &est, uint32_t &flags)
{
    if (nat < g && up < 0.5) {
        const float a = 2u * nat < g ? log1pf(-(float)nat / (float)g) : logf((float)(g - nat)) - logf((float)g);
        const float d = a - b_up;
        const float e = -(float)g * d;
        if (d < 0.0f && fabsf(d) >= 0.5f * fmaxf(fabsf(a), fabsf(b_up)) &&
            fabsf(e - (float)theta) > 1e-3f * (float)theta) {
            est = e;
            flags = e >= (float)theta ? ASSE_SP_REPORTED : 0u;
            return;
        }
    }
    eq4(g, theta, nat, up, est, flags);
}

// UP of a frame (Sec. 4.3): product over rows of |AAT(k',i,j)| / (g 2^c).
__device__ __forceinline__ double frame_up(const Params &P, const unsigned long long *aat, uint32_t frame)
{
    const double denom = __dmul_rn((double)P.g, (double)(P.cmask + 1));
    double up = 1.0;
    for (uint32_t i = 0; i < P.r; i++)
        up = __dmul_rn(up, __ddiv_rn((double)aat[(size_t)i * P.nf + frame], denom));
    return up;
}

__device__ __forceinline__ void emit(Status *st, asse_superpoint *csip, asse_superpoint *report, uint64_t out_cap,
                                     const asse_superpoint &sp)
{
    const unsigned long long p = atomicAdd(&st->n_csip, 1ull);
    if (p < out_cap)
        csip[p] = sp;
    if (sp.flags & ASSE_SP_REPORTED) {
        const unsigned long long p2 = atomicAdd(&st->n_report, 1ull);
        if (p2 < out_cap)
            report[p2] = sp;
    }
}

constexpr int RESTORE_THREADS = 512;
constexpr uint32_t RESTORE_SMEM_TUPLES = 640;  // per level; the rest of a level spills to the global scratch
constexpr uint32_t RESTORE_SMEM_COLS = 512;    // columns of each row's SA list placed in shared memory

__device__ __forceinline__ void overflow(Status *st, uint32_t needed)
{
    atomicExch(&st->overflow, 1u);
    atomicMax(&st->needed, (unsigned long long)needed);
}

// Tuple a of a level: the first RESTORE_SMEM_TUPLES in shared memory, the rest
// in this frame's part of the global scratch.
__device__ __forceinline__ Tuple *tuple_at(Tuple *sm, Tuple *gl, uint32_t a)
{
    return a < RESTORE_SMEM_TUPLES ? sm + a : gl + a;
}

__global__ void __launch_bounds__(RESTORE_THREADS) restore_kernel(Params P, ScanOut o, Tuple *scratch, uint32_t cap,
                                                                  asse_superpoint *csip, asse_superpoint *report,
                                                                  uint64_t out_cap, SliceCtl *advance)
{
    // the scan of this close has read the slice state; open the next slice
    if (advance != nullptr && blockIdx.x == 0)
        open_next_slice(P, advance);
    __shared__ uint32_t n_sa[8];
    __shared__ double p_row[8];  // |AAT(k',i,j)| / (g 2^c) of each row (Sec. 4.3)
    __shared__ uint32_t n_next;
    __shared__ Tuple sm_t[2][RESTORE_SMEM_TUPLES];
    __shared__ uint2 sm_x[4][RESTORE_SMEM_COLS];  // (bits, positions) of the columns of rows 0..3
    const uint32_t j = blockIdx.x;
    const uint32_t cols = P.cmask + 1;
    const int tid = threadIdx.x;
    // every row's list length and load (one division per thread), and the
    // columns of rows 0..3 placed on LBS positions, all in one pass
    if (tid < (int)P.r) {
        const uint32_t i = tid;
        n_sa[i] = o.sa_n[i * P.nf + j];
        p_row[i] = __ddiv_rn((double)o.aat[(size_t)i * P.nf + j], __dmul_rn((double)P.g, (double)(P.cmask + 1)));
    }
    for (uint32_t e = tid; e < 4 * RESTORE_SMEM_COLS; e += RESTORE_THREADS) {
        const uint32_t i = e / RESTORE_SMEM_COLS, b = e - i * RESTORE_SMEM_COLS;
        if (i < P.r && b < o.sa_n[i * P.nf + j]) {
            uint32_t v, m;
            place(P, o.sa_x[((size_t)i * P.nf + j) * cols + b], (int)i, v, m);
            sm_x[i][b] = make_uint2(v, m);
        }
    }
    if (tid == 0)
        n_next = 0;
    __syncthreads();
    for (uint32_t i = 0; i < P.r; i++)
        if (n_sa[i] == 0)
            return;
    Tuple *cur_g = scratch + (size_t)j * 2 * cap;
    Tuple *nxt_g = cur_g + cap;
    Tuple *cur_s = sm_t[0], *nxt_s = sm_t[1];
    uint32_t n_cur = n_sa[0];
    if (n_cur > cap) {
        if (tid == 0)
            overflow(o.status, n_cur);
        return;
    }
    // level 0: the columns of SA(0, j)
    for (uint32_t a = tid; a < n_cur; a += RESTORE_THREADS) {
        Tuple t;
        if (a < RESTORE_SMEM_COLS) {
            t.L = sm_x[0][a].x;
            t.known = sm_x[0][a].y;
        } else {
            place(P, o.sa_x[(size_t)j * cols + a], 0, t.L, t.known);
        }
        t.slot[0] = (uint16_t)a;
        *tuple_at(cur_s, cur_g, a) = t;
    }
    __syncthreads();
    // levels 1..r-1: keep a column of row i if it agrees with the tuple on
    // every position already covered
    for (uint32_t i = 1; i < P.r; i++) {
        const uint32_t ni = n_sa[i];
        const uint32_t *xs = o.sa_x + ((size_t)i * P.nf + j) * cols;
        // a warp takes one tuple at a time, its lanes the row's columns;
        // survivors are counted with one shared-memory atomic per warp round
        const int lane = tid & 31, warp = tid >> 5;
        const unsigned lt = (1u << lane) - 1u;
        for (uint32_t a = warp; a < n_cur; a += RESTORE_THREADS / 32) {
            const Tuple t = *tuple_at(cur_s, cur_g, a);
            for (uint32_t b0 = 0; b0 < ni; b0 += 32) {
                const uint32_t b = b0 + lane;
                bool keep = false;
                uint32_t v = 0, m = 0;
                if (b < ni) {
                    if (i < 4 && b < RESTORE_SMEM_COLS) {
                        const uint2 vm = sm_x[i][b];
                        v = vm.x;
                        m = vm.y;
                    } else {
                        place(P, xs[b], (int)i, v, m);
                    }
                    keep = ((t.L ^ v) & m & t.known) == 0;
                }
                const unsigned mk = __ballot_sync(FULL_MASK, keep);
                if (mk == 0)
                    continue;
                uint32_t base = 0;
                if (lane == 0)
                    base = atomicAdd(&n_next, (uint32_t)__popc(mk));
                base = __shfl_sync(FULL_MASK, base, 0);
                if (keep) {
                    const uint32_t p = base + __popc(mk & lt);
                    if (p < cap) {
                        Tuple t2 = t;
                        t2.L = t.L | v;
                        t2.known = t.known | m;
                        t2.slot[i] = (uint16_t)b;
                        *tuple_at(nxt_s, nxt_g, p) = t2;
                    }
                }
            }
        }
        __syncthreads();
        n_cur = n_next;
        if (n_cur > cap) {
            if (tid == 0)
                overflow(o.status, n_cur);
            return;
        }
        Tuple *tmp = cur_s;
        cur_s = nxt_s;
        nxt_s = tmp;
        tmp = cur_g;
        cur_g = nxt_g;
        nxt_g = tmp;
        __syncthreads();  // every thread has read n_next before it is reset
        if (tid == 0)
            n_next = 0;
        __syncthreads();
    }
    const int lane = tid & 31, warp = tid >> 5;
    for (uint32_t t = warp; t < n_cur; t += RESTORE_THREADS / 32) {
        const Tuple tu = *tuple_at(cur_s, cur_g, t);
        uint32_t nat = 0;
        for (uint32_t m = lane; m < P.mw; m += 32) {
            uint32_t acc = FULL_MASK;
            for (uint32_t i = 0; i < P.r; i++)
                acc &= o.sa_mask[(((size_t)i * P.nf + j) * cols + tu.slot[i]) * P.mw + m];
            nat += __popc(acc);
        }
        nat = __reduce_add_sync(FULL_MASK, nat);
        if (lane == 0) {
            // UP of the frame: the product over the rows, in row order
            double up = 1.0;
            for (uint32_t i = 0; i < P.r; i++)
                up = __dmul_rn(up, p_row[i]);
            const uint32_t y = (uint32_t)(((uint64_t)tu.L << P.u) | j);
            asse_superpoint sp;
            sp.aip = unmangle(P.Ainv, y);
            sp.nat = nat;
            eq4_fast(P.g, P.theta, nat, up, log1pf(-(float)up), sp.est, sp.flags);
            emit(o.status, csip, report, out_cap, sp);
        }
    }
}

// Sec. 4.3 for given hosts: one warp per host; NAT as the AND over the r rows
// of the active fields of each word, Eq. 4 with the frame's UP.
template <int WB>
__global__ void __launch_bounds__(256) estimate_kernel(Params P, const uint32_t *pool, uint32_t c0, uint32_t kp,
                                                       const unsigned long long *aat, const uint32_t *aips,
                                                       uint64_t n, asse_superpoint *out)
{
    constexpr uint32_t F = 32 / WB;
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
    const uint32_t nwords = (P.g + F - 1) / F;
    for (uint64_t t = (uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); t < n; t += warps) {
        const uint32_t aip = aips[t];
        const uint32_t f = mangle(P.A, aip);
        const uint32_t z = f & (P.nf - 1);
        const uint64_t LL = lbs_twice(P, f);
        uint32_t nat = 0;
        for (uint32_t q = lane; q < nwords; q += 32) {
            uint32_t acc = FULL_MASK;
            for (uint32_t i = 0; i < P.r; i++) {
                const uint64_t atv = ((uint64_t)i << P.E_log2) + ((z << P.c) | column(P, LL, (int)i));
                acc &= active_fields<WB>(P, pool[atv * P.Wd + q], q, c0, kp);
            }
            nat += __popc(acc);
        }
        nat = __reduce_add_sync(FULL_MASK, nat);
        if (lane == 0) {
            asse_superpoint sp;
            sp.aip = aip;
            sp.nat = nat;
            eq4(P.g, P.theta, nat, frame_up(P, aat, z), sp.est, sp.flags);
            out[t] = sp;
        }
    }
}

}  // namespace

cudaError_t launch_restore(const Params &P, const ScanOut &o, Tuple *scratch, uint32_t cap, asse_superpoint *csip,
                           asse_superpoint *report, uint64_t out_cap, cudaStream_t s, uint64_t *launches,
                           SliceCtl *advance)
{
    *launches += 1;
    restore_kernel<<<P.nf, RESTORE_THREADS, 0, s>>>(P, o, scratch, cap, csip, report, out_cap, advance);
    return cudaGetLastError();
}

cudaError_t launch_estimate(const Params &P, uint32_t w, const uint32_t *pool, uint32_t c0, uint32_t kp,
                            const unsigned long long *aat, const uint32_t *aips, uint64_t n, asse_superpoint *out,
                            int sms, cudaStream_t s, uint64_t *launches)
{
    if (n == 0)
        return cudaSuccess;
    const uint64_t want = (n + 7) / 8;
    const unsigned grid = (unsigned)(want > (uint64_t)sms * 8 ? (uint64_t)sms * 8 : want);
    *launches += 1;
    return dispatch_w(w, [&](auto wb) {
        constexpr int WB = decltype(wb)::value;
        estimate_kernel<WB><<<grid, 256, 0, s>>>(P, pool, c0, kp, aat, aips, n, out);
        return cudaGetLastError();
    });
}

}  // namespace asse
