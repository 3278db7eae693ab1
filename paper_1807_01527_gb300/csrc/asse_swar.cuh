// SWAR activity tests on packed AT words, shared by the scan (asse_scan.cu)
// and the feature rows of the learned estimator (asse_features.cu).
//
// The active values of a block form the cyclic window act-k'+1 .. act (mod
// 2k), i.e. at most two plain ranges.  The even and the odd fields of a word
// are tested separately, each field then having w free bits above it; with
// a guard bit just above each field, (v | guard) - lo keeps the guard iff
// v >= lo and (hi | guard) - v keeps it iff v <= hi, with no borrow between
// fields.  Per-position constants carry each field's own range, so words
// that straddle two ACT blocks and the fields past g (empty ranges) need no
// special case.  Byte-wide fields holding seven-bit values have the guard
// bit inside the field and are tested all four at once (asse_bytes.h).
#pragma once

#include <cstdint>

#include "asse_bytes.h"
#include "asse_device.cuh"

namespace asse {

// Layout of the even/odd field groups of a word of WB-bit fields.
template <int WB>
struct Swar {
    static constexpr uint32_t F = 32 / WB;
    static constexpr uint32_t FM = (1u << WB) - 1;
    // position of field j inside its group (the odd group is shifted down by WB)
    static __host__ __device__ constexpr uint32_t pos(uint32_t j) { return (j >> 1) * 2 * WB; }
    static __host__ __device__ constexpr uint32_t group_fields(uint32_t odd)
    {
        uint32_t m = 0;
        for (uint32_t j = odd; j < F; j += 2)
            m |= FM << pos(j);
        return m;
    }
    static __host__ __device__ constexpr uint32_t group_guards(uint32_t odd)
    {
        uint32_t m = 0;
        for (uint32_t j = odd; j < F; j += 2)
            m |= 1u << (pos(j) + WB);
        return m;
    }
    static __host__ __device__ constexpr uint32_t group_ones(uint32_t odd)
    {
        uint32_t m = 0;
        for (uint32_t j = odd; j < F; j += 2)
            m |= 1u << pos(j);
        return m;
    }
    static constexpr uint32_t ME = group_fields(0);
    static constexpr uint32_t HE = group_guards(0);
    static constexpr uint32_t HO = group_guards(1);
};

// Per word position: for the even (e) and odd (o) field groups, the low ends
// lo and the high ends with guards hih = hi | guard of two value ranges.
struct RangeDesc {
    uint32_t lo1e, hih1e, lo1o, hih1o, lo2e, hih2e, lo2o, hih2o;
};

template <int WB>
__device__ __forceinline__ void put_range(RangeDesc &d, uint32_t j, uint32_t l1, uint32_t h1, uint32_t l2, uint32_t h2)
{
    using S = Swar<WB>;
    const uint32_t p = S::pos(j), g = 1u << (p + WB);
    if (j & 1) {
        d.lo1o |= l1 << p;
        d.hih1o |= (h1 << p) | g;
        d.lo2o |= l2 << p;
        d.hih2o |= (h2 << p) | g;
    } else {
        d.lo1e |= l1 << p;
        d.hih1e |= (h1 << p) | g;
        d.lo2e |= l2 << p;
        d.hih2e |= (h2 << p) | g;
    }
}

// The active-value ranges of every field of word position q.
template <int WB>
__device__ RangeDesc count_desc(const Params &P, uint32_t q, uint32_t c0, uint32_t kp)
{
    using S = Swar<WB>;
    RangeDesc d = {0, 0, 0, 0, 0, 0, 0, 0};
    for (uint32_t j = 0; j < S::F; j++) {
        const uint32_t h = q * S::F + j;
        uint32_t l1 = S::FM, h1 = 0, l2 = S::FM, h2 = 0;  // empty ranges
        if (h < P.g) {
            if (P.ace) {
                l1 = P.k + 1 - kp;
                h1 = P.k;
            } else {
                const uint32_t act = act_of(P, c0, pos_block(P, h));
                if (act + 1 >= kp) {
                    l1 = act + 1 - kp;
                    h1 = act;
                } else {  // the window wraps past 0 to the top of 0..2k-1
                    l1 = 0;
                    h1 = act;
                    l2 = act + P.k2 + 1 - kp;
                    h2 = P.k2 - 1;
                }
            }
        }
        put_range<WB>(d, j, l1, h1, l2, h2);
    }
    return d;
}

// The value ranges Algorithm 2 clears in every field of word position q when
// block 0 has ACT c0n.
template <int WB>
__device__ RangeDesc refresh_desc(const Params &P, uint32_t q, uint32_t c0n)
{
    using S = Swar<WB>;
    RangeDesc d = {0, 0, 0, 0, 0, 0, 0, 0};
    for (uint32_t j = 0; j < S::F; j++) {
        const uint32_t h = q * S::F + j;
        uint32_t l1 = S::FM, h1 = 0, l2 = S::FM, h2 = 0;
        if (h < P.g && !P.ace) {
            const uint32_t act = act_of(P, c0n, pos_block(P, h));
            if (act == 0) {
                l1 = 0;
                h1 = P.k;
            } else if (act == P.k) {
                l1 = P.k;
                h1 = P.k2 - 1;
                l2 = 0;
                h2 = 0;
            }
        }
        put_range<WB>(d, j, l1, h1, l2, h2);
    }
    return d;
}

__device__ __forceinline__ RangeDesc load_desc(const uint4 *lo, const uint4 *hi, uint32_t x)
{
    const uint4 a = lo[x], b = hi[x];
    return RangeDesc{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
}

// Guard bits of the fields of word w whose value lies in one of the ranges.
template <int WB>
__device__ __forceinline__ void in_ranges(uint32_t w, const RangeDesc &d, uint32_t &ge_bits, uint32_t &go_bits)
{
    using S = Swar<WB>;
    const uint32_t xe = w & S::ME, xo = (w >> WB) & S::ME;
    const uint32_t xeh = xe | S::HE, xoh = xo | S::HO;
    ge_bits = (((xeh - d.lo1e) & (d.hih1e - xe)) | ((xeh - d.lo2e) & (d.hih2e - xe))) & S::HE;
    go_bits = (((xoh - d.lo1o) & (d.hih1o - xo)) | ((xoh - d.lo2o) & (d.hih2o - xo))) & S::HO;
}

template <int WB>
__device__ __forceinline__ uint32_t count_word(uint32_t w, const RangeDesc &d)
{
    uint32_t e, o;
    in_ranges<WB>(w, d, e, o);
    return __popc(e) + __popc(o);
}

// Field j (bit j) set iff field j of w is in one of the ranges.
template <int WB>
__device__ __forceinline__ uint32_t field_bits(uint32_t w, const RangeDesc &d)
{
    using S = Swar<WB>;
    uint32_t e, o, am = 0;
    in_ranges<WB>(w, d, e, o);
#pragma unroll
    for (uint32_t j = 0; j < S::F; j++)
        am |= ((((j & 1) ? o : e) >> (S::pos(j) + WB)) & 1u) << j;
    return am;
}

// Algorithm 2 on a word: the fields in the refresh ranges become 2k.
template <int WB>
__device__ __forceinline__ uint32_t refresh_swar(const Params &P, uint32_t w, const RangeDesc &d)
{
    using S = Swar<WB>;
    uint32_t e, o;
    in_ranges<WB>(w, d, e, o);
    const uint32_t fm = ((e >> WB) * S::FM) | (((o >> WB) * S::FM) << WB);
    uint32_t k2rep = 0;
#pragma unroll
    for (uint32_t j = 0; j < S::F; j++)
        k2rep |= P.k2 << (j * WB);
    return (w & ~fm) | (k2rep & fm);
}

// Aging counters: every non-zero field of w loses one.
template <int WB>
__device__ __forceinline__ uint32_t decay_swar(uint32_t w)
{
    using S = Swar<WB>;
    const uint32_t xe = w & S::ME, xo = (w >> WB) & S::ME;
    const uint32_t nz_e = ((xe | S::HE) - S::group_ones(0)) & S::HE;  // guard kept iff the field is >= 1
    const uint32_t nz_o = ((xo | S::HO) - S::group_ones(1)) & S::HO;
    return w - (nz_e >> WB) - ((nz_o >> WB) << WB);  // no borrow: each decremented field is >= 1
}

// ---------------------------------------------------------------------------
// Byte-wide fields with values below 128 (asse_bytes.h): the range entries of
// every word position, built like count_desc / refresh_desc but as four byte
// lanes of one word each.

// The count ranges of word position q (one ACT block per word is not
// assumed: a word whose fields fall in two blocks gets per-byte ranges).
__device__ __forceinline__ uint4 count_desc_bytes(const Params &P, uint32_t q, uint32_t c0, uint32_t kp)
{
    uint4 d = make_uint4(0, 0, 0, 0);
    for (uint32_t j = 0; j < 4; j++) {
        const uint32_t h = q * 4 + j;
        uint32_t l1 = 127, h1 = 0, l2 = 127, h2 = 0;  // empty ranges
        if (h < P.g) {
            if (P.ace) {
                l1 = P.k + 1 - kp;
                h1 = P.k;
            } else {
                const uint32_t act = act_of(P, c0, pos_block(P, h));
                if (act + 1 >= kp) {
                    l1 = act + 1 - kp;
                    h1 = act;
                } else {  // the window wraps past 0 to the top of 0..2k-1
                    l1 = 0;
                    h1 = act;
                    l2 = act + P.k2 + 1 - kp;
                    h2 = P.k2 - 1;
                }
            }
        }
        d.x |= l1 << (8 * j);
        d.y |= (h1 | 0x80u) << (8 * j);
        d.z |= l2 << (8 * j);
        d.w |= (h2 | 0x80u) << (8 * j);
    }
    return d;
}

// The ranges Algorithm 2 clears in every byte of word position q when block 0
// has ACT c0n.
__device__ __forceinline__ uint4 refresh_desc_bytes(const Params &P, uint32_t q, uint32_t c0n)
{
    uint4 d = make_uint4(0, 0, 0, 0);
    for (uint32_t j = 0; j < 4; j++) {
        const uint32_t h = q * 4 + j;
        uint32_t l1 = 127, h1 = 0, l2 = 127, h2 = 0;
        if (h < P.g && !P.ace) {
            const uint32_t act = act_of(P, c0n, pos_block(P, h));
            if (act == 0) {
                l1 = 0;
                h1 = P.k;
            } else if (act == P.k) {
                l1 = P.k;
                h1 = P.k2 - 1;
                l2 = 0;
                h2 = 0;
            }
        }
        d.x |= l1 << (8 * j);
        d.y |= (h1 | 0x80u) << (8 * j);
        d.z |= l2 << (8 * j);
        d.w |= (h2 | 0x80u) << (8 * j);
    }
    return d;
}

}  // namespace asse
