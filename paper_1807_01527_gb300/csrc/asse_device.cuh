// Device-side arithmetic of the ASSE hot path: exact IP mangling modulo
// p = 2^32 + 15, the column split of RRH, the bip hash BH, ACT blocks and the
// per-field activity test.  Everything here is integer arithmetic that the
// kernels keep in registers.
#pragma once

#include <cstdint>
#include <type_traits>

#include "asse_internal.h"

namespace asse {

constexpr uint64_t kP = 4294967311ull;  // 2^32 + 15 (Sec. 4.1: prime above 2^32)

// x mod p for any 64-bit x, from 2^32 = -15 (mod p): two folds, no division.
__device__ __forceinline__ uint64_t mod_p(uint64_t x)
{
    const uint64_t hi = x >> 32, lo = x & 0xffffffffull;
    // lo - 15*hi + 15*p: congruent to x and positive (hi < 2^32), below 2^36 + 2^32.
    const uint64_t v = lo + 15ull * ((1ull << 32) - hi) + 225ull;
    const int64_t r = (int64_t)(v & 0xffffffffull) - 15ll * (int64_t)(v >> 32);
    return r < 0 ? (uint64_t)(r + (int64_t)kP) : (uint64_t)r;
}

// a*b mod p for a, b < p (either may have bit 32 set).
__device__ __forceinline__ uint64_t mulmod_p(uint64_t a, uint64_t b)
{
    const uint64_t ah = a >> 32, bh = b >> 32;  // 0 or 1
    const uint64_t al = a & 0xffffffffull, bl = b & 0xffffffffull;
    uint64_t r = mod_p(al * bl);
    if (ah | bh) {
        // a*b = ah*bh*2^64 + (ah*bl + bh*al)*2^32 + al*bl with 2^32 = -15, 2^64 = 225.
        const uint64_t neg = 15ull * (ah * bl + bh * al);  // < 30 * 2^32 < 30 p
        r = mod_p(r + 225ull * (ah & bh) + 30ull * kP - neg);
    }
    return r;
}

// f(aip) = A*aip mod p, walked until it is below 2^32 (one-to-one on uint32).
__device__ __forceinline__ uint32_t mangle(uint32_t A, uint32_t aip)
{
    uint64_t y = mod_p((uint64_t)A * aip);
    while (y >> 32)
        y = mulmod_p(A, y);
    return (uint32_t)y;
}

// f^-1(y) = A^-1 * y mod p with the same walk.
__device__ __forceinline__ uint32_t unmangle(uint64_t Ainv, uint32_t y)
{
    uint64_t x = mulmod_p(Ainv, y);
    while (x >> 32)
        x = mulmod_p(Ainv, x);
    return (uint32_t)x;
}

// BH(bip): top 32 bits of bh_a*bip + bh_b (mod 2^64), scaled to [0, g).
__device__ __forceinline__ uint32_t bip_hash(const Params &P, uint32_t bip)
{
    const uint64_t h = P.bh_a * (uint64_t)bip + P.bh_b;
    return __umulhi((uint32_t)(h >> 32), P.g);
}

// Column index x_i: c bits of the W-bit LBS starting at position s*i (MSB
// first, wrapping).  LL holds LBS twice side by side, so the wrapped window
// is one shift of LL.
__device__ __forceinline__ uint32_t column(const Params &P, uint64_t LL, int i)
{
    return (uint32_t)(LL >> P.xshift[i]) & P.cmask;
}

__device__ __forceinline__ uint64_t lbs_twice(const Params &P, uint32_t f)
{
    const uint64_t L = (uint64_t)(f >> P.u);
    return (L << P.W) | L;
}

// Place column index x of row i back onto its positions of the W-bit LBS.
__device__ __forceinline__ void place(const Params &P, uint32_t x, int i, uint32_t &val, uint32_t &mask)
{
    const uint64_t wmask = (P.W == 32) ? 0xffffffffull : ((1ull << P.W) - 1);
    const uint64_t V = (uint64_t)x << P.xshift[i];
    const uint64_t M = (uint64_t)P.cmask << P.xshift[i];
    val = (uint32_t)((V >> P.W) | (V & wmask));
    mask = (uint32_t)((M >> P.W) | (M & wmask));
}

// ACT block of AT h: min(h / a, 2k-1), h / a by a multiply-high that is exact
// for h, a < 2^16.
__device__ __forceinline__ uint32_t act_block(const Params &P, uint32_t h)
{
    const uint32_t b = (uint32_t)(((uint64_t)h * P.blk_magic) >> 32);
    return b < P.k2 - 1 ? b : P.k2 - 1;
}

// ACT block of the AT stored at position p of an ATV (block_slot order when
// P.paired).
__device__ __forceinline__ uint32_t pos_block(const Params &P, uint32_t p)
{
    const uint32_t s = act_block(P, p);
    return P.paired ? slot_block(P.k, s) : s;
}

// Storage position of AT h (h itself unless P.paired).
__device__ __forceinline__ uint32_t at_pos(const Params &P, uint32_t h)
{
    if (!P.paired)
        return h;
    const uint32_t b = act_block(P, h);
    return h - b * P.blk + block_slot(P.k, b) * P.blk;
}

// The AT stored at position p (the inverse of at_pos).
__device__ __forceinline__ uint32_t pos_at(const Params &P, uint32_t p)
{
    if (!P.paired)
        return p;
    const uint32_t s = act_block(P, p);
    return p - s * P.blk + slot_block(P.k, s) * P.blk;
}

// ACT of block b in the slice whose block 0 has ACT c0.
__device__ __forceinline__ uint32_t act_of(const Params &P, uint32_t c0, uint32_t b)
{
    const uint32_t a = c0 + b;
    return a >= P.k2 ? a - P.k2 : a;
}

// Algorithm 1 (AT) / aging-counter test (ACE) for one field value.
__device__ __forceinline__ bool field_active(const Params &P, uint32_t v, uint32_t act, uint32_t kp)
{
    if (P.ace)
        return v + kp >= P.k + 1;  // v >= k - k' + 1
    if (v >= P.k2)
        return false;
    uint32_t dis = act + P.k2 - v;
    dis = dis >= P.k2 ? dis - P.k2 : dis;
    return dis + 1 <= kp;
}

// Algorithm 2 on one field whose new ACT is act (only 0 and k act).
__device__ __forceinline__ uint32_t preserve(const Params &P, uint32_t v, uint32_t act)
{
    if (act == 0)
        return v <= P.k ? P.k2 : v;
    if (act == P.k)
        return (v == 0 || (v >= P.k && v < P.k2)) ? P.k2 : v;
    return v;
}

// Bit mask of the active fields of one packed word (bit j = field j),
// fields at or past g excluded.
template <int WB>
__device__ __forceinline__ uint32_t active_fields(const Params &P, uint32_t word, uint32_t q, uint32_t c0,
                                                  uint32_t kp)
{
    constexpr int F = 32 / WB;
    constexpr uint32_t FM = (1u << WB) - 1;
    const uint32_t h0 = q * F;
    uint32_t am = 0;
    if (P.ace) {
#pragma unroll
        for (int j = 0; j < F; j++) {
            const uint32_t v = (word >> (j * WB)) & FM;
            am |= (uint32_t)(v + kp >= P.k + 1) << j;
        }
    } else {
        const uint32_t b0 = pos_block(P, h0), b1 = pos_block(P, h0 + F - 1);
        if (b0 == b1) {
            // one ACT for the whole word: active values are the cyclic window
            // act, act-1, ..., act-k'+1 (mod 2k)
            const uint32_t act = act_of(P, c0, b0);
#pragma unroll
            for (int j = 0; j < F; j++) {
                const uint32_t v = (word >> (j * WB)) & FM;
                uint32_t dis = act + P.k2 - v;
                dis = dis >= P.k2 ? dis - P.k2 : dis;
                am |= (uint32_t)((v < P.k2) & (dis < kp)) << j;
            }
        } else {
#pragma unroll 1
            for (int j = 0; j < F; j++) {
                const uint32_t v = (word >> (j * WB)) & FM;
                am |= (uint32_t)field_active(P, v, act_of(P, c0, pos_block(P, h0 + j)), kp) << j;
            }
        }
    }
    if (h0 + F > P.g)
        am &= (P.g > h0) ? ((1u << (P.g - h0)) - 1) : 0u;
    return am;
}

constexpr unsigned FULL_MASK = 0xffffffffu;

__device__ __forceinline__ uint32_t u4get(const uint4 &v, int e)
{
    return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
}

// Calls fn(std::integral_constant<int, w>) for the packed field width w (1..8
// but not 7, which packed_width stores in 8 bits), so that the field layout
// is a compile-time constant in every kernel.
template <typename Fn>
cudaError_t dispatch_w(uint32_t w, Fn &&fn)
{
    switch (w) {
    case 1: return fn(std::integral_constant<int, 1>());
    case 2: return fn(std::integral_constant<int, 2>());
    case 3: return fn(std::integral_constant<int, 3>());
    case 4: return fn(std::integral_constant<int, 4>());
    case 5: return fn(std::integral_constant<int, 5>());
    case 6: return fn(std::integral_constant<int, 6>());
    case 8: return fn(std::integral_constant<int, 8>());
    default: return cudaErrorInvalidValue;
    }
}

// Threads a kernel can keep resident per SM (grid sizing of the persistent
// grid-stride kernels).
template <typename K>
int resident_blocks(K kernel, int threads, size_t smem)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess || n < 1)
        n = 1;
    return n;
}

}  // namespace asse
