// Word-level tests on byte-wide counter fields whose values stay below 128:
// the packed layout of seven-bit counters, which packed_width
// (asse_internal.h) stores in eight bits, four fields to a 32-bit word.  Bit
// 7 of every byte is 0 in the pool, so it serves as the guard bit in place:
// one subtraction tests all four fields against a bound, with no borrow
// from one byte into the next.  Host and device code (the host build checks
// these functions exhaustively against per-byte definitions).
#pragma once

#include <cstdint>

#include <vector_types.h>

#if defined(__CUDACC__)
#define ASSE_BYTES_FN __host__ __device__ __forceinline__
#else
#define ASSE_BYTES_FN inline
#endif

namespace asse {

constexpr uint32_t BYTE_GUARDS = 0x80808080u;
constexpr uint32_t BYTE_ONES = 0x01010101u;

// A range entry holds, per byte, the low end lo and the high end with the
// guard, hi | 0x80, of two value ranges: (x, y) = (lo1, hih1) and (z, w) =
// (lo2, hih2).  lo <= 127; an empty range is lo = 127, hi = 0.

// Bit 7 of every byte of w whose value lies in one of the ranges of d:
// (v | 0x80) - lo keeps bit 7 iff v >= lo, (hi | 0x80) - v keeps it iff
// v <= hi, and neither borrows from the next byte (v, lo, hi <= 127).
ASSE_BYTES_FN uint32_t in_ranges_bytes(uint32_t w, const uint4 &d)
{
    const uint32_t wh = w | BYTE_GUARDS;
    return (((wh - d.x) & (d.y - w)) | ((wh - d.z) & (d.w - w))) & BYTE_GUARDS;
}

// Field j (bit j) set iff byte j of w is in one of the ranges.
ASSE_BYTES_FN uint32_t field_bits_bytes(uint32_t w, const uint4 &d)
{
    const uint32_t m = in_ranges_bytes(w, d);
    return ((m >> 7) | (m >> 14) | (m >> 21) | (m >> 28)) & 0xFu;
}

// Algorithm 2 on a word: the bytes in the refresh ranges become 2k (k2).
ASSE_BYTES_FN uint32_t refresh_bytes(uint32_t k2, uint32_t w, const uint4 &d)
{
    const uint32_t fm = (in_ranges_bytes(w, d) >> 7) * 0xFFu;
    return (w & ~fm) | ((k2 * BYTE_ONES) & fm);
}

// Aging counters: every non-zero byte of w loses one.
ASSE_BYTES_FN uint32_t decay_bytes(uint32_t w)
{
    const uint32_t nz = ((w | BYTE_GUARDS) - BYTE_ONES) & BYTE_GUARDS;  // bit 7 kept iff the byte is >= 1
    return w - (nz >> 7);
}

}  // namespace asse
