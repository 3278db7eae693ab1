// Exhaustive host check of the word-level tests on byte-wide counter fields
// (csrc/asse_bytes.h) against their per-byte definitions: every value v,
// every range [lo, hi] with v, lo, hi in 0..127, in every byte position of
// the word, next to other bytes that would expose a borrow or a carry.
// Prints the number of mismatches and "ok" when there are none.
#include <cstdio>
#include <cstdint>

#include <cuda_runtime.h>

#include "asse_bytes.h"

using namespace asse;

static uint32_t rng_state = 12345u;
static uint32_t next_byte()
{
    rng_state = rng_state * 1664525u + 1013904223u;
    return (rng_state >> 24) & 0x7Fu;  // 0..127: a valid neighbour value
}

int main()
{
    long bad = 0, checked = 0;
    for (uint32_t pos = 0; pos < 4; pos++) {
        const uint32_t sh = 8 * pos;
        for (uint32_t lo = 0; lo < 128; lo++)
            for (uint32_t hi = 0; hi < 128; hi++) {
                // range [lo, hi] in this byte, empty ranges in the others;
                // the second range empty everywhere
                uint4 d;
                d.x = (127u * BYTE_ONES & ~(0xFFu << sh)) | (lo << sh);
                d.y = (0x80u * BYTE_ONES & ~(0xFFu << sh)) | ((hi | 0x80u) << sh);
                d.z = 127u * BYTE_ONES;
                d.w = 0x80u * BYTE_ONES;
                // the same range as the second one, the first empty
                uint4 e = make_uint4(d.z, d.w, d.x, d.y);
                for (uint32_t v = 0; v < 128; v++) {
                    uint32_t w = 0;
                    for (uint32_t j = 0; j < 4; j++)
                        w |= (j == pos ? v : next_byte()) << (8 * j);
                    const bool want = lo <= v && v <= hi;
                    const uint32_t m1 = in_ranges_bytes(w, d), m2 = in_ranges_bytes(w, e);
                    const uint32_t mbit = 0x80u << sh;
                    if (((m1 & mbit) != 0) != want || ((m2 & mbit) != 0) != want || (m1 & ~mbit) || (m2 & ~mbit))
                        bad++;
                    if (field_bits_bytes(w, d) != (want ? 1u << pos : 0u))
                        bad++;
                    // Algorithm 2 with k2 = 120: the byte becomes 120 iff in range, others unchanged
                    const uint32_t r = refresh_bytes(120u, w, d);
                    const uint32_t want_r = want ? (w & ~(0xFFu << sh)) | (120u << sh) : w;
                    if (r != want_r)
                        bad++;
                    checked++;
                }
            }
        // decay: every non-zero byte loses one, whatever its neighbours hold
        for (uint32_t v = 0; v < 128; v++)
            for (int rep = 0; rep < 64; rep++) {
                uint32_t w = 0, want = 0;
                for (uint32_t j = 0; j < 4; j++) {
                    const uint32_t b = j == pos ? v : next_byte();
                    w |= b << (8 * j);
                    want |= (b ? b - 1 : 0u) << (8 * j);
                }
                if (decay_bytes(w) != want)
                    bad++;
                checked++;
            }
    }
    // two ranges at once in all four bytes, random
    for (int it = 0; it < 2000000; it++) {
        uint4 d = make_uint4(0, 0, 0, 0);
        uint32_t w = 0, want = 0;
        for (uint32_t j = 0; j < 4; j++) {
            uint32_t l1 = next_byte(), h1 = next_byte(), l2 = next_byte(), h2 = next_byte(), v = next_byte();
            d.x |= l1 << (8 * j);
            d.y |= (h1 | 0x80u) << (8 * j);
            d.z |= l2 << (8 * j);
            d.w |= (h2 | 0x80u) << (8 * j);
            w |= v << (8 * j);
            if ((l1 <= v && v <= h1) || (l2 <= v && v <= h2))
                want |= 0x80u << (8 * j);
        }
        if (in_ranges_bytes(w, d) != want)
            bad++;
        checked++;
    }
    std::printf("%ld %ld %s\n", checked, bad, bad ? "MISMATCH" : "ok");
    return bad ? 1 : 0;
}
