// Internal declarations shared by the host API (asse_api.cu) and the
// kernels (asse_kernels.cu).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/asse.h"

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
    uint64_t blk_magic; // ceil(2^32 / floor(g/2k))
    uint64_t Ainv;      // A^-1 mod p (may exceed 2^32)
    uint64_t bh_a, bh_b;
    uint32_t xshift[8]; // 2W - c - s*i: shift of the doubled LBS giving x_i
};

// Device-resident status of one close, reset by every scan.
struct Status {
    unsigned long long n_csip;    // candidates restored (Algorithm 4)
    unsigned long long n_report;  // candidates with estimate >= theta
    unsigned long long needed;    // tuples the overflowing join level needed
    unsigned int overflow;        // a frame exceeded the restore capacity
    unsigned int pad;
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

struct ScanOut {
    uint16_t *cnt;
    unsigned long long *aat;
    uint32_t *sa_n, *sa_x, *sa_mask;
    Status *status;
};

// Kernel launchers (asse_kernels.cu).  Each returns the cudaError_t of its
// launch and adds the number of kernels it launched to *launches.
cudaError_t launch_ingest(const Params &P, uint32_t w, uint32_t *pool, const uint32_t *pairs, uint64_t n,
                          uint32_t c0, int sms, cudaStream_t s, uint64_t *launches);
cudaError_t launch_scan(const Params &P, uint32_t w, uint32_t *pool, uint32_t c0, uint32_t kp, const Refresh *fuse,
                        const ScanOut &o, int sms, cudaStream_t s, uint64_t *launches);
cudaError_t launch_refresh(const Params &P, uint32_t w, uint32_t *pool, const Refresh &R, int sms, cudaStream_t s,
                           uint64_t *launches);
cudaError_t launch_restore(const Params &P, const ScanOut &o, Tuple *scratch, uint32_t cap, asse_superpoint *csip,
                           asse_superpoint *report, uint64_t out_cap, cudaStream_t s, uint64_t *launches);
cudaError_t launch_estimate(const Params &P, uint32_t w, const uint32_t *pool, uint32_t c0, uint32_t kp,
                            const unsigned long long *aat, const uint32_t *aips, uint64_t n, asse_superpoint *out,
                            int sms, cudaStream_t s, uint64_t *launches);

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
int pool_fail(asse_pool *p, int code, const std::string &msg);

}  // namespace asse
