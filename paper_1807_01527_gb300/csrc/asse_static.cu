// asse_restore_static: the restore of the last scan (the join, NAT and the
// estimate of every candidate) for callers that must not allocate device
// memory while they run it.
//
// Who needs this: a packet pipeline that closes slices on a latency budget
// cannot afford cudaMalloc/cudaFree on its path, because those calls may
// synchronise the whole device and stall the other streams feeding it, and
// some hosts hand all device memory to another allocator up front so that no
// later allocation may happen at all.  Such a caller already owns its output
// buffers; the only extra memory the restore needs is the scratch where the
// row-by-row join keeps its partial column tuples, and here that scratch is
// a fixed array compiled into the library instead of memory obtained at run
// time.
#include <cuda_runtime.h>

#include <cstddef>
#include <mutex>
#include <string>

#include "asse_internal.h"

namespace {

// The join scratch: 2^u frames x 2 levels x tuples_per_frame tuples must fit.
// 131,072 tuples of 24 bytes = 3 MiB of device memory, held by every GPU that
// loads the library until the process exits.
static __device__ __align__(256) asse::Tuple g_restore_scratch[ASSE_STATIC_RESTORE_TUPLES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
asse::Tuple *g_scratch_addr[kMaxDevices] = {};

// The device address of g_restore_scratch on the current device.  In host
// code the array's name only stands in for the symbol, so the address is
// looked up once per device (with that device current) and cached.
int scratch_address(asse_pool *pool, asse::Tuple **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return asse::pool_fail(pool, ASSE_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return asse::pool_fail(pool, ASSE_EINVAL, "device ordinal beyond the static scratch table");
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_scratch_addr[dev] == nullptr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_restore_scratch);
        if (e != cudaSuccess || p == nullptr)
            return asse::pool_fail(pool, ASSE_ECUDA,
                                   std::string("cudaGetSymbolAddress of the restore scratch: ") +
                                       cudaGetErrorString(e));
        g_scratch_addr[dev] = static_cast<asse::Tuple *>(p);
    }
    *out = g_scratch_addr[dev];
    return ASSE_OK;
}

}  // namespace

extern "C" int asse_restore_static(asse_pool *pool, uint32_t tuples_per_frame, asse_superpoint *candidates,
                                   asse_superpoint *reported, uint64_t cap, uint64_t *counters)
{
    if (!pool)
        return ASSE_EINVAL;
    if (!candidates || !reported || !counters || cap == 0)
        return asse::pool_fail(pool, ASSE_EINVAL, "asse_restore_static needs two output lists and counters");
    asse::RestoreView v;
    if (int rc = asse::pool_restore_view(pool, &v))
        return rc;
    const uint64_t need = (uint64_t)tuples_per_frame * 2u * v.P.nf;
    if (tuples_per_frame == 0 || need > ASSE_STATIC_RESTORE_TUPLES)
        return asse::pool_fail(pool, ASSE_EINVAL,
                               "tuples_per_frame x 2 x 2^u = " + std::to_string(need) +
                                   " exceeds the static restore scratch of " +
                                   std::to_string(ASSE_STATIC_RESTORE_TUPLES) + " tuples");
    asse::Tuple *scratch = nullptr;
    if (int rc = scratch_address(pool, &scratch))
        return rc;
    // The scratch is fully written by each frame's join before it is read, so
    // only the counters have to start at zero.
    // the caller's counters are the first four 64-bit words of the status the
    // restore kernel writes; it never touches the fields after them
    static_assert(offsetof(asse::Status, overflow) + sizeof(unsigned int) <= 4 * sizeof(uint64_t),
                  "restore counters must fit in 4 x uint64");
    cudaError_t e = cudaMemsetAsync(counters, 0, 4 * sizeof(uint64_t), v.stream);
    if (e != cudaSuccess)
        return asse::pool_fail(pool, ASSE_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    asse::ScanOut o = v.o;
    o.status = reinterpret_cast<asse::Status *>(counters);
    e = asse::launch_restore(v.P, o, scratch, tuples_per_frame, candidates, reported, cap, v.stream, v.launches);
    if (e != cudaSuccess)
        return asse::pool_fail(pool, ASSE_ECUDA, std::string("restore launch: ") + cudaGetErrorString(e));
    return ASSE_OK;
}
