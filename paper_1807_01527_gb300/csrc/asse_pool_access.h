// Host-side reads of a pool's bookkeeping (kept in asse_api.cu) for entry
// points defined in other files.
#pragma once

#include <cstdint>

struct asse_pool;

namespace asse {

// Capacity, in records, of the pool's candidate and report lists
// (restore_cap x 2^u): no restore returns more candidates than this.
uint64_t pool_list_cap(const asse_pool *p);

}  // namespace asse
