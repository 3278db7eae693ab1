// Host build (g++) of the CUDA library's key-table helpers (csrc/asse_internal.h):
//   "M aip h"                          -> key_mix(aip, h)
//   "S n_atv pool_bytes l2_bytes mode" -> key_table_log2(...)
// one answer per input line, for checks on a machine without a GPU.
#include <cstdio>

#include "asse_internal.h"

int main()
{
    char op;
    while (std::scanf(" %c", &op) == 1) {
        if (op == 'M') {
            unsigned aip, h;
            if (std::scanf("%u %u", &aip, &h) != 2)
                return 1;
            std::printf("%llu\n", asse::key_mix(aip, h));
        } else if (op == 'S') {
            unsigned long long n_atv, pool_bytes, l2;
            unsigned mode;
            if (std::scanf("%llu %llu %llu %u", &n_atv, &pool_bytes, &l2, &mode) != 4)
                return 1;
            std::printf("%u\n", asse::key_table_log2(n_atv, pool_bytes, l2, mode));
        } else {
            return 1;
        }
    }
    return 0;
}
