// Prints the word ranges the CUDA library's slice control gives Algorithm 2
// (refresh_for in csrc/asse_internal.h) for each "k g blk F t_new paired"
// line of standard input: "c0n n_ranges lo0 hi0 lo1 hi1".  Host-only build (g++), so
// the range logic can be checked on a machine without a GPU.
#include <cstdio>

#include "asse_internal.h"

int main()
{
    unsigned k, g, blk, F, paired;
    unsigned long long t;
    while (std::scanf("%u %u %u %u %llu %u", &k, &g, &blk, &F, &t, &paired) == 6) {
        const asse::Refresh R = asse::refresh_for(k, g, blk, F, t, paired != 0);
        std::printf("%u %u %u %u %u %u\n", R.c0n, R.n_ranges, R.q_lo[0], R.q_hi[0], R.q_lo[1], R.q_hi[1]);
    }
    return 0;
}
