// Host-side rules of the CUDA library, printed for test_host_logic.py:
// the Gram row chunk, the Gram CTA sizes, the shared-memory budgets and the
// round-robin table of the step kernels, the sizes of the delta-form update
// tiles (no GPU needed).
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "../paper_1907_08560_gb300/csrc/hz_launch.h"
#include "../paper_1907_08560_gb300/csrc/hz_pivot.cuh"
#include "../paper_1907_08560_gb300/csrc/hz_delta.cuh"

int main(int argc, char **argv)
{
    if (argc >= 2 && !strcmp(argv[1], "chunk") && argc == 6) {
        printf("%d\n", hz::gram_chunk_rows(atoi(argv[2]), atoi(argv[3]), atoi(argv[4]), atoi(argv[5])));
        return 0;
    }
    if (argc == 2 && !strcmp(argv[1], "sizes")) {
        printf("smem update16 %zu update8 %zu inner16 %zu inner8 %zu\n", hz::update_smem(16),
               hz::update_smem(8), hz::inner_smem_bytes(16), hz::inner_smem_bytes(8));
        for (int kk = 2; kk <= hz::KKMAX; kk += 2)
            printf("threads %d %d %d\n", kk, hz::gram_threads(kk), hz::gram_threads_c128(kk));
        return 0;
    }
    if (argc == 2 && !strcmp(argv[1], "delta")) {
        printf("%zu %zu %zu %d %d %.17g %.17g\n", hz::delta64_smem(), hz::df64_smem(), hz::update_smem(16),
               hz::UPD_R, hz::DF_R, hz::DELTA_E, hz::DF_E);
        return 0;
    }
    if (argc == 3 && !strcmp(argv[1], "rr")) {
        const int N = atoi(argv[2]);
        for (int r = 0; r < N - 1; ++r)
            for (int k = 0; k < N / 2; ++k) {
                int a, b;
                hz::rr_pair(N, r, k, &a, &b);
                printf("%d %d %d %d\n", r, k, a, b);
            }
        return 0;
    }
    return 2;
}
