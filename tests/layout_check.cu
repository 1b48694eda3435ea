// Test-only host program (compiled and run by tests/test_kernel_resources.py,
// no GPU needed): the slot map of the paired spectrum layout is a bijection
// from (row j < V, bin m < M/2) onto [0, V M/2), for even and odd row counts,
// and the two rows of a pair share each 128-byte line four bins at a time.
#include <cstdio>
#include <vector>

#include "bst_stages.cuh"

int main() {
    const int Ms[] = {16, 48, 512, 768, 4096};
    const int Vs[] = {2, 3, 7, 8, 57, 2000, 2048, 2049};
    for (int M : Ms)
        for (int V : Vs) {
            const int H = M / 2;
            std::vector<int> seen((size_t)V * H, 0);
            for (int j = 0; j < V; ++j)
                for (int m = 0; m < H; ++m) {
                    const int s = bst::paired_slot(j, m, H, V);
                    if (s < 0 || s >= V * H || seen[s]++) {
                        std::printf("FAIL M=%d V=%d j=%d m=%d slot=%d\n", M, V, j, m, s);
                        return 1;
                    }
                    if (j + 1 < (V & ~1) && (j % 2) == 0 && bst::paired_slot(j + 1, m, H, V) / 8 != s / 8) {
                        std::printf("FAIL line sharing M=%d V=%d j=%d m=%d\n", M, V, j, m);
                        return 1;
                    }
                }
        }
    std::printf("OK\n");
    return 0;
}
