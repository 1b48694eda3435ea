// Test-only host program (compiled and run by tests/test_kernel_resources.py,
// no GPU needed): the slot map of the paired spectrum layout is a bijection
// from (row j < V, bin m < M/2) onto [0, V M/2), for even and odd row counts,
// the two rows of a pair share each 128-byte line four bins at a time, and
// the offsets between neighbouring bins and rows that the gather relies on.
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
                    // the offsets the gather uses away from the seam: next bin and next row
                    if (j + 1 < (V & ~1)) {
                        const int dr = (j & 1) ? 2 * H - 4 : 4;
                        if (bst::paired_slot(j + 1, m, H, V) != s + dr) {
                            std::printf("FAIL row offset M=%d V=%d j=%d m=%d\n", M, V, j, m);
                            return 1;
                        }
                        if (m + 1 < H && bst::paired_slot(j, m + 1, H, V) != s + ((m & 3) == 3 ? 5 : 1)) {
                            std::printf("FAIL bin offset M=%d V=%d j=%d m=%d\n", M, V, j, m);
                            return 1;
                        }
                    }
                }
        }
    std::printf("OK\n");
    return 0;
}
