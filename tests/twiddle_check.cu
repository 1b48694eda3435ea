// Test-only host program (compiled and run by tests/test_kernel_resources.py,
// no GPU needed): the twiddle allocation of a plan (make_twiddles in
// bst_twiddle.h) for every supported FFT length.  The radices of each
// schedule multiply to M; the per-pass tables of both schedules tile the
// allocation after the base table exactly once, at the offsets the FFT
// kernels read (pass_tab_base); and every entry (s - 1) NS + k of a pass
// equals exp(-2 pi i k s / (NS R)) to float rounding.
#include <cmath>
#include <cstdio>
#include <vector>

#include "bst_twiddle.h"

int main() {
    const int Ms[] = {16, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048, 3072, 4096};
    for (int M : Ms) {
        const std::vector<float2> tw = bst::make_twiddles(M);
        if ((int)tw.size() != bst::tw_alloc_len(M)) {
            std::printf("FAIL size M=%d\n", M);
            return 1;
        }
        std::vector<int> owner(tw.size(), 0);
        for (int maxr : {16, 8}) {
            const int P = bst::pass_count(M, maxr);
            int prod = 1;
            for (int p = 0; p < P; ++p) {
                if (bst::pass_ns(M, p, maxr) != prod) {
                    std::printf("FAIL ns M=%d maxr=%d p=%d\n", M, maxr, p);
                    return 1;
                }
                prod *= bst::radix_of(M, p, maxr);
            }
            if (prod != M) {
                std::printf("FAIL radices M=%d maxr=%d\n", M, maxr);
                return 1;
            }
            for (int p = 1; p < P; ++p) {
                const int R = bst::radix_of(M, p, maxr), NS = bst::pass_ns(M, p, maxr);
                const int base = bst::pass_tab_base(M, maxr, p);
                for (int s = 1; s < R; ++s)
                    for (int k = 0; k < NS; ++k) {
                        const int i = base + (s - 1) * NS + k;
                        if (i < M || i >= (int)tw.size()) {
                            std::printf("FAIL range M=%d maxr=%d p=%d\n", M, maxr, p);
                            return 1;
                        }
                        ++owner[i];
                        const double a = -2.0 * M_PI * (double)k * s / ((double)NS * R);
                        if (std::fabs(tw[i].x - std::cos(a)) > 1e-7 || std::fabs(tw[i].y - std::sin(a)) > 1e-7) {
                            std::printf("FAIL value M=%d maxr=%d p=%d s=%d k=%d\n", M, maxr, p, s, k);
                            return 1;
                        }
                    }
            }
        }
        for (size_t i = M; i < owner.size(); ++i)
            if (owner[i] != 1) {
                std::printf("FAIL coverage M=%d entry %zu used %d times\n", M, i, owner[i]);
                return 1;
            }
    }
    std::printf("OK\n");
    return 0;
}
