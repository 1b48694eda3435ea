// bst_twiddle.h -- host construction of a plan's twiddle allocation: the base
// table tw[m] = exp(-2 pi i m / M), m < M, computed in double precision, then
// the per-pass tables of both radix schedules (largest radix 16, then 8), at
// the offsets that bst_fft.cuh's pass_tab_base gives: entry (s - 1) NS + k of
// pass p (radix R, sub-transform length NS) is w^(k s), w = exp(-2 pi i /
// (NS R)), i.e. tw[k s M / (NS R)].
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "bst_fft.cuh"

namespace bst {

inline std::vector<float2> make_twiddles(int M) {
    std::vector<float2> tw(tw_alloc_len(M));
    for (int m = 0; m < M; ++m) {
        const double a = -2.0 * M_PI * (double)m / (double)M;
        tw[m] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    for (int maxr : {16, 8})
        for (int pp = 1; pp < pass_count(M, maxr); ++pp) {
            const int R = radix_of(M, pp, maxr), NS = pass_ns(M, pp, maxr);
            const int base = pass_tab_base(M, maxr, pp), step = M / (NS * R);
            for (int s = 1; s < R; ++s)
                for (int k = 0; k < NS; ++k) tw[base + (s - 1) * NS + k] = tw[k * s * step];
        }
    return tw;
}

}  // namespace bst
