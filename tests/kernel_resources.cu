// Test-only translation unit (compiled by tests/test_kernel_resources.py, never
// linked): instantiates the forward kernels of the 2048^3 workload
// (M = 4096 at pad factor 2, N = 2048, radix-16 schedule) so that a CPU test
// can read their register and spill figures from ptxas.
#include "bst_forward.cuh"

template __global__ void bst::k_ray_fft<4096, 256, 2, 16, 2048, true>(const float*, int, int, int, int, int,
                                                                       const float*, float, float2*, const float2*);
template __global__ void bst::k_grid_col<4096, 256, 1, 16, 2048>(const float2*, int, int, const int*, const float2*,
                                                                  float2*, const float2*, int);
template __global__ void bst::k_grid_col_paired<4096, 256, 1, 16, 2048>(const float2*, int, int, const int*,
                                                                         const float2*, float2*, const float2*, int);
template __global__ void bst::k_row_ifft<4096, 256, 1, 16, 2048>(const float2*, int, int, int, float, float*,
                                                                  const float2*, const float*);
template __global__ void bst::k_grid_col_xchg<4096, 256, 16, 2048, 2>(const float2*, int, int, const int*,
                                                                       const float2*, float2*, const float2*, int);
