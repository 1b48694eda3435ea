// bst_forward.cuh -- the kernels of the BST forward path,
// templated on the FFT length M, the radix schedule MAXR and the ray count NC
// (N as a compile-time constant, 0 for the runtime value).  With NC known the
// padded rays' zero half and the transforms' dropped outputs are known per
// index group, so the first and last Stockham passes skip them.  Instantiated
// per pad factor by fbp_pad1.cu and fbp_pad2.cu (two translation units that
// compile in parallel); fbp.cu holds the plan-level entry points.
//
// Per pair of slices (packed as the real and imaginary parts of one complex
// line, so every FFT is a full complex transform with no waste):
//
//   k_ray_fft   stages P2 + P3 + P4: load each angle's rays with centre-aligned
//               zero padding to M, forward FFT along t in shared memory,
//               multiply by the weight W[|k|], write Z[V][M].
//   k_grid_col  stages P0 + P5 + the column half of P6: for one Cartesian
//               column c' and its mirror -c', compute the polar coordinates of
//               every point once, gather the four bilinear taps from Z for both
//               points (gather form, no atomics), inverse FFT along r' in
//               shared memory, keep the N central rows, write T.
//   k_grid_col_paired  the same from the paired layout of Z (one 16-byte
//               slot (Z[k], Z[-k]) per bin serves a point and its mirror),
//               which the ray kernel writes when the plan asks for it.
//   k_grid_col_xchg  the same for one column pair per block with the first
//               FFT pass of both columns fed from registers (partner lanes
//               swap the halves of their gathered point pairs).
//   k_row_ifft  the row half of P6 + P7 + P8: inverse FFT along c' for four
//               rows at a time, keep the N central columns, scale by
//               dt dw^2 = N / (2 M^2), write Re to slice a and Im to slice b.
//
// Z and T live in a caller-provided workspace sized for a chunk of pairs
// that fits in L2 where possible (one pair at N = 2048: 2 x 64 MiB).
// This header holds device code only; the host launcher is bst_launch.cuh.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "bst_stages.cuh"

namespace bst {

// ---------------------------------------------------------------------------
// per-size kernels: one slice pair per blockIdx.y of a chunk

// ILV: the block's LPC angle rows interleaved over its lanes (ray_unit)
template <int M, int TPL, int LPC, int MAXR, int NC = 0, bool ILV = false>
__global__ void __launch_bounds__(TPL * LPC, (TPL * LPC <= 1024) ? 1024 / (TPL * LPC) : 1)
    k_ray_fft(const float* __restrict__ sino, int slices, int pair0, int N, int V, int mode,
              const float* __restrict__ g, float two_alpha, float2* __restrict__ Z, const float2* __restrict__ tw) {
    extern __shared__ float2 smem[];
    const int pl = blockIdx.y;
    const int sa = 2 * (pair0 + pl), sb = sa + 1;
    ray_unit<M, TPL, LPC, MAXR, NC, BlockSync, ILV, true>(smem, blockIdx.x * LPC, V, N, sino + (size_t)sa * V * N,
                                                    sb < slices ? sino + (size_t)sb * V * N : nullptr, mode, g,
                                                    two_alpha, Z + (size_t)pl * V * M, tw);
}

template <int M, int TPL, int LPC, int MAXR, int NC = 0>
__global__ void __launch_bounds__(TPL * LPC, (TPL * LPC <= 1024) ? 1024 / (TPL * LPC) : 1)
    k_ray_fft_prep(const float* __restrict__ sino, int slices, int pair0, int N, int V, PrepArgs pa, int mode,
                   const float* __restrict__ g, float two_alpha, float2* __restrict__ Z,
                   const float2* __restrict__ tw) {
    extern __shared__ float2 smem[];
    const int pl = blockIdx.y;
    const int sa = 2 * (pair0 + pl), sb = sa + 1;
    const bool hb = sb < slices;
    ray_unit_prep<M, TPL, LPC, MAXR, NC>(
        smem, blockIdx.x * LPC, V, N, sino + (size_t)sa * V * N, hb ? sino + (size_t)sb * V * N : nullptr,
        pa.dark ? pa.dark + (size_t)sa * N : nullptr, (pa.dark && hb) ? pa.dark + (size_t)sb * N : nullptr,
        pa.flat ? pa.flat + (size_t)sa * N : nullptr, (pa.flat && hb) ? pa.flat + (size_t)sb * N : nullptr, pa, mode,
        g, two_alpha, Z + (size_t)pl * V * M, tw);
}

// gridding launches: grid (column groups, pairs), or with pair_fast
// (pairs, column groups) so that the blocks of one column group for all the
// chunk's pairs run together and share the group's geometry-table reads in L2
template <int M, int TPL, int CPC, int MAXR, int NC = 0>
__global__ void __launch_bounds__(TPL * CPC, (TPL * CPC <= 256) ? 1024 / (TPL * CPC) : 1)
    k_grid_col(const float2* __restrict__ Z, int V, int N, const int* __restrict__ gJ,
               const float2* __restrict__ gF, float2* __restrict__ T, const float2* __restrict__ tw, int pair_fast) {
    extern __shared__ float2 smem[];
    const int pl = pair_fast ? blockIdx.x : blockIdx.y;
    const int cg = pair_fast ? blockIdx.y : blockIdx.x;
    grid_unit<M, TPL, CPC, MAXR, NC>(smem, cg * CPC, V, N, Z + (size_t)pl * V * M, gJ, gF,
                                 T + (size_t)pl * ((N + 3) / 4) * 4 * M, tw);
}

// the same stages from the paired spectrum layout (grid_unit_paired)
template <int M, int TPL, int CPC, int MAXR, int NC = 0>
__global__ void __launch_bounds__(2 * TPL * CPC, (2 * TPL * CPC <= 1024) ? 1024 / (2 * TPL * CPC) : 1)
    k_grid_col_paired(const float2* __restrict__ Z, int V, int N, const int* __restrict__ gJ,
                      const float2* __restrict__ gF, float2* __restrict__ T, const float2* __restrict__ tw,
                      int pair_fast) {
    extern __shared__ float2 smem[];
    const int pl = pair_fast ? blockIdx.x : blockIdx.y;
    const int cg = pair_fast ? blockIdx.y : blockIdx.x;
    grid_unit_paired<M, TPL, CPC, MAXR, NC>(smem, cg * CPC, V, N,
                                            reinterpret_cast<const float4*>(Z + (size_t)pl * V * M), gJ, gF,
                                            T + (size_t)pl * ((N + 3) / 4) * 4 * M, tw);
}

// the same for one column pair per block, the first FFT pass of both columns
// fed from registers (grid_unit_xchg)
template <int M, int TPL, int MAXR, int NC = 0, int PS = 2>
__global__ void __launch_bounds__(2 * TPL, (2 * TPL <= 1024) ? 1024 / (2 * TPL) : 1)
    k_grid_col_xchg(const float2* __restrict__ Z, int V, int N, const int* __restrict__ gJ,
                    const float2* __restrict__ gF, float2* __restrict__ T, const float2* __restrict__ tw,
                    int pair_fast) {
    extern __shared__ float2 smem[];
    const int pl = pair_fast ? blockIdx.x : blockIdx.y;
    const int cq = pair_fast ? blockIdx.y : blockIdx.x;
    grid_unit_xchg<M, TPL, MAXR, NC, PS>(smem, cq, V, N, reinterpret_cast<const float4*>(Z + (size_t)pl * V * M), gJ,
                                         gF, T + (size_t)pl * ((N + 3) / 4) * 4 * M, tw);
}

template <int M, int TPL, int TPC, int MAXR, int NC = 0>
__global__ void __launch_bounds__(4 * TPL * TPC)
    k_row_ifft(const float2* __restrict__ T, int slices, int pair0, int N, float scale, float* __restrict__ vol,
               const float2* __restrict__ tw, const float* __restrict__ dk) {
    extern __shared__ float2 smem[];
    const int pl = blockIdx.y;
    const int sa = 2 * (pair0 + pl), sb = sa + 1;
    row_unit<M, TPL, TPC, MAXR, NC>(smem, blockIdx.x * TPC, N, T + (size_t)pl * ((N + 3) / 4) * 4 * M,
                                vol + (size_t)sa * N * N, sb < slices ? vol + (size_t)sb * N * N : nullptr, scale,
                                tw, dk);
}

}  // namespace bst
