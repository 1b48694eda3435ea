// bst_forward.cuh -- the kernels of the BST forward path and their launcher,
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
//   k_row_ifft  the row half of P6 + P7 + P8: inverse FFT along c' for four
//               rows at a time, keep the N central columns, scale by
//               dt dw^2 = N / (2 M^2), write Re to slice a and Im to slice b.
//
// Z and T live in a caller-provided workspace sized for a chunk of pairs
// that fits in L2 where possible (one pair at N = 2048: 2 x 64 MiB).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "bst_stages.cuh"

namespace bst {

// ---------------------------------------------------------------------------
// per-size kernels: one slice pair per blockIdx.y of a chunk

template <int M, int TPL, int LPC, int MAXR, int NC = 0>
__global__ void __launch_bounds__(TPL * LPC)
    k_ray_fft(const float* __restrict__ sino, int slices, int pair0, int N, int V, int mode,
              const float* __restrict__ g, float two_alpha, float2* __restrict__ Z, const float2* __restrict__ tw) {
    extern __shared__ float2 smem[];
    const int pl = blockIdx.y;
    const int sa = 2 * (pair0 + pl), sb = sa + 1;
    ray_unit<M, TPL, LPC, MAXR, NC>(smem, blockIdx.x * LPC, V, N, sino + (size_t)sa * V * N,
                                sb < slices ? sino + (size_t)sb * V * N : nullptr, mode, g, two_alpha,
                                Z + (size_t)pl * V * M, tw);
}

template <int M, int TPL, int LPC, int MAXR, int NC = 0>
__global__ void __launch_bounds__(TPL * LPC)
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

template <int M, int TPL, int CPC, int MAXR, int NC = 0>
__global__ void __launch_bounds__(TPL * CPC, (TPL * CPC <= 256) ? 1024 / (TPL * CPC) : 1)
    k_grid_col(const float2* __restrict__ Z, int V, int N, const int* __restrict__ gJ,
               const float2* __restrict__ gF, float2* __restrict__ T, const float2* __restrict__ tw) {
    extern __shared__ float2 smem[];
    const int pl = blockIdx.y;
    grid_unit<M, TPL, CPC, MAXR, NC>(smem, blockIdx.x * CPC, V, N, Z + (size_t)pl * V * M, gJ, gF,
                                 T + (size_t)pl * ((N + 3) / 4) * 4 * M, tw);
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

// ---------------------------------------------------------------------------
// host launcher

template <class K>
static bool set_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return true;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess;
}

template <int M> struct FwdCfg {
    static constexpr int TPL = tpl_of<M>();
    static constexpr int LPC1 = (256 / TPL) > 1 ? 256 / TPL : 1;
    static constexpr int CPC = (128 / TPL) > 1 ? 128 / TPL : 1;
    static constexpr int TPC = (128 / (4 * TPL)) > 1 ? 128 / (4 * TPL) : 1;
    static constexpr size_t S1 = (size_t)LPC1 * smem_line_len(M) * sizeof(float2);
    static constexpr size_t S2 = (size_t)CPC * smem_line_len(M) * sizeof(float2);
    static constexpr size_t S3 = (size_t)4 * TPC * row_line_stride<M>() * sizeof(float2);
};

template <int M, int MAXR, int NC>
bst_status_t launch_forward_M(bst_plan_s* p, const float* sino, int slices, int mode, const float* g, float* vol,
                              void* ws, cudaStream_t st, int max_chunk, int lanes, const PrepArgs* prep) {
    using C = FwdCfg<M>;
    static std::atomic<unsigned long long> attr_done{0};
    if (!bsth::once_per_device(attr_done, [] {
            return set_smem(k_ray_fft<M, C::TPL, C::LPC1, MAXR, NC>, C::S1) &&
                   set_smem(k_ray_fft_prep<M, C::TPL, C::LPC1, MAXR, NC>, C::S1) &&
                   set_smem(k_grid_col<M, C::TPL, C::CPC, MAXR, NC>, C::S2) &&
                   set_smem(k_row_ifft<M, C::TPL, C::TPC, MAXR, NC>, C::S3);
        }))
        return BST_ERR_CUDA;
    const int N = p->N, V = p->V;
    const int pairs = (slices + 1) / 2;
    const int chunk = std::min(pairs, max_chunk);
    const int nchunks = (pairs + chunk - 1) / chunk;
    // chunks rotate over up to kMaxLanes streams (each with its own part of the
    // workspace) so that one chunk's gridding overlaps the next chunk's FFTs;
    // per-stage timing keeps everything on the caller's stream
    int nl = std::min(std::min(lanes, nchunks), bsth::kMaxLanes);
    if (nl < 2 || p->timing || !bst_ensure_lanes(p)) nl = 1;
    const size_t lane_elems = (size_t)chunk * (V + (size_t)((N + 3) / 4) * 4) * M;
    const float scale = (float)((double)N / (2.0 * (double)M * (double)M));
    const float two_alpha = (float)(2 * p->alpha);
    const int row_tiles = (N + 3) / 4;
    const bool kbg = p->grid_kind == BST_GRID_KAISER_BESSEL;
    if (kbg && mode != BSTK_RAW) mode |= BSTK_KBW;
    const float* dk = kbg ? p->kb_dk : nullptr;
    if (nl > 1) {
        if (cudaEventRecord(p->ev_fork, st) != cudaSuccess) return BST_ERR_CUDA;
        for (int l = 0; l < nl; ++l)
            if (cudaStreamWaitEvent(p->lane[l], p->ev_fork, 0) != cudaSuccess) return BST_ERR_CUDA;
    }
    for (int c = 0; c < nchunks; ++c) {
        const int p0 = c * chunk;
        const int np = std::min(chunk, pairs - p0);
        const int l = c % nl;
        cudaStream_t s = nl > 1 ? p->lane[l] : st;
        float2* Z = (float2*)ws + (size_t)l * lane_elems;
        float2* T = Z + (size_t)chunk * V * M;
        bst_timing_mark(p, s, -1);
        if (prep)
            k_ray_fft_prep<M, C::TPL, C::LPC1, MAXR, NC>
                <<<dim3((V + C::LPC1 - 1) / C::LPC1, np), C::TPL * C::LPC1, C::S1, s>>>(
                    sino, slices, p0, N, V, *prep, mode, g, two_alpha, Z, p->tw);
        else
            k_ray_fft<M, C::TPL, C::LPC1, MAXR, NC><<<dim3((V + C::LPC1 - 1) / C::LPC1, np), C::TPL * C::LPC1, C::S1, s>>>(
                sino, slices, p0, N, V, mode, g, two_alpha, Z, p->tw);
        bst_timing_mark(p, s, 0);
        if (kbg) {
            const bst_status_t ks = bst_launch_kb_col(p, Z, T, np, s);
            if (ks != BST_OK) return ks;
        } else {
            k_grid_col<M, C::TPL, C::CPC, MAXR, NC><<<dim3((M / 2 + C::CPC - 1) / C::CPC, np), C::TPL * C::CPC, C::S2, s>>>(
                Z, V, N, p->geo_J, p->geo_f, T, p->tw);
        }
        bst_timing_mark(p, s, 1);
        k_row_ifft<M, C::TPL, C::TPC, MAXR, NC><<<dim3((row_tiles + C::TPC - 1) / C::TPC, np), 4 * C::TPL * C::TPC, C::S3, s>>>(
            T, slices, p0, N, scale, vol, p->tw, dk);
        bst_timing_mark(p, s, 2);
    }
    if (nl > 1) {
        for (int l = 0; l < nl; ++l) {
            if (cudaEventRecord(p->ev_join[l], p->lane[l]) != cudaSuccess) return BST_ERR_CUDA;
            if (cudaStreamWaitEvent(st, p->ev_join[l], 0) != cudaSuccess) return BST_ERR_CUDA;
        }
    }
    return cudaGetLastError() == cudaSuccess ? BST_OK : BST_ERR_CUDA;
}

}  // namespace bst
