// bst_launch.cuh -- host launcher of the BST forward path (the kernels are
// in bst_forward.cuh): per chunk of slice pairs, the ray, gridding and row
// kernels on one of up to two plan-owned streams, with the plan's launch
// shape (radix schedule, spectrum layout, chunk, block order, lanes).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "bst_forward.cuh"

namespace bst {

// ---------------------------------------------------------------------------
// host launcher

template <class K>
static bool set_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return true;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess;
}

template <int M> struct FwdCfg {
    static constexpr int TPL = tpl_of<M>();
    // ray kernel: 256 threads a block, or, for lengths whose line takes 256
    // threads, two interleaved angle rows in 512 (whole lines of the paired
    // layout per warp store)
    static constexpr bool ILV1 = TPL >= 256;
    static constexpr int LPC1 = ILV1 ? 2 : ((256 / TPL) > 1 ? 256 / TPL : 1);
    static constexpr int CPC = (128 / TPL) > 1 ? 128 / TPL : 1;
    static constexpr int TPC = (128 / (4 * TPL)) > 1 ? 128 / (4 * TPL) : 1;
    static constexpr size_t S1 = (size_t)LPC1 * ray_line_stride<M, ILV1>() * sizeof(float2);
    static constexpr size_t S2 = (size_t)CPC * smem_line_len(M) * sizeof(float2);
    static constexpr int CPCP = paired_cpc<M>();
    static constexpr size_t S2P = (size_t)2 * CPCP * smem_line_len(M) * sizeof(float2);
    // the register-fed gridding kernel: half-warps of 16 consecutive threads of a column
    static constexpr bool XCHG_OK = TPL % 16 == 0;
    static constexpr size_t S2X = (size_t)2 * smem_line_len(M) * sizeof(float2);
    static constexpr size_t S3 = (size_t)4 * TPC * row_line_stride<M>() * sizeof(float2);
};

// the shared-memory opt-in of the register-fed gridding kernel, where it exists
template <int M, int MAXR, int NC>
static bool set_smem_xchg() {
    using C = FwdCfg<M>;
    if constexpr (C::XCHG_OK) return set_smem(k_grid_col_xchg<M, C::TPL, MAXR, NC>, C::S2X);
    return true;
}

template <int M, int MAXR, int NC>
bst_status_t launch_forward_M(bst_plan_s* p, const float* sino, int slices, int mode, const float* g, float* vol,
                              void* ws, cudaStream_t st, int max_chunk, int lanes, const PrepArgs* prep) {
    using C = FwdCfg<M>;
    static std::atomic<unsigned long long> attr_done{0};
    if (!bsth::once_per_device(attr_done, [] {
            return set_smem(k_ray_fft<M, C::TPL, C::LPC1, MAXR, NC, C::ILV1>, C::S1) &&
                   set_smem(k_ray_fft_prep<M, C::TPL, C::LPC1, MAXR, NC>, C::S1) &&
                   set_smem(k_grid_col<M, C::TPL, C::CPC, MAXR, NC>, C::S2) &&
                   set_smem(k_grid_col_paired<M, C::TPL, C::CPCP, MAXR, NC>, C::S2P) &&
                   set_smem_xchg<M, MAXR, NC>() &&
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
    int nl = std::min(std::min(std::min(lanes, nchunks), bsth::kMaxLanes), std::max(p->max_lanes, 1));
    if (nl < 2 || p->timing || !bst_ensure_lanes(p)) nl = 1;
    const size_t lane_elems = (size_t)chunk * (V + (size_t)((N + 3) / 4) * 4) * M;
    const float scale = (float)((double)N / (2.0 * (double)M * (double)M));
    const float two_alpha = (float)(2 * p->alpha);
    const int row_tiles = (N + 3) / 4;
    const bool kbg = p->grid_kind == BST_GRID_KAISER_BESSEL;
    if (kbg && mode != BSTK_RAW) mode |= BSTK_KBW;
    // the paired spectrum layout serves the bilinear gridding kernel only
    const bool paired = !kbg && mode != BSTK_RAW && p->fwd_layout == BST_LAYOUT_PAIRED;
    if (paired) mode |= BSTK_PAIRED;
    const int pf = p->pair_fast ? 1 : 0;
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
            k_ray_fft<M, C::TPL, C::LPC1, MAXR, NC, C::ILV1><<<dim3((V + C::LPC1 - 1) / C::LPC1, np), C::TPL * C::LPC1, C::S1, s>>>(
                sino, slices, p0, N, V, mode, g, two_alpha, Z, p->tw);
        bst_timing_mark(p, s, 0);
        if (kbg) {
            const bst_status_t ks = bst_launch_kb_col(p, Z, T, np, s);
            if (ks != BST_OK) return ks;
        } else if (paired && C::XCHG_OK && p->grid_xchg) {
            if constexpr (C::XCHG_OK) {
                k_grid_col_xchg<M, C::TPL, MAXR, NC><<<pf ? dim3(np, M / 2) : dim3(M / 2, np), 2 * C::TPL, C::S2X, s>>>(
                    Z, V, N, p->geo_J, p->geo_f, T, p->tw, pf);
            }
        } else if (paired) {
            const int ncg = (M / 2 + C::CPCP - 1) / C::CPCP;
            k_grid_col_paired<M, C::TPL, C::CPCP, MAXR, NC>
                <<<pf ? dim3(np, ncg) : dim3(ncg, np), 2 * C::TPL * C::CPCP, C::S2P, s>>>(
                    Z, V, N, p->geo_J, p->geo_f, T, p->tw, pf);
        } else {
            const int ncg = (M / 2 + C::CPC - 1) / C::CPC;
            k_grid_col<M, C::TPL, C::CPC, MAXR, NC><<<pf ? dim3(np, ncg) : dim3(ncg, np), C::TPL * C::CPC, C::S2, s>>>(
                Z, V, N, p->geo_J, p->geo_f, T, p->tw, pf);
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
