// fbp.cu -- the BST forward path (bst_fbp, bst_backproject) on sm_103a.
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
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "bst_stages.cuh"

namespace bst {

// ---------------------------------------------------------------------------
// per-size kernels: one slice pair per blockIdx.y of a chunk

template <int M, int TPL, int LPC, int MAXR>
__global__ void __launch_bounds__(TPL * LPC)
    k_ray_fft(const float* __restrict__ sino, int slices, int pair0, int N, int V, int mode,
              const float* __restrict__ g, float two_alpha, float2* __restrict__ Z, const float2* __restrict__ tw) {
    extern __shared__ float2 smem[];
    const int pl = blockIdx.y;
    const int sa = 2 * (pair0 + pl), sb = sa + 1;
    ray_unit<M, TPL, LPC, MAXR>(smem, blockIdx.x * LPC, V, N, sino + (size_t)sa * V * N,
                                sb < slices ? sino + (size_t)sb * V * N : nullptr, mode, g, two_alpha,
                                Z + (size_t)pl * V * M, tw);
}

// Plan set-up: the angular part of the geometry of every point (q, r') of the
// half grid q in [0, M/2) (the mirror half shares it), bracket -2 for points
// that are zero (outside the band, or the origin, which takes the DC mean).
__global__ void k_geo_table(Geo geo, int M, int* __restrict__ gJ, float2* __restrict__ gF) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)(M / 2) * M) return;
    const int q = (int)(idx / M), ridx = (int)(idx % M);
    const int ry = signed_freq(ridx, M);
    Polar P;
    int jk = (int)(-2 * 65536);
    float2 f = make_float2(0.f, 0.f);
    if (!(q == 0 && ry == 0) && polar_of(q, ry, geo, P)) {
        jk = P.J * 65536 + P.k0;
        f = make_float2(P.fth, P.frac);
    }
    gJ[idx] = jk;
    gF[idx] = f;
}

template <int M, int TPL, int LPC, int MAXR>
__global__ void __launch_bounds__(TPL * LPC)
    k_ray_fft_prep(const float* __restrict__ sino, int slices, int pair0, int N, int V, PrepArgs pa, int mode,
                   const float* __restrict__ g, float two_alpha, float2* __restrict__ Z,
                   const float2* __restrict__ tw) {
    extern __shared__ float2 smem[];
    const int pl = blockIdx.y;
    const int sa = 2 * (pair0 + pl), sb = sa + 1;
    const bool hb = sb < slices;
    ray_unit_prep<M, TPL, LPC, MAXR>(
        smem, blockIdx.x * LPC, V, N, sino + (size_t)sa * V * N, hb ? sino + (size_t)sb * V * N : nullptr,
        pa.dark ? pa.dark + (size_t)sa * N : nullptr, (pa.dark && hb) ? pa.dark + (size_t)sb * N : nullptr,
        pa.flat ? pa.flat + (size_t)sa * N : nullptr, (pa.flat && hb) ? pa.flat + (size_t)sb * N : nullptr, pa, mode,
        g, two_alpha, Z + (size_t)pl * V * M, tw);
}

template <int M, int TPL, int CPC, int MAXR>
__global__ void __launch_bounds__(TPL * CPC, (TPL * CPC <= 256) ? 1024 / (TPL * CPC) : 1)
    k_grid_col(const float2* __restrict__ Z, int V, int N, const int* __restrict__ gJ,
               const float2* __restrict__ gF, float2* __restrict__ T, const float2* __restrict__ tw) {
    extern __shared__ float2 smem[];
    const int pl = blockIdx.y;
    grid_unit<M, TPL, CPC, MAXR>(smem, blockIdx.x * CPC, V, N, Z + (size_t)pl * V * M, gJ, gF,
                                 T + (size_t)pl * ((N + 3) / 4) * 4 * M, tw);
}

template <int M, int TPL, int TPC, int MAXR>
__global__ void __launch_bounds__(4 * TPL * TPC)
    k_row_ifft(const float2* __restrict__ T, int slices, int pair0, int N, float scale, float* __restrict__ vol,
               const float2* __restrict__ tw, const float* __restrict__ dk) {
    extern __shared__ float2 smem[];
    const int pl = blockIdx.y;
    const int sa = 2 * (pair0 + pl), sb = sa + 1;
    row_unit<M, TPL, TPC, MAXR>(smem, blockIdx.x * TPC, N, T + (size_t)pl * ((N + 3) / 4) * 4 * M,
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

template <int M, int MAXR>
bst_status_t launch_forward_M(bst_plan_s* p, const float* sino, int slices, int mode, const float* g, float* vol,
                              void* ws, cudaStream_t st, int max_chunk, int lanes, const PrepArgs* prep) {
    using C = FwdCfg<M>;
    static bool attr_ok = set_smem(k_ray_fft<M, C::TPL, C::LPC1, MAXR>, C::S1) &&
                          set_smem(k_ray_fft_prep<M, C::TPL, C::LPC1, MAXR>, C::S1) &&
                          set_smem(k_grid_col<M, C::TPL, C::CPC, MAXR>, C::S2) &&
                          set_smem(k_row_ifft<M, C::TPL, C::TPC, MAXR>, C::S3);
    if (!attr_ok) return BST_ERR_CUDA;
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
            k_ray_fft_prep<M, C::TPL, C::LPC1, MAXR>
                <<<dim3((V + C::LPC1 - 1) / C::LPC1, np), C::TPL * C::LPC1, C::S1, s>>>(
                    sino, slices, p0, N, V, *prep, mode, g, two_alpha, Z, p->tw);
        else
            k_ray_fft<M, C::TPL, C::LPC1, MAXR><<<dim3((V + C::LPC1 - 1) / C::LPC1, np), C::TPL * C::LPC1, C::S1, s>>>(
                sino, slices, p0, N, V, mode, g, two_alpha, Z, p->tw);
        bst_timing_mark(p, s, 0);
        if (kbg) {
            const bst_status_t ks = bst_launch_kb_col(p, Z, T, np, s);
            if (ks != BST_OK) return ks;
        } else {
            k_grid_col<M, C::TPL, C::CPC, MAXR><<<dim3((M / 2 + C::CPC - 1) / C::CPC, np), C::TPL * C::CPC, C::S2, s>>>(
                Z, V, N, p->geo_J, p->geo_f, T, p->tw);
        }
        bst_timing_mark(p, s, 1);
        k_row_ifft<M, C::TPL, C::TPC, MAXR><<<dim3((row_tiles + C::TPC - 1) / C::TPC, np), 4 * C::TPL * C::TPC, C::S3, s>>>(
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

#define BST_FOR_EACH_M(X) \
    X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096) X(48) X(96) X(192) X(384) X(768) X(1536) X(3072)

static bst_status_t forward_dispatch(bst_plan_s* p, const float* sino, int slices, int mode, const float* g,
                                     float* vol, void* ws, cudaStream_t st, int max_chunk, int lanes,
                                     const bst::PrepArgs* prep) {
    switch (p->M) {
#define BST_CASE(m)                                                                                         \
    case m:                                                                                                 \
        return p->maxr == 8                                                                                 \
                   ? bst::launch_forward_M<m, 8>(p, sino, slices, mode, g, vol, ws, st, max_chunk, lanes, prep) \
                   : bst::launch_forward_M<m, 16>(p, sino, slices, mode, g, vol, ws, st, max_chunk, lanes, prep);
        BST_FOR_EACH_M(BST_CASE)
#undef BST_CASE
    }
    return BST_ERR_UNSUPPORTED_SIZE;
}

bst_status_t bst_launch_forward_chunked(bst_plan_s* p, const float* sino, int slices, int mode, const float* g,
                                        float* vol, void* ws, cudaStream_t st, int max_chunk, int lanes) {
    return forward_dispatch(p, sino, slices, mode, g, vol, ws, st, max_chunk, lanes, nullptr);
}

bst_status_t bst_launch_forward_prep(bst_plan_s* p, const float* sino, int slices, const bst::PrepArgs& prep,
                                     const float* g, float* vol, void* ws, size_t ws_bytes, cudaStream_t st) {
    const int pairs = (slices + 1) / 2;
    const int chunk = std::min(pairs, p->chunk_pairs);
    const int lanes = (int)std::min<size_t>(bsth::kMaxLanes, ws_bytes / ((size_t)chunk * bsth::fwd_bytes_per_pair(p)));
    return forward_dispatch(p, sino, slices, BSTK_FILTER, g, vol, ws, st, p->chunk_pairs, lanes, &prep);
}

bst_status_t bst_launch_forward(bst_plan_s* p, const float* sino, int slices, int mode, const float* g, float* vol,
                                void* ws, size_t ws_bytes, cudaStream_t st) {
    const int pairs = (slices + 1) / 2;
    const int chunk = std::min(pairs, p->chunk_pairs);
    const int lanes = (int)std::min<size_t>(bsth::kMaxLanes, ws_bytes / ((size_t)chunk * bsth::fwd_bytes_per_pair(p)));
    return bst_launch_forward_chunked(p, sino, slices, mode, g, vol, ws, st, p->chunk_pairs, lanes);
}

namespace bst {
template <int M>
bst_status_t launch_ray_spectrum_M(bst_plan_s* p, const float* sino, int slices, int p0, int np, float2* Y,
                                   cudaStream_t st) {
    using C = FwdCfg<M>;
    static bool attr_ok = set_smem(k_ray_fft<M, C::TPL, C::LPC1, 16>, C::S1);
    if (!attr_ok) return BST_ERR_CUDA;
    bst_timing_mark(p, st, -1);
    k_ray_fft<M, C::TPL, C::LPC1, 16><<<dim3((p->V + C::LPC1 - 1) / C::LPC1, np), C::TPL * C::LPC1, C::S1, st>>>(
        sino, slices, p0, p->N, p->V, BSTK_RAW, nullptr, 0.f, Y, p->tw);
    bst_timing_mark(p, st, 0);
    return BST_OK;
}
}  // namespace bst

// Y[pair][V][M] = unscaled DFT of the padded rays of pairs [p0, p0 + np), no weight
bst_status_t bst_launch_ray_spectrum(bst_plan_s* p, const float* sino, int slices, int p0, int np, float2* Y,
                                     cudaStream_t st) {
    switch (p->M) {
#define BST_CASE(m) \
    case m: return bst::launch_ray_spectrum_M<m>(p, sino, slices, p0, np, Y, st);
        BST_FOR_EACH_M(BST_CASE)
#undef BST_CASE
    }
    return BST_ERR_UNSUPPORTED_SIZE;
}

bst_status_t bst_build_geo_table(bst_plan_s* p) {
    const size_t n = (size_t)(p->M / 2) * p->M;
    if (cudaMalloc((void**)&p->geo_J, n * sizeof(int)) != cudaSuccess) return BST_ERR_OUT_OF_MEMORY;
    if (cudaMalloc((void**)&p->geo_f, n * sizeof(float2)) != cudaSuccess) return BST_ERR_OUT_OF_MEMORY;
    bst::k_geo_table<<<(unsigned)((n + 255) / 256), 256>>>(p->geo(), p->M, p->geo_J, p->geo_f);
    if (cudaGetLastError() != cudaSuccess) return BST_ERR_CUDA;
    return cudaDeviceSynchronize() == cudaSuccess ? BST_OK : BST_ERR_CUDA;
}

extern "C" bst_status_t bst_fbp_prep(bst_plan_t p, const float* d_sino, int slices, const float* d_dark,
                                     const float* d_flat, float shift, float kb_beta, float kb_halfwidth,
                                     const float* d_g, float* d_volume, void* d_ws, size_t ws_bytes,
                                     bst_stream_t stream) {
    if (!p || !d_sino || !d_volume || slices <= 0) return BST_ERR_INVALID_ARGUMENT;
    if (d_dark && !d_flat) return BST_ERR_INVALID_ARGUMENT;
    if (!std::isfinite(shift) || std::fabs(shift) >= (float)p->N) return BST_ERR_INVALID_ARGUMENT;
    if (!(kb_beta >= 0.f) || !std::isfinite(kb_beta) || (kb_beta > 0.f && !(kb_halfwidth > 0.f)))
        return BST_ERR_INVALID_ARGUMENT;
    const size_t ns = (size_t)slices * p->V * p->N * sizeof(float), nv = (size_t)slices * p->N * p->N * sizeof(float);
    const uintptr_t a0 = (uintptr_t)d_sino, b0 = (uintptr_t)d_volume;
    if (a0 < b0 + nv && b0 < a0 + ns) return BST_ERR_INVALID_ARGUMENT;
    if (!d_ws || ws_bytes < bst_workspace_bytes(p, slices)) return BST_ERR_WORKSPACE_TOO_SMALL;
    bst::PrepArgs pa;
    pa.dark = d_dark;
    pa.flat = d_flat;
    pa.shift = shift;
    pa.shift_int = (int)std::floor(shift);
    pa.shift_frac = (float)((double)shift - std::floor((double)shift));
    pa.kb_beta = kb_beta;
    pa.kb_inv_half = kb_beta > 0.f ? 1.f / kb_halfwidth : 0.f;
    pa.kb_norm = kb_beta > 0.f ? (float)(1.0 / bst_bessel_i0((double)kb_beta)) : 1.f;
    return bst_launch_forward_prep(p, d_sino, slices, pa, d_g, d_volume, d_ws, ws_bytes, (cudaStream_t)stream);
}
