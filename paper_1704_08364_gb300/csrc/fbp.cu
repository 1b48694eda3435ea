// fbp.cu -- plan-level entry points of the BST forward path: the plan's
// geometry table, the dispatch of bst_fbp / bst_backproject / bst_fbp_prep on
// the FFT length and the pad factor (the kernels are in bst_forward.cuh,
// instantiated by fbp_pad1.cu and fbp_pad2.cu), the raw ray spectrum used by
// the adjoint, and bst_fbp_prep.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "bst_launch.cuh"

namespace bst {

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

}  // namespace bst

#define BST_FOR_EACH_M(X) \
    X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096) X(48) X(96) X(192) X(384) X(768) X(1536) X(3072)

static bst_status_t forward_dispatch(bst_plan_s* p, const float* sino, int slices, int mode, const float* g,
                                     float* vol, void* ws, cudaStream_t st, int max_chunk, int lanes,
                                     const bst::PrepArgs* prep) {
    return p->alpha == 2 ? bst_forward_pad2(p, sino, slices, mode, g, vol, ws, st, max_chunk, lanes, prep)
                         : bst_forward_pad1(p, sino, slices, mode, g, vol, ws, st, max_chunk, lanes, prep);
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
    static std::atomic<unsigned long long> attr_done{0};
    if (!bsth::once_per_device(attr_done, [] { return set_smem(k_ray_fft<M, C::TPL, C::LPC1, 16, 0>, C::S1); }))
        return BST_ERR_CUDA;
    bst_timing_mark(p, st, -1);
    k_ray_fft<M, C::TPL, C::LPC1, 16, 0><<<dim3((p->V + C::LPC1 - 1) / C::LPC1, np), C::TPL * C::LPC1, C::S1, st>>>(
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
    if (!bsth::on_plan_device(p)) return BST_ERR_INVALID_ARGUMENT;
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
