// brute.cu -- slant-stack backprojection (brute_backproject), the O(N^3)
// per-slice comparator of Sec. 2, with an optional ramp-type prefilter.
//
//   k_ss_filter  per angle and slice pair: zero-pad to M, FFT along t,
//                multiply by h_k / M (h_k = |sigma_k| g[k], h_0 = dsigma/4 g[0],
//                h_{M/2} = 0), inverse FFT, crop to N samples.
//   k_ss_bp      Eq. 2 as a Riemann sum: b[r][c] = sum_j w_j y_j(i_f) with
//                i_f = (c - N/2) cos t_j + (r - N/2) sin t_j + N/2 and linear
//                interpolation (zero outside [0, N-1]).  One 16 x 16 pixel tile
//                and Q slices per block (the Q slices share the geometry, as the
//                paper's blocks of Q sinograms do); batches of angles are staged
//                in shared memory with zero fill, so the inner loop has no bounds
//                tests.  The tile origin's detector coordinate is computed in
//                double precision, the per-pixel offset (< 25 samples) in float.
#include <cuda_runtime.h>

#include <algorithm>

#include "bst_fft.cuh"
#include "bst_internal.h"

namespace bst {

template <int M> __host__ __device__ constexpr int brute_tpl() { return (M % 3 == 0) ? M / 12 : M / 16; }

struct SsRaySrc {
    const float* ya;
    const float* yb;
    int N, M;
    bool live;
    static constexpr bool kSmem = false;
    __device__ __forceinline__ float2 load(int m) const {
        int i = m + (N >> 1);
        if (i >= M) i -= M;
        if (!live || i >= N) return make_float2(0.f, 0.f);
        return make_float2(__ldg(ya + i), yb ? __ldg(yb + i) : 0.f);
    }
};

// multiply the spectrum by h_k / M while storing it back into shared memory
struct RampSmem {
    float2* p;
    const float* g;
    int M;
    float dsig;
    static constexpr bool kSmem = true;
    __device__ __forceinline__ void store(int k, float2 v) const {
        const int ak = k <= (M >> 1) ? k : M - k;
        float h;
        if (ak == (M >> 1)) h = 0.f;
        else {
            const float gk = g ? __ldg(g + ak) : 1.f;
            h = (ak == 0 ? 0.25f * dsig : (float)ak * dsig) * gk;
        }
        h = h / (float)M;
        p[k + (k >> 4)] = make_float2(v.x * h, v.y * h);
    }
    __device__ __forceinline__ float2 load(int i) const { return p[i + (i >> 4)]; }
};

struct CropDst {
    float* qa;
    float* qb;
    int N, M;
    bool live;
    static constexpr bool kSmem = false;
    __device__ __forceinline__ void store(int m, float2 v) const {
        if (!live) return;
        const int i = signed_freq(m, M) + (N >> 1);
        if (i < 0 || i >= N) return;
        qa[i] = v.x;
        if (qb) qb[i] = v.y;
    }
};

template <int M, int TPL, int LPC>
__global__ void __launch_bounds__(TPL * LPC)
    k_ss_filter(const float* __restrict__ sino, int slices, int N, int V, const float* __restrict__ g, float dsig,
                float* __restrict__ q, const float2* __restrict__ tw) {
    extern __shared__ float2 smem[];
    const int line = threadIdx.x / TPL, t = threadIdx.x % TPL;
    const int j = blockIdx.x * LPC + line;
    const int sa = 2 * blockIdx.y, sb = sa + 1;
    const bool live = j < V;
    const int jj = live ? j : 0;
    SsRaySrc src{sino + ((size_t)sa * V + jj) * N, sb < slices ? sino + ((size_t)sb * V + jj) * N : nullptr, N, M,
                 live};
    float2* base = smem + line * smem_line_len(M);
    RampSmem mid{base, g, M, dsig};
    SmemLine sm{base};
    fft_line<M, TPL, false>(t, src, mid, sm, tw);
    __syncthreads();
    CropDst dst{q + ((size_t)sa * V + jj) * N, sb < slices ? q + ((size_t)sb * V + jj) * N : nullptr, N, M, live};
    fft_line<M, TPL, true>(t, sm, dst, sm, tw);
}

constexpr int SS_TILE = 16;
constexpr int SS_AB = 16;   // angles per staged batch
constexpr int SS_W = 28;    // staged samples per angle and slice (>= 15 (|cos| + |sin|) + 4)

template <int Q>
__global__ void __launch_bounds__(256)
    k_ss_bp(const float* __restrict__ y, int S, int V, int N, const double2* __restrict__ cs64,
            const float2* __restrict__ cs32, const float* __restrict__ wq, float* __restrict__ vol) {
    __shared__ float seg[SS_AB][Q][SS_W];
    __shared__ float bfrac[SS_AB];
    __shared__ int blo[SS_AB];
    __shared__ float2 bcs[SS_AB];
    __shared__ float bw[SS_AB];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int c0 = blockIdx.x * SS_TILE, r0 = blockIdx.y * SS_TILE;
    const int s0 = blockIdx.z * Q;
    float acc[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) acc[q] = 0.f;
    for (int jb = 0; jb < V; jb += SS_AB) {
        __syncthreads();
        if (threadIdx.x < SS_AB) {
            const int j = jb + threadIdx.x;
            if (j < V) {
                const double2 cs = cs64[j];
                const double fo = (double)(c0 - N / 2) * cs.x + (double)(r0 - N / 2) * cs.y + (double)(N / 2);
                const double mn = fo + fmin(0.0, (SS_TILE - 1) * cs.x) + fmin(0.0, (SS_TILE - 1) * cs.y);
                const int lo = (int)floor(mn) - 1;
                blo[threadIdx.x] = lo;
                bfrac[threadIdx.x] = (float)(fo - (double)lo);
                bcs[threadIdx.x] = cs32[j];
                bw[threadIdx.x] = wq[j];
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < SS_AB * Q * SS_W; e += 256) {
            const int a = e / (Q * SS_W);
            const int rem = e - a * (Q * SS_W);
            const int qq = rem / SS_W, w = rem - qq * SS_W;
            const int j = jb + a, s = s0 + qq;
            float v = 0.f;
            if (j < V && s < S) {
                const int i = blo[a] + w;
                if (i >= 0 && i < N) v = __ldg(y + ((size_t)s * V + j) * N + i) * bw[a];
            }
            seg[a][qq][w] = v;
        }
        __syncthreads();
        const int na = min(SS_AB, V - jb);
        for (int a = 0; a < na; ++a) {
            const float2 cs = bcs[a];
            const float v = fmaf((float)tx, cs.x, fmaf((float)ty, cs.y, bfrac[a]));
            const float fl = floorf(v);
            const int i0 = (int)fl;
            const float f = v - fl;
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const float y0 = seg[a][q][i0], y1 = seg[a][q][i0 + 1];
                acc[q] += fmaf(f, y1 - y0, y0);
            }
        }
    }
    const int r = r0 + ty, c = c0 + tx;
    if (r < N && c < N) {
#pragma unroll
        for (int q = 0; q < Q; ++q)
            if (s0 + q < S) vol[((size_t)(s0 + q) * N + r) * N + c] = acc[q];
    }
}

template <int M>
bst_status_t launch_ss_filter_M(bst_plan_s* p, const float* sino, int slices, const float* g, float* q,
                                cudaStream_t st) {
    constexpr int TPL = brute_tpl<M>();
    constexpr int LPC = (256 / TPL) > 1 ? 256 / TPL : 1;
    constexpr size_t S = (size_t)LPC * smem_line_len(M) * sizeof(float2);
    static std::atomic<unsigned long long> attr_done{0};
    if (!bsth::once_per_device(attr_done, [] {
            return S <= 48 * 1024 || cudaFuncSetAttribute(k_ss_filter<M, TPL, LPC>,
                                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                          (int)S) == cudaSuccess;
        }))
        return BST_ERR_CUDA;
    const int pairs = (slices + 1) / 2;
    const float dsig = (float)((double)p->N / (2.0 * (double)M));
    bst_timing_mark(p, st, -1);
    k_ss_filter<M, TPL, LPC><<<dim3((p->V + LPC - 1) / LPC, pairs), TPL * LPC, S, st>>>(sino, slices, p->N, p->V, g,
                                                                                        dsig, q, p->tw);
    bst_timing_mark(p, st, 3);
    return BST_OK;
}

}  // namespace bst

size_t bst_brute_ws(const bst_plan_s* p, int slices, int filtered) {
    if (!filtered) return 0;
    return (size_t)slices * p->V * p->N * sizeof(float);
}

#define BST_FOR_EACH_M(X) \
    X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096) X(48) X(96) X(192) X(384) X(768) X(1536) X(3072)

bst_status_t bst_launch_brute(bst_plan_s* p, const float* sino, int slices, const float* g, float* vol, void* ws,
                              size_t /*ws_bytes*/, cudaStream_t st) {
    const float* y = sino;
    if (g) {
        float* q = (float*)ws;
        bst_status_t s = BST_ERR_UNSUPPORTED_SIZE;
        switch (p->M) {
#define BST_CASE(m) \
    case m: s = bst::launch_ss_filter_M<m>(p, sino, slices, g, q, st); break;
            BST_FOR_EACH_M(BST_CASE)
#undef BST_CASE
        }
        if (s != BST_OK) return s;
        y = q;
    }
    constexpr int Q = 8;
    const int N = p->N;
    dim3 grid((N + bst::SS_TILE - 1) / bst::SS_TILE, (N + bst::SS_TILE - 1) / bst::SS_TILE, (slices + Q - 1) / Q);
    bst_timing_mark(p, st, -1);
    bst::k_ss_bp<Q><<<grid, 256, 0, st>>>(y, slices, p->V, N, p->cs64, p->cs32, p->wq, vol);
    bst_timing_mark(p, st, 4);
    return cudaGetLastError() == cudaSuccess ? BST_OK : BST_ERR_CUDA;
}
