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

#include "bst_fft.cuh"
#include "bst_geo.cuh"
#include "bst_internal.h"

namespace bst {

// threads per line: 16 elements per thread (12 for lengths 3 * 2^a)
template <int M> __host__ __device__ constexpr int tpl_of() { return (M % 3 == 0) ? M / 12 : M / 16; }

// ---------------------------------------------------------------------------
// k_ray_fft

struct RaySrc {
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

struct SpecDst {
    float2* z;
    const float* g;
    int M, mode;
    float two_alpha;
    bool live;
    static constexpr bool kSmem = false;
    __device__ __forceinline__ void store(int k, float2 v) const {
        if (!live) return;
        const int ak = k <= (M >> 1) ? k : M - k;
        float w;
        if (mode == BSTK_RAW) w = 1.f;
        else if (ak == (M >> 1)) w = 0.f;
        else if (mode == BSTK_FILTER) w = g ? __ldg(g + ak) : 1.f;
        else w = ak == 0 ? 0.f : __fdiv_rn(two_alpha, (float)ak);
        z[k] = make_float2(v.x * w, v.y * w);
    }
};

template <int M, int TPL, int LPC>
__global__ void __launch_bounds__(TPL * LPC)
    k_ray_fft(const float* __restrict__ sino, int slices, int pair0, int N, int V, int mode,
              const float* __restrict__ g, float two_alpha, float2* __restrict__ Z, const float2* __restrict__ tw) {
    extern __shared__ float2 smem[];
    const int line = threadIdx.x / TPL, t = threadIdx.x % TPL;
    const int j = blockIdx.x * LPC + line;
    const int pl = blockIdx.y;
    const int sa = 2 * (pair0 + pl), sb = sa + 1;
    const bool live = j < V;
    const int jj = live ? j : 0;
    RaySrc src{sino + ((size_t)sa * V + jj) * N, sb < slices ? sino + ((size_t)sb * V + jj) * N : nullptr, N, M,
               live};
    SpecDst dst{Z + ((size_t)pl * V + jj) * M, g, M, mode, two_alpha, live};
    SmemLine sm{smem + line * smem_line_len(M)};
    fft_line<M, TPL, false>(t, src, dst, sm, tw);
}

// ---------------------------------------------------------------------------
// k_grid_col

// T layout per pair: [ceil(N/4)][M][4] complex, row r of the kept band at
// (r / 4, c', r % 4): a column write fills whole 32-byte sectors and a
// four-row block is contiguous for k_row_ifft.
struct ColDst {
    float2* T;
    int N, M, cidx;
    bool rev, live;
    static constexpr bool kSmem = false;
    __device__ __forceinline__ void store(int p, float2 v) const {
        if (!live) return;
        const int q = rev ? (p == 0 ? 0 : M - p) : p;
        const int r = signed_freq(q, M) + (N >> 1);
        if (r < 0 || r >= N) return;
        T[((size_t)(r >> 2) * M + cidx) * 4 + (r & 3)] = v;
    }
};

// Plan set-up: the angular part of the geometry of every point (q, r') of the
// half grid q in [0, M/2) (the mirror half shares it), bracket -2 for points
// that are zero (outside the band, or the origin, which takes the DC mean).
__global__ void k_geo_table(Geo geo, int M, short* __restrict__ gJ, float* __restrict__ gF) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)(M / 2) * M) return;
    const int q = (int)(idx / M), ridx = (int)(idx % M);
    const int ry = signed_freq(ridx, M);
    Polar P;
    short J = -2;
    float f = 0.f;
    if (!(q == 0 && ry == 0) && polar_of(q, ry, geo, P)) {
        J = (short)P.J;
        f = P.fth;
    }
    gJ[idx] = J;
    gF[idx] = f;
}

// Bilinear gather of one side of a column pair: plus = true for the point
// (q, r') itself (kappa = +rho when P.up), false for its mirror (-q, -r').
// Two points per step; all eight tap loads are issued before any is used.
template <int M, int TPL, int PPT>
__device__ __forceinline__ void gather_side(const float2* __restrict__ Zp, int V, int q, bool live, int t,
                                            const short* __restrict__ gJq, const float* __restrict__ gFq,
                                            bool mirror, const SmemLine& sm) {
    constexpr int H = M >> 1;
    const float2 zero = make_float2(0.f, 0.f);
#pragma unroll 1
    for (int i = 0; i < PPT; i += 2) {
        float2 z[2][4];
        float wk[2], wt[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int ridx = t + (i + u) * TPL;
            const int ry = signed_freq(ridx, M);
            const int Jt = __ldg(gJq + ridx);
            wt[u] = __ldg(gFq + ridx);
            // a table bracket >= -1 means the point is inside the band and not the origin
            const bool ok = live && Jt >= -1;
            const int rho2 = q * q + ry * ry;
            const float rf = __fsqrt_rn((float)rho2);
            int k0 = (int)rf;
            if (k0 * k0 > rho2) --k0;
            else if ((k0 + 1) * (k0 + 1) <= rho2) ++k0;
            const float frac = __fdividef((float)(rho2 - k0 * k0), rf + (float)k0);
            // kappa = +rho for q >= 0 when r' >= 0; the mirror point has -kappa
            const bool plus = (ry >= 0) != mirror;
            int K0;
            if (plus) {
                K0 = k0;
                wk[u] = frac;
            } else if (frac > 0.f) {
                K0 = -k0 - 1;
                wk[u] = 1.f - frac;
            } else {
                K0 = -k0;
                wk[u] = 0.f;
            }
            int o00, o01, o10, o11;
            bool v00, v01, v10, v11;
            if (ok && Jt >= 0 && Jt <= V - 2 && K0 > -H && K0 < H - 1) {
                // common case: no seam row, both radial taps inside the band
                const int k0m = K0 < 0 ? K0 + M : K0;
                const int k1m = k0m + 1 == M ? 0 : k0m + 1;
                o00 = Jt * M + k0m;
                o01 = Jt * M + k1m;
                o10 = o00 + M;
                o11 = o01 + M;
                v00 = v01 = v10 = v11 = true;
            } else {
                // rows of the bracket; virtual rows -1 and V read rows V-1 and 0 at -k
                const int J = ok ? Jt : 0;
                const int rowA = J < 0 ? V - 1 : J;
                const int sA = J < 0 ? -1 : 1;
                const int rowB = J + 1 >= V ? 0 : J + 1;
                const int sB = J + 1 >= V ? -1 : 1;
                const int b00 = sA * K0, b01 = sA * (K0 + 1), b10 = sB * K0, b11 = sB * (K0 + 1);
                v00 = ok && b00 < H && b00 > -H;
                v01 = ok && b01 < H && b01 > -H;
                v10 = ok && b10 < H && b10 > -H;
                v11 = ok && b11 < H && b11 > -H;
                o00 = v00 ? rowA * M + (b00 < 0 ? b00 + M : b00) : 0;
                o01 = v01 ? rowA * M + (b01 < 0 ? b01 + M : b01) : 0;
                o10 = v10 ? rowB * M + (b10 < 0 ? b10 + M : b10) : 0;
                o11 = v11 ? rowB * M + (b11 < 0 ? b11 + M : b11) : 0;
            }
            const float2 a00 = __ldg(Zp + o00), a01 = __ldg(Zp + o01);
            const float2 a10 = __ldg(Zp + o10), a11 = __ldg(Zp + o11);
            z[u][0] = v00 ? a00 : zero;
            z[u][1] = v01 ? a01 : zero;
            z[u][2] = v10 ? a10 : zero;
            z[u][3] = v11 ? a11 : zero;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const float fk = wk[u], ft = wt[u];
            const float2 z00 = z[u][0], z01 = z[u][1], z10 = z[u][2], z11 = z[u][3];
            const float2 a = make_float2(fmaf(fk, z01.x - z00.x, z00.x), fmaf(fk, z01.y - z00.y, z00.y));
            const float2 b = make_float2(fmaf(fk, z11.x - z10.x, z10.x), fmaf(fk, z11.y - z10.y, z10.y));
            sm.store(t + (i + u) * TPL, make_float2(fmaf(ft, b.x - a.x, a.x), fmaf(ft, b.y - a.y, a.y)));
        }
    }
}

template <int M, int TPL, int CPC>
__global__ void __launch_bounds__(TPL * CPC, (TPL * CPC <= 256) ? 1024 / (TPL * CPC) : 1)
    k_grid_col(const float2* __restrict__ Z, int V, int N, const short* __restrict__ gJ,
               const float* __restrict__ gF, float2* __restrict__ T, const float2* __restrict__ tw) {
    extern __shared__ float2 smem[];
    constexpr int PPT = M / TPL;   // Cartesian points per thread and column
    static_assert(PPT % 2 == 0, "points per thread");
    const int pl = blockIdx.y;
    const float2* Zp = Z + (size_t)pl * V * M;
    float2* Tp = T + (size_t)pl * ((N + 3) / 4) * 4 * M;
    const int cp = threadIdx.x / TPL;
    const int t = threadIdx.x % TPL;
    const int q = blockIdx.x * CPC + cp;
    const bool live = q < (M >> 1);
    const SmemLine sm{smem + cp * smem_line_len(M)};
    const short* gJq = gJ + (size_t)(live ? q : 0) * M;
    const float* gFq = gF + (size_t)(live ? q : 0) * M;
    // P0 + P5 then the column inverse FFT, first for column q, then for its
    // mirror -q (the same angular geometry; stored index-reversed, its
    // transform is read back reversed; column -M/2 pairs with q = 0 and is
    // zero).  Consecutive lanes take consecutive rows, so a warp's taps fall
    // on neighbouring polar samples.
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {
        if (side == 0 || q != 0) {
            gather_side<M, TPL, PPT>(Zp, V, q, live, t, gJq, gFq, side == 1, sm);
        } else {
            for (int i = 0; i < PPT; ++i) sm.store(t + i * TPL, make_float2(0.f, 0.f));
        }
        // the origin is single-valued: mean over angles of the DC bin
        if (side == 0 && live && q == 0) {
            if constexpr (TPL >= 32) {
                if (t < 32) {
                    float sx = 0.f, sy = 0.f;
                    for (int j = t; j < V; j += 32) {
                        const float2 zz = __ldg(Zp + (size_t)j * M);
                        sx += zz.x;
                        sy += zz.y;
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        sx += __shfl_xor_sync(0xffffffffu, sx, o);
                        sy += __shfl_xor_sync(0xffffffffu, sy, o);
                    }
                    if (t == 0) sm.store(0, make_float2(sx / (float)V, sy / (float)V));
                }
            } else {
                if (t == 0) {
                    float sx = 0.f, sy = 0.f;
                    for (int j = 0; j < V; ++j) {
                        const float2 zz = __ldg(Zp + (size_t)j * M);
                        sx += zz.x;
                        sy += zz.y;
                    }
                    sm.store(0, make_float2(sx / (float)V, sy / (float)V));
                }
            }
        }
        __syncthreads();
        const ColDst dst{Tp, N, M, side == 0 ? q : (q == 0 ? (M >> 1) : M - q), side == 1 && q != 0, live};
        fft_line<M, TPL, true>(t, sm, dst, sm, tw);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// k_row_ifft

struct TileSrc {
    const float2* T;
    int M, rb, line;
    bool live;
    static constexpr bool kSmem = false;
    __device__ __forceinline__ float2 load(int c) const {
        return live ? __ldg(T + ((size_t)rb * M + c) * 4 + line) : make_float2(0.f, 0.f);
    }
};

struct VolDst {
    float* va;
    float* vb;
    int N, M;
    float scale;
    bool live;
    static constexpr bool kSmem = false;
    __device__ __forceinline__ void store(int p, float2 v) const {
        if (!live) return;
        const int c = signed_freq(p, M) + (N >> 1);
        if (c < 0 || c >= N) return;
        va[c] = v.x * scale;
        if (vb) vb[c] = v.y * scale;
    }
};

template <int M> __host__ __device__ constexpr int row_line_stride() { return smem_line_len(M) + 4; }

template <int M, int TPL, int TPC>
__global__ void __launch_bounds__(4 * TPL * TPC)
    k_row_ifft(const float2* __restrict__ T, int slices, int pair0, int N, float scale, float* __restrict__ vol,
               const float2* __restrict__ tw) {
    extern __shared__ float2 smem[];
    const int pl = blockIdx.y;
    const int tile = threadIdx.x / (4 * TPL);
    const int w = threadIdx.x % (4 * TPL);
    const int line = w & 3, t = w >> 2;
    const int rb = blockIdx.x * TPC + tile;
    const int r = rb * 4 + line;
    const bool live = r < N;
    const int rr = live ? r : 0;
    const float2* Tp = T + (size_t)pl * ((N + 3) / 4) * 4 * M;
    const int sa = 2 * (pair0 + pl), sb = sa + 1;
    TileSrc src{Tp, M, live ? rb : 0, line, live};
    VolDst dst{vol + ((size_t)sa * N + rr) * N, sb < slices ? vol + ((size_t)sb * N + rr) * N : nullptr, N, M,
               scale, live};
    SmemLine sm{smem + (tile * 4 + line) * row_line_stride<M>()};
    fft_line<M, TPL, true>(t, src, dst, sm, tw);
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

template <int M>
bst_status_t launch_forward_M(bst_plan_s* p, const float* sino, int slices, int mode, const float* g, float* vol,
                              void* ws, cudaStream_t st, int max_chunk, int lanes) {
    using C = FwdCfg<M>;
    static bool attr_ok = set_smem(k_ray_fft<M, C::TPL, C::LPC1>, C::S1) &&
                          set_smem(k_grid_col<M, C::TPL, C::CPC>, C::S2) &&
                          set_smem(k_row_ifft<M, C::TPL, C::TPC>, C::S3);
    if (!attr_ok) return BST_ERR_CUDA;
    const int N = p->N, V = p->V;
    const int pairs = (slices + 1) / 2;
    const int chunk = std::min(pairs, max_chunk);
    const int nchunks = (pairs + chunk - 1) / chunk;
    // chunks alternate between two streams (each with its own half of the
    // workspace) so that one chunk's gridding overlaps the next chunk's FFTs;
    // per-stage timing keeps everything on the caller's stream
    const int nl = (lanes >= 2 && nchunks >= 2 && !p->timing && bst_ensure_lanes(p)) ? 2 : 1;
    const size_t lane_elems = (size_t)chunk * (V + (size_t)((N + 3) / 4) * 4) * M;
    const float scale = (float)((double)N / (2.0 * (double)M * (double)M));
    const float two_alpha = (float)(2 * p->alpha);
    const int row_tiles = (N + 3) / 4;
    if (nl == 2) {
        if (cudaEventRecord(p->ev_fork, st) != cudaSuccess) return BST_ERR_CUDA;
        for (int l = 0; l < 2; ++l)
            if (cudaStreamWaitEvent(p->lane[l], p->ev_fork, 0) != cudaSuccess) return BST_ERR_CUDA;
    }
    for (int c = 0; c < nchunks; ++c) {
        const int p0 = c * chunk;
        const int np = std::min(chunk, pairs - p0);
        const int l = c % nl;
        cudaStream_t s = nl == 2 ? p->lane[l] : st;
        float2* Z = (float2*)ws + (size_t)l * lane_elems;
        float2* T = Z + (size_t)chunk * V * M;
        bst_timing_mark(p, s, -1);
        k_ray_fft<M, C::TPL, C::LPC1><<<dim3((V + C::LPC1 - 1) / C::LPC1, np), C::TPL * C::LPC1, C::S1, s>>>(
            sino, slices, p0, N, V, mode, g, two_alpha, Z, p->tw);
        bst_timing_mark(p, s, 0);
        k_grid_col<M, C::TPL, C::CPC><<<dim3((M / 2 + C::CPC - 1) / C::CPC, np), C::TPL * C::CPC, C::S2, s>>>(
            Z, V, N, p->geo_J, p->geo_f, T, p->tw);
        bst_timing_mark(p, s, 1);
        k_row_ifft<M, C::TPL, C::TPC><<<dim3((row_tiles + C::TPC - 1) / C::TPC, np), 4 * C::TPL * C::TPC, C::S3, s>>>(
            T, slices, p0, N, scale, vol, p->tw);
        bst_timing_mark(p, s, 2);
    }
    if (nl == 2) {
        for (int l = 0; l < 2; ++l) {
            if (cudaEventRecord(p->ev_join[l], p->lane[l]) != cudaSuccess) return BST_ERR_CUDA;
            if (cudaStreamWaitEvent(st, p->ev_join[l], 0) != cudaSuccess) return BST_ERR_CUDA;
        }
    }
    return cudaGetLastError() == cudaSuccess ? BST_OK : BST_ERR_CUDA;
}

}  // namespace bst

#define BST_FOR_EACH_M(X) \
    X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096) X(48) X(96) X(192) X(384) X(768) X(1536) X(3072)

bst_status_t bst_launch_forward_chunked(bst_plan_s* p, const float* sino, int slices, int mode, const float* g,
                                        float* vol, void* ws, cudaStream_t st, int max_chunk, int lanes) {
    switch (p->M) {
#define BST_CASE(m) \
    case m: return bst::launch_forward_M<m>(p, sino, slices, mode, g, vol, ws, st, max_chunk, lanes);
        BST_FOR_EACH_M(BST_CASE)
#undef BST_CASE
    }
    return BST_ERR_UNSUPPORTED_SIZE;
}

bst_status_t bst_launch_forward(bst_plan_s* p, const float* sino, int slices, int mode, const float* g, float* vol,
                                void* ws, size_t ws_bytes, cudaStream_t st) {
    const int pairs = (slices + 1) / 2;
    const int chunk = std::min(pairs, p->chunk_pairs);
    const int lanes = ws_bytes >= 2 * (size_t)chunk * bsth::fwd_bytes_per_pair(p) ? 2 : 1;
    return bst_launch_forward_chunked(p, sino, slices, mode, g, vol, ws, st, p->chunk_pairs, lanes);
}

namespace bst {
template <int M>
bst_status_t launch_ray_spectrum_M(bst_plan_s* p, const float* sino, int slices, int p0, int np, float2* Y,
                                   cudaStream_t st) {
    using C = FwdCfg<M>;
    static bool attr_ok = set_smem(k_ray_fft<M, C::TPL, C::LPC1>, C::S1);
    if (!attr_ok) return BST_ERR_CUDA;
    bst_timing_mark(p, st, -1);
    k_ray_fft<M, C::TPL, C::LPC1><<<dim3((p->V + C::LPC1 - 1) / C::LPC1, np), C::TPL * C::LPC1, C::S1, st>>>(
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
    if (cudaMalloc((void**)&p->geo_J, n * sizeof(short)) != cudaSuccess) return BST_ERR_OUT_OF_MEMORY;
    if (cudaMalloc((void**)&p->geo_f, n * sizeof(float)) != cudaSuccess) return BST_ERR_OUT_OF_MEMORY;
    bst::k_geo_table<<<(unsigned)((n + 255) / 256), 256>>>(p->geo(), p->M, p->geo_J, p->geo_f);
    if (cudaGetLastError() != cudaSuccess) return BST_ERR_CUDA;
    return cudaDeviceSynchronize() == cudaSuccess ? BST_OK : BST_ERR_CUDA;
}
