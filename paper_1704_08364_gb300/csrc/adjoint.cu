// adjoint.cu -- the exact transpose of the discrete BST operator
// (radon_adjoint) and the gradient with respect to the filter taps
// (bst_fbp_filter_grad).
//
// Read backwards, the BST chain is a Fourier-slice projector (the FST dual of
// the BST, Sec. 2).  For a slice pair packed as f_a + i f_b:
//
//   k_adj_row_fft   transpose of the crop and the row inverse FFT: zero-extend
//                   each image row to M and FFT it (opposite exponent).
//   k_adj_col_fft   transpose of the column inverse FFT: zero-extend each
//                   column to M and FFT it, giving the full Cartesian spectrum.
//   k_adj_polar     transpose of the bilinear gridding in gather form: every
//                   polar sample (j, k) sums the weighted Cartesian values of
//                   the gridding cells that tap it (cell lists built once per
//                   plan, with the forward path's own coordinate function, so
//                   the weights are bitwise those of the forward gridding);
//                   plus the transpose of the DC mean; then the weight W and
//                   the inverse FFT along t, cropped to the N detector samples,
//                   scaled by dt dw^2, Re -> slice a, Im -> slice b.
//
// The filter gradient recomputes the ray spectrum Y (no weight) and the
// polar pull-back lambda of the image gradient, and reduces
// Re(conj(lambda) Y) over angles, slices and +-k in a fixed order.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "bst_fft.cuh"
#include "bst_geo.cuh"
#include "bst_internal.h"

namespace bst {

template <int M> __host__ __device__ constexpr int adj_tpl() { return (M % 3 == 0) ? M / 12 : M / 16; }
template <int M> __host__ __device__ constexpr int adj_row_stride() { return smem_line_len(M) + 4; }

// ---------------------------------------------------------------------------
// k_adj_row_fft

struct ImgRowSrc {
    const float* fa;
    const float* fb;
    int N, M;
    bool live;
    static constexpr bool kSmem = false;
    __device__ __forceinline__ float2 load(int p) const {
        const int c = signed_freq(p, M) + (N >> 1);
        if (!live || c < 0 || c >= N) return make_float2(0.f, 0.f);
        return make_float2(__ldg(fa + c), fb ? __ldg(fb + c) : 0.f);
    }
};

struct TileDst {
    float2* T;
    int M, rb, line;
    bool live;
    static constexpr bool kSmem = false;
    __device__ __forceinline__ void store(int k, float2 v) const {
        if (live) T[((size_t)rb * M + k) * 4 + line] = v;
    }
};

template <int M, int TPL, int TPC>
__global__ void __launch_bounds__(4 * TPL * TPC)
    k_adj_row_fft(const float* __restrict__ vol, int slices, int pair0, int N, float2* __restrict__ T,
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
    const int sa = 2 * (pair0 + pl), sb = sa + 1;
    ImgRowSrc src{vol + ((size_t)sa * N + rr) * N, sb < slices ? vol + ((size_t)sb * N + rr) * N : nullptr, N, M,
                  live};
    TileDst dst{T + (size_t)pl * ((N + 3) / 4) * 4 * M, M, rb, line, rb * 4 < N};
    SmemLine sm{smem + (tile * 4 + line) * adj_row_stride<M>()};
    fft_line<M, TPL, false>(t, src, dst, sm, tw);
}

// ---------------------------------------------------------------------------
// k_adj_col_fft

struct TileColSrc {
    const float2* T;
    int N, M, cidx;
    static constexpr bool kSmem = false;
    __device__ __forceinline__ float2 load(int p) const {
        const int r = signed_freq(p, M) + (N >> 1);
        if (r < 0 || r >= N) return make_float2(0.f, 0.f);
        return __ldg(T + ((size_t)(r >> 2) * M + cidx) * 4 + (r & 3));
    }
};

struct ColOut {
    float2* X;
    bool live;
    static constexpr bool kSmem = false;
    __device__ __forceinline__ void store(int k, float2 v) const {
        if (live) X[k] = v;
    }
};

template <int M, int TPL, int LPC>
__global__ void __launch_bounds__(TPL * LPC)
    k_adj_col_fft(const float2* __restrict__ T, int N, float2* __restrict__ X, const float2* __restrict__ tw) {
    extern __shared__ float2 smem[];
    const int pl = blockIdx.y;
    const int line = threadIdx.x / TPL, t = threadIdx.x % TPL;
    const int c = blockIdx.x * LPC + line;
    const bool live = c < M;
    const int cc = live ? c : 0;
    TileColSrc src{T + (size_t)pl * ((N + 3) / 4) * 4 * M, N, M, cc};
    ColOut dst{X + ((size_t)pl * M + cc) * M, live};
    SmemLine sm{smem + line * smem_line_len(M)};
    fft_line<M, TPL, false>(t, src, dst, sm, tw);
}

// ---------------------------------------------------------------------------
// k_adj_polar

struct Cells {
    const int* __restrict__ start;   // [(V+1) M + 1]
    const int* __restrict__ pts;     // index c * M + r into the spectrum
    const float2* __restrict__ w;    // (fth, fk) of each point
};

// Weighted sum of the Cartesian values of the cell (J, K0) for its tap `tap`
// (0: (J, K0), 1: (J, K0+1), 2: (J+1, K0), 3: (J+1, K0+1)).
__device__ __forceinline__ float2 cell_sum(const Cells& cl, const float2* __restrict__ X, int M, int J, int K0,
                                           int tap) {
    float2 acc = make_float2(0.f, 0.f);
    if (K0 < -(M >> 1) || K0 > (M >> 1) - 1) return acc;
    const int cell = (J + 1) * M + (K0 + (M >> 1));
    const int b = __ldg(cl.start + cell), e = __ldg(cl.start + cell + 1);
    for (int i = b; i < e; ++i) {
        const float2 fw = __ldg(cl.w + i);
        const float wt = (tap & 2 ? fw.x : 1.f - fw.x) * (tap & 1 ? fw.y : 1.f - fw.y);
        const float2 x = __ldg(X + __ldg(cl.pts + i));
        acc.x = fmaf(wt, x.x, acc.x);
        acc.y = fmaf(wt, x.y, acc.y);
    }
    return acc;
}

// Weighted sum over the cells (J, K0 - 1) (tap `hi`: its radial weight is fk)
// and (J, K0) (tap `lo`: 1 - fk), which are adjacent in the cell lists, with
// angular weight fth (rows J + 1 of the bracket) or 1 - fth (row J).
__device__ __forceinline__ float2 cell_pair_sum(const Cells& cl, const float2* __restrict__ X, int M, int J, int K0,
                                                bool upper) {
    float2 acc = make_float2(0.f, 0.f);
    const int cell = (J + 1) * M + (K0 + (M >> 1));
    const int b = __ldg(cl.start + cell - 1), mid = __ldg(cl.start + cell), e = __ldg(cl.start + cell + 1);
    for (int i = b; i < e; ++i) {
        const float2 fw = __ldg(cl.w + i);
        const float wt = (upper ? fw.x : 1.f - fw.x) * (i < mid ? fw.y : 1.f - fw.y);
        const float2 x = __ldg(X + __ldg(cl.pts + i));
        acc.x = fmaf(wt, x.x, acc.x);
        acc.y = fmaf(wt, x.y, acc.y);
    }
    return acc;
}

// lambda_j[K]: transpose of the gridding (every cell tap that lands on (j, K))
__device__ __forceinline__ float2 polar_pullback(const Cells& cl, const float2* __restrict__ X, int V, int M, int j,
                                                 int K) {
    float2 s = make_float2(0.f, 0.f);
    if (K <= -(M >> 1)) return s;
    float2 v;
    // taps (j, K) of the cells (j, K) [weight 1 - fk] and (j, K - 1) [weight fk], bracket row J = j
    v = cell_pair_sum(cl, X, M, j, K, false);
    s.x += v.x; s.y += v.y;
    // the same from bracket J = j - 1, whose upper row J + 1 is j
    v = cell_pair_sum(cl, X, M, j - 1, K, true);
    s.x += v.x; s.y += v.y;
    if (j == 0) {  // seam: the J+1 = V taps of bracket V-1 read row 0 at -k
        v = cell_sum(cl, X, M, V - 1, -K, 2);
        s.x += v.x; s.y += v.y;
        v = cell_sum(cl, X, M, V - 1, -K - 1, 3);
        s.x += v.x; s.y += v.y;
    }
    if (j == V - 1) {  // the J = -1 taps of bracket -1 read row V-1 at -k
        v = cell_sum(cl, X, M, -1, -K, 0);
        s.x += v.x; s.y += v.y;
        v = cell_sum(cl, X, M, -1, -K - 1, 1);
        s.x += v.x; s.y += v.y;
    }
    return s;
}

struct SinoCrop {
    float* ya;
    float* yb;
    int N, M;
    float scale;
    bool live;
    static constexpr bool kSmem = false;
    __device__ __forceinline__ void store(int m, float2 v) const {
        if (!live) return;
        const int i = signed_freq(m, M) + (N >> 1);
        if (i < 0 || i >= N) return;
        ya[i] = v.x * scale;
        if (yb) yb[i] = v.y * scale;
    }
};

// mode: BSTK_FILTER / BSTK_BACKPROJECT: weight, inverse FFT, crop -> sino;
//       BSTK_RAW: no sinogram.
// lam (may be null in the first two modes): lambda (no weight) to lam[pair][V][M]
template <int M, int TPL, int LPC>
__global__ void __launch_bounds__(TPL * LPC)
    k_adj_polar(const float2* __restrict__ X, Cells cl, int V, int N, int slices, int pair0, int mode,
                const float* __restrict__ g, float two_alpha, float scale, float* __restrict__ sino,
                float2* __restrict__ lam, const float2* __restrict__ tw) {
    extern __shared__ float2 smem[];
    const int pl = blockIdx.y;
    const int line = threadIdx.x / TPL, t = threadIdx.x % TPL;
    const int j = blockIdx.x * LPC + line;
    const bool live = j < V;
    const int jj = live ? j : 0;
    const float2* Xp = X + (size_t)pl * M * M;
    const SmemLine sm{smem + line * smem_line_len(M)};
    const float2 origin = __ldg(Xp);   // spectrum value at (0, 0)
    for (int k = t; k < M; k += TPL) {
        float2 v = make_float2(0.f, 0.f);
        if (live) {
            v = polar_pullback(cl, Xp, V, M, jj, signed_freq(k, M));
            if (k == 0) {
                v.x += origin.x / (float)V;
                v.y += origin.y / (float)V;
            }
        }
        if (lam && live) lam[((size_t)pl * V + jj) * M + k] = v;
        if (mode != BSTK_RAW) {
            const int ak = k <= (M >> 1) ? k : M - k;
            float w;
            if (ak == (M >> 1)) w = 0.f;
            else if (mode == BSTK_FILTER) w = g ? __ldg(g + ak) : 1.f;
            else w = ak == 0 ? 0.f : __fdiv_rn(two_alpha, (float)ak);
            sm.store(k, make_float2(v.x * w, v.y * w));
        }
    }
    if (mode == BSTK_RAW) return;   // uniform across the block
    __syncthreads();
    const int sa = 2 * (pair0 + pl), sb = sa + 1;
    SinoCrop dst{sino + ((size_t)sa * V + jj) * N, sb < slices ? sino + ((size_t)sb * V + jj) * N : nullptr, N, M,
                 scale, live};
    fft_line<M, TPL, true>(t, sm, dst, sm, tw);
}

// ---------------------------------------------------------------------------
// cell lists of the gridding (plan set-up)

__global__ void k_cell_keys(Geo geo, int M, int* __restrict__ key, float2* __restrict__ wt) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)M * M) return;
    const int cidx = (int)(idx / M), ridx = (int)(idx % M);
    const int cx = signed_freq(cidx, M), ry = signed_freq(ridx, M);
    int k = -1;
    float2 w = make_float2(0.f, 0.f);
    Polar P;
    if (!(cx == 0 && ry == 0) && polar_of(cx, ry, geo, P)) {
        int K0;
        float fk;
        radial_bin(P, P.up, K0, fk);
        k = (P.J + 1) * M + (K0 + (M >> 1));
        w = make_float2(P.fth, fk);
    }
    key[idx] = k;
    wt[idx] = w;
}

// ---------------------------------------------------------------------------
// filter gradient reductions

// part[pair][k] = sum_j Re(conj(lam_j[k]) Y_j[k])
// part[pair][k] = sum_j Re(conj(lam_j[k]) Y_j[k]): a block takes 32 bins k and
// splits the angles over 8 groups of its threads (j = g, g + 8, ...), whose
// sums are then added in a fixed order (deterministic)
constexpr int FG_K = 32, FG_G = 8;
__global__ void __launch_bounds__(FG_K * FG_G)
    k_fg_partial(const float2* __restrict__ lam, const float2* __restrict__ Y, int V, int M, int pair0,
                 float* __restrict__ part) {
    __shared__ float red[FG_G][FG_K];
    const int kl = threadIdx.x % FG_K, grp = threadIdx.x / FG_K;
    const int k = blockIdx.x * FG_K + kl;
    const int pl = blockIdx.y;
    float s = 0.f;
    if (k < M) {
        const float2* l = lam + (size_t)pl * V * M + k;
        const float2* y = Y + (size_t)pl * V * M + k;
        for (int j = grp; j < V; j += FG_G) {
            const float2 a = __ldg(l + (size_t)j * M), b = __ldg(y + (size_t)j * M);
            s = fmaf(a.x, b.x, fmaf(a.y, b.y, s));
        }
    }
    red[grp][kl] = s;
    __syncthreads();
    if (grp == 0 && k < M) {
        float t = 0.f;
#pragma unroll
        for (int g = 0; g < FG_G; ++g) t += red[g][kl];
        part[(size_t)(pair0 + pl) * M + k] = t;
    }
}

// grad[m] = scale * sum over pairs of part[k = m] + part[k = M - m] (m = 1..M/2-1), fixed order;
// scale = dt dw^2 restores the constants the unscaled transforms leave out
__global__ void k_fg_final(const float* __restrict__ part, int pairs, int M, float scale, float* __restrict__ grad) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M / 2) return;
    float s = 0.f;
    for (int p = 0; p < pairs; ++p) {
        const float* q = part + (size_t)p * M;
        s += q[m];
        if (m != 0) s += q[M - m];
    }
    grad[m] = s * scale;
}

// ---------------------------------------------------------------------------
// host side

template <class K>
static bool set_smem_a(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return true;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess;
}

template <int M> struct AdjCfg {
    static constexpr int TPL = adj_tpl<M>();
    static constexpr int TPC = (128 / (4 * TPL)) > 1 ? 128 / (4 * TPL) : 1;
    static constexpr int LPC = (256 / TPL) > 1 ? 256 / TPL : 1;
    static constexpr size_t S1 = (size_t)4 * TPC * adj_row_stride<M>() * sizeof(float2);
    static constexpr size_t S2 = (size_t)LPC * smem_line_len(M) * sizeof(float2);
};

struct AdjLayout {
    int chunk;
    float2 *T, *X, *lam, *Y;
    float* part;
};

static size_t adj_bytes_per_pair(const bst_plan_s* p) {
    const size_t rows_t = (size_t)((p->N + 3) / 4) * 4;
    return (rows_t * p->M + (size_t)p->M * p->M + 2 * (size_t)p->V * p->M) * sizeof(float2);
}

static int adj_chunk(const bst_plan_s* p, int pairs) {
    const size_t budget = (size_t)256 << 20;
    return (int)std::max<size_t>(1, std::min<size_t>((size_t)pairs, budget / adj_bytes_per_pair(p)));
}

static AdjLayout adj_layout(const bst_plan_s* p, int pairs, void* ws) {
    AdjLayout L;
    L.chunk = adj_chunk(p, pairs);
    const size_t rows_t = (size_t)((p->N + 3) / 4) * 4;
    float2* b = (float2*)ws;
    L.T = b;
    b += (size_t)L.chunk * rows_t * p->M;
    L.X = b;
    b += (size_t)L.chunk * p->M * p->M;
    L.lam = b;
    b += (size_t)L.chunk * p->V * p->M;
    L.Y = b;
    b += (size_t)L.chunk * p->V * p->M;
    L.part = (float*)b;
    return L;
}

template <int M>
static bst_status_t adjoint_chunk(bst_plan_s* p, const AdjLayout& L, const float* vol, int slices, int p0, int np,
                                  int mode, const float* g, float* sino, bool keep_lam, cudaStream_t st) {
    using C = AdjCfg<M>;
    static std::atomic<unsigned long long> attr_done{0};
    if (!bsth::once_per_device(attr_done, [] {
            return set_smem_a(k_adj_row_fft<M, C::TPL, C::TPC>, C::S1) &&
                   set_smem_a(k_adj_col_fft<M, C::TPL, C::LPC>, C::S2) &&
                   set_smem_a(k_adj_polar<M, C::TPL, C::LPC>, C::S2);
        }))
        return BST_ERR_CUDA;
    const int N = p->N, V = p->V;
    const int row_tiles = (N + 3) / 4;
    bst_timing_mark(p, st, -1);
    k_adj_row_fft<M, C::TPL, C::TPC><<<dim3((row_tiles + C::TPC - 1) / C::TPC, np), 4 * C::TPL * C::TPC, C::S1, st>>>(
        vol, slices, p0, N, L.T, p->tw);
    bst_timing_mark(p, st, 5);
    k_adj_col_fft<M, C::TPL, C::LPC><<<dim3((M + C::LPC - 1) / C::LPC, np), C::TPL * C::LPC, C::S2, st>>>(
        L.T, N, L.X, p->tw);
    bst_timing_mark(p, st, 6);
    Cells cl{p->cell_start, p->cell_pts, p->cell_w};
    const float scale = (float)((double)N / (2.0 * (double)M * (double)M));
    k_adj_polar<M, C::TPL, C::LPC><<<dim3((V + C::LPC - 1) / C::LPC, np), C::TPL * C::LPC, C::S2, st>>>(
        L.X, cl, V, N, slices, p0, mode, g, (float)(2 * p->alpha), scale, sino, keep_lam ? L.lam : nullptr, p->tw);
    bst_timing_mark(p, st, 7);
    return BST_OK;
}

}  // namespace bst

#define BST_FOR_EACH_M(X) \
    X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096) X(48) X(96) X(192) X(384) X(768) X(1536) X(3072)

size_t bst_adjoint_ws(const bst_plan_s* p, int slices) {
    const int pairs = (slices + 1) / 2;
    return (size_t)bst::adj_chunk(p, pairs) * bst::adj_bytes_per_pair(p) + (size_t)pairs * p->M * sizeof(float) + 256;
}

bst_status_t bst_build_cells(bst_plan_s* p, cudaStream_t st) {
    if (p->cells_built) return BST_OK;
    const int M = p->M;
    const size_t n = (size_t)M * M;
    int* d_key = nullptr;
    float2* d_w = nullptr;
    if (cudaMalloc((void**)&d_key, n * sizeof(int)) != cudaSuccess) return BST_ERR_OUT_OF_MEMORY;
    if (cudaMalloc((void**)&d_w, n * sizeof(float2)) != cudaSuccess) {
        cudaFree(d_key);
        return BST_ERR_OUT_OF_MEMORY;
    }
    bst::k_cell_keys<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p->geo(), M, d_key, d_w);
    std::vector<int> key(n);
    std::vector<float2> w(n);
    bool ok = cudaMemcpyAsync(key.data(), d_key, n * sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
              cudaMemcpyAsync(w.data(), d_w, n * sizeof(float2), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
              cudaStreamSynchronize(st) == cudaSuccess;
    cudaFree(d_key);
    cudaFree(d_w);
    if (!ok) return BST_ERR_CUDA;
    const size_t ncell = (size_t)(p->V + 1) * M;
    std::vector<int> start(ncell + 1, 0);
    for (size_t i = 0; i < n; ++i)
        if (key[i] >= 0) ++start[(size_t)key[i] + 1];
    for (size_t c = 0; c < ncell; ++c) start[c + 1] += start[c];
    const int total = start[ncell];
    std::vector<int> pts(std::max(total, 1));
    std::vector<float2> pw(std::max(total, 1));
    std::vector<int> cur(start.begin(), start.end() - 1);
    for (size_t i = 0; i < n; ++i) {   // stable: ascending point index within a cell
        if (key[i] < 0) continue;
        const int pos = cur[key[i]]++;
        pts[pos] = (int)i;
        pw[pos] = w[i];
    }
    if (cudaMalloc((void**)&p->cell_start, start.size() * sizeof(int)) != cudaSuccess ||
        cudaMalloc((void**)&p->cell_pts, pts.size() * sizeof(int)) != cudaSuccess ||
        cudaMalloc((void**)&p->cell_w, pw.size() * sizeof(float2)) != cudaSuccess)
        return BST_ERR_OUT_OF_MEMORY;
    if (cudaMemcpy(p->cell_start, start.data(), start.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->cell_pts, pts.data(), pts.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->cell_w, pw.data(), pw.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess)
        return BST_ERR_CUDA;
    p->cell_n = total;
    p->cells_built = true;
    return BST_OK;
}

static bst_status_t adjoint_chunk_dispatch(bst_plan_s* p, const bst::AdjLayout& L, const float* vol, int slices,
                                           int p0, int np, int mode, const float* g, float* sino, bool keep_lam,
                                           cudaStream_t st) {
    switch (p->M) {
#define BST_CASE(m) \
    case m: return bst::adjoint_chunk<m>(p, L, vol, slices, p0, np, mode, g, sino, keep_lam, st);
        BST_FOR_EACH_M(BST_CASE)
#undef BST_CASE
    }
    return BST_ERR_UNSUPPORTED_SIZE;
}

bst_status_t bst_launch_adjoint(bst_plan_s* p, int mode, const float* g, const float* vol, int slices, float* sino,
                                void* ws, size_t /*ws_bytes*/, cudaStream_t st) {
    bst_status_t s = bst_build_cells(p, st);
    if (s != BST_OK) return s;
    const int pairs = (slices + 1) / 2;
    const bst::AdjLayout L = bst::adj_layout(p, pairs, ws);
    for (int p0 = 0; p0 < pairs; p0 += L.chunk) {
        const int np = std::min(L.chunk, pairs - p0);
        s = adjoint_chunk_dispatch(p, L, vol, slices, p0, np, mode, g, sino, false, st);
        if (s != BST_OK) return s;
    }
    return cudaGetLastError() == cudaSuccess ? BST_OK : BST_ERR_CUDA;
}

// the raw ray spectrum (no weight) of pairs [p0, p0+np) into Y, from fbp.cu
bst_status_t bst_launch_ray_spectrum(bst_plan_s* p, const float* sino, int slices, int p0, int np, float2* Y,
                                     cudaStream_t st);

// Both gradients of <grad_vol, FBP(sino; g)>: grad_sino = the adjoint applied to
// grad_vol (taps g; skipped when null), grad_g = sum Re(conj(lambda) Y) (skipped
// when null), from one pull-back lambda per chunk.
bst_status_t bst_launch_backward(bst_plan_s* p, const float* sino, const float* gvol, int slices, const float* g,
                                 float* grad_sino, float* grad_g, void* ws, cudaStream_t st) {
    bst_status_t s = bst_build_cells(p, st);
    if (s != BST_OK) return s;
    const int pairs = (slices + 1) / 2;
    const bst::AdjLayout L = bst::adj_layout(p, pairs, ws);
    const int M = p->M, V = p->V;
    for (int p0 = 0; p0 < pairs; p0 += L.chunk) {
        const int np = std::min(L.chunk, pairs - p0);
        s = adjoint_chunk_dispatch(p, L, gvol, slices, p0, np, grad_sino ? BSTK_FILTER : BSTK_RAW, g, grad_sino,
                                   grad_g != nullptr, st);
        if (s != BST_OK) return s;
        if (grad_g) {
            s = bst_launch_ray_spectrum(p, sino, slices, p0, np, L.Y, st);
            if (s != BST_OK) return s;
            bst::k_fg_partial<<<dim3((M + bst::FG_K - 1) / bst::FG_K, np), bst::FG_K * bst::FG_G, 0, st>>>(
                L.lam, L.Y, V, M, p0, L.part);
        }
    }
    if (grad_g) {
        const float scale = (float)((double)p->N / (2.0 * (double)M * (double)M));
        bst::k_fg_final<<<(M / 2 + 255) / 256, 256, 0, st>>>(L.part, pairs, M, scale, grad_g);
    }
    return cudaGetLastError() == cudaSuccess ? BST_OK : BST_ERR_CUDA;
}

bst_status_t bst_launch_filter_grad(bst_plan_s* p, const float* sino, const float* gvol, int slices, float* grad_g,
                                    void* ws, size_t /*ws_bytes*/, cudaStream_t st) {
    return bst_launch_backward(p, sino, gvol, slices, nullptr, nullptr, grad_g, ws, st);
}
