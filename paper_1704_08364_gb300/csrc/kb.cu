// kb.cu -- Kaiser-Bessel gridding for stage P5: plan tables (kernel polynomial,
// deapodization, per-strip sample lists), the gridding + column-FFT kernel
// and bst_plan_set_gridding.
//
// The paper leaves the interpolation kernel of P5 open.  With KB gridding the
// path computes, up to the gridding error, the polar quadrature of the inverse
// 2D Fourier integral x(u) = sum_{j,k} a_jk exp(2 pi i omega_jk . u) with
// a_jk = dtheta_j dsigma |sigma_k| W[|k|] Y_j[k] (Eq. 3 with the filter of
// P4), where bilinear interpolation in (kappa, theta) loses several digits.
// Kernel shape: beta = pi sqrt((W / alpha)^2 (alpha - 1/2)^2 - 0.8) for the
// grid oversampling alpha = M / N (Beatty, Nishimura and Pauly, 2005).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "bst_kb.cuh"

namespace bst {

template <int M, int MAXR>
__global__ void __launch_bounds__(kb_threads<M>(), 1)
    k_kb_col(const float2* __restrict__ Z, int V, int N, KbArgs kb, float2* __restrict__ T,
             const float2* __restrict__ tw) {
    extern __shared__ float2 smem[];
    const int pl = blockIdx.y;
    // strips nearest the column c' = 0 carry the most samples: start there
    const int b = blockIdx.x;
    const int strip = (b & 1) ? kb.nstrips - 1 - (b >> 1) : (b >> 1);
    kb_col_unit<M, tpl_of<M>(), MAXR>(smem, strip, V, N, Z + (size_t)pl * V * M, kb,
                                      T + (size_t)pl * ((N + 3) / 4) * 4 * M, tw);
}

template <int M, int MAXR>
bst_status_t launch_kb_col_M(bst_plan_s* p, const float2* Z, float2* T, int np, cudaStream_t st) {
    constexpr size_t smem = kb_smem_bytes<M>();
    static std::atomic<unsigned long long> attr_done{0};
    if (!bsth::once_per_device(attr_done, [] {
            return cudaFuncSetAttribute(k_kb_col<M, MAXR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
                   cudaSuccess;
        }))
        return BST_ERR_CUDA;
    KbArgs a;
    static_assert(sizeof(a.poly) == sizeof(p->kb_poly), "polynomial size");
    for (int i = 0; i <= KB_POLY; ++i) a.poly[i] = p->kb_poly[i];
    a.t_scale = 8.f / (float)(p->kb_w * p->kb_w);
    a.istart = p->kb_start;
    a.items = p->kb_items;
    a.list = p->kb_list;
    a.dir = p->dir;
    a.wq = p->wq;
    a.W = p->kb_w;
    a.nstrips = p->kb_nstrips;
    k_kb_col<M, MAXR><<<dim3(p->kb_nstrips, np), kb_threads<M>(), smem, st>>>(Z, p->V, p->N, a, T, p->tw);
    return BST_OK;
}

}  // namespace bst

#define BST_FOR_EACH_M(X) \
    X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096) X(48) X(96) X(192) X(384) X(768) X(1536) X(3072)

bst_status_t bst_launch_kb_col(bst_plan_s* p, const float2* Z, float2* T, int np, cudaStream_t st) {
    switch (p->M) {
#define BST_CASE(m)                                                                            \
    case m:                                                                                    \
        return p->maxr == 8 ? bst::launch_kb_col_M<m, 8>(p, Z, T, np, st)                      \
                            : bst::launch_kb_col_M<m, 16>(p, Z, T, np, st);
        BST_FOR_EACH_M(BST_CASE)
#undef BST_CASE
    }
    return BST_ERR_UNSUPPORTED_SIZE;
}

double bst_bessel_i0(double x) {
    double term = 1.0, sum = 1.0;
    const double q = 0.25 * x * x;
    for (int k = 1; k < 500 && term > 1e-18 * sum; ++k) {
        term *= q / ((double)k * (double)k);
        sum += term;
    }
    return sum;
}

void bst_free_kb(bst_plan_s* p) {
    cudaFree(p->kb_dk);
    cudaFree(p->kb_start);
    cudaFree(p->kb_list);
    cudaFree(p->kb_items);
    p->kb_dk = nullptr;
    for (float& c : p->kb_poly) c = 0.f;
    p->kb_start = p->kb_list = nullptr;
    p->kb_items = nullptr;
    p->kb_w = 0;
    p->kb_n = 0;
    p->kb_nstrips = 0;
}

template <class T>
static bool upload_vec(T** d, const std::vector<T>& h) {
    if (cudaMalloc((void**)d, std::max<size_t>(h.size(), 1) * sizeof(T)) != cudaSuccess) return false;
    return h.empty() || cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) == cudaSuccess;
}

// Tables of KB gridding of width W for the plan, host-built in double:
//   the kernel polynomial and the deapodization;
//   per strip of four columns, every sample (j, k), k != 0, -M/2, whose
//   footprint (the W columns c' - c_s in (-W/2, W/2]) meets the strip, sorted
//   by the first row of its footprint (r' - r_s > -W/2, taken mod M);
//   per band of four rows of the strip, the range of that list whose footprint
//   meets the band (two ranges at the wrap), cut into work items of at most
//   KB_ITEM entries; a strip's items ordered longest first.
static bst_status_t build_kb(bst_plan_s* p, int W) {
    using bst::KB_CS;
    using bst::KB_ITEM;
    using bst::KB_RB;
    const int M = p->M, V = p->V, N = p->N;
    const int ns = M / KB_CS, nb = M / KB_RB;
    const double alpha = (double)M / (double)N;
    const double beta = M_PI * std::sqrt((W / alpha) * (W / alpha) * (alpha - 0.5) * (alpha - 0.5) - 0.8);
    const double i0b = bst_bessel_i0(beta);

    // phi(x) = (I0(beta sqrt(1 - (2x/W)^2)) - 1) / (I0(beta) - 1): the KB kernel
    // without its pedestal, zero at |x| = W/2, so that a footprint edge falling
    // exactly on a grid point adds nothing and the gridded spectrum of a real
    // slice stays Hermitian (the pair packing relies on it)
    // evaluated on the GPU as a polynomial of degree KB_POLY in t = 2u - 1,
    // u = (2x/W)^2 in [0, 1] (phi is an entire function of u): interpolation
    // at the Chebyshev nodes of t, then the Chebyshev series rewritten in
    // powers of t (all in double; the monomial coefficients stay below 1 in
    // magnitude, so Horner's rule in float loses only a few ulp)
    constexpr int DMAX = bst::KB_POLY;
    const int D = bst::kb_degree(W);
    double cheb[DMAX + 1] = {0};
    for (int i = 0; i <= D; ++i) {
        const double th = M_PI * (i + 0.5) / (D + 1);
        const double t = std::cos(th);
        const double u = 0.5 * (t + 1.0);
        const double f = (bst_bessel_i0(beta * std::sqrt(std::max(1.0 - u, 0.0))) - 1.0) / (i0b - 1.0);
        for (int k = 0; k <= D; ++k) cheb[k] += f * std::cos(k * th) * (2.0 / (D + 1));
    }
    cheb[0] *= 0.5;
    double mono[DMAX + 1] = {0}, tk[DMAX + 1] = {0}, tkm1[DMAX + 1] = {0};
    tkm1[0] = 1.0;                       // T_0
    tk[1] = 1.0;                         // T_1
    mono[0] += cheb[0];
    mono[1] += cheb[1];
    for (int k = 2; k <= D; ++k) {       // T_k = 2 t T_{k-1} - T_{k-2}
        double nx[DMAX + 1] = {0};
        for (int m = 0; m <= D; ++m) {
            if (m > 0) nx[m] += 2.0 * tk[m - 1];
            nx[m] -= tkm1[m];
        }
        for (int m = 0; m <= D; ++m) {
            tkm1[m] = tk[m];
            tk[m] = nx[m];
            mono[m] += cheb[k] * nx[m];
        }
    }

    // 1 / C(nu), C(nu) = W (sinh(z) / z - sinc(W nu)) / (I0(beta) - 1),
    // z = sqrt(beta^2 - (pi W nu)^2), sinc(x) = sin(pi x) / (pi x)
    std::vector<float> dk(N);
    for (int i = 0; i < N; ++i) {
        const double nu = (double)(i - N / 2) / (double)M;
        const double z2 = beta * beta - (M_PI * W * nu) * (M_PI * W * nu);
        const double z = std::sqrt(std::fabs(z2));
        const double r = z < 1e-8 ? 1.0 : (z2 >= 0 ? std::sinh(z) / z : std::sin(z) / z);
        const double a = M_PI * W * nu;
        const double sn = a == 0.0 ? 1.0 : std::sin(a) / a;
        dk[i] = (float)((i0b - 1.0) / (W * (r - sn)));
    }

    // footprint starts (first column and first row, mod M) of every sample
    std::vector<double> cth(V), sth(V);
    for (int j = 0; j < V; ++j) {
        cth[j] = std::cos(p->theta[j]);
        sth[j] = std::sin(p->theta[j]);
    }
    auto first = [&](double x) {
        const int f = (int)std::floor(x - 0.5 * W) + 1;
        return f < 0 ? f + M : (f >= M ? f - M : f);
    };
    // pass 1: entries per (strip, first row)
    std::vector<int> cnt((size_t)ns * M + 1, 0);
    auto strips_of = [&](int fc, auto&& fn) {
        int last = -1;
        for (int d = 0; d < W; ++d) {
            int c = fc + d;
            if (c >= M) c -= M;
            const int s = c / KB_CS;
            if (s != last) {
                fn(s);
                last = s;
            }
        }
    };
    for (int j = 0; j < V; ++j)
        for (int kidx = 1; kidx < M; ++kidx) {
            if (kidx == M / 2) continue;
            const double k = (double)(kidx < M / 2 ? kidx : kidx - M);
            const int fc = first(k * cth[j]), fr = first(k * sth[j]);
            strips_of(fc, [&](int s) { ++cnt[(size_t)s * M + fr + 1]; });
        }
    for (size_t i = 0; i < (size_t)ns * M; ++i) cnt[i + 1] += cnt[i];
    const size_t n = (size_t)cnt[(size_t)ns * M];
    if (n >= (size_t)INT32_MAX) return BST_ERR_UNSUPPORTED_SIZE;
    // pass 2: the lists, sorted by (strip, first row)
    std::vector<int> list(n);
    {
        std::vector<int> fill(cnt.begin(), cnt.end() - 1);
        for (int j = 0; j < V; ++j)
            for (int kidx = 1; kidx < M; ++kidx) {
                if (kidx == M / 2) continue;
                const double k = (double)(kidx < M / 2 ? kidx : kidx - M);
                const int fc = first(k * cth[j]), fr = first(k * sth[j]);
                strips_of(fc, [&](int s) { list[fill[(size_t)s * M + fr]++] = j * M + kidx; });
            }
    }
    // work items: band b of strip s needs first rows in [KB_RB b - W + 1, KB_RB b + KB_RB - 1] (mod M)
    std::vector<int4> items;
    std::vector<int> istart(ns + 1, 0);
    auto row_pos = [&](int s, int r) { return cnt[(size_t)s * M + r]; };   // first entry with first row >= r
    auto emit = [&](int b, int lo, int hi) {
        for (int e = lo; e < hi; e += KB_ITEM) items.push_back(make_int4(b, e, std::min(hi, e + KB_ITEM), 0));
    };
    for (int s = 0; s < ns; ++s) {
        for (int b = 0; b < nb; ++b) {
            const int lo = KB_RB * b - W + 1, hi = KB_RB * b + KB_RB;   // rows [lo, hi)
            if (lo >= 0) {
                emit(b, row_pos(s, lo), row_pos(s, hi));
            } else {
                emit(b, row_pos(s, lo + M), row_pos(s, M));
                emit(b, row_pos(s, 0), row_pos(s, hi));
            }
        }
        // longest first: the lanes of a warp then take items of about the same
        // length, and the block's last round of items is its shortest
        std::stable_sort(items.begin() + istart[s], items.end(),
                         [](const int4& a, const int4& b) { return a.z - a.y > b.z - b.y; });
        istart[s + 1] = (int)items.size();
    }

    bst_free_kb(p);
    bool ok = upload_vec(&p->kb_dk, dk) && upload_vec(&p->kb_start, istart) &&
              upload_vec(&p->kb_list, list) && upload_vec(&p->kb_items, items);
    if (!ok) {
        cudaGetLastError();
        bst_free_kb(p);
        return BST_ERR_OUT_OF_MEMORY;
    }
    for (int i = 0; i <= DMAX; ++i) p->kb_poly[i] = i <= D ? (float)mono[i] : 0.f;
    p->kb_w = W;
    p->kb_n = n;
    p->kb_nstrips = ns;
    return BST_OK;
}

extern "C" {

bst_status_t bst_plan_set_gridding(bst_plan_t p, int kind, int width) {
    if (!p) return BST_ERR_INVALID_ARGUMENT;
    if (!bsth::on_plan_device(p)) return BST_ERR_INVALID_ARGUMENT;
    if (kind == BST_GRID_BILINEAR) {
        cudaDeviceSynchronize();
        bst_free_kb(p);
        p->grid_kind = BST_GRID_BILINEAR;
        return BST_OK;
    }
    if (kind != BST_GRID_KAISER_BESSEL || width < 2 || width > bst::KB_WMAX || width % 2 != 0)
        return BST_ERR_INVALID_ARGUMENT;
    if (p->grid_kind == BST_GRID_KAISER_BESSEL && p->kb_w == width) return BST_OK;
    cudaDeviceSynchronize();
    const bst_status_t s = build_kb(p, width);
    if (s != BST_OK) {
        p->grid_kind = BST_GRID_BILINEAR;
        return s;
    }
    p->grid_kind = BST_GRID_KAISER_BESSEL;
    return BST_OK;
}

bst_status_t bst_plan_get_gridding(bst_plan_t p, int* kind, int* width) {
    if (!p || !kind || !width) return BST_ERR_INVALID_ARGUMENT;
    *kind = p->grid_kind;
    *width = p->grid_kind == BST_GRID_KAISER_BESSEL ? p->kb_w : 2;
    return BST_OK;
}

}  // extern "C"
