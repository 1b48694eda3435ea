// bst_stages.cuh -- the three stages of the BST forward path as device
// functions over "units" (a few lines of one slice pair), shared by the
// per-size kernels of bst_forward.cuh and the persistent ragged kernel of ragged.cu.
//
//   ray_unit   stages P2 + P3 + P4 for LPC angles j0.. of a pair: centre-aligned
//              zero padding of the rays to M, forward FFT along t, weight W[|k|],
//              written to Z[V][M] (natural order).
//   grid_unit  stages P0 + P5 + the column half of P6 for CPC Cartesian column
//              pairs (q, -q), q = q0..: bilinear gather from Z with the plan's
//              angular geometry table, inverse FFT along r', the N central rows
//              written to T.
//   row_unit   the row half of P6 + P7 + P8 for TPC blocks of four rows: inverse
//              FFT along c', the N central columns scaled by dt dw^2 = N/(2 M^2)
//              (and by the deapodization of KB gridding when it is used),
//              Re to slice a and Im to slice b.
//
// Every thread of the block calls the unit (the FFT passes contain barriers).
// MAXR is the radix schedule (largest radix 16 or 8) chosen per FFT length.
#pragma once
#include <cuda_runtime.h>

#include "bst_fft.cuh"
#include "bst_geo.cuh"
#include "bst_internal.h"

namespace bst {

// threads per line: 16 elements per thread (12 for lengths 3 * 2^a)
template <int M> __host__ __device__ constexpr int tpl_of() { return (M % 3 == 0) ? M / 12 : M / 16; }

// NC: the ray count N as a compile-time constant (0: the runtime value).  With
// it, the padded samples that are always zero are known per index group.
template <int NC = 0>
struct RaySrc {
    const float* ya;
    const float* yb;
    int N, M;
    bool live;
    static constexpr bool kSmem = false;
    // every padded index m in [lo, hi) lies in the zero padding
    static __host__ __device__ constexpr bool zero_group(int lo, int hi, int Mc) {
        return NC > 0 && lo >= NC / 2 && hi <= Mc - NC / 2;
    }
    __device__ __forceinline__ float2 load(int m) const {
        const int n = NC > 0 ? NC : N;
        int i = m + (n >> 1);
        if (i >= M) i -= M;
        if (!live || i >= n) return make_float2(0.f, 0.f);
        return make_float2(__ldg(ya + i), yb ? __ldg(yb + i) : 0.f);
    }
};

// Slot of bin m of row j in the paired layout of one pair's spectrum (V rows
// of M/2 slots of 16 bytes, slot (Z[j][m], Z[j][-m])): rows are stored two by
// two, each 128-byte line holding bins 4i .. 4i + 3 of rows 2p and 2p + 1, so
// the two rows of a bilinear bracket often share a line and the taps of a
// warp fall on about a fifth fewer lines than with whole rows; with V odd the
// last row is stored whole after the pairs.
__host__ __device__ __forceinline__ int paired_slot(int j, int m, int H, int V) {
    const int ve = V & ~1;
    return j < ve ? ((((j >> 1) * (H >> 2)) + (m >> 2)) << 3) + ((j & 1) << 2) + (m & 3) : ve * H + m;
}

// Store the weighted spectrum value of bin k of row j of one pair's spectrum
// z (the pair's base).  Packed layout: z[j M + k], k in [0, M).  Paired
// layout (mode flag BSTK_PAIRED): slot m of row j holds (Z[m], Z[-m]) for
// m in [0, M/2), placed by paired_slot, so that the two taps of a Cartesian
// point and of its mirror point (which reads bin -k) are one 16-byte load;
// bin 0 fills both halves of slot 0, the Nyquist bin (weight 0) is not stored.
__device__ __forceinline__ void spec_store(float2* z, int j, int V, int M, int mode, int k, float2 v) {
    if (!(mode & BSTK_PAIRED)) {
        z[(size_t)j * M + k] = v;
        return;
    }
    const int h = M >> 1;
    if (k < h) {
        const int s = paired_slot(j, k, h, V);
        z[2 * s] = v;
        if (k == 0) z[2 * s + 1] = v;
    } else if (k > h) {
        z[2 * paired_slot(j, M - k, h, V) + 1] = v;
    }
}

struct SpecDst {
    float2* z;      // the pair's spectrum
    int j, V;       // row (angle) of this line, rows of the pair
    const float* g;
    int M, mode;
    float two_alpha;
    bool live;
    static constexpr bool kSmem = false;
    __device__ __forceinline__ void store(int k, float2 v) const {
        if (!live) return;
        const int ak = k <= (M >> 1) ? k : M - k;
        const int md = mode & 7;
        float w;
        if (md == BSTK_RAW) w = 1.f;
        else if (ak == (M >> 1)) w = 0.f;
        else if (md == BSTK_FILTER) w = g ? __ldg(g + ak) : 1.f;
        else w = ak == 0 ? 0.f : __fdiv_rn(two_alpha, (float)ak);
        if (mode & BSTK_KBW) w *= ak == 0 ? 0.25f : (float)ak;
        spec_store(z, j, V, M, mode, k, make_float2(v.x * w, v.y * w));
    }
};

// T layout per pair: [ceil(N/4)][M][4] complex, row r of the kept band at
// (r / 4, c', r % 4): a column write fills whole 32-byte sectors and a
// four-row block is contiguous for k_row_ifft.
template <int NC = 0>
struct ColDst {
    float2* T;
    int N, M, cidx;
    bool rev, live;
    static constexpr bool kSmem = false;
    // no output index p in [lo, hi) is kept (in either reading direction)
    static __host__ __device__ constexpr bool drop_group(int lo, int hi, int Mc) {
        return NC > 0 && lo >= NC / 2 + 1 && hi <= Mc - NC / 2;
    }
    __device__ __forceinline__ void store(int p, float2 v) const {
        if (!live) return;
        const int n = NC > 0 ? NC : N;
        const int q = rev ? (p == 0 ? 0 : M - p) : p;
        const int r = signed_freq(q, M) + (n >> 1);
        if (r < 0 || r >= n) return;
        T[((size_t)(r >> 2) * M + cidx) * 4 + (r & 3)] = v;
    }
};

// Bilinear gather of one side of a column pair: plus = true for the point
// (q, r') itself (kappa = +rho when P.up), false for its mirror (-q, -r').
// Thread t gathers rows t + i TPL into x[i], the first FFT pass's inputs.  PS
// points per step; all 4 PS tap loads of a step are issued before any is used.
template <int M, int TPL, int PPT, int PS = 2>
__device__ __forceinline__ void gather_side(const float2* __restrict__ Zp, int V, int q, bool live, int t,
                                            const int* __restrict__ gJq, const float2* __restrict__ gFq,
                                            bool mirror, float2 (&x)[PPT]) {
    static_assert(PPT % PS == 0, "points per step");
    constexpr int H = M >> 1;
    const float2 zero = make_float2(0.f, 0.f);
    // the plan's table (bracket and floor(rho) packed; angle and radius
    // fractions), prefetched two steps ahead so that each step waits on the
    // tap loads only
    int jn[2 * PS];
    float2 fn[2 * PS];
#pragma unroll
    for (int u = 0; u < 2 * PS; ++u) {
        jn[u] = __ldg(gJq + t + (u < PPT ? u : 0) * TPL);
        fn[u] = __ldg(gFq + t + (u < PPT ? u : 0) * TPL);
    }
#pragma unroll
    for (int i = 0; i < PPT; i += PS) {
        float2 z[PS][4];
        float wk[PS], wt[PS];
        int jc[PS];
        float2 fc[PS];
#pragma unroll
        for (int u = 0; u < PS; ++u) {
            jc[u] = jn[u];
            fc[u] = fn[u];
            jn[u] = jn[PS + u];
            fn[u] = fn[PS + u];
        }
        if (i + 2 * PS < PPT) {
#pragma unroll
            for (int u = 0; u < PS; ++u) {
                jn[PS + u] = __ldg(gJq + t + (i + 2 * PS + u) * TPL);
                fn[PS + u] = __ldg(gFq + t + (i + 2 * PS + u) * TPL);
            }
        }
#pragma unroll
        for (int u = 0; u < PS; ++u) {
            const int ridx = t + (i + u) * TPL;
            const int ry = signed_freq(ridx, M);
            const int jk = jc[u];
            const float2 fw = fc[u];
            const int Jt = jk >> 16;
            const int k0 = jk & 0xffff;
            const float frac = fw.y;
            wt[u] = fw.x;
            // a table bracket >= -1 means the point is inside the band and not the origin
            const bool ok = live && Jt >= -1;
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
            // taps outside the band (about a fifth of the grid's points lie
            // beyond rho = M/2, mostly in whole warps) issue no load
            z[u][0] = v00 ? __ldg(Zp + o00) : zero;
            z[u][1] = v01 ? __ldg(Zp + o01) : zero;
            z[u][2] = v10 ? __ldg(Zp + o10) : zero;
            z[u][3] = v11 ? __ldg(Zp + o11) : zero;
        }
#pragma unroll
        for (int u = 0; u < PS; ++u) {
            const float fk = wk[u], ft = wt[u];
            const float2 z00 = z[u][0], z01 = z[u][1], z10 = z[u][2], z11 = z[u][3];
            const float2 a = make_float2(fmaf(fk, z01.x - z00.x, z00.x), fmaf(fk, z01.y - z00.y, z00.y));
            const float2 b = make_float2(fmaf(fk, z11.x - z10.x, z10.x), fmaf(fk, z11.y - z10.y, z10.y));
            x[i + u] = make_float2(fmaf(ft, b.x - a.x, a.x), fmaf(ft, b.y - a.y, a.y));
        }
    }
}

// row r of the kept band of T (layout [ceil(N/4)][M][4])
struct TileSrc {
    const float2* T;
    int M, r;
    bool live;
    static constexpr bool kSmem = false;
    __device__ __forceinline__ float2 load(int c) const {
        return live ? __ldg(T + ((size_t)(r >> 2) * M + c) * 4 + (r & 3)) : make_float2(0.f, 0.f);
    }
};

template <int NC = 0>
struct VolDst {
    float* va;
    float* vb;
    int N, M;
    float scale;
    bool live;
    const float* dk;    // per-column deapodization of KB gridding, or null
    static constexpr bool kSmem = false;
    // no output index p in [lo, hi) falls inside the N kept columns
    static __host__ __device__ constexpr bool drop_group(int lo, int hi, int Mc) {
        return NC > 0 && lo >= NC / 2 && hi <= Mc - NC / 2;
    }
    __device__ __forceinline__ void store(int p, float2 v) const {
        if (!live) return;
        const int n = NC > 0 ? NC : N;
        const int c = signed_freq(p, M) + (n >> 1);
        if (c < 0 || c >= n) return;
        const float s = dk ? scale * __ldg(dk + c) : scale;
        va[c] = v.x * s;
        if (vb) vb[c] = v.y * s;
    }
};

template <int M> __host__ __device__ constexpr int row_line_stride() { return smem_line_len(M) + 4; }

// ---- pre-reconstruction stages fused into the ray load and the weight ------
//
// Normalization (Sec. 1 (a)): y = -log[(I - D)/(I0 - D)] from counts I with the
// slice's flat row I0 and dark row D (both differences clamped to >= 1e-6).
// Window (stage P1): y_i *= w(t_i - shift dt), a Kaiser-Bessel window
// I0(b sqrt(1 - (t/h)^2)) / I0(b) for |t| <= h.  Centering (Sec. 1 (b)): the
// spectrum is multiplied by exp(+2 pi i k shift / M), the exact shift of the
// padded ray by `shift` samples.
struct PrepArgs {
    const float* dark;    // [S][N] or null (0)
    const float* flat;    // [S][N] or null (input is already y)
    float shift;          // centering shift in detector samples
    int shift_int;        // its integer part ...
    float shift_frac;     // ... and fraction (exact phase reduction)
    float kb_beta;        // window shape (0: no window)
    float kb_inv_half;    // 1 / half-width (detector units)
    float kb_norm;        // 1 / I0(kb_beta)
};

template <int NC = 0>
struct RaySrcPrep {
    const float* ya;
    const float* yb;
    const float* da;
    const float* db;
    const float* fa;
    const float* fb;
    int N, M;
    bool live;
    PrepArgs pa;
    static constexpr bool kSmem = false;
    static __host__ __device__ constexpr bool zero_group(int lo, int hi, int Mc) {
        return NC > 0 && lo >= NC / 2 && hi <= Mc - NC / 2;
    }
    __device__ __forceinline__ float sample(const float* y, const float* d, const float* f, int i) const {
        float v = __ldg(y + i);
        if (f) {
            const float dk = d ? __ldg(d + i) : 0.f;
            v = -logf(fmaxf(v - dk, 1e-6f) / fmaxf(__ldg(f + i) - dk, 1e-6f));
        }
        return v;
    }
    __device__ __forceinline__ float2 load(int m) const {
        const int n = NC > 0 ? NC : N;
        int i = m + (n >> 1);
        if (i >= M) i -= M;
        if (!live || i >= n) return make_float2(0.f, 0.f);
        float w = 1.f;
        if (pa.kb_beta > 0.f) {
            const float t = ((float)(i - (n >> 1)) - pa.shift) * (2.f / (float)n);
            const float u = t * pa.kb_inv_half;
            w = fabsf(u) <= 1.f ? cyl_bessel_i0f(pa.kb_beta * sqrtf(fmaxf(1.f - u * u, 0.f))) * pa.kb_norm : 0.f;
        }
        return make_float2(w * sample(ya, da, fa, i), yb ? w * sample(yb, db, fb, i) : 0.f);
    }
};

struct SpecDstShift {
    float2* z;      // the pair's spectrum
    int j, V;       // row (angle) of this line, rows of the pair
    const float* g;
    int M, mode;
    float two_alpha;
    bool live;
    PrepArgs pa;
    static constexpr bool kSmem = false;
    __device__ __forceinline__ void store(int k, float2 v) const {
        if (!live) return;
        const int ak = k <= (M >> 1) ? k : M - k;
        const int md = mode & 7;
        float w;
        if (ak == (M >> 1)) w = 0.f;
        else if (md == BSTK_FILTER) w = g ? __ldg(g + ak) : 1.f;
        else w = ak == 0 ? 0.f : __fdiv_rn(two_alpha, (float)ak);
        if (mode & BSTK_KBW) w *= ak == 0 ? 0.25f : (float)ak;
        if (pa.shift != 0.f) {
            // exp(+2 pi i k s / M) with s = s_int + s_frac; the integer part reduced exactly mod M
            const int ks = signed_freq(k, M);
            int m = (int)(((long long)ks * pa.shift_int) % M);
            if (m < 0) m += M;
            float s1, c1, s2, c2;
            sincospif(2.f * (float)m / (float)M, &s1, &c1);
            sincospif(2.f * (float)ks * pa.shift_frac / (float)M, &s2, &c2);
            const float c = c1 * c2 - s1 * s2, sn = s1 * c2 + c1 * s2;
            v = make_float2(v.x * c - v.y * sn, v.x * sn + v.y * c);
        }
        spec_store(z, j, V, M, mode, k, make_float2(v.x * w, v.y * w));
    }
};

// ray_unit with the pre-reconstruction stages (slice rows da/db, fa/fb of the
// dark and flat fields, or null)
template <int M, int TPL, int LPC, int MAXR, int NC = 0>
__device__ __forceinline__ void ray_unit_prep(float2* smem, int j0, int V, int N, const float* __restrict__ ya,
                                              const float* __restrict__ yb, const float* da, const float* db,
                                              const float* fa, const float* fb, const PrepArgs& pa, int mode,
                                              const float* __restrict__ g, float two_alpha,
                                              float2* __restrict__ Zp, const float2* __restrict__ tw) {
    const int line = threadIdx.x / TPL, t = threadIdx.x % TPL;
    const int j = j0 + line;
    const bool live = j < V;
    const int jj = live ? j : 0;
    RaySrcPrep<NC> src{ya + (size_t)jj * N, yb ? yb + (size_t)jj * N : nullptr, da, db, fa, fb, N, M, live, pa};
    SpecDstShift dst{Zp, jj, V, g, M, mode, two_alpha, live, pa};
    SmemLine sm{smem + line * smem_line_len(M)};
    fft_line<M, TPL, false, MAXR>(t, src, dst, sm, tw);
}

// Shared-memory stride between the lines of a ray unit: with the lines
// interleaved over the lanes (ILV), the lines are skewed by 16 banks so that
// lanes of two lines at the same offset do not share a bank.
template <int M, bool ILV> __host__ __device__ constexpr int ray_line_stride() { return smem_line_len(M) + (ILV ? 8 : 0); }

// P2 + P3 + P4 for lines j0 .. j0 + LPC - 1 of one slice pair (TPL * LPC
// threads; tid the thread's index among them, -1: threadIdx.x; `sync` the
// barrier that covers them; TWT: twiddles from the per-pass tables).  ILV: thread tid works on line tid % LPC, so a
// warp holds the same bins of LPC consecutive angle rows, whose slots the
// paired layout keeps in the same 128-byte lines.
template <int M, int TPL, int LPC, int MAXR, int NC = 0, class SYNC = BlockSync, bool ILV = false, bool TWT = false>
__device__ __forceinline__ void ray_unit(float2* smem, int j0, int V, int N, const float* __restrict__ ya,
                                         const float* __restrict__ yb, int mode, const float* __restrict__ g,
                                         float two_alpha, float2* __restrict__ Zp, const float2* __restrict__ tw,
                                         const SYNC& sync = SYNC(), int tid = -1) {
    if (tid < 0) tid = threadIdx.x;
    const int line = ILV ? tid % LPC : tid / TPL, t = ILV ? tid / LPC : tid % TPL;
    const int j = j0 + line;
    const bool live = j < V;
    const int jj = live ? j : 0;
    RaySrc<NC> src{ya + (size_t)jj * N, yb ? yb + (size_t)jj * N : nullptr, N, M, live};
    SpecDst dst{Zp, jj, V, g, M, mode, two_alpha, live};
    SmemLine sm{smem + line * ray_line_stride<M, ILV>()};
    fft_line<M, TPL, false, MAXR, TWT>(t, src, dst, sm, tw, sync);
}

// P0 + P5 + column P6 for column pairs q0 .. q0 + CPC - 1 (blockDim = TPL * CPC):
// first column q, then its mirror -q (the same angular geometry; stored
// index-reversed, its transform is read back reversed; column -M/2 pairs with
// q = 0 and is zero).  Consecutive lanes take consecutive rows, so a warp's taps
// fall on neighbouring polar samples.
template <int M, int TPL, int CPC, int MAXR, int NC = 0>
__device__ __forceinline__ void grid_unit(float2* smem, int q0, int V, int N, const float2* __restrict__ Zp,
                                          const int* __restrict__ gJ, const float2* __restrict__ gF,
                                          float2* __restrict__ Tp, const float2* __restrict__ tw) {
    constexpr int PPT = M / TPL;   // Cartesian points per thread and column
    static_assert(PPT % 2 == 0, "points per thread");
    const int cp = threadIdx.x / TPL;
    const int t = threadIdx.x % TPL;
    const int q = q0 + cp;
    const bool live = q < (M >> 1);
    const SmemLine sm{smem + cp * smem_line_len(M)};
    const int* gJq = gJ + (size_t)(live ? q : 0) * M;
    const float2* gFq = gF + (size_t)(live ? q : 0) * M;
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {
        float2 x[PPT];
        if (side == 0 || q != 0) {
            gather_side<M, TPL, PPT>(Zp, V, q, live, t, gJq, gFq, side == 1, x);
        } else {
#pragma unroll
            for (int i = 0; i < PPT; ++i) x[i] = make_float2(0.f, 0.f);
        }
        // the origin is single-valued: mean over angles of the DC bin (row 0 of
        // thread 0's rows)
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
                    if (t == 0) x[0] = make_float2(sx / (float)V, sy / (float)V);
                }
            } else {
                if (t == 0) {
                    float sx = 0.f, sy = 0.f;
                    for (int j = 0; j < V; ++j) {
                        const float2 zz = __ldg(Zp + (size_t)j * M);
                        sx += zz.x;
                        sy += zz.y;
                    }
                    x[0] = make_float2(sx / (float)V, sy / (float)V);
                }
            }
        }
        // side 0's last pass may still read the line
        if (side == 1) __syncthreads();
        const ColDst<NC> dst{Tp, N, M, side == 0 ? q : (q == 0 ? (M >> 1) : M - q), side == 1 && q != 0, live};
        fft_line_regs<M, TPL, true, MAXR>(t, x, dst, sm, tw);
    }
}

// Column pairs per block of the paired gridding unit: blocks of at least 256
// threads (2 TPL threads per column pair).
template <int M> __host__ __device__ constexpr int paired_cpc() {
    return (128 / tpl_of<M>()) > 1 ? 128 / tpl_of<M>() : 1;
}

// P0 + P5 + column P6 for CPC column pairs (q, -q), q = q0 + g, from the
// paired spectrum layout Z2[V][M/2] (float4 slot (Z[j][k], Z[j][-k]), see
// spec_store).  A Cartesian point (q, r') and its mirror (-q, -r') share the
// polar geometry and read the same four slots: at signed radius kappa = +rho
// the point takes the Z[.][+k] halves and the mirror the Z[.][-k] halves
// (swapped for kappa = -rho, and again on a seam row, which reads row V-1 or
// 0 at -k).  The radial taps are always bins floor(rho) and floor(rho) + 1
// with fraction rho - floor(rho) (the two signed-radius brackets of the
// packed form give the same value).  2 TPL threads per column pair gather
// M / (2 TPL) point pairs each into the two shared-memory lines, then
// threads [0, TPL) of the pair run the inverse FFT of column q and
// [TPL, 2 TPL) that of column -q (stored index-reversed; column -M/2 pairs
// with q = 0 and is zero).  PS point pairs per gather step.
template <int M, int TPL, int CPC, int MAXR, int NC = 0, int PS = 2, class SYNC = BlockSync>
__device__ __forceinline__ void grid_unit_paired(float2* smem, int q0, int V, int N, const float4* __restrict__ Z2,
                                                 const int* __restrict__ gJ, const float2* __restrict__ gF,
                                                 float2* __restrict__ Tp, const float2* __restrict__ tw,
                                                 const SYNC& sync = SYNC(), int tid = -1) {
    constexpr int H = M >> 1;
    constexpr int NT = 2 * TPL;
    constexpr int PPT = M / NT;   // point pairs per thread
    static_assert(PPT % PS == 0, "point pairs per step");
    static_assert(PPT % 2 == 0 && (PPT / 2) * NT == (M >> 1), "half the rows of a column per half of the steps");
    static_assert(NT < 32 || NT % 32 == 0, "groups of 32 or more threads are whole warps");
    if (tid < 0) tid = threadIdx.x;
    const int g = tid / NT;
    const int lt = tid % NT;
    const int q = q0 + g;
    const bool live = q < H;
    const SmemLine l0{smem + 2 * g * smem_line_len(M)};
    const SmemLine l1{smem + (2 * g + 1) * smem_line_len(M)};
    const int* gJq = gJ + (size_t)(live ? q : 0) * M;
    const float2* gFq = gF + (size_t)(live ? q : 0) * M;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    int jn[PS];
    float2 fn[PS];
#pragma unroll
    for (int u = 0; u < PS; ++u) {
        jn[u] = __ldg(gJq + lt + u * NT);
        fn[u] = __ldg(gFq + lt + u * NT);
    }
#pragma unroll
    for (int i = 0; i < PPT; i += PS) {
        int jc[PS];
        float2 fc[PS];
#pragma unroll
        for (int u = 0; u < PS; ++u) {
            jc[u] = jn[u];
            fc[u] = fn[u];
        }
        if (i + PS < PPT) {
#pragma unroll
            for (int u = 0; u < PS; ++u) {
                jn[u] = __ldg(gJq + lt + (i + PS + u) * NT);
                fn[u] = __ldg(gFq + lt + (i + PS + u) * NT);
            }
        }
        float4 z[PS][4];
        bool selA[PS], selB[PS];
#pragma unroll
        for (int u = 0; u < PS; ++u) {
            const int Jt = jc[u] >> 16;
            const int k0 = jc[u] & 0xffff;
            // a table bracket >= -1 means the point is inside the band and not the origin
            const bool ok = live && Jt >= -1;
            // kappa = +rho for the point (q, r'), q >= 0, iff r' >= 0, i.e. its row
            // index lt + (i + u) NT < M/2: with 0 <= lt < NT that is exactly
            // (i + u) NT < M/2, fixed per unrolled step
            const bool up = (i + u) < PPT / 2;
            const int J = ok ? Jt : 0;
            const bool sA = J < 0, sB = J + 1 >= V;
            const int rowA = sA ? V - 1 : J;
            const int rowB = sB ? 0 : J + 1;
            // the point takes the +k halves of a row when up, unless the row is a seam row
            selA[u] = up != sA;
            selB[u] = up != sB;
            const bool k1ok = ok && k0 + 1 < H;
            // slots of the four taps: away from the seam both rows lie in the
            // paired storage and the other three are fixed offsets from the
            // first (next bin: +1, or +5 into the next group of four; next
            // row: +4 within a line, 2H - 4 from an odd row to the next line)
            int a0, a1, b0, b1;
            if (!sA && !sB && rowA + 1 < (V & ~1)) {
                a0 = paired_slot(rowA, k0, H, V);
                a1 = a0 + ((k0 & 3) == 3 ? 5 : 1);
                const int dr = (rowA & 1) ? 2 * H - 4 : 4;
                b0 = a0 + dr;
                b1 = a1 + dr;
            } else {
                const int k1 = k1ok ? k0 + 1 : k0;
                a0 = paired_slot(rowA, k0, H, V);
                a1 = paired_slot(rowA, k1, H, V);
                b0 = paired_slot(rowB, k0, H, V);
                b1 = paired_slot(rowB, k1, H, V);
            }
            z[u][0] = ok ? __ldg(Z2 + a0) : zero4;
            z[u][1] = k1ok ? __ldg(Z2 + a1) : zero4;
            z[u][2] = ok ? __ldg(Z2 + b0) : zero4;
            z[u][3] = k1ok ? __ldg(Z2 + b1) : zero4;
        }
#pragma unroll
        for (int u = 0; u < PS; ++u) {
            const int ridx = lt + (i + u) * NT;
            const float ft = fc[u].x, fk = fc[u].y;
            // radial interpolation of whole slots (both halves: Z[.][+k] and
            // Z[.][-k]), then the halves of each row for the point (p) and its
            // mirror (m)
            const float4 a0 = z[u][0], a1 = z[u][1], b0 = z[u][2], b1 = z[u][3];
            const float4 A = make_float4(fmaf(fk, a1.x - a0.x, a0.x), fmaf(fk, a1.y - a0.y, a0.y),
                                         fmaf(fk, a1.z - a0.z, a0.z), fmaf(fk, a1.w - a0.w, a0.w));
            const float4 B = make_float4(fmaf(fk, b1.x - b0.x, b0.x), fmaf(fk, b1.y - b0.y, b0.y),
                                         fmaf(fk, b1.z - b0.z, b0.z), fmaf(fk, b1.w - b0.w, b0.w));
            const float2 pA = selA[u] ? make_float2(A.x, A.y) : make_float2(A.z, A.w);
            const float2 mA = selA[u] ? make_float2(A.z, A.w) : make_float2(A.x, A.y);
            const float2 pB = selB[u] ? make_float2(B.x, B.y) : make_float2(B.z, B.w);
            const float2 mB = selB[u] ? make_float2(B.z, B.w) : make_float2(B.x, B.y);
            l0.store(ridx, make_float2(fmaf(ft, pB.x - pA.x, pA.x), fmaf(ft, pB.y - pA.y, pA.y)));
            l1.store(ridx, q == 0 ? make_float2(0.f, 0.f)
                                  : make_float2(fmaf(ft, mB.x - mA.x, mA.x), fmaf(ft, mB.y - mA.y, mA.y)));
        }
    }
    // the origin is single-valued: mean over angles of the DC bin (the gather
    // stored 0 there, from thread 0 of the group, which also writes the mean).
    // A group of 32 or more threads starts on a warp boundary (NT is then a
    // multiple of 32), so its first warp reduces with a full-warp shuffle;
    // smaller groups share a warp with other groups and sum serially.
    if constexpr (NT >= 32) {
        if (live && q == 0 && lt < 32) {
            float sx = 0.f, sy = 0.f;
            for (int j = lt; j < V; j += 32) {
                const float4 zz = __ldg(Z2 + paired_slot(j, 0, H, V));
                sx += zz.x;
                sy += zz.y;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                sx += __shfl_xor_sync(0xffffffffu, sx, o);
                sy += __shfl_xor_sync(0xffffffffu, sy, o);
            }
            if (lt == 0) l0.store(0, make_float2(sx / (float)V, sy / (float)V));
        }
    } else {
        if (live && q == 0 && lt == 0) {
            float sx = 0.f, sy = 0.f;
            for (int j = 0; j < V; ++j) {
                const float4 zz = __ldg(Z2 + paired_slot(j, 0, H, V));
                sx += zz.x;
                sy += zz.y;
            }
            l0.store(0, make_float2(sx / (float)V, sy / (float)V));
        }
    }
    sync();
    const int half = lt / TPL, t = lt % TPL;
    const SmemLine& line = half ? l1 : l0;
    const ColDst<NC> dst{Tp, N, M, half == 0 ? q : (q == 0 ? H : M - q), half == 1 && q != 0, live};
    fft_line<M, TPL, true, MAXR>(t, line, dst, line, tw, sync);
}

// P0 + P5 + column P6 for one column pair (q, -q) from the paired spectrum
// layout (2 TPL threads), with the first FFT pass of both columns fed from
// registers instead of through shared memory.  Thread (warp w, lane l) is
// thread t = 16 w + l % 16 of column q (l < 16) or of column -q (l >= 16,
// stored index-reversed), so a warp holds the same 16 consecutive t of both
// columns.  The first pass of thread t needs rows t + i TPL, i < M / TPL, of
// its column (fft_line_regs); the lane of column q gathers the point pairs of
// the even i, its partner lane l ^ 16 those of the odd i.  Each point pair
// gives the value of column q (the point) and of column -q (its mirror): a
// lane keeps its own column's value and swaps the other with its partner
// (shfl.xor 16), so that each lane then holds all its first-pass inputs.
// The taps of a quarter-warp (the unit in which 16-byte loads are served)
// are those of 8 consecutive rows of one column, as in grid_unit_paired.
// PS point pairs per gather step.
template <int M, int TPL, int MAXR, int NC = 0, int PS = 2>
__device__ __forceinline__ void grid_unit_xchg(float2* smem, int q, int V, int N, const float4* __restrict__ Z2,
                                               const int* __restrict__ gJ, const float2* __restrict__ gF,
                                               float2* __restrict__ Tp, const float2* __restrict__ tw) {
    constexpr int H = M >> 1;
    constexpr int PPL = M / TPL;   // first-pass inputs per thread (16, or 12 for lengths 3 * 2^a)
    constexpr int PPT = PPL / 2;   // point pairs gathered per thread
    static_assert(TPL % 16 == 0, "half-warps of 16 consecutive threads of a column");
    static_assert(PPL % 4 == 0 && PPT % PS == 0, "steps of the upper and lower half rows");
    const int lane = threadIdx.x & 31;
    const int h = lane >> 4;                                   // 0: column q, 1: column -q
    const int t = ((threadIdx.x >> 5) << 4) + (lane & 15);     // thread index within the column
    const bool live = q < H;
    const int* gJq = gJ + (size_t)(live ? q : 0) * M;
    const float2* gFq = gF + (size_t)(live ? q : 0) * M;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    // xe[i] = input 2 i, xo[i] = input 2 i + 1 of the thread's first pass
    float2 xe[PPT], xo[PPT];
    int jn[PS];
    float2 fn[PS];
#pragma unroll
    for (int u = 0; u < PS; ++u) {
        jn[u] = __ldg(gJq + t + (2 * u + h) * TPL);
        fn[u] = __ldg(gFq + t + (2 * u + h) * TPL);
    }
#pragma unroll
    for (int i = 0; i < PPT; i += PS) {
        int jc[PS];
        float2 fc[PS];
#pragma unroll
        for (int u = 0; u < PS; ++u) {
            jc[u] = jn[u];
            fc[u] = fn[u];
        }
        if (i + PS < PPT) {
#pragma unroll
            for (int u = 0; u < PS; ++u) {
                jn[u] = __ldg(gJq + t + (2 * (i + PS + u) + h) * TPL);
                fn[u] = __ldg(gFq + t + (2 * (i + PS + u) + h) * TPL);
            }
        }
        float4 z[PS][4];
        bool selA[PS], selB[PS];
#pragma unroll
        for (int u = 0; u < PS; ++u) {
            const int Jt = jc[u] >> 16;
            const int k0 = jc[u] & 0xffff;
            const bool ok = live && Jt >= -1;
            // the row t + (2 (i + u) + h) TPL is below M/2 (kappa = +rho for
            // the point) iff 2 (i + u) + h < PPL / 2, i.e. i + u < PPL / 4 for
            // both h: fixed per unrolled step
            const bool up = (i + u) < PPL / 4;
            const int J = ok ? Jt : 0;
            const bool sA = J < 0, sB = J + 1 >= V;
            const int rowA = sA ? V - 1 : J;
            const int rowB = sB ? 0 : J + 1;
            selA[u] = up != sA;
            selB[u] = up != sB;
            const bool k1ok = ok && k0 + 1 < H;
            int a0, a1, b0, b1;
            if (!sA && !sB && rowA + 1 < (V & ~1)) {
                a0 = paired_slot(rowA, k0, H, V);
                a1 = a0 + ((k0 & 3) == 3 ? 5 : 1);
                const int dr = (rowA & 1) ? 2 * H - 4 : 4;
                b0 = a0 + dr;
                b1 = a1 + dr;
            } else {
                const int k1 = k1ok ? k0 + 1 : k0;
                a0 = paired_slot(rowA, k0, H, V);
                a1 = paired_slot(rowA, k1, H, V);
                b0 = paired_slot(rowB, k0, H, V);
                b1 = paired_slot(rowB, k1, H, V);
            }
            z[u][0] = ok ? __ldg(Z2 + a0) : zero4;
            z[u][1] = k1ok ? __ldg(Z2 + a1) : zero4;
            z[u][2] = ok ? __ldg(Z2 + b0) : zero4;
            z[u][3] = k1ok ? __ldg(Z2 + b1) : zero4;
        }
#pragma unroll
        for (int u = 0; u < PS; ++u) {
            const float ft = fc[u].x, fk = fc[u].y;
            const float4 a0 = z[u][0], a1 = z[u][1], b0 = z[u][2], b1 = z[u][3];
            const float4 A = make_float4(fmaf(fk, a1.x - a0.x, a0.x), fmaf(fk, a1.y - a0.y, a0.y),
                                         fmaf(fk, a1.z - a0.z, a0.z), fmaf(fk, a1.w - a0.w, a0.w));
            const float4 B = make_float4(fmaf(fk, b1.x - b0.x, b0.x), fmaf(fk, b1.y - b0.y, b0.y),
                                         fmaf(fk, b1.z - b0.z, b0.z), fmaf(fk, b1.w - b0.w, b0.w));
            const float2 pA = selA[u] ? make_float2(A.x, A.y) : make_float2(A.z, A.w);
            const float2 mA = selA[u] ? make_float2(A.z, A.w) : make_float2(A.x, A.y);
            const float2 pB = selB[u] ? make_float2(B.x, B.y) : make_float2(B.z, B.w);
            const float2 mB = selB[u] ? make_float2(B.z, B.w) : make_float2(B.x, B.y);
            const float2 P = make_float2(fmaf(ft, pB.x - pA.x, pA.x), fmaf(ft, pB.y - pA.y, pA.y));
            const float2 Q = q == 0 ? make_float2(0.f, 0.f)
                                    : make_float2(fmaf(ft, mB.x - mA.x, mA.x), fmaf(ft, mB.y - mA.y, mA.y));
            // keep the own column's value, swap the other with the partner lane
            const float2 own = h ? Q : P, oth = h ? P : Q;
            const float2 rcv = make_float2(__shfl_xor_sync(0xffffffffu, oth.x, 16),
                                           __shfl_xor_sync(0xffffffffu, oth.y, 16));
            xe[i + u] = h ? rcv : own;
            xo[i + u] = h ? own : rcv;
        }
    }
    float2 x[PPL];
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
        x[2 * i] = xe[i];
        x[2 * i + 1] = xo[i];
    }
    // the origin (row 0 of column q = 0, input 0 of thread 0, the gather gave 0
    // there) is single-valued: mean over angles of the DC bin, by warp 0
    if (live && q == 0 && threadIdx.x < 32) {
        float sx = 0.f, sy = 0.f;
        for (int j = lane; j < V; j += 32) {
            const float4 zz = __ldg(Z2 + paired_slot(j, 0, H, V));
            sx += zz.x;
            sy += zz.y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sx += __shfl_xor_sync(0xffffffffu, sx, o);
            sy += __shfl_xor_sync(0xffffffffu, sy, o);
        }
        if (lane == 0) x[0] = make_float2(sx / (float)V, sy / (float)V);
    }
    const SmemLine sm{smem + h * smem_line_len(M)};
    const ColDst<NC> dst{Tp, N, M, h == 0 ? q : (q == 0 ? H : M - q), h == 1 && q != 0, live};
    fft_line_regs<M, TPL, true, MAXR>(t, x, dst, sm, tw);
}

// row P6 + P7 + P8 for row tiles rb0 .. rb0 + TPC - 1 of RPT rows each (RPT TPL
// TPC threads; tid and sync as for ray_unit): tile b holds rows RPT b ..
// RPT b + RPT - 1.  RPT = 4 reads T in whole 32-byte groups of four rows; a
// worker too small for four lines takes RPT = 2.  va, vb: the [N][N] images
// of slices a and b (vb may be null)
template <int M, int TPL, int TPC, int MAXR, int NC = 0, class SYNC = BlockSync, int RPT = 4, bool TWT = false>
__device__ __forceinline__ void row_unit(float2* smem, int rb0, int N, const float2* __restrict__ Tp,
                                         float* __restrict__ va, float* __restrict__ vb, float scale,
                                         const float2* __restrict__ tw, const float* __restrict__ dk = nullptr,
                                         const SYNC& sync = SYNC(), int tid = -1) {
    static_assert(RPT == 4 || RPT == 2, "rows per tile");
    if (tid < 0) tid = threadIdx.x;
    const int tile = tid / (RPT * TPL);
    const int w = tid % (RPT * TPL);
    const int line = w % RPT, t = w / RPT;
    const int r = (rb0 + tile) * RPT + line;
    const bool live = r < N;
    const int rr = live ? r : 0;
    TileSrc src{Tp, M, rr, live};
    VolDst<NC> dst{va + (size_t)rr * N, vb ? vb + (size_t)rr * N : nullptr, N, M,
               dk ? scale * __ldg(dk + rr) : scale, live, dk};
    SmemLine sm{smem + (tile * RPT + line) * row_line_stride<M>()};
    fft_line<M, TPL, true, MAXR, TWT>(t, src, dst, sm, tw, sync);
}

}  // namespace bst
