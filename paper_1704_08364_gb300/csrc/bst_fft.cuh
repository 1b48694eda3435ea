// bst_fft.cuh -- shared-memory Stockham FFT engine for one line of length M.
//
// Used by every stage of the BST path that transforms along a line: the 1D
// FFT along the detector (stage P3), the column and row passes of the 2D
// inverse FFT (stage P6) and their adjoints.  A line of M complex64 values
// is transformed by TPL threads in log_R(M) radix-R Stockham passes
// (out-of-order autosort: no bit reversal), in place in shared memory with a
// barrier between the loads and the stores of each pass.  The first pass may
// read from any source (global memory, a gather) and the last may write to
// any sink, so loads and stores fuse with the neighbouring stage.
//
// Pass with sub-transform length NS and radix R, butterfly j in [0, M/R):
//   inputs   x[j + s M/R],  s = 0..R-1
//   twiddle  x_s *= w^(k s),  k = j mod NS,  w = exp(-+ 2 pi i / (NS R))
//   DFT_R in registers
//   outputs  y[(j / NS) NS R + k + s NS]
// Forward transforms use exp(-2 pi i k m / M), inverse ones exp(+...), both
// unnormalised.  Twiddles come from a table tw[m] = exp(-2 pi i m / M)
// computed in double precision on the host.
#pragma once
#include <cuda_runtime.h>

namespace bst {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// a * (sigma i), sigma = -1 forward, +1 inverse
template <bool INV> __device__ __forceinline__ float2 mul_si(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
// a * (c + sigma i d): multiplication by exp(sigma i phi) with c = cos phi, d = sin phi
template <bool INV> __device__ __forceinline__ float2 mul_w(float2 a, float c, float d) {
    const float sd = INV ? d : -d;
    return make_float2(fmaf(a.x, c, -a.y * sd), fmaf(a.y, c, a.x * sd));
}

// cos and sin of pi/4, pi/8, 3 pi/8 and sqrt(3)/2
#define BST_R2 0.70710678118654752440f
#define BST_C8 0.92387953251128675613f
#define BST_S8 0.38268343236508977173f
#define BST_H3 0.86602540378443864676f

template <int R, bool INV> struct Dft;

template <bool INV> struct Dft<2, INV> {
    __device__ __forceinline__ static void run(float2* a) {
        const float2 t = a[1];
        a[1] = csub(a[0], t);
        a[0] = cadd(a[0], t);
    }
};

template <bool INV> struct Dft<3, INV> {
    __device__ __forceinline__ static void run(float2* a) {
        const float2 t = cadd(a[1], a[2]);
        const float2 u = csub(a[1], a[2]);
        const float2 m = make_float2(fmaf(-0.5f, t.x, a[0].x), fmaf(-0.5f, t.y, a[0].y));
        const float2 v = mul_si<INV>(cscale(u, BST_H3));
        a[0] = cadd(a[0], t);
        a[1] = cadd(m, v);
        a[2] = csub(m, v);
    }
};

template <bool INV> struct Dft<4, INV> {
    __device__ __forceinline__ static void run(float2* a) {
        const float2 a0 = cadd(a[0], a[2]), a1 = csub(a[0], a[2]);
        const float2 b0 = cadd(a[1], a[3]), b1 = mul_si<INV>(csub(a[1], a[3]));
        a[0] = cadd(a0, b0);
        a[2] = csub(a0, b0);
        a[1] = cadd(a1, b1);
        a[3] = csub(a1, b1);
    }
};

template <bool INV> struct Dft<8, INV> {
    __device__ __forceinline__ static void run(float2* a) {
        float2 e[4] = {a[0], a[2], a[4], a[6]};
        float2 o[4] = {a[1], a[3], a[5], a[7]};
        Dft<4, INV>::run(e);
        Dft<4, INV>::run(o);
        o[1] = mul_w<INV>(o[1], BST_R2, BST_R2);
        o[2] = mul_si<INV>(o[2]);
        o[3] = mul_w<INV>(o[3], -BST_R2, BST_R2);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            a[k] = cadd(e[k], o[k]);
            a[k + 4] = csub(e[k], o[k]);
        }
    }
};

// 16 = 4 x 4: four DFT4 over the inputs of stride 4, internal twiddles
// W16^(n2 k1), four DFT4 over the results (fewer multiplications than 2 x 8)
template <bool INV> struct Dft<16, INV> {
    __device__ __forceinline__ static void run(float2* a) {
        float2 b[4][4];
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
            float2 c[4] = {a[n2], a[n2 + 4], a[n2 + 8], a[n2 + 12]};
            Dft<4, INV>::run(c);
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) b[n2][k1] = c[k1];
        }
        // W16^(n2 k1) for n2, k1 = 1..3: exponents 1 2 3 / 2 4 6 / 3 6 9
        b[1][1] = mul_w<INV>(b[1][1], BST_C8, BST_S8);
        b[1][2] = mul_w<INV>(b[1][2], BST_R2, BST_R2);
        b[1][3] = mul_w<INV>(b[1][3], BST_S8, BST_C8);
        b[2][1] = mul_w<INV>(b[2][1], BST_R2, BST_R2);
        b[2][2] = mul_si<INV>(b[2][2]);
        b[2][3] = mul_w<INV>(b[2][3], -BST_R2, BST_R2);
        b[3][1] = mul_w<INV>(b[3][1], BST_S8, BST_C8);
        b[3][2] = mul_w<INV>(b[3][2], -BST_R2, BST_R2);
        b[3][3] = mul_w<INV>(b[3][3], -BST_C8, -BST_S8);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            float2 c[4] = {b[0][k1], b[1][k1], b[2][k1], b[3][k1]};
            Dft<4, INV>::run(c);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) a[k1 + 4 * k2] = c[k2];
        }
    }
};

// ---- radix schedule --------------------------------------------------------

__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x / 2); }
// Radix of pass p for length M = 3^b 2^a (b <= 1) with radices at most MAXR
// (16 or 8): one radix-3 pass first, then ceil(a / log2 MAXR) power-of-two
// passes of as equal a size as possible.  The maximum radix is the schedule
// the autotuner chooses between.
__host__ __device__ constexpr int radix_of(int M, int p, int MAXR = 16) {
    const bool three = (M % 3 == 0);
    if (three && p == 0) return 3;
    const int a = ilog2c(three ? M / 3 : M);
    const int rb = ilog2c(MAXR);
    const int passes = (a + rb - 1) / rb;
    const int q = p - (three ? 1 : 0);
    const int bits = a / passes + (q < a % passes ? 1 : 0);
    return 1 << bits;
}

// ---- per-pass twiddle tables ---------------------------------------------------
//
// Beside the base table tw[m] = exp(-2 pi i m / M), m < M, the plan stores for
// each radix schedule (largest radix 16, then 8) and each pass p >= 1 (radix
// R, sub-transform length NS) the pass's twiddles w^(k s), w = exp(-2 pi i /
// (NS R)), at entry (s - 1) NS + k (s = 1..R-1, k < NS): the R - 1 twiddles of
// butterfly k are NS apart, so the lanes of a warp (consecutive k) read them
// coalesced.  Each entry equals tw[k s M / (NS R)].

// sub-transform length before pass p of the schedule
__host__ __device__ constexpr int pass_ns(int M, int p, int MAXR) {
    return p == 0 ? 1 : pass_ns(M, p - 1, MAXR) * radix_of(M, p - 1, MAXR);
}
// entries of the tables of passes 1 .. p - 1 of the schedule
__host__ __device__ constexpr int pass_tab_prefix(int M, int p, int MAXR) {
    return p <= 1 ? 0 : pass_tab_prefix(M, p - 1, MAXR) + (radix_of(M, p - 1, MAXR) - 1) * pass_ns(M, p - 1, MAXR);
}
// passes of the schedule
__host__ __device__ constexpr int pass_count(int M, int MAXR, int p = 0) {
    return pass_ns(M, p, MAXR) >= M ? p : pass_count(M, MAXR, p + 1);
}
// offset in tw of the table of pass p of the schedule (16 first, then 8)
__host__ __device__ constexpr int pass_tab_base(int M, int MAXR, int p) {
    return M + (MAXR == 8 ? pass_tab_prefix(M, pass_count(M, 16), 16) : 0) + pass_tab_prefix(M, p, MAXR);
}
// complex64 entries of the whole twiddle allocation
__host__ __device__ constexpr int tw_alloc_len(int M) {
    return M + pass_tab_prefix(M, pass_count(M, 16), 16) + pass_tab_prefix(M, pass_count(M, 8), 8);
}

// ---- barriers ----------------------------------------------------------------

// Barrier between the passes of a line: the whole block (__syncthreads), or a
// named barrier shared by the n threads (a multiple of 32) of one worker of a
// block, so that workers of one block run independent lines.
struct BlockSync {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
struct WorkerSync {
    int id;   // barrier 1..15 (0 is the block's __syncthreads barrier)
    int n;    // threads of the worker
    __device__ __forceinline__ void operator()() const {
        asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
    }
};

// ---- line storage ----------------------------------------------------------

// Shared-memory line with one padding slot per 16 elements (bank-conflict free
// for the strided stores of the early passes).
__host__ __device__ constexpr int smem_line_len(int M) { return M + M / 16; }

struct SmemLine {
    float2* p;
    static constexpr bool kSmem = true;
    static constexpr bool kPlain = true;   // load/store are exactly p[i + i/16]
    __device__ __forceinline__ float2 load(int i) const { return p[i + (i >> 4)]; }
    __device__ __forceinline__ void store(int i, float2 v) const { p[i + (i >> 4)] = v; }
};

// ---- passes ----------------------------------------------------------------

// Sources that know index groups of always-zero input (S::zero_group) and
// destinations that know index groups of outputs they drop (D::drop_group):
// the first pass then loads nothing there and the last pass stores nothing
// there, and the compiler removes the arithmetic that only fed them.
template <class T, class = void> struct zero_group_trait { static constexpr bool value = false; };
template <class T>
struct zero_group_trait<T, decltype(void(T::zero_group(0, 0, 0)))> { static constexpr bool value = true; };
template <class T, class = void> struct drop_group_trait { static constexpr bool value = false; };
template <class T>
struct drop_group_trait<T, decltype(void(T::drop_group(0, 0, 0)))> { static constexpr bool value = true; };

template <class S, int M>
__device__ __forceinline__ constexpr bool src_zero_group(int lo, int hi) {
    if constexpr (zero_group_trait<S>::value) return S::zero_group(lo, hi, M);
    return false;
}
template <class D, int M>
__device__ __forceinline__ constexpr bool dst_drop_group(int lo, int hi) {
    if constexpr (drop_group_trait<D>::value) return D::drop_group(lo, hi, M);
    return false;
}

// true for a plain SmemLine (no weighting or remapping in load/store)
template <class T, class = void> struct plain_line_trait { static constexpr bool value = false; };
template <class T> struct plain_line_trait<T, decltype(void(T::kPlain))> { static constexpr bool value = T::kPlain; };
template <class T> __host__ __device__ constexpr bool is_plain_line() { return plain_line_trait<T>::value; }

// w[s] = tw[s * b] for s = 1..R-1 (b = k M / (NS R)): the powers of two of the
// base root come from the table, the others are products of at most three
// table values (error a few ulp), which quarters the table loads of a pass.
template <int R>
__device__ __forceinline__ void twiddles(const float2* __restrict__ tw, int b, float2* w) {
    if constexpr (R == 2) {
        w[1] = __ldg(tw + b);
    } else if constexpr (R == 3) {
        w[1] = __ldg(tw + b);
        w[2] = __ldg(tw + 2 * b);
    } else if constexpr (R == 4) {
        w[1] = __ldg(tw + b);
        w[2] = __ldg(tw + 2 * b);
        w[3] = cmul(w[1], w[2]);
    } else if constexpr (R == 8) {
        w[1] = __ldg(tw + b);
        w[2] = __ldg(tw + 2 * b);
        w[4] = __ldg(tw + 4 * b);
        w[3] = cmul(w[1], w[2]);
        w[5] = cmul(w[1], w[4]);
        w[6] = cmul(w[2], w[4]);
        w[7] = cmul(w[3], w[4]);
    } else {
        static_assert(R == 16, "radix");
        w[1] = __ldg(tw + b);
        w[2] = __ldg(tw + 2 * b);
        w[4] = __ldg(tw + 4 * b);
        w[8] = __ldg(tw + 8 * b);
        w[3] = cmul(w[1], w[2]);
        w[5] = cmul(w[1], w[4]);
        w[6] = cmul(w[2], w[4]);
        w[7] = cmul(w[3], w[4]);
#pragma unroll
        for (int s = 1; s < 8; ++s) w[8 + s] = cmul(w[s], w[8]);
    }
}

// a[s] *= w[s] (conjugated for the inverse) with w[s] = tw[s * b].  For R = 16
// the upper half is applied as (w[s] w[8]) a[8 + s], the same products as the
// table of twiddles() but never more than eight twiddles live at once.
template <int R, bool INV>
__device__ __forceinline__ void apply_twiddles(const float2* __restrict__ tw, int b, float2* a) {
    if constexpr (R == 16) {
        float2 w[8];
        w[1] = __ldg(tw + b);
        w[2] = __ldg(tw + 2 * b);
        w[4] = __ldg(tw + 4 * b);
        w[3] = cmul(w[1], w[2]);
        w[5] = cmul(w[1], w[4]);
        w[6] = cmul(w[2], w[4]);
        w[7] = cmul(w[3], w[4]);
#pragma unroll
        for (int s = 1; s < 8; ++s) a[s] = INV ? cmulc(a[s], w[s]) : cmul(a[s], w[s]);
        const float2 w8 = __ldg(tw + 8 * b);
        a[8] = INV ? cmulc(a[8], w8) : cmul(a[8], w8);
#pragma unroll
        for (int s = 1; s < 8; ++s) {
            const float2 ws = cmul(w[s], w8);
            a[8 + s] = INV ? cmulc(a[8 + s], ws) : cmul(a[8 + s], ws);
        }
    } else {
        float2 w[R];
        twiddles<R>(tw, b, w);
#pragma unroll
        for (int s = 1; s < R; ++s) a[s] = INV ? cmulc(a[s], w[s]) : cmul(a[s], w[s]);
    }
}

// TWT: the twiddles of a pass with NS > 1 come from the pass's own table
// (TB: its offset in tw), one coalesced load each, instead of from the base
// table with products
template <int M, int R, int NS, int TPL, bool INV, bool TWT, int TB, class Src, class Dst, class SYNC>
__device__ __forceinline__ void stockham_pass(int t, const Src& src, const Dst& dst,
                                              const float2* __restrict__ tw, bool sync_mid, const SYNC& sync) {
    constexpr int NB = M / R;
    constexpr int IT = (NB + TPL - 1) / TPL;
    float2 a[IT][R];
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        const int j = t + it * TPL;
        if ((NB % TPL) == 0 || j < NB) {
            if constexpr (is_plain_line<Src>() && NB % 16 == 0) {
                // padded index of j + s NB is (j + j/16) + s (NB + NB/16): one base, constant offsets
                const float2* p = src.p + j + (j >> 4);
#pragma unroll
                for (int s = 0; s < R; ++s) a[it][s] = p[s * (NB + NB / 16)];
            } else {
#pragma unroll
                for (int s = 0; s < R; ++s)
                    a[it][s] = src_zero_group<Src, M>(s * NB, (s + 1) * NB) ? make_float2(0.f, 0.f)
                                                                              : src.load(j + s * NB);
            }
        }
    }
    if (sync_mid) sync();
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        const int j = t + it * TPL;
        if ((NB % TPL) == 0 || j < NB) {
            const int k = (NS == 1) ? 0 : (j % NS);
            if (NS > 1) {
                if constexpr (TWT) {
                    const float2* tp = tw + TB + k;
#pragma unroll
                    for (int s = 1; s < R; ++s) {
                        const float2 w = __ldg(tp + (s - 1) * NS);
                        a[it][s] = INV ? cmulc(a[it][s], w) : cmul(a[it][s], w);
                    }
                } else {
                    constexpr int STEP = M / (NS * R);
                    apply_twiddles<R, INV>(tw, k * STEP, a[it]);
                }
            }
            Dft<R, INV>::run(a[it]);
            const int base = (j / NS) * NS * R + k;
            if constexpr (is_plain_line<Dst>() && (NS % 16 == 0 || (NS == 1 && 16 % R == 0))) {
                // the R outputs base + s NS stay in one 16-group (NS = 1, base a multiple
                // of R) or move by whole groups (NS a multiple of 16): constant offsets
                float2* p = dst.p + base + (base >> 4);
                constexpr int PS = NS == 1 ? 1 : NS + NS / 16;
#pragma unroll
                for (int s = 0; s < R; ++s) p[s * PS] = a[it][s];
            } else {
                // in the last pass base = j < NS, so output s covers indices [s NS, (s + 1) NS)
                constexpr bool LASTP = NS * R == M;
#pragma unroll
                for (int s = 0; s < R; ++s)
                    if (!(LASTP && dst_drop_group<Dst, M>(s * NS, (s + 1) * NS))) dst.store(base + s * NS, a[it][s]);
            }
        }
    }
}

// Run passes PIDX.. of the length-M transform.  Pass 0 reads `src`, the last
// pass writes `dst`; the others go through the shared-memory line `sm`.
// Every thread that `sync` covers must call this (it contains barriers).
template <int M, int TPL, bool INV, int MAXR, int PIDX, int NS, bool TWT, class Src, class Dst, class SYNC>
__device__ __forceinline__ void fft_run(int t, const Src& src, const Dst& dst, const SmemLine& sm,
                                        const float2* __restrict__ tw, const SYNC& sync) {
    constexpr int R = radix_of(M, PIDX, MAXR);
    constexpr bool LAST = (NS * R == M);
    constexpr int TB = pass_tab_base(M, MAXR, PIDX);
    if constexpr (PIDX == 0) {
        if constexpr (LAST) {
            stockham_pass<M, R, NS, TPL, INV, TWT, TB>(t, src, dst, tw, Src::kSmem && Dst::kSmem, sync);
        } else {
            stockham_pass<M, R, NS, TPL, INV, TWT, TB>(t, src, sm, tw, Src::kSmem, sync);
            sync();
            fft_run<M, TPL, INV, MAXR, PIDX + 1, NS * R, TWT>(t, src, dst, sm, tw, sync);
        }
    } else {
        if constexpr (LAST) {
            stockham_pass<M, R, NS, TPL, INV, TWT, TB>(t, sm, dst, tw, Dst::kSmem, sync);
        } else {
            stockham_pass<M, R, NS, TPL, INV, TWT, TB>(t, sm, sm, tw, true, sync);
            sync();
            fft_run<M, TPL, INV, MAXR, PIDX + 1, NS * R, TWT>(t, src, dst, sm, tw, sync);
        }
    }
}

// TWT: twiddles from the per-pass tables (one coalesced load each) instead of
// four base-table loads and products per butterfly
template <int M, int TPL, bool INV, int MAXR = 16, bool TWT = false, class Src, class Dst, class SYNC = BlockSync>
__device__ __forceinline__ void fft_line(int t, const Src& src, const Dst& dst, const SmemLine& sm,
                                         const float2* __restrict__ tw, const SYNC& sync = SYNC()) {
    fft_run<M, TPL, INV, MAXR, 0, 1, TWT>(t, src, dst, sm, tw, sync);
}

// The transform of a line whose values thread t already holds in registers,
// x[i] = line[t + i TPL] for i < M / TPL (the order in which a gather fills the
// line).  These are exactly the first pass's inputs of butterflies
// j = t + it TPL: element j + s M/R is x[it + s IT].  So pass 0 runs on them
// directly and only its outputs go to the shared-memory line `sm`; the later
// passes are those of fft_line.  Call with every thread of the block; `sm`
// must be free for writing (the caller's barrier).
template <int M, int TPL, bool INV, int MAXR = 16, class Dst, class SYNC = BlockSync, bool TWT = false>
__device__ __forceinline__ void fft_line_regs(int t, float2 (&x)[M / TPL], const Dst& dst, const SmemLine& sm,
                                              const float2* __restrict__ tw, const SYNC& sync = SYNC()) {
    constexpr int R = radix_of(M, 0, MAXR);
    constexpr int NB = M / R;
    static_assert(NB % TPL == 0, "one or more whole first-pass butterflies per thread");
    constexpr int IT = NB / TPL;
    if constexpr (R == M) {
        // a single pass: one thread holds the whole line
        Dft<R, INV>::run(x);
#pragma unroll
        for (int s = 0; s < R; ++s)
            if (!dst_drop_group<Dst, M>(s, s + 1)) dst.store(s, x[s]);
        return;
    }
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        float2 a[R];
#pragma unroll
        for (int s = 0; s < R; ++s) a[s] = x[it + s * IT];
        Dft<R, INV>::run(a);
        const int base = (t + it * TPL) * R;
        if constexpr (16 % R == 0) {
            // base is a multiple of R, so the R outputs stay in one 16-group
            float2* p = sm.p + base + (base >> 4);
#pragma unroll
            for (int s = 0; s < R; ++s) p[s] = a[s];
        } else {
#pragma unroll
            for (int s = 0; s < R; ++s) sm.store(base + s, a[s]);
        }
    }
    if constexpr (R < M) {
        sync();
        fft_run<M, TPL, INV, MAXR, 1, R, TWT>(t, sm, dst, sm, tw, sync);
    }
}

// signed frequency of natural-order index p
__device__ __forceinline__ int signed_freq(int p, int M) { return p < (M >> 1) ? p : p - M; }

}  // namespace bst
