// bst_kb.cuh -- stage P5 as Kaiser-Bessel convolution gridding, fused with the
// column half of P6 (device part).
//
// Every polar sample Y_j[k] (k != 0, -M/2) carries the area of its polar cell:
// the ray stage has multiplied it by |k| W[|k|] (W[0] / 4 for the DC cell, the
// cell average of |k|) and the angular weight dtheta_j is applied here.  It sits
// at (c_s, r_s) = k (cos theta_j, sin theta_j) bins and is spread onto the W x W
// Cartesian points c' - c_s, r' - r_s in (-W/2, W/2] with the separable kernel
// phi(x) = (I0(beta sqrt(1 - (2x/W)^2)) - 1) / (I0(beta) - 1) (the KB kernel
// without its pedestal, zero at the support edge), on the M-periodic grid.
// The division by phi's transform (deapodization) happens in the row stage.
//
// One block owns a strip of CS consecutive Cartesian columns (storage order),
// kept in shared memory as CS padded FFT lines: it zeroes them, spreads the
// strip's samples (the plan lists, per strip, every sample whose footprint
// touches it) with shared-memory atomics, then runs the inverse FFT along r'
// of each column in place and writes the N central rows to T exactly as the
// bilinear gather does.  The V samples of the DC bin all sit at the origin;
// one warp sums them (with their angular weights) and spreads the sum once.
//
// Positions are exact to float rounding of a number below one: k cos(theta)
// is split into the nearest integer and a remainder with the double-float
// direction table and FMA, so the kernel weights do not lose the ~1e-4 bin
// that a plain float product loses at radius 2048.
#pragma once
#include <cuda_runtime.h>

#include "bst_stages.cuh"

namespace bst {

constexpr int KB_TAB = 8192;   // table intervals over [0, W/2]
constexpr int KB_WMAX = 8;

struct KbArgs {
    const float* tab;      // [KB_TAB + 2] phi(i W / (2 KB_TAB)); the last entry repeats
    const int* start;      // [nstrips + 1] CSR offsets of the strips' sample lists
    const int* list;       // sample ids j M + kidx (natural-order bin index)
    const float4* dir;     // [V + 2] (cos_hi, cos_lo, sin_hi, sin_lo) of theta_{j}, at j + 1
    const float* wq;       // [V] angular weights dtheta_j
    int W;                 // kernel width in bins (even, <= KB_WMAX)
    float tab_scale;       // KB_TAB / (W / 2)
    int nstrips;
};

// columns per strip: CS lines of TPL threads fill a 1024-thread block
template <int M> __host__ __device__ constexpr int kb_strip_cols() {
    return (1024 / tpl_of<M>()) < M ? 1024 / tpl_of<M>() : M;
}

template <int M> __host__ __device__ constexpr size_t kb_smem_bytes() {
    return (size_t)kb_strip_cols<M>() * smem_line_len(M) * sizeof(float2) + (size_t)(KB_TAB + 2) * sizeof(float);
}

__device__ __forceinline__ float kb_phi(const float* tab, float x, float scale) {
    const float u = fabsf(x) * scale;
    int i = (int)u;
    i = i < KB_TAB ? i : KB_TAB;
    const float f = u - (float)i;
    const float a = tab[i];
    return fmaf(f, tab[i + 1] - a, a);
}

// k * (hi + lo) = n + d with n an integer (as float) and |d| <= ~0.5
__device__ __forceinline__ void kb_split(float k, float hi, float lo, float& n, float& d) {
    const float p = __fmul_rn(k, hi);
    const float e = fmaf(k, lo, fmaf(k, hi, -p));
    n = rintf(p);
    d = __fadd_rn(__fsub_rn(p, n), e);
}

// Spread one sample of value z at (nc + dc, nr + dr) bins into the strip's
// columns [c0, c0 + CS).  Strip-local lines of length LL (padded index).
template <int M, int CS>
__device__ __forceinline__ void kb_spread(float2* smem, const float* tab, const KbArgs& kb, int c0, float nc,
                                          float dc, float nr, float dr, float2 z) {
    constexpr int LL = smem_line_len(M);
    const int hw = kb.W >> 1;
    const int fc0 = (int)nc - hw + (dc < 0.f ? 0 : 1);
    const int fr0 = (int)nr - hw + (dr < 0.f ? 0 : 1);
    const float xc0 = (float)(fc0 - (int)nc) - dc;
    const float xr0 = (float)(fr0 - (int)nr) - dr;
    float wr[KB_WMAX];
#pragma unroll
    for (int i = 0; i < KB_WMAX; ++i) wr[i] = i < kb.W ? kb_phi(tab, xr0 + (float)i, kb.tab_scale) : 0.f;
#pragma unroll
    for (int ic = 0; ic < KB_WMAX; ++ic) {
        if (ic >= kb.W) break;
        const int fc = fc0 + ic;
        const int lc = (fc < 0 ? fc + M : fc) - c0;
        if ((unsigned)lc >= (unsigned)CS) continue;
        const float wc = kb_phi(tab, xc0 + (float)ic, kb.tab_scale);
        const float2 zc = make_float2(wc * z.x, wc * z.y);
        float* line = reinterpret_cast<float*>(smem + lc * LL);
#pragma unroll
        for (int ir = 0; ir < KB_WMAX; ++ir) {
            if (ir >= kb.W) break;
            const int fr = fr0 + ir;
            const int rr = fr < 0 ? fr + M : fr;
            const int o = 2 * (rr + (rr >> 4));
            atomicAdd(line + o, wr[ir] * zc.x);
            atomicAdd(line + o + 1, wr[ir] * zc.y);
        }
    }
}

// P5 (KB gridding) + column P6 for the strip of CS columns starting at c0 of
// one slice pair (blockDim = TPL * CS).
template <int M, int TPL, int MAXR>
__device__ __forceinline__ void kb_col_unit(float2* smem, int strip, int V, int N, const float2* __restrict__ Zp,
                                            const KbArgs& kb, float2* __restrict__ Tp,
                                            const float2* __restrict__ tw) {
    constexpr int CS = kb_strip_cols<M>();
    constexpr int NT = TPL * CS;
    constexpr int LL = smem_line_len(M);
    float* tab = reinterpret_cast<float*>(smem + CS * LL);
    const int tid = threadIdx.x;
    for (int i = tid; i < KB_TAB + 2; i += NT) tab[i] = __ldg(kb.tab + i);
    for (int i = tid; i < CS * LL; i += NT) smem[i] = make_float2(0.f, 0.f);
    __syncthreads();
    const int c0 = strip * CS;

    // the strip's samples; lanes of a warp take entries NT / 32 apart so that
    // their footprints (neighbouring samples of one ray overlap) rarely collide
    const int e0 = __ldg(kb.start + strip), e1 = __ldg(kb.start + strip + 1);
    const int slot = (NT % 32 == 0) ? (tid & 31) * (NT / 32) + (tid >> 5) : tid;
    for (int base = e0; base < e1; base += NT) {
        const int e = base + slot;
        if (e >= e1) continue;
        const int s = __ldg(kb.list + e);
        const int j = s / M;
        const int kidx = s - j * M;
        const float k = (float)(kidx < (M >> 1) ? kidx : kidx - M);
        const float4 d = __ldg(kb.dir + j + 1);
        float nc, dc, nr, dr;
        kb_split(k, d.x, d.y, nc, dc);
        kb_split(k, d.z, d.w, nr, dr);
        const float2 zz = __ldg(Zp + s);
        const float wa = __ldg(kb.wq + j);
        kb_spread<M, CS>(smem, tab, kb, c0, nc, dc, nr, dr, make_float2(wa * zz.x, wa * zz.y));
    }

    // the DC bin of every angle sits at the origin: one weighted sum, spread once
    {
        const int hw = kb.W >> 1;
        bool here = false;
        for (int ic = 0; ic < kb.W; ++ic) {
            const int fc = ic - hw + 1;
            here |= (unsigned)((fc < 0 ? fc + M : fc) - c0) < (unsigned)CS;
        }
        if (here) {
            if constexpr (NT >= 32) {
                if (tid < 32) {
                    float sx = 0.f, sy = 0.f;
                    for (int j = tid; j < V; j += 32) {
                        const float w = __ldg(kb.wq + j);
                        const float2 zz = __ldg(Zp + (size_t)j * M);
                        sx = fmaf(w, zz.x, sx);
                        sy = fmaf(w, zz.y, sy);
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        sx += __shfl_xor_sync(0xffffffffu, sx, o);
                        sy += __shfl_xor_sync(0xffffffffu, sy, o);
                    }
                    if (tid == 0) kb_spread<M, CS>(smem, tab, kb, c0, 0.f, 0.f, 0.f, 0.f, make_float2(sx, sy));
                }
            } else {
                if (tid == 0) {
                    float sx = 0.f, sy = 0.f;
                    for (int j = 0; j < V; ++j) {
                        const float w = __ldg(kb.wq + j);
                        const float2 zz = __ldg(Zp + (size_t)j * M);
                        sx = fmaf(w, zz.x, sx);
                        sy = fmaf(w, zz.y, sy);
                    }
                    kb_spread<M, CS>(smem, tab, kb, c0, 0.f, 0.f, 0.f, 0.f, make_float2(sx, sy));
                }
            }
        }
    }
    __syncthreads();

    // inverse FFT along r' of each column in place; the N central rows go to T
    const int line = tid / TPL, t = tid % TPL;
    const SmemLine sm{smem + line * LL};
    const ColDst dst{Tp, N, M, c0 + line, false, true};
    fft_line<M, TPL, true, MAXR>(t, sm, dst, sm, tw);
}

}  // namespace bst
