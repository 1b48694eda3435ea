// bst_kb.cuh -- stage P5 as Kaiser-Bessel convolution gridding, fused with the
// column half of P6 (device part).
//
// Every polar sample Y_j[k] (k != 0, -M/2) carries the area of its polar cell:
// the ray stage has multiplied it by |k| W[|k|] (W[0] / 4 for the DC cell, the
// cell average of |k|) and the angular weight dtheta_j is applied here.  It sits
// at (c_s, r_s) = k (cos theta_j, sin theta_j) bins and is spread onto the W x W
// Cartesian points c' - c_s, r' - r_s in (-W/2, W/2] with the separable kernel
// phi(x) = (I0(beta sqrt(1 - (2x/W)^2)) - 1) / (I0(beta) - 1) (the KB kernel
// without its pedestal, zero at the support edge), on the M-periodic grid;
// phi is evaluated as a per-plan polynomial (KbArgs::poly).
// The division by phi's transform (deapodization) happens in the row stage.
//
// One block owns a strip of four consecutive Cartesian columns (storage
// order), kept in shared memory as four padded FFT lines.  The plan lists, per
// strip, every sample whose footprint touches it, sorted by the first row of
// the footprint, and cuts the strip into bands of four rows: a band's samples
// are then one contiguous range of that list (two at the periodic wrap), which
// the plan splits into work items of at most KB_ITEM entries.  A thread takes
// an item, accumulates the 4 x 4 cell of its band in registers (the weight of
// every sample at every cell point, zero outside the footprint) and adds the
// cell to shared memory once, so heavy bands near the origin are shared by
// many threads and the atomics are one per cell point and item, not per
// sample.  Then the inverse FFT along r' of each column runs in place and the
// N central rows go to T exactly as with the bilinear gather.  The V samples
// of the DC bin all sit at the origin; one warp sums them (with their angular
// weights) and spreads the sum once.
//
// Positions are exact to float rounding of a number below one: k cos(theta)
// is split into the nearest integer and a remainder with the double-float
// direction table and FMA, so the kernel weights do not lose the ~1e-4 bin
// that a plain float product loses at radius 2048.  Weights come from the
// exact distance to each cell point, so which samples the plan lists (in
// double precision) only has to be a superset of the float footprints up to
// the kernel's zero edge.
#pragma once
#include <cuda_runtime.h>

#include "bst_stages.cuh"

namespace bst {

constexpr int KB_POLY = 12;    // degree of the kernel polynomial (see KbArgs::poly)
constexpr int KB_WMAX = 8;
constexpr int KB_CS = 4;       // columns per strip
constexpr int KB_RB = 4;       // rows per band
constexpr int KB_ITEM = 64;    // entries per work item at most (16 and 128 measured slower)

struct KbArgs {
    // phi as a polynomial of degree kb_degree(W) <= KB_POLY in
    // t = 2 (2x/W)^2 - 1 (Chebyshev interpolation of phi at degree + 1 nodes,
    // built per plan in double precision; monomial coefficients, Horner in
    // float: absolute error below 3e-7 for every supported width and pad
    // factor); coefficients above the degree are zero
    float poly[KB_POLY + 1];
    float t_scale;         // 8 / W^2, so that t = x^2 t_scale - 1
    const int* istart;     // [nstrips + 1] offsets of the strips' work items
    const int4* items;     // (band, first entry, end entry, 0)
    const int* list;       // sample ids j M + kidx (natural-order bin index)
    const float4* dir;     // [V + 2] (cos_hi, cos_lo, sin_hi, sin_lo) of theta_{j}, at j + 1
    const float* wq;       // [V] angular weights dtheta_j
    int W;                 // kernel width in bins (even, <= KB_WMAX)
    int nstrips;
};

template <int M> __host__ __device__ constexpr int kb_threads() { return KB_CS * tpl_of<M>(); }

template <int M> __host__ __device__ constexpr size_t kb_smem_bytes() {
    return (size_t)KB_CS * smem_line_len(M) * sizeof(float2);
}

// phi(x): the plan's polynomial of degree DEG in t = 2 (2x/W)^2 - 1 on the
// support, zero for |x| >= W/2 (t >= 1).  Arithmetic only (the coefficients
// are kernel arguments), so the weights cost FMA issue instead of
// shared-memory lookups.  DEG = 10 serves W <= 6 (interpolation error below
// 1e-7), DEG = 12 all widths (the plan fits the degree it will use).
template <int DEG = KB_POLY>
__device__ __forceinline__ float kb_phi(const KbArgs& kb, float x) {
    const float t = fmaf(x * x, kb.t_scale, -1.f);
    float h = kb.poly[DEG];
#pragma unroll
    for (int i = DEG - 1; i >= 0; --i) h = fmaf(h, t, kb.poly[i]);
    return t < 1.f ? h : 0.f;
}

// degree of the kernel polynomial for width W
__host__ __device__ constexpr int kb_degree(int W) { return W <= 6 ? 10 : KB_POLY; }

// k * (hi + lo) = n + d with n an integer (as float) and |d| <= ~0.5
__device__ __forceinline__ void kb_split(float k, float hi, float lo, float& n, float& d) {
    const float p = __fmul_rn(k, hi);
    const float e = fmaf(k, lo, fmaf(k, hi, -p));
    n = rintf(p);
    d = __fadd_rn(__fsub_rn(p, n), e);
}

// signed distance (in bins, periodic in M) from the sample at n + d to grid index g
template <int M>
__device__ __forceinline__ float kb_dist(int g, float n, float d) {
    int q = g - (int)n;
    q = q >= (M >> 1) ? q - M : (q < -(M >> 1) ? q + M : q);
    return (float)q - d;
}

// accumulate the samples of entries [lo, hi) into the 4 x 4 cell (rows r0..r0+3,
// columns c0..c0+3) and add the cell to the strip's shared-memory lines.  The
// loads of the next entry (its sample's direction, value and angular weight;
// the sample id one entry further) are issued before the current entry's
// arithmetic, so their latency overlaps it.
template <int M, int DEG>
__device__ __forceinline__ void kb_item(float2* smem, const KbArgs& kb, const float2* __restrict__ Zp,
                                        int c0, int r0, int lo, int hi) {
    constexpr int LL = smem_line_len(M);
    float ax[KB_CS][KB_RB], ay[KB_CS][KB_RB];
#pragma unroll
    for (int c = 0; c < KB_CS; ++c)
#pragma unroll
        for (int r = 0; r < KB_RB; ++r) ax[c][r] = ay[c][r] = 0.f;
    int sn = lo < hi ? __ldg(kb.list + lo) : 0;          // sample id of entry e
    int sn2 = lo + 1 < hi ? __ldg(kb.list + lo + 1) : 0; // ... of entry e + 1
    float4 dn = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 zn = make_float2(0.f, 0.f);
    float wn = 0.f;
    if (lo < hi) {
        const int j = sn / M;
        dn = __ldg(kb.dir + j + 1);
        zn = __ldg(Zp + sn);
        wn = __ldg(kb.wq + j);
    }
    for (int e = lo; e < hi; ++e) {
        const int s = sn;
        const float4 d = dn;
        const float2 zz = zn;
        const float wa = wn;
        if (e + 1 < hi) {
            sn = sn2;
            sn2 = e + 2 < hi ? __ldg(kb.list + e + 2) : 0;
            const int jn = sn / M;
            dn = __ldg(kb.dir + jn + 1);
            zn = __ldg(Zp + sn);
            wn = __ldg(kb.wq + jn);
        }
        const int j = s / M;
        const int kidx = s - j * M;
        const float k = (float)(kidx < (M >> 1) ? kidx : kidx - M);
        float nc, dc, nr, dr;
        kb_split(k, d.x, d.y, nc, dc);
        kb_split(k, d.z, d.w, nr, dr);
        // distances to the band's rows and the strip's columns: the first one
        // with the periodic wrap, the others one bin further each (a wrap
        // inside a run of four points only moves points that are at least
        // M/2 - 4 >= W/2 bins away, where phi is zero either way)
        const float xr = kb_dist<M>(r0, nr, dr), xc = kb_dist<M>(c0, nc, dc);
        float wr[KB_RB];
#pragma unroll
        for (int r = 0; r < KB_RB; ++r) wr[r] = kb_phi<DEG>(kb, xr + (float)r);
#pragma unroll
        for (int c = 0; c < KB_CS; ++c) {
            const float wc = wa * kb_phi<DEG>(kb, xc + (float)c);
            const float zx = wc * zz.x, zy = wc * zz.y;
#pragma unroll
            for (int r = 0; r < KB_RB; ++r) {
                ax[c][r] = fmaf(wr[r], zx, ax[c][r]);
                ay[c][r] = fmaf(wr[r], zy, ay[c][r]);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < KB_CS; ++c) {
        float* line = reinterpret_cast<float*>(smem + c * LL);
#pragma unroll
        for (int r = 0; r < KB_RB; ++r) {
            const int rr = r0 + r;
            const int o = 2 * (rr + (rr >> 4));
            atomicAdd(line + o, ax[c][r]);
            atomicAdd(line + o + 1, ay[c][r]);
        }
    }
}

// the DC sample at the origin (value z) into the strip's columns
template <int M>
__device__ __forceinline__ void kb_spread_dc(float2* smem, const KbArgs& kb, int c0, float2 z) {
    constexpr int LL = smem_line_len(M);
    const int hw = kb.W >> 1;
    for (int c = 0; c < KB_CS; ++c) {
        const float x = kb_dist<M>(c0 + c, 0.f, 0.f);
        if (fabsf(x) >= (float)hw) continue;
        const float wc = kb_phi(kb, x);
        float* line = reinterpret_cast<float*>(smem + c * LL);
        for (int r = -hw + 1; r < hw; ++r) {
            const int rr = r < 0 ? r + M : r;
            const float w = wc * kb_phi(kb, (float)r);
            const int o = 2 * (rr + (rr >> 4));
            atomicAdd(line + o, w * z.x);
            atomicAdd(line + o + 1, w * z.y);
        }
    }
}

// P5 (KB gridding) + column P6 for the strip of four columns starting at
// c0 = 4 strip of one slice pair (blockDim = 4 TPL)
template <int M, int TPL, int MAXR>
__device__ __forceinline__ void kb_col_unit(float2* smem, int strip, int V, int N, const float2* __restrict__ Zp,
                                            const KbArgs& kb, float2* __restrict__ Tp,
                                            const float2* __restrict__ tw) {
    constexpr int NT = KB_CS * TPL;
    constexpr int LL = smem_line_len(M);
    __shared__ int next_item;
    const int tid = threadIdx.x;
    for (int i = tid; i < KB_CS * LL; i += NT) smem[i] = make_float2(0.f, 0.f);
    const int c0 = strip * KB_CS;
    const int i0 = __ldg(kb.istart + strip), i1 = __ldg(kb.istart + strip + 1);
    if (tid == 0) next_item = i0 + NT;
    __syncthreads();

    // items are ordered longest first; each thread takes the next free one
    // when it finishes (greedy longest-first), which evens out the threads'
    // work before the barrier of the column transform
    if (kb.W <= 6) {
        for (int i = i0 + tid; i < i1; i = atomicAdd(&next_item, 1)) {
            const int4 it = __ldg(kb.items + i);
            kb_item<M, kb_degree(6)>(smem, kb, Zp, c0, KB_RB * it.x, it.y, it.z);
        }
    } else {
        for (int i = i0 + tid; i < i1; i = atomicAdd(&next_item, 1)) {
            const int4 it = __ldg(kb.items + i);
            kb_item<M, kb_degree(8)>(smem, kb, Zp, c0, KB_RB * it.x, it.y, it.z);
        }
    }

    // the DC bin of every angle sits at the origin: one weighted sum, spread once
    if (c0 < (kb.W >> 1) || c0 + KB_CS > M - (kb.W >> 1)) {
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
                if (tid == 0) kb_spread_dc<M>(smem, kb, c0, make_float2(sx, sy));
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
                kb_spread_dc<M>(smem, kb, c0, make_float2(sx, sy));
            }
        }
    }
    __syncthreads();

    // inverse FFT along r' of each column in place; the N central rows go to T
    const int line = tid / TPL, t = tid % TPL;
    const SmemLine sm{smem + line * LL};
    const ColDst<> dst{Tp, N, M, c0 + line, false, true};
    fft_line<M, TPL, true, MAXR>(t, sm, dst, sm, tw);
}

}  // namespace bst
