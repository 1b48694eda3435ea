// bst_geo.cuh -- polar coordinates of Cartesian frequency points (stage P5).
//
// The 2D spectrum of the backprojection is known on the polar grid
// (sigma_k, theta_j) through Eq. 3; stage P5 interpolates it onto the
// Cartesian grid omega = (c', r') dw.  In bins, the point (c', r') has radius
// rho = sqrt(c'^2 + r'^2) and lies on the line through the origin at angle
// theta in [0, pi): signed radius kappa = +rho when r' > 0 or (r' = 0 and
// c' >= 0), else kappa = -rho with the direction flipped (the signed-radius
// form of P0: y(-t, theta) = y(t, theta + pi)).  The value is the bilinear
// interpolation of the polar samples in (kappa, theta) with the angle bracket
// theta_J <= theta < theta_{J+1}, J = -1..V-1, theta_{-1} = theta_{V-1} - pi,
// theta_V = theta_0 + pi; a tap on the virtual rows -1 or V reads row V-1 or 0
// at bin -k.  Points with rho >= M/2 and taps at |k| >= M/2 are zero.
//
// FP32 accuracy: the radius fraction is computed from the exact integer
// rho^2 as (rho^2 - k0^2) / (rho + k0), and the angle offset from theta_J as
// atan(cross / dot) with the cross product evaluated in double-float
// arithmetic (cos and sin of theta_J as hi + lo float pairs, leading products
// split with FMA), so that the interpolation weights are accurate to a few
// ulp even at radius M/2 = 2048 bins.
#pragma once
#include <cuda_runtime.h>

namespace bst {

struct Geo {
    const float4* __restrict__ dir;    // [V+2] (cos_hi, cos_lo, sin_hi, sin_lo) of theta_J, J = -1..V
    const float* __restrict__ invdth;  // [V+1] 1 / (theta_{J+1} - theta_J), J = -1..V-1
    const int* __restrict__ lut;       // [L] largest J with theta_J <= b pi / L (or -1)
    int V, M, L;
    float lut_scale;                   // L / pi
    int uniform;                       // angles evenly spaced: bracket estimate by arithmetic
    float th0, inv_step;               // theta_0 and 1 / spacing (uniform estimate only)
};

struct Polar {
    int J;       // angle bracket, -1..V-1
    float fth;   // fraction in the bracket, [0, 1]
    int k0;      // floor(rho)
    float frac;  // rho - k0, [0, 1)
    bool up;     // kappa = +rho (else -rho)
};

// (ch + cl) uy - (sh + sl) ux with the products of the leading parts split
// exactly by FMA; no contraction across the explicit roundings.
__device__ __forceinline__ float cross_df(float4 d, float ux, float uy) {
    const float p1 = __fmul_rn(d.x, uy);
    const float p2 = __fmul_rn(d.z, ux);
    const float e1 = fmaf(d.x, uy, -p1);
    const float e2 = fmaf(d.z, ux, -p2);
    const float lo = __fadd_rn(__fsub_rn(e1, e2), __fsub_rn(__fmul_rn(d.y, uy), __fmul_rn(d.w, ux)));
    return __fadd_rn(__fsub_rn(p1, p2), lo);
}

// Angle of (ux, uy), uy >= 0, to within ~5e-6 rad: an odd polynomial of
// degree 11 in the octant ratio (coefficients fitted by weighted least
// squares to atan on [0, 1]).  Only an estimate: the bracket it selects is
// verified with exact cross products.
__device__ __forceinline__ float angle_estimate(float ux, float uy) {
    const float ax = fabsf(ux);
    const float mn = fminf(ax, uy), mx = fmaxf(ax, uy);
    const float t = __fdividef(mn, mx);
    const float t2 = t * t;
    float p = fmaf(t2, -0.01017310842871666f, 0.04828116297721863f);
    p = fmaf(t2, p, -0.11188798397779465f);
    p = fmaf(t2, p, 0.19143280386924744f);
    p = fmaf(t2, p, -0.33220672607421875f);
    p = fmaf(t2, p, 0.9999518394470215f);
    float a = t * p;
    if (uy > ax) a = 1.57079632679489662f - a;
    if (ux < 0.f) a = 3.14159265358979324f - a;
    return a;
}

// Radial part of the polar coordinates of (cx, ry): rho = sqrt(cx^2 + ry^2)
// as k0 = floor(rho) and frac = rho - k0 (from the exact integer rho^2), and
// the sign of kappa.  Returns false when rho >= M/2 (the point is zero).
__device__ __forceinline__ bool polar_radius(int cx, int ry, int M, Polar& P) {
    const int rho2 = cx * cx + ry * ry;
    const int half = M >> 1;
    if (rho2 >= half * half) return false;
    P.up = (ry > 0) || (ry == 0 && cx >= 0);
    const float rf = __fsqrt_rn((float)rho2);   // rho2 < 2^24 is exact in float
    int k0 = (int)rf;
    if (k0 * k0 > rho2) --k0;
    else if ((k0 + 1) * (k0 + 1) <= rho2) ++k0;
    P.frac = __fdividef((float)(rho2 - k0 * k0), rf + (float)k0);
    P.k0 = k0;
    return true;
}

// Angular part: bracket J and fraction fth of the direction (ux, uy), uy >= 0.
__device__ __forceinline__ void polar_angle(float ux, float uy, const Geo& g, Polar& P) {
    const float th = angle_estimate(ux, uy);
    int J;
    if (g.uniform) {
        J = __float2int_rd((th - g.th0) * g.inv_step);
    } else {
        int b = (int)(th * g.lut_scale);
        b = b < 0 ? 0 : (b >= g.L ? g.L - 1 : b);
        J = __ldg(g.lut + b);
    }
    J = J < -1 ? -1 : (J > g.V - 1 ? g.V - 1 : J);
    while (J < g.V - 1 && cross_df(__ldg(g.dir + J + 2), ux, uy) >= 0.f) ++J;
    float4 d = __ldg(g.dir + J + 1);
    float cr = cross_df(d, ux, uy);
    while (J >= 0 && cr < 0.f) {
        --J;
        d = __ldg(g.dir + J + 1);
        cr = cross_df(d, ux, uy);
    }
    const float dt = fmaf(d.x, ux, d.z * uy);
    float delta;
    if (fabsf(cr) <= 0.0625f * dt) {
        // atan(q) = q (1 - q^2/3 + q^4/5 - q^6/7), truncation < 1e-10 relative for |q| <= 1/16
        const float q = __fdividef(cr, dt);
        const float q2 = q * q;
        delta = q * fmaf(q2, fmaf(q2, fmaf(q2, -1.0f / 7.0f, 0.2f), -1.0f / 3.0f), 1.0f);
    } else {
        delta = atan2f(cr, dt);
    }
    const float f = delta * __ldg(g.invdth + J + 1);
    P.fth = fminf(fmaxf(f, 0.f), 1.f);
    P.J = J;
}

// Polar coordinates of the Cartesian point (cx, ry), origin excluded.
// Returns false when rho >= M/2 (the point is zero).
__device__ __forceinline__ bool polar_of(int cx, int ry, const Geo& g, Polar& P) {
    if (!polar_radius(cx, ry, g.M, P)) return false;
    const float ux = (float)(P.up ? cx : -cx);
    const float uy = (float)(P.up ? ry : -ry);
    polar_angle(ux, uy, g, P);
    return true;
}

// Polar sample (virtual row Jv, signed bin K) of the spectrum Z[V][M] (natural order).
__device__ __forceinline__ float2 polar_tap(const float2* __restrict__ Z, int V, int M, int Jv, int K) {
    int row = Jv, bin = K;
    if (Jv < 0) {
        row = V - 1;
        bin = -K;
    } else if (Jv >= V) {
        row = 0;
        bin = -K;
    }
    const int half = M >> 1;
    if (bin >= half || bin <= -half) return make_float2(0.f, 0.f);
    if (bin < 0) bin += M;
    return __ldg(Z + (size_t)row * M + bin);
}

// Bilinear interpolation at (bracket J, fraction fth; radial bin K0, fraction fk).
__device__ __forceinline__ float2 polar_gather(const float2* __restrict__ Z, int V, int M, int J, float fth,
                                               int K0, float fk) {
    const float2 z00 = polar_tap(Z, V, M, J, K0);
    const float2 z01 = polar_tap(Z, V, M, J, K0 + 1);
    const float2 z10 = polar_tap(Z, V, M, J + 1, K0);
    const float2 z11 = polar_tap(Z, V, M, J + 1, K0 + 1);
    const float2 a = make_float2(fmaf(fk, z01.x - z00.x, z00.x), fmaf(fk, z01.y - z00.y, z00.y));
    const float2 b = make_float2(fmaf(fk, z11.x - z10.x, z10.x), fmaf(fk, z11.y - z10.y, z10.y));
    return make_float2(fmaf(fth, b.x - a.x, a.x), fmaf(fth, b.y - a.y, a.y));
}

// Signed radial bin and fraction of the point (kappa = +rho if plus, else -rho).
__device__ __forceinline__ void radial_bin(const Polar& P, bool plus, int& K0, float& fk) {
    if (plus) {
        K0 = P.k0;
        fk = P.frac;
    } else if (P.frac > 0.f) {
        K0 = -P.k0 - 1;
        fk = 1.f - P.frac;
    } else {
        K0 = -P.k0;
        fk = 0.f;
    }
}

}  // namespace bst
