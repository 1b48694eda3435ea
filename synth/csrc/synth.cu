// synth.cu -- device-side generator of large synthetic sinogram workloads.
//
// Input generation only (it holds none of the backprojection method): the
// closed-form parallel-beam projection of a sum of ellipses (the paper's
// analytic ellipsoid workload, Sec. 4 footnote, after Kak & Slaney), plus
// additive Gaussian noise with sigma = frac * max|y| of each slice, drawn
// with the counter-based Philox4x32-10 generator (Salmon, Moraes, Dror and
// Shaw, SC 2011) and the Box-Muller transform.  Used where a workload is too
// large to generate on the host (2048 slices x 2048 x 2048 is 32 GiB).
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

__global__ void k_ellipse_rows(const float* __restrict__ ell, const int* __restrict__ cnt, int kmax,
                               const float* __restrict__ theta, int V, int N, float* __restrict__ y) {
    extern __shared__ float sh[];  // per ellipse: a_th^2, c . xi, 2 rho a b
    const int j = blockIdx.x, s = blockIdx.y;
    const int K = cnt[s];
    const float th = theta[j];
    float c, sn;
    sincosf(th, &sn, &c);
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const float* e = ell + ((size_t)s * kmax + k) * 6;
        float cp, sp;
        sincosf(th - e[4], &sp, &cp);
        sh[3 * k + 0] = e[2] * e[2] * cp * cp + e[3] * e[3] * sp * sp;
        sh[3 * k + 1] = e[0] * c + e[1] * sn;
        sh[3 * k + 2] = 2.f * e[5] * e[2] * e[3];
    }
    __syncthreads();
    const float dt = 2.f / (float)N;
    float* row = y + ((size_t)s * V + j) * N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const float t = (float)(i - N / 2) * dt;
        float acc = 0.f;
        for (int k = 0; k < K; ++k) {
            const float a2 = sh[3 * k], d = t - sh[3 * k + 1];
            const float r = a2 - d * d;
            if (r > 0.f) acc += sh[3 * k + 2] * sqrtf(r) / a2;
        }
        row[i] = acc;
    }
}

__global__ void k_slice_absmax(const float* __restrict__ y, size_t per_slice, float* __restrict__ out) {
    const float* p = y + (size_t)blockIdx.x * per_slice;
    float m = 0.f;
    for (size_t i = threadIdx.x; i < per_slice; i += blockDim.x) m = fmaxf(m, fabsf(p[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float w[32];
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? w[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) out[blockIdx.x] = m;
    }
}

// Philox4x32-10: ten rounds of the multiply-xor bijection with a Weyl key schedule
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// counter of element pair e: e + pair0, pair0 = the pairs of the slices before
// this block, so that a block of slices gets the same noise as those slices of
// the whole volume
__global__ void k_add_noise(float* __restrict__ y, int V, int N, int S, const float* __restrict__ smax, float frac,
                            unsigned long long seed, unsigned long long pair0) {
    const size_t per_slice = (size_t)V * N;
    const size_t total = per_slice * S;
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; 2 * e < total; e += (size_t)gridDim.x * blockDim.x) {
        const unsigned long long c = e + pair0;
        const uint4 r = philox4x32_10(make_uint4((uint32_t)c, (uint32_t)(c >> 32), 0x5eedu, 0u), key);
        const float u1 = ((float)(r.x >> 8) + 1.f) * (1.f / 16777216.f);
        const float u2 = (float)(r.y >> 8) * (1.f / 16777216.f);
        const float rad = sqrtf(-2.f * logf(u1));
        float sn, cs;
        sincospif(2.f * u2, &sn, &cs);
        for (int h = 0; h < 2; ++h) {
            const size_t idx = 2 * e + h;
            if (idx < total) {
                const float sigma = frac * smax[idx / per_slice];
                y[idx] += sigma * rad * (h ? sn : cs);
            }
        }
    }
}

}  // namespace

extern "C" {

// y[S][V][N] = closed-form projections of the per-slice ellipses
// ell[S][kmax][6] = (cx, cy, a, b, psi, rho), cnt[S] ellipses each, at angles theta[V].
int synth_ellipse_sinogram(const float* ell, const int* cnt, int kmax, const float* theta, int S, int V, int N,
                           float* y, void* stream) {
    if (!ell || !cnt || !theta || !y || S <= 0 || V <= 0 || N <= 0 || kmax <= 0) return 1;
    k_ellipse_rows<<<dim3(V, S), 256, 3 * kmax * sizeof(float), (cudaStream_t)stream>>>(ell, cnt, kmax, theta, V, N,
                                                                                          y);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

// y += N(0, (frac * max|y_s|)^2) per slice s; smax_scratch: S floats of device memory.
// first_slice: index of y's first slice in the whole volume (first_slice * V * N even).
int synth_add_gaussian_noise(float* y, int S, int V, int N, float frac, unsigned long long seed, long long first_slice,
                             float* smax_scratch, void* stream) {
    if (!y || !smax_scratch || S <= 0 || V <= 0 || N <= 0 || first_slice < 0) return 1;
    const unsigned long long before = (unsigned long long)first_slice * V * N;
    if (before & 1) return 1;
    cudaStream_t st = (cudaStream_t)stream;
    k_slice_absmax<<<S, 1024, 0, st>>>(y, (size_t)V * N, smax_scratch);
    k_add_noise<<<152 * 16, 256, 0, st>>>(y, V, N, S, smax_scratch, frac, seed, before / 2);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

}  // extern "C"
