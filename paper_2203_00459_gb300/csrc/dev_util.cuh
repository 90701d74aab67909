// Device helpers shared by the forward and adjoint kernels: warp/block reductions, the
// Hermitian half-plane magnitude lookup, and the error-free rotation coordinates of Rotate.
#pragma once
#include <cfloat>

#include "common.cuh"

namespace fmbym {

// ---------------------------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------------------------

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Sum (or max) over a block whose size is a multiple of 32; every thread gets the result.
template <bool MAX>
__device__ __forceinline__ float block_reduce(float v, float* red) {
    v = MAX ? warp_max(v) : warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        float r = lane < nw ? red[lane] : (MAX ? -FLT_MAX : 0.f);
        r = MAX ? warp_max(r) : warp_sum(r);
        if (lane == 0) red[0] = r;
    }
    __syncthreads();
    return red[0];
}

// |F| at integer frequency (vi, ui) of the N-periodic spectrum, read from the u-major half plane
// m[u][v] (u <= N/2) through |F(-v,-u)| = |F(v,u)|.
// Block-wide sums of K values at once (two barriers in all); red holds 32 K floats.  Every thread
// receives the sums in v.  Fixed order, so the result does not depend on timing.
template <int K>
__device__ __forceinline__ void block_sum_n(float (&v)[K], float* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) red[wid * K + k] = v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float t = 0.f;
        for (int w = 0; w < nw; ++w) t += red[w * K + k];
        v[k] = t;
    }
}

// The (f, g) magnitude pair at (vi, ui) of the N-periodic spectrum from the u-major half plane of
// interleaved pairs (the Hermitian mirror for ui > N/2).
__device__ __forceinline__ float2 mag2_at(const float2* __restrict__ m, int n, int vi, int ui) {
    if (n & 1) {   // odd N (the paper's 127, 255, 511): reduce by division; the half plane has u <= (N-1)/2
        vi = (vi % n + n) % n;
        ui = (ui % n + n) % n;
        if (ui > (n >> 1)) {
            vi = vi == 0 ? 0 : n - vi;
            ui = n - ui;
        }
        return __ldg(&m[ui * n + vi]);
    }
    vi &= n - 1;
    ui &= n - 1;
    if (ui > (n >> 1)) {
        vi = (n - vi) & (n - 1);
        ui = n - ui;
    }
    return __ldg(&m[ui * n + vi]);
}

__device__ __forceinline__ float mag_at(const float* __restrict__ m, int n, int vi, int ui) {
    vi &= n - 1;
    ui &= n - 1;
    if (ui > (n >> 1)) {
        vi = (n - vi) & (n - 1);
        ui = n - ui;
    }
    return __ldg(&m[ui * n + vi]);
}

// Bluestein's chirp convolution of one length-N sequence (element i at buf[spad(i) * es]) by
// thread j < M/16 of its group.  With w[n] = exp(i pi n^2 / N), n k = (n^2 + k^2 - (k - n)^2) / 2
// gives X[k] = sum_n x[n] exp(-2 pi i n k / N) = conj(w[k]) sum_n (x[n] conj(w[n])) w[k - n], a
// linear convolution that the M-point FFTs (M >= 2N - 1) evaluate as
// y = IFFT_M(FFT_M(a) * bh) with bh = FFT_M(b) / M of the circular filter b.  On return buf holds
// y; X[k] = conj(w[k]) y[k] for k < N is the caller's.  load(n) gives x[n] for n < N.  Every
// thread of the CTA must call it (it contains barriers).
template <int M, class Load>
__device__ __forceinline__ void bluestein(float2* buf, int es, int j, int n, const DevPlan& p, Load load) {
    constexpr int T = FftPlan<M>::T;
    first_pass_global<M>(buf, es, j, [&](int m) {
        return m < n ? c_cjmul(__ldg(&p.chirp[m]), load(m)) : make_float2(0.f, 0.f);
    });
    __syncthreads();
    fft_passes_from<M, -1, 2>(buf, es, j, p.tw_m);
    for (int k = j; k < M; k += T) buf[spad(k) * es] = c_mul(buf[spad(k) * es], __ldg(&p.bh[k]));
    __syncthreads();
    fft<M, +1>(buf, es, j, true, p.tw_m);
}

// Exact fixed-point sampling coordinates of the Rotate step: with C = cos(theta) 2^40 and
// S = sin(theta) 2^40 rounded to integers (from the double cosine and sine the splits carry), the
// sample of output pixel (X, Y) sits at p = c + R(-theta)((X, Y) - c), i.e.
//   px 2^40 = c 2^40 + C (X - c) + S (Y - c),   py 2^40 = c 2^40 - S (X - c) + C (Y - c),
// integers below 2^50 for N <= 512, so every pixel's coordinates are exact to 2^-40 px and cost
// one 64-bit multiply-add each.
struct RotFixed {
    long long C, S, px0, py0;   // px0, py0: the coordinates of (X, Y) = (0, 0)
};

__device__ __forceinline__ RotFixed rot_fixed(float ch, float cl, float sh, float sl, int n) {
    const double one = 1099511627776.0;   // 2^40
    RotFixed r;
    r.C = __double2ll_rn(((double)ch + (double)cl) * one);
    r.S = __double2ll_rn(((double)sh + (double)sl) * one);
    // centre c = n/2 (a half-integer for odd n): c 2^40 = n 2^39, and C c = (C n) / 2, exact for even n
    // and within 2^-41 px for odd n
    const long long c = (long long)n << 39, Cc = (r.C * n) >> 1, Sc = (r.S * n) >> 1;
    r.px0 = c - Cc - Sc;
    r.py0 = c + Sc - Cc;
    return r;
}

// Bilinear f at fixed-point (px, py), zero outside the scan (Alg. 1 Rotate).
__device__ __forceinline__ float rotated_sample_fixed(const float* __restrict__ src, int n, long long px,
                                                      long long py) {
    const int x0 = (int)(px >> 40), y0 = (int)(py >> 40);
    const float fx = (float)(int)((px >> 16) & 0xFFFFFF) * (1.f / 16777216.f);
    const float fy = (float)(int)((py >> 16) & 0xFFFFFF) * (1.f / 16777216.f);
    float v = 0.f;
    if ((unsigned)x0 < (unsigned)(n - 1) && (unsigned)y0 < (unsigned)(n - 1)) {
        // all four taps inside (the same sum, in the same order, without the bounds tests)
        const float* r = src + (size_t)y0 * n + x0;
        v += (1.f - fy) * (1.f - fx) * __ldg(r);
        v += (1.f - fy) * fx * __ldg(r + 1);
        v += fy * (1.f - fx) * __ldg(r + n);
        v += fy * fx * __ldg(r + n + 1);
        return v;
    }
    const bool xin0 = (unsigned)x0 < (unsigned)n, xin1 = (unsigned)(x0 + 1) < (unsigned)n;
    if ((unsigned)y0 < (unsigned)n) {
        const float* r = src + (size_t)y0 * n;
        if (xin0) v += (1.f - fy) * (1.f - fx) * __ldg(r + x0);
        if (xin1) v += (1.f - fy) * fx * __ldg(r + x0 + 1);
    }
    if ((unsigned)(y0 + 1) < (unsigned)n) {
        const float* r = src + (size_t)(y0 + 1) * n;
        if (xin0) v += fy * (1.f - fx) * __ldg(r + x0);
        if (xin1) v += fy * fx * __ldg(r + x0 + 1);
    }
    return v;
}

// Combines per-block (mean, M2, max, count) statistics of the translation scores into the mean,
// population std and maximum over all `total` scores (Chan's update).  With equal block counts
// (even N) the mean is the mean of the block means; the blocks of an odd N's frame hold different
// counts (the left-out lag), and the mean is weighted by them.  Run by one full warp; every lane
// returns the results.
__device__ __forceinline__ void xy_stats_warp(const float* __restrict__ s, int nblk, float total, float& mu,
                                              float& sd, float& cmax, bool weighted = false) {
    const int lane = threadIdx.x & 31;
    float lsum = 0.f, lmax = -FLT_MAX;
    for (int i = lane; i < nblk; i += 32) {
        lsum += weighted ? s[4 * i] * s[4 * i + 3] : s[4 * i];
        lmax = fmaxf(lmax, s[4 * i + 2]);
    }
    mu = weighted ? warp_sum(lsum) / total : warp_sum(lsum) / nblk;
    cmax = warp_max(lmax);
    float lm2 = 0.f;
    for (int i = lane; i < nblk; i += 32) {
        const float d = s[4 * i] - mu;
        lm2 += s[4 * i + 1] + s[4 * i + 3] * d * d;
    }
    sd = sqrtf(warp_sum(lm2) / total);
}

}  // namespace fmbym
