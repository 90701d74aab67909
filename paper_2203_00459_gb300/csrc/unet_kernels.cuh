// Kernels of the masking network h_alpha (Sec. III-D, Eq. 10-12, Tab. II): bf16 tensor-core
// convolutions with float32 accumulation, BatchNorm, ReLU, max-pool, bilinear x2, the sigmoid
// head with the mask multiply, their adjoints, and Adam.
//
// Tensors are NHWC.  Activations after BN + ReLU, max-pool and upsampling are bf16; convolution
// outputs before BN, and every gradient that is summed, are float32.  Convolutions are implicit
// GEMMs on mma.sync.m16n8k16 (bf16 in, f32 accumulate): M = 16 output pixels of one image row,
// N = 8 output channels, K = 16 input channels of one 3x3 tap.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace fmbym {
namespace unet {

typedef __nv_bfloat16 bf16;

constexpr int kTH = 8, kTW = 32;          // output tile of a conv CTA: 8 rows x 32 columns
constexpr int kTileH = kTH + 2, kTileW = kTW + 2;
constexpr float kEps = 1e-5f, kMomentum = 0.1f;

__device__ __forceinline__ void mma16816(float* c, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// ---------------------------------------------------------------------------------------------
// 3x3 convolution (zero padding 1): forward, or dgrad with the flipped transposed kernel
// ---------------------------------------------------------------------------------------------
//
// Input: the channel concatenation [in0 (c0 channels), in1 (c1 channels)] of two bf16 NHWC
// tensors, or (planes != 0) two float32 planes f, g as the 2 channels of the first layer.
// Weights: bf16 [COUT][9][cinp], cinp = channels rounded up to 16 (zero padded).
// Output: float32 NHWC split at channel `split`: channels [0, split) go to out0 (row stride
// split), [split, COUT) to out1 (row stride COUT - split); acc0/acc1 add instead of store.
// stats (forward only): per CTA and channel (mean, sum of squared deviations) of the outputs.
template <int COUT>
__global__ void __launch_bounds__(256) k_conv3x3(const bf16* __restrict__ in0, int c0, const bf16* __restrict__ in1,
                                                 int c1, const float* __restrict__ pf, const float* __restrict__ pg,
                                                 const bf16* __restrict__ wt, int cinp, float* __restrict__ out0,
                                                 float* __restrict__ out1, int split, int acc0, int acc1,
                                                 float2* __restrict__ stats, int H, int W) {
    constexpr int NT = COUT / 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ps = cinp + 8;                      // pixel stride of the input tile (bf16)
    bf16* tile = reinterpret_cast<bf16*>(smem_raw);
    bf16* ws = tile + kTileH * kTileW * ps;       // weights [COUT][9][ps]
    const int tx0 = blockIdx.x * kTW, ty0 = blockIdx.y * kTH, b = blockIdx.z;
    const int tid = threadIdx.x;
    // input tile with halo; channel groups of 8 (16 bytes)
    const int groups = cinp / 8;
    for (int idx = tid; idx < kTileH * kTileW * groups; idx += 256) {
        const int gq = idx % groups, pix = idx / groups, ty = pix / kTileW, tx = pix % kTileW;
        const int y = ty0 + ty - 1, x = tx0 + tx - 1;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (y >= 0 && y < H && x >= 0 && x < W) {
            const size_t pidx = ((size_t)b * H + y) * W + x;
            const int ch = gq * 8;
            if (pf) {
                if (gq == 0) {
                    const bf16 a = __float2bfloat16_rn(pf[pidx]), c = __float2bfloat16_rn(pg[pidx]);
                    v.x = pack2(a, c);
                }
            } else if (ch < c0) {
                v = *reinterpret_cast<const uint4*>(in0 + pidx * c0 + ch);
            } else if (ch < c0 + c1) {
                v = *reinterpret_cast<const uint4*>(in1 + pidx * c1 + (ch - c0));
            }
        }
        *reinterpret_cast<uint4*>(tile + pix * ps + gq * 8) = v;
    }
    for (int idx = tid; idx < COUT * 9 * groups; idx += 256) {
        const int gq = idx % groups, row = idx / groups;
        *reinterpret_cast<uint4*>(ws + row * ps + gq * 8) =
            *reinterpret_cast<const uint4*>(wt + (size_t)row * cinp + gq * 8);
    }
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    float acc[2][NT][4];
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int n = 0; n < NT; ++n)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[m][n][k] = 0.f;
    const uint32_t* tile32 = reinterpret_cast<const uint32_t*>(tile);
    const uint32_t* ws32 = reinterpret_cast<const uint32_t*>(ws);
    const int ps32 = ps / 2;
    for (int tap = 0; tap < 9; ++tap) {
        const int ky = tap / 3, kx = tap % 3;
        for (int kc = 0; kc < cinp; kc += 16) {
            uint32_t a[2][4];
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const int p0 = (warp + ky) * kTileW + m * 16 + g + kx;
                const int base0 = p0 * ps32 + (kc >> 1) + t, base1 = (p0 + 8) * ps32 + (kc >> 1) + t;
                a[m][0] = tile32[base0];
                a[m][1] = tile32[base1];
                a[m][2] = tile32[base0 + 4];
                a[m][3] = tile32[base1 + 4];
            }
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                const int wb = ((n * 8 + g) * 9 + tap) * ps32 + (kc >> 1) + t;
                uint32_t bb[2] = {ws32[wb], ws32[wb + 4]};
                mma16816(acc[0][n], a[0], bb);
                mma16816(acc[1][n], a[1], bb);
            }
        }
    }
    // store
    const int y = ty0 + warp;
#pragma unroll
    for (int m = 0; m < 2; ++m) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int x = tx0 + m * 16 + g + 8 * h;
            const size_t pidx = ((size_t)b * H + y) * W + x;
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                const int ch = n * 8 + 2 * t;
                const float v0 = acc[m][n][2 * h], v1 = acc[m][n][2 * h + 1];
                if (ch < split) {
                    float2* o = reinterpret_cast<float2*>(out0 + pidx * split + ch);
                    if (acc0) {
                        float2 old = *o;
                        *o = make_float2(old.x + v0, old.y + v1);
                    } else {
                        *o = make_float2(v0, v1);
                    }
                } else {
                    float2* o = reinterpret_cast<float2*>(out1 + pidx * (COUT - split) + (ch - split));
                    if (acc1) {
                        float2 old = *o;
                        *o = make_float2(old.x + v0, old.y + v1);
                    } else {
                        *o = make_float2(v0, v1);
                    }
                }
            }
        }
    }
    if (stats) {
        // per-channel mean and sum of squared deviations over the CTA's 256 outputs: lanes with the
        // same t hold the same channels; reduce over g, then over warps in a fixed order
        __shared__ float red[8][COUT];
        __shared__ float mean_s[COUT];
#pragma unroll
        for (int n = 0; n < NT; ++n) {
            float s0 = acc[0][n][0] + acc[0][n][2] + acc[1][n][0] + acc[1][n][2];
            float s1 = acc[0][n][1] + acc[0][n][3] + acc[1][n][1] + acc[1][n][3];
#pragma unroll
            for (int o = 4; o < 32; o <<= 1) {
                s0 += __shfl_xor_sync(0xffffffffu, s0, o);
                s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            }
            if (g == 0) {
                red[warp][n * 8 + 2 * t] = s0;
                red[warp][n * 8 + 2 * t + 1] = s1;
            }
        }
        __syncthreads();
        if (tid < COUT) {
            float s = 0.f;
            for (int w = 0; w < 8; ++w) s += red[w][tid];
            mean_s[tid] = s * (1.f / (kTH * kTW));
        }
        __syncthreads();
#pragma unroll
        for (int n = 0; n < NT; ++n) {
            const float mu0 = mean_s[n * 8 + 2 * t], mu1 = mean_s[n * 8 + 2 * t + 1];
            float q0 = 0.f, q1 = 0.f;
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                q0 += (acc[m][n][0] - mu0) * (acc[m][n][0] - mu0) + (acc[m][n][2] - mu0) * (acc[m][n][2] - mu0);
                q1 += (acc[m][n][1] - mu1) * (acc[m][n][1] - mu1) + (acc[m][n][3] - mu1) * (acc[m][n][3] - mu1);
            }
#pragma unroll
            for (int o = 4; o < 32; o <<= 1) {
                q0 += __shfl_xor_sync(0xffffffffu, q0, o);
                q1 += __shfl_xor_sync(0xffffffffu, q1, o);
            }
            __syncthreads();
            if (g == 0) {
                red[warp][n * 8 + 2 * t] = q0;
                red[warp][n * 8 + 2 * t + 1] = q1;
            }
        }
        __syncthreads();
        if (tid < COUT) {
            float s = 0.f;
            for (int w = 0; w < 8; ++w) s += red[w][tid];
            const int cta = (b * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
            stats[(size_t)cta * COUT + tid] = make_float2(mean_s[tid], s);
        }
    }
}

inline size_t conv_smem(int cout, int cinp) {
    return (size_t)(kTileH * kTileW + cout * 9) * (cinp + 8) * sizeof(bf16);
}

// ---------------------------------------------------------------------------------------------
// BatchNorm
// ---------------------------------------------------------------------------------------------

// Combines the per-CTA (mean, M2) partials of one channel (equal counts, fixed-order Chan
// updates), updates the running statistics (momentum 0.1, unbiased variance) and writes
// bn[c] = (mean, 1/sqrt(var + eps)) for the batch statistics.  One block per channel.
__global__ void __launch_bounds__(256) k_bn_finalize(const float2* __restrict__ stats, int ncta, int C,
                                                     float cnt_per_cta, float* __restrict__ run_mean,
                                                     float* __restrict__ run_var, float2* __restrict__ bn) {
    __shared__ double sn[256], sm[256], sq[256];
    const int c = blockIdx.x;
    double n = 0.0, mu = 0.0, m2 = 0.0;
    for (int i = threadIdx.x; i < ncta; i += 256) {
        const float2 s = stats[(size_t)i * C + c];
        const double nb = cnt_per_cta, d = (double)s.x - mu, tot = n + nb;
        mu += d * nb / tot;
        m2 += (double)s.y + d * d * n * nb / tot;
        n = tot;
    }
    sn[threadIdx.x] = n;
    sm[threadIdx.x] = mu;
    sq[threadIdx.x] = m2;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            const double na = sn[threadIdx.x], nb = sn[threadIdx.x + o], tot = na + nb;
            if (nb > 0) {
                const double d = sm[threadIdx.x + o] - sm[threadIdx.x];
                sm[threadIdx.x] += d * nb / tot;
                sq[threadIdx.x] += sq[threadIdx.x + o] + d * d * na * nb / tot;
                sn[threadIdx.x] = tot;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double N = sn[0], mean = sm[0], var = sq[0] / N;
        run_mean[c] = (float)((1.0 - kMomentum) * run_mean[c] + kMomentum * mean);
        run_var[c] = (float)((1.0 - kMomentum) * run_var[c] + kMomentum * var * N / (N > 1 ? N - 1 : 1));
        bn[c] = make_float2((float)mean, (float)(1.0 / sqrt(var + kEps)));
    }
}

// Evaluation: bn[c] = (running mean, 1/sqrt(running var + eps)).
__global__ void k_bn_eval(const float* __restrict__ run_mean, const float* __restrict__ run_var, int C,
                          float2* __restrict__ bn) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < C) bn[c] = make_float2(run_mean[c], 1.f / sqrtf(run_var[c] + kEps));
}

// a = bf16(relu((y - mean) invstd gamma + beta)), 8 channels per thread.
__global__ void k_bn_relu(const float* __restrict__ y, const float2* __restrict__ bn, const float* __restrict__ gamma,
                          const float* __restrict__ beta, bf16* __restrict__ a, long long n8, int C) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n8) return;
    const int c0 = (int)((i * 8) % C);
    const float4 v0 = reinterpret_cast<const float4*>(y)[2 * i], v1 = reinterpret_cast<const float4*>(y)[2 * i + 1];
    const float vin[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
    uint32_t o[4];
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
        float r[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = c0 + k + h;
            const float2 s = bn[c];
            r[h] = fmaxf(0.f, fmaf((vin[k + h] - s.x) * s.y, gamma[c], beta[c]));
        }
        o[k / 2] = pack2(__float2bfloat16_rn(r[0]), __float2bfloat16_rn(r[1]));
    }
    reinterpret_cast<uint4*>(a)[i] = make_uint4(o[0], o[1], o[2], o[3]);
}

// Adjoint of a = relu(xhat gamma + beta) with batch statistics, part 1: per-CTA partial sums over a
// slab of pixels of dpre = da [pre > 0] and dpre xhat per channel (fixed order).  C <= 64.
__global__ void __launch_bounds__(256) k_bn_bwd_reduce(const float* __restrict__ y, const float* __restrict__ da,
                                                       const float2* __restrict__ bn,
                                                       const float* __restrict__ gamma,
                                                       const float* __restrict__ beta, long long npix, int C,
                                                       int pix_per_cta, float2* __restrict__ part) {
    __shared__ float s1[256], s2[256];
    const int lanes = 256 / C * C;  // threads used: a multiple of C
    const int c = threadIdx.x % C, r = threadIdx.x / C, rows = 256 / C;
    float a1 = 0.f, a2 = 0.f;
    if ((int)threadIdx.x < lanes) {
        const float2 s = bn[c];
        const float gm = gamma[c], bt = beta[c];
        const long long p0 = (long long)blockIdx.x * pix_per_cta;
        for (long long p = p0 + r; p < p0 + pix_per_cta && p < npix; p += rows) {
            const float yv = y[p * C + c];
            const float xh = (yv - s.x) * s.y;
            const float pre = fmaf(xh, gm, bt);
            const float dp = pre > 0.f ? da[p * C + c] : 0.f;
            a1 += dp;
            a2 += dp * xh;
        }
    }
    s1[threadIdx.x] = a1;
    s2[threadIdx.x] = a2;
    __syncthreads();
    if ((int)threadIdx.x < C) {
        float t1 = 0.f, t2 = 0.f;
        for (int k = 0; k < rows; ++k) {
            t1 += s1[k * C + threadIdx.x];
            t2 += s2[k * C + threadIdx.x];
        }
        part[(size_t)blockIdx.x * C + threadIdx.x] = make_float2(t1, t2);
    }
}

// Part 2: sums the partials in order -> d beta = sum dpre, d gamma = sum dpre xhat (written to the
// gradient array) and the per-channel means used by the dy kernel: sums[c] = (mean dpre, mean dpre xhat).
__global__ void k_bn_bwd_finalize(const float2* __restrict__ part, int nparts, int C, float inv_n,
                                  float* __restrict__ dgamma, float* __restrict__ dbeta, float2* __restrict__ sums) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    double t1 = 0.0, t2 = 0.0;
    for (int i = 0; i < nparts; ++i) {
        const float2 v = part[(size_t)i * C + c];
        t1 += v.x;
        t2 += v.y;
    }
    dbeta[c] = (float)t1;
    dgamma[c] = (float)t2;
    sums[c] = make_float2((float)(t1 * inv_n), (float)(t2 * inv_n));
}

// Part 3: dy = gamma invstd (dpre - mean dpre - xhat mean(dpre xhat)), rounded to bf16 for the
// tensor-core dgrad and wgrad.
__global__ void k_bn_bwd_dy(const float* __restrict__ y, const float* __restrict__ da, const float2* __restrict__ bn,
                            const float* __restrict__ gamma, const float* __restrict__ beta,
                            const float2* __restrict__ sums, bf16* __restrict__ dy, long long n, int C) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = (int)(i % C);
    const float2 s = bn[c];
    const float xh = (y[i] - s.x) * s.y;
    const float pre = fmaf(xh, gamma[c], beta[c]);
    const float dp = pre > 0.f ? da[i] : 0.f;
    const float2 m = sums[c];
    dy[i] = __float2bfloat16_rn(gamma[c] * s.y * (dp - m.x - xh * m.y));
}

// ---------------------------------------------------------------------------------------------
// max-pool 2x2 and bilinear x2 (align_corners = False) with their adjoints
// ---------------------------------------------------------------------------------------------

__global__ void k_maxpool(const bf16* __restrict__ a, bf16* __restrict__ p, int B, int H, int W, int C) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int Ho = H / 2, Wo = W / 2;
    if (i >= (long long)B * Ho * Wo * C) return;
    const int c = (int)(i % C);
    long long r = i / C;
    const int x = (int)(r % Wo);
    r /= Wo;
    const int y = (int)(r % Ho);
    const int b = (int)(r / Ho);
    const bf16* base = a + (((size_t)b * H + 2 * y) * W + 2 * x) * C + c;
    float m = __bfloat162float(base[0]);
    m = fmaxf(m, __bfloat162float(base[C]));
    m = fmaxf(m, __bfloat162float(base[(size_t)W * C]));
    m = fmaxf(m, __bfloat162float(base[(size_t)W * C + C]));
    p[i] = __float2bfloat16_rn(m);
}

// Routes d p to the first maximum of its window in row-major order (strict >), added to da.
__global__ void k_maxpool_bwd(const bf16* __restrict__ a, const float* __restrict__ dp, float* __restrict__ da,
                              int B, int H, int W, int C) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int Ho = H / 2, Wo = W / 2;
    if (i >= (long long)B * Ho * Wo * C) return;
    const int c = (int)(i % C);
    long long r = i / C;
    const int x = (int)(r % Wo);
    r /= Wo;
    const int y = (int)(r % Ho);
    const int b = (int)(r / Ho);
    const size_t off[4] = {0, (size_t)C, (size_t)W * C, (size_t)W * C + C};
    const size_t base = (((size_t)b * H + 2 * y) * W + 2 * x) * C + c;
    int best = 0;
    float m = __bfloat162float(a[base]);
#pragma unroll
    for (int k = 1; k < 4; ++k) {
        const float v = __bfloat162float(a[base + off[k]]);
        if (v > m) {
            m = v;
            best = k;
        }
    }
    da[base + off[best]] += dp[i];
}

// Source row/column of the bilinear x2 upsampling with align_corners = False: output index o
// reads input i0 with weight l0 and i1 with weight l1 (the input index is clamped at 0 and at
// the last row, as the library routine does).
__device__ __forceinline__ void up_src(int o, int n, int& i0, int& i1, float& l0, float& l1) {
    float s = 0.5f * (o + 0.5f) - 0.5f;
    if (s < 0.f) s = 0.f;
    i0 = (int)s;
    i1 = i0 < n - 1 ? i0 + 1 : i0;
    l1 = s - (float)i0;
    l0 = 1.f - l1;
}

__global__ void k_upsample(const bf16* __restrict__ a, bf16* __restrict__ u, int B, int h, int w, int C) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int H = 2 * h, W = 2 * w;
    if (i >= (long long)B * H * W * C) return;
    const int c = (int)(i % C);
    long long r = i / C;
    const int X = (int)(r % W);
    r /= W;
    const int Y = (int)(r % H);
    const int b = (int)(r / H);
    int y0, y1, x0, x1;
    float ly0, ly1, lx0, lx1;
    up_src(Y, h, y0, y1, ly0, ly1);
    up_src(X, w, x0, x1, lx0, lx1);
    const bf16* base = a + (size_t)b * h * w * C + c;
    auto at = [&](int yy, int xx) { return __bfloat162float(base[((size_t)yy * w + xx) * C]); };
    const float v = ly0 * (lx0 * at(y0, x0) + lx1 * at(y0, x1)) + ly1 * (lx0 * at(y1, x0) + lx1 * at(y1, x1));
    u[i] = __float2bfloat16_rn(v);
}

// Weight that the forward assigns from input index k to output index o (both taps if clamped).
__device__ __forceinline__ float up_w(int o, int k, int n) {
    int i0, i1;
    float l0, l1;
    up_src(o, n, i0, i1, l0, l1);
    return (i0 == k ? l0 : 0.f) + (i1 == k ? l1 : 0.f);
}

// Transpose of the upsampling in gather form: d a[k] = sum over outputs o in [2k-2, 2k+2] of the
// forward weights times d u[o]; written (not added) to da.
__global__ void k_upsample_bwd(const float* __restrict__ du, float* __restrict__ da, int B, int h, int w, int C) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int H = 2 * h, W = 2 * w;
    if (i >= (long long)B * h * w * C) return;
    const int c = (int)(i % C);
    long long r = i / C;
    const int x = (int)(r % w);
    r /= w;
    const int y = (int)(r % h);
    const int b = (int)(r / h);
    float s = 0.f;
    for (int Y = max(0, 2 * y - 2); Y <= min(H - 1, 2 * y + 2); ++Y) {
        const float wy = up_w(Y, y, h);
        if (wy == 0.f) continue;
        for (int X = max(0, 2 * x - 2); X <= min(W - 1, 2 * x + 2); ++X) {
            const float wx = up_w(X, x, w);
            if (wx == 0.f) continue;
            s += wy * wx * du[(((size_t)b * H + Y) * W + X) * C + c];
        }
    }
    da[i] = s;
}

// ---------------------------------------------------------------------------------------------
// head: 1x1 convolution C -> 2 with bias, sigmoid, mask multiply (Eq. 10-11), and its adjoint
// ---------------------------------------------------------------------------------------------

template <int C>
__global__ void k_head(const bf16* __restrict__ a, const float* __restrict__ hw, const float* __restrict__ hb,
                       const float* __restrict__ f, const float* __restrict__ g, float* __restrict__ fo,
                       float* __restrict__ go, float* __restrict__ masks, long long npix, int HW) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npix) return;
    float z0 = hb[0], z1 = hb[1];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const float v = __bfloat162float(a[i * C + c]);
        z0 = fmaf(__bfloat162float(__float2bfloat16_rn(hw[c])), v, z0);
        z1 = fmaf(__bfloat162float(__float2bfloat16_rn(hw[C + c])), v, z1);
    }
    const float m0 = 1.f / (1.f + expf(-z0)), m1 = 1.f / (1.f + expf(-z1));
    if (fo) fo[i] = f[i] * m0;
    if (go) go[i] = g[i] * m1;
    if (masks) {
        const long long b = i / HW, p = i % HW;
        masks[(b * 2) * HW + p] = m0;
        masks[(b * 2 + 1) * HW + p] = m1;
    }
}

// d z_o = d(out_o) scan_o m_o (1 - m_o); d a[c] = sum_o W[o][c] d z_o; per-block partial sums of
// d W[o][c] = sum d z_o a[c] and d b[o] = sum d z_o (2 C + 2 values, fixed order).
template <int C>
__global__ void __launch_bounds__(256) k_head_bwd(const bf16* __restrict__ a, const float* __restrict__ hw,
                                                  const float* __restrict__ hb, const float* __restrict__ f,
                                                  const float* __restrict__ g, const float* __restrict__ dfo,
                                                  const float* __restrict__ dgo, float* __restrict__ da,
                                                  float* __restrict__ part, long long npix) {
    __shared__ float red[8][2 * C + 2];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float loc[2 * C + 2];
#pragma unroll
    for (int k = 0; k < 2 * C + 2; ++k) loc[k] = 0.f;
    if (i < npix) {
        float av[C], w0[C], w1[C];
        float z0 = hb[0], z1 = hb[1];
#pragma unroll
        for (int c = 0; c < C; ++c) {
            av[c] = __bfloat162float(a[i * C + c]);
            w0[c] = __bfloat162float(__float2bfloat16_rn(hw[c]));
            w1[c] = __bfloat162float(__float2bfloat16_rn(hw[C + c]));
            z0 = fmaf(w0[c], av[c], z0);
            z1 = fmaf(w1[c], av[c], z1);
        }
        const float m0 = 1.f / (1.f + expf(-z0)), m1 = 1.f / (1.f + expf(-z1));
        const float d0 = dfo[i] * f[i] * m0 * (1.f - m0), d1 = dgo[i] * g[i] * m1 * (1.f - m1);
#pragma unroll
        for (int c = 0; c < C; ++c) {
            da[i * C + c] = w0[c] * d0 + w1[c] * d1;
            loc[c] = d0 * av[c];
            loc[C + c] = d1 * av[c];
        }
        loc[2 * C] = d0;
        loc[2 * C + 1] = d1;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 2 * C + 2; ++k) {
        float v = loc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 2 * C + 2) {
        float s = 0.f;
        for (int w = 0; w < 8; ++w) s += red[w][threadIdx.x];
        part[(size_t)blockIdx.x * (2 * C + 2) + threadIdx.x] = s;
    }
}

// Sums per-block partials column by column in a fixed order into out (added to out if acc).
__global__ void k_sum_parts(const float* __restrict__ part, int nparts, int width, float* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= width) return;
    double s = 0.0;
    for (int i = 0; i < nparts; ++i) s += part[(size_t)i * width + k];
    out[k] = (float)s;
}

// ---------------------------------------------------------------------------------------------
// weight gradient of a 3x3 convolution
// ---------------------------------------------------------------------------------------------
//
// dW[co][tap][ci] = sum over pixels of dy[p][co] in[p + tap][ci], an implicit GEMM with M = 16
// output channels, N = 8 input channels, K = 16 pixels of a tile row.  A CTA owns one block of 16
// output channels and up to 64 input channels (one block of 8 per warp, all 9 taps in registers)
// and walks a chunk of 8 x 32 pixel tiles; its partial dW goes to part[chunk] and k_wgrad_reduce
// sums the chunks in order.  Tiles are stored channel-major in shared memory.
__global__ void __launch_bounds__(256) k_wgrad(const bf16* __restrict__ dy, int cout, const bf16* __restrict__ in0,
                                               int c0, const bf16* __restrict__ in1, int c1,
                                               const float* __restrict__ pf, const float* __restrict__ pg, int B,
                                               int H, int W, int tiles_per_chunk, float* __restrict__ part) {
    constexpr int DS = kTH * kTW + 8;          // channel stride of the dy tile
    constexpr int IS = kTileH * kTileW + 4;    // channel stride of the input tile
    extern __shared__ __align__(16) unsigned char smem_w[];
    bf16* dys = reinterpret_cast<bf16*>(smem_w);
    bf16* ins = dys + 16 * DS;
    const int cin = pf ? 2 : c0 + c1;
    const int co0 = blockIdx.y * 16, ci_base = blockIdx.z * 64;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    const int ci0 = ci_base + warp * 8;
    float acc[9][4];
#pragma unroll
    for (int k = 0; k < 9; ++k)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[k][j] = 0.f;
    const int tiles_x = W / kTW, tiles_y = H / kTH, ntiles = B * tiles_x * tiles_y;
    const uint16_t* dys16 = reinterpret_cast<const uint16_t*>(dys);
    const uint16_t* ins16 = reinterpret_cast<const uint16_t*>(ins);
    for (int tt = 0; tt < tiles_per_chunk; ++tt) {
        const int tile = blockIdx.x * tiles_per_chunk + tt;
        if (tile >= ntiles) break;
        const int b = tile / (tiles_x * tiles_y), rem = tile % (tiles_x * tiles_y);
        const int ty0 = (rem / tiles_x) * kTH, tx0 = (rem % tiles_x) * kTW;
        __syncthreads();
        for (int idx = tid; idx < 16 * kTH * kTW; idx += 256) {
            const int co = idx % 16, pix = idx / 16, y = ty0 + pix / kTW, x = tx0 + pix % kTW;
            bf16 v = __float2bfloat16_rn(0.f);
            if (co0 + co < cout) v = dy[(((size_t)b * H + y) * W + x) * cout + co0 + co];
            dys[co * DS + pix] = v;
        }
        for (int idx = tid; idx < 64 * kTileH * kTileW; idx += 256) {
            const int ci = idx % 64, pix = idx / 64, y = ty0 + pix / kTileW - 1, x = tx0 + pix % kTileW - 1;
            const int c = ci_base + ci;
            bf16 v = __float2bfloat16_rn(0.f);
            if (c < cin && y >= 0 && y < H && x >= 0 && x < W) {
                const size_t p = ((size_t)b * H + y) * W + x;
                if (pf) v = __float2bfloat16_rn(c == 0 ? pf[p] : pg[p]);
                else if (c < c0) v = in0[p * c0 + c];
                else v = in1[p * c1 + (c - c0)];
            }
            ins[ci * IS + pix] = v;
        }
        __syncthreads();
        if (ci0 < cin) {
            for (int row = 0; row < kTH; ++row) {
                for (int xs = 0; xs < kTW; xs += 16) {
                    const int p0 = row * kTW + xs;
                    uint32_t a[4];
                    const uint32_t* d32 = reinterpret_cast<const uint32_t*>(dys16 + g * DS + p0);
                    const uint32_t* d32b = reinterpret_cast<const uint32_t*>(dys16 + (g + 8) * DS + p0);
                    a[0] = d32[t];
                    a[1] = d32b[t];
                    a[2] = d32[t + 4];
                    a[3] = d32b[t + 4];
#pragma unroll
                    for (int tap = 0; tap < 9; ++tap) {
                        const int ky = tap / 3, kx = tap % 3;
                        const uint16_t* ib = ins16 + (warp * 8 + g) * IS + (row + ky) * kTileW + xs + kx;
                        uint32_t bb[2];
                        bb[0] = (uint32_t)ib[2 * t] | ((uint32_t)ib[2 * t + 1] << 16);
                        bb[1] = (uint32_t)ib[2 * t + 8] | ((uint32_t)ib[2 * t + 9] << 16);
                        mma16816(acc[tap], a, bb);
                    }
                }
            }
        }
    }
    // acc[tap]: rows co0 + g (+8), columns ci0 + 2t (+1)
    if (ci0 < cin) {
        float* o = part + (size_t)blockIdx.x * cout * 9 * cin;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int co = co0 + g + 8 * h;
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int ci = ci0 + 2 * t + j;
                    if (co < cout && ci < cin) o[((size_t)co * 9 + tap) * cin + ci] = acc[tap][2 * h + j];
                }
            }
        }
    }
}

constexpr size_t kWgradSmem = (size_t)(16 * (kTH * kTW + 8) + 64 * (kTileH * kTileW + 4)) * sizeof(bf16);

// dW (PyTorch layout [co][ci][3][3]) = sum over chunks of part[chunk][co][tap][ci], fixed order.
__global__ void k_wgrad_reduce(const float* __restrict__ part, int nchunks, int cout, int cin,
                               float* __restrict__ dw) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int total = cout * 9 * cin;
    if (k >= total) return;
    const int ci = k % cin, tap = (k / cin) % 9, co = k / (9 * cin);
    float s = 0.f;
    for (int i = 0; i < nchunks; ++i) s += part[(size_t)i * total + k];
    dw[((size_t)co * cin + ci) * 9 + tap] = s;
}

// ---------------------------------------------------------------------------------------------
// weights and optimiser
// ---------------------------------------------------------------------------------------------

// From the float32 master weight [co][ci][3][3]: the forward layout bf16 [co][tap][cinp] and the
// dgrad layout bf16 [ci][8 - tap][coutp] (flipped taps, transposed channels), zero padded.
__global__ void k_prep_weights(const float* __restrict__ w, int cout, int cin, int cinp, int coutp,
                               bf16* __restrict__ wf, bf16* __restrict__ wd) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int nf = cout * 9 * cinp, nd = cin * 9 * coutp;
    if (k < nf) {
        const int ci = k % cinp, tap = (k / cinp) % 9, co = k / (9 * cinp);
        wf[k] = __float2bfloat16_rn(ci < cin ? w[((size_t)co * cin + ci) * 9 + tap] : 0.f);
    }
    if (wd && k < nd) {
        const int co = k % coutp, tp = (k / coutp) % 9, ci = k / (9 * coutp);
        wd[k] = __float2bfloat16_rn(co < cout ? w[((size_t)co * cin + ci) * 9 + (8 - tp)] : 0.f);
    }
}

// Adam (Kingma & Ba) on the float32 master parameters.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ gr, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = gr[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace unet
}  // namespace fmbym
