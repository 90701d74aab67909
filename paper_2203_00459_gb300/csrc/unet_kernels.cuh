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

constexpr int kTilePx = kTH * kTW, kHaloPx = kTileH * kTileW;   // pixels of a tile, and with its halo

// 16-byte global -> shared copies (zero-filled when !valid), and their group waits
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gsrc), "r"(valid ? 16 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_n(int n) {   // wait until at most n groups are pending
    if (n >= 2) asm volatile("cp.async.wait_group 2;\n" ::: "memory");
    else if (n == 1) asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    else asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// ldmatrix: eight 16-byte rows per 8x8 matrix, row addresses from lanes 8 i .. 8 i + 7 for matrix i
__device__ __forceinline__ void ldsm_x4(uint32_t* r, const void* row_addr) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(row_addr);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(s));
}
__device__ __forceinline__ void ldsm_x2(uint32_t* r, const void* row_addr) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(row_addr);
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r[0]), "=r"(r[1]) : "r"(s));
}
__device__ __forceinline__ void ldsm_x4_trans(uint32_t* r, const void* row_addr) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(row_addr);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(s));
}

// ---------------------------------------------------------------------------------------------
// 3x3 convolution (zero padding 1): forward, or dgrad with the flipped transposed kernel
// ---------------------------------------------------------------------------------------------
//
// Input: the channel concatenation [in0 (c0 channels), in1 (c1 channels)] of two bf16 NHWC
// tensors, or (pf != NULL) two float32 planes f, g as the 2 channels of the first layer; G groups
// of 8 channels (zero padded).  Weights: bf16 [COUT][9 G][8], i.e. [COUT][tap][8 G], taps
// row-major.  Output: float32 NHWC split at channel `split`: channels [0, split) go to out0 (row
// stride split), [split, COUT) to out1 (row stride COUT - split); acc0/acc1 add instead of store.
// stats (forward only): per CTA and channel (mean, sum of squared deviations) of its outputs: each
// tile's pair is taken over its 256 R pixels and merged into the CTA's running pair by Chan's
// update, in tile order.
//
// An implicit GEMM on mma.sync.m16n8k16: M = 16 output pixels of a tile row, N = 8 output
// channels, and each K = 16 step takes two (tap, channel group) items, so 8-channel layers waste
// no K.  The CTA is persistent over tiles: the whole weight array sits in shared memory, the
// input tiles (with halo) arrive by cp.async in the NHWC byte order -- one 16-byte row per pixel
// and channel group -- through a ring of `nstage` buffers, and ldmatrix reads the A fragments at
// shifted row addresses (the tap) and the B fragments from the weight rows.  A CTA tile is 8 R rows
// x 32 columns (each warp R rows), R = 4 for narrow layers so that the per-tile work outweighs the
// per-tile bookkeeping.
__host__ __device__ constexpr int conv_items_padded(int G) { return (9 * G + 1) / 2 * 2; }
__host__ __device__ inline size_t conv_weight_bytes(int cout, int G) {
    return (size_t)cout * (conv_items_padded(G) + 1) * 16;
}
// input tile with halo of a CTA tile of 8 R rows x 32 columns
__host__ __device__ inline size_t conv_tile_bytes(int G, int R) { return (size_t)G * (8 * R + 2) * kTileW * 16; }
constexpr int kConvMaxItems = 9 * 16 + 1;

template <int COUT, int R>
__global__ void __launch_bounds__(256) k_conv3x3(const bf16* __restrict__ in0, int c0, const bf16* __restrict__ in1,
                                                 int c1, const float* __restrict__ pf, const float* __restrict__ pg,
                                                 const bf16* __restrict__ wt, int G, int nstage,
                                                 float* __restrict__ out0, float* __restrict__ out1, int split,
                                                 int acc0, int acc1, float2* __restrict__ stats, int B, int H,
                                                 int W) {
    constexpr int NT = COUT / 8, TH = 8 * R, HALO = (TH + 2) * kTileW;
    extern __shared__ __align__(128) unsigned char smem_c[];
    __shared__ int item_off[kConvMaxItems];       // per item: group * halo + ky * row + kx (pixels)
    __shared__ float2 wstat[8][COUT];            // per warp (R tile rows): (mean, M2) of each channel
    const int NI = 9 * G, NIp = conv_items_padded(G), WS = NIp + 1;   // weight row stride (odd: no conflicts)
    unsigned char* ws = smem_c;
    unsigned char* ring = smem_c + (size_t)COUT * WS * 16;
    const size_t TB = conv_tile_bytes(G, R);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    for (int i = tid; i < COUT * NIp; i += 256) {
        const int co = i / NIp, it = i % NIp;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (it < NI) v = *reinterpret_cast<const uint4*>(wt + ((size_t)co * NI + it) * 8);
        *reinterpret_cast<uint4*>(ws + ((size_t)co * WS + it) * 16) = v;
    }
    for (int i = tid; i < NIp; i += 256) {
        const int it = min(i, NI - 1), tap = it / G, grp = it % G;   // the odd pad item repeats a real one
        item_off[i] = grp * HALO + (tap / 3) * kTileW + tap % 3;      // (its weights are zero)
    }
    const int tiles_x = W / kTW, tiles_y = H / TH, tiles_img = tiles_x * tiles_y, ntiles = B * tiles_img;
    const int n = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    auto stage = [&](int k) {   // the k-th tile of this CTA into ring slot k % nstage
        unsigned char* buf = ring + (size_t)(k % nstage) * TB;
        const int tile = blockIdx.x + k * gridDim.x;
        const int b = tile / tiles_img, rem = tile - b * tiles_img;
        const int ty = rem / tiles_x;
        const int ty0 = ty * TH, tx0 = (rem - ty * tiles_x) * kTW;
        for (int pix = tid; pix < HALO; pix += 256) {
            const int hy = pix / kTileW;
            const int y = ty0 + hy - 1, x = tx0 + (pix - hy * kTileW) - 1;
            const bool inside = y >= 0 && y < H && x >= 0 && x < W;
            const size_t p = inside ? ((size_t)b * H + y) * W + x : 0;
            if (pf) {
                uint4 v = make_uint4(0, 0, 0, 0);
                if (inside) v.x = pack2(__float2bfloat16_rn(pf[p]), __float2bfloat16_rn(pg[p]));
                *reinterpret_cast<uint4*>(buf + (size_t)pix * 16) = v;
            } else {
                const bf16* s0 = in0 + p * c0;
                const bf16* s1 = in1 + p * c1 - c0;
                for (int grp = 0; grp < G; ++grp) {
                    const int ch = grp * 8;
                    cp_async16(buf + (size_t)(grp * HALO + pix) * 16, ch < c0 ? s0 + ch : s1 + ch, inside);
                }
            }
        }
    };

    // per-lane ldmatrix rows: A matrices (pixels 0-7 | 8-15) x (item 2s | 2s+1); B matrices
    // (channel block n | n+1) x (item 2s | 2s+1), eight output channels each
    const int mi = lane >> 3, r8 = lane & 7;
    const int a_px = warp * R * kTileW + (mi & 1) * 8 + r8, a_item = mi >> 1;
    const int b_row = (mi >> 1) * 8 + r8, b_item = mi & 1;
    float run_mean = 0.f, run_m2 = 0.f;   // the CTA's statistics so far (threads tid < COUT)
    for (int k = 0; k < nstage - 1; ++k) {
        if (k < n) stage(k);
        cp_async_commit();
    }
    for (int it = 0; it < n; ++it) {
        if (it + nstage - 1 < n) stage(it + nstage - 1);
        cp_async_commit();
        cp_async_wait_n(nstage - 1);
        __syncthreads();
        const unsigned char* tb = ring + (size_t)(it % nstage) * TB;
        float acc[R][2][NT][4];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int m = 0; m < 2; ++m)
#pragma unroll
                for (int q = 0; q < NT; ++q)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[r][m][q][j] = 0.f;
        for (int s = 0; s < NIp / 2; ++s) {
            const unsigned char* ab = tb + (size_t)(item_off[2 * s + a_item] + a_px) * 16;
            uint32_t a[R][2][4];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                ldsm_x4(a[r][0], ab + (size_t)r * kTileW * 16);
                ldsm_x4(a[r][1], ab + (size_t)(r * kTileW + 16) * 16);
            }
#pragma unroll
            for (int q = 0; q < NT; q += 2) {
                if (q + 1 < NT) {
                    uint32_t bq[4];
                    ldsm_x4(bq, ws + ((size_t)(q * 8 + b_row) * WS + 2 * s + b_item) * 16);
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        mma16816(acc[r][0][q], a[r][0], bq);
                        mma16816(acc[r][1][q], a[r][1], bq);
                        mma16816(acc[r][0][q + 1], a[r][0], bq + 2);
                        mma16816(acc[r][1][q + 1], a[r][1], bq + 2);
                    }
                } else {
                    uint32_t bq[2];
                    ldsm_x2(bq, ws + ((size_t)(q * 8 + r8) * WS + 2 * s + b_item) * 16);
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        mma16816(acc[r][0][q], a[r][0], bq);
                        mma16816(acc[r][1][q], a[r][1], bq);
                    }
                }
            }
        }
        // epilogue: rows g (+8) of the m-block are pixels, columns 2t (+1) channels
        const int tile = blockIdx.x + it * gridDim.x;
        const int b = tile / tiles_img, rem = tile - b * tiles_img;
        const int ty = rem / tiles_x;
        const int y0 = ty * TH + warp * R, tx0 = (rem - ty * tiles_x) * kTW;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const size_t prow = ((size_t)b * H + y0 + r) * W + tx0;
#pragma unroll
            for (int m = 0; m < 2; ++m) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const size_t pidx = prow + m * 16 + g + 8 * h;
#pragma unroll
                    for (int q = 0; q < NT; ++q) {
                        const int ch = q * 8 + 2 * t;
                        const float v0 = acc[r][m][q][2 * h], v1 = acc[r][m][q][2 * h + 1];
                        if (ch < split) {
                            float2* o = reinterpret_cast<float2*>(out0 + pidx * split + ch);
                            if (acc0) {
                                const float2 old = *o;
                                *o = make_float2(old.x + v0, old.y + v1);
                            } else {
                                *o = make_float2(v0, v1);
                            }
                        } else {
                            float2* o = reinterpret_cast<float2*>(out1 + pidx * (COUT - split) + (ch - split));
                            if (acc1) {
                                const float2 old = *o;
                                *o = make_float2(old.x + v0, old.y + v1);
                            } else {
                                *o = make_float2(v0, v1);
                            }
                        }
                    }
                }
            }
        }
        if (stats) {
            // per channel: each warp's 32 R outputs (its tile rows) give a (mean, M2) pair by
            // shuffles over g; the 8 warps' pairs (equal counts) give the tile's, which is merged
            // into the CTA's running pair by Chan's update
            constexpr float kWarpPx = 32.f * R;
#pragma unroll
            for (int q = 0; q < NT; ++q) {
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    float sm = 0.f;
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        sm += acc[r][0][q][j] + acc[r][0][q][j + 2] + acc[r][1][q][j] + acc[r][1][q][j + 2];
#pragma unroll
                    for (int o = 4; o < 32; o <<= 1) sm += __shfl_xor_sync(0xffffffffu, sm, o);
                    const float mu = sm * (1.f / kWarpPx);
                    float m2 = 0.f;
#pragma unroll
                    for (int r = 0; r < R; ++r)
#pragma unroll
                        for (int m = 0; m < 2; ++m)
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const float d = acc[r][m][q][2 * h + j] - mu;
                                m2 = fmaf(d, d, m2);
                            }
#pragma unroll
                    for (int o = 4; o < 32; o <<= 1) m2 += __shfl_xor_sync(0xffffffffu, m2, o);
                    if (g == 0) wstat[warp][q * 8 + 2 * t + j] = make_float2(mu, m2);
                }
            }
            __syncthreads();
            if (tid < COUT) {
                float mu = 0.f;
#pragma unroll
                for (int w = 0; w < 8; ++w) mu += wstat[w][tid].x;
                mu *= 0.125f;
                float m2 = 0.f;
#pragma unroll
                for (int w = 0; w < 8; ++w) {
                    const float d = wstat[w][tid].x - mu;
                    m2 += wstat[w][tid].y + kWarpPx * d * d;
                }
                // merge (8 kWarpPx, mu, m2) into (it * 8 kWarpPx, run_mean, run_m2)
                const float d = mu - run_mean, f = 1.f / (float)(it + 1);
                run_mean = fmaf(d, f, run_mean);
                run_m2 += m2 + d * d * (8.f * kWarpPx) * (float)it * f;
            }
        }
        __syncthreads();
    }
    if (stats && tid < COUT && n > 0) stats[(size_t)blockIdx.x * COUT + tid] = make_float2(run_mean, run_m2);
}

// ---------------------------------------------------------------------------------------------
// 3x3 convolution as a flat GEMM over pixels: the deep levels of the network, whose images are
// narrower than a tile or whose weights do not fit in shared memory
// ---------------------------------------------------------------------------------------------
//
// out[p][co] = sum_k A[p][k] W[co][k] over the flattened pixels p = (b, y, x) and k = (tap, ci),
// A the im2col of the input, gathered on the fly.  A CTA owns MT pixels and NT output channels
// (blockIdx.y) and walks K in chunks of kGK items (tap, 8-channel group); each chunk's A rows
// (pixel, item) and B rows (output channel, item) arrive by cp.async, 16 bytes each (zero-filled
// outside the image and past the last item), through a ring of kGStages slots, and ldmatrix
// reads both.  Each thread gathers for one pixel, decoded once.  Warps: 4 along pixels x 2 along
// output channels, (MT / 4) x (NT / 2) each.  Inputs, weights, the output split and the
// statistics are those of k_conv3x3; the statistics are per CTA (MT pixels) and channel.
// Requires B H W to be a multiple of MT and cout of NT.
constexpr int kGK = 8, kGStages = 4;
__host__ __device__ constexpr size_t gemm_conv_smem(int MT, int NT) { return kGStages * (size_t)(MT + NT) * kGK * 16; }

template <int MT, int NT>
__global__ void __launch_bounds__(256) k_conv3x3_gemm(const bf16* __restrict__ in0, int c0,
                                                      const bf16* __restrict__ in1, int c1,
                                                      const float* __restrict__ pf, const float* __restrict__ pg,
                                                      const bf16* __restrict__ wt, int G, int cout,
                                                      float* __restrict__ out0, float* __restrict__ out1, int split,
                                                      int acc0, int acc1, float2* __restrict__ stats, int B, int H,
                                                      int W) {
    constexpr int MB = MT / 64, NB = NT / 16;          // m-blocks and n-blocks per warp
    constexpr int TPP = 256 / MT;                       // threads per pixel in the gather
    constexpr size_t SLOT = (size_t)(MT + NT) * kGK * 16;
    extern __shared__ __align__(128) unsigned char smem_g[];
    __shared__ float2 wstat[4][NT];
    const int NI = 9 * G, nchunk = (NI + kGK - 1) / kGK, HW = H * W;
    const int p0 = blockIdx.x * MT, co0 = blockIdx.y * NT;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    const int wm = warp & 3, wn = warp >> 2;
    // this thread's gather pixel and first item slot
    const int gpx = tid % MT, gli = tid / MT;
    int gb, gy, gx;
    {
        const int p = p0 + gpx;
        gb = p / HW;
        const int r = p - gb * HW;
        gy = r / W;
        gx = r - gy * W;
    }

    auto stage = [&](int kc) {   // K chunk kc into ring slot kc % kGStages
        unsigned char* As = smem_g + (size_t)(kc % kGStages) * SLOT;
        unsigned char* Bs = As + (size_t)kGK * MT * 16;
        const int it0 = kc * kGK;
#pragma unroll
        for (int li = gli; li < kGK; li += TPP) {
            const int item = it0 + li;
            const int tap = item < NI ? item / G : 0, grp = item - tap * G;
            const int yy = gy + tap / 3 - 1, xx = gx + tap % 3 - 1;
            const bool inside = item < NI && yy >= 0 && yy < H && xx >= 0 && xx < W;
            const size_t q = inside ? ((size_t)gb * H + yy) * W + xx : 0;
            unsigned char* dst = As + (size_t)(li * MT + gpx) * 16;
            if (pf) {
                uint4 v = make_uint4(0, 0, 0, 0);
                if (inside) v.x = pack2(__float2bfloat16_rn(pf[q]), __float2bfloat16_rn(pg[q]));
                *reinterpret_cast<uint4*>(dst) = v;
            } else {
                const int ch = inside ? grp * 8 : 0;
                cp_async16(dst, ch < c0 ? in0 + q * c0 + ch : in1 + q * c1 + (ch - c0), inside);
            }
        }
        for (int e = tid; e < kGK * NT; e += 256) {
            const int li = e / NT, co = e - li * NT, item = it0 + li;
            const bool ok = item < NI;
            cp_async16(Bs + (size_t)e * 16, wt + ((size_t)(co0 + co) * NI + (ok ? item : 0)) * 8, ok);
        }
    };

    float acc[MB][NB][4];
#pragma unroll
    for (int m = 0; m < MB; ++m)
#pragma unroll
        for (int nb = 0; nb < NB; ++nb)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[m][nb][j] = 0.f;
    const int mi = lane >> 3, r8 = lane & 7;
    const int a_px = wm * (MT / 4) + (mi & 1) * 8 + r8, a_item = mi >> 1;
    const int b_co = wn * (NT / 2) + (mi >> 1) * 8 + r8, b_item = mi & 1;
    for (int k = 0; k < kGStages - 1; ++k) {
        if (k < nchunk) stage(k);
        cp_async_commit();
    }
    for (int kc = 0; kc < nchunk; ++kc) {
        if (kc + kGStages - 1 < nchunk) stage(kc + kGStages - 1);
        cp_async_commit();
        cp_async_wait_n(kGStages - 1);
        __syncthreads();
        const unsigned char* As = smem_g + (size_t)(kc % kGStages) * SLOT;
        const unsigned char* Bs = As + (size_t)kGK * MT * 16;
#pragma unroll
        for (int s = 0; s < kGK / 2; ++s) {
            uint32_t a[MB][4];
#pragma unroll
            for (int m = 0; m < MB; ++m)
                ldsm_x4(a[m], As + (size_t)((2 * s + a_item) * MT + a_px + 16 * m) * 16);
#pragma unroll
            for (int nb = 0; nb < NB; nb += 2) {
                uint32_t bq[4];
                ldsm_x4(bq, Bs + (size_t)((2 * s + b_item) * NT + b_co + 8 * nb) * 16);
#pragma unroll
                for (int m = 0; m < MB; ++m) {
                    mma16816(acc[m][nb], a[m], bq);
                    mma16816(acc[m][nb + 1], a[m], bq + 2);
                }
            }
        }
        __syncthreads();
    }
    // acc[m][nb][j]: pixel p0 + wm MT/4 + 16 m + g (+8 for j >= 2), channel co0 + wn NT/2 + 8 nb + 2 t + (j & 1)
#pragma unroll
    for (int m = 0; m < MB; ++m) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const size_t p = (size_t)p0 + wm * (MT / 4) + 16 * m + g + 8 * h;
#pragma unroll
            for (int nb = 0; nb < NB; ++nb) {
                const int ch = co0 + wn * (NT / 2) + nb * 8 + 2 * t;
                const float v0 = acc[m][nb][2 * h], v1 = acc[m][nb][2 * h + 1];
                if (ch < split) {
                    float2* o = reinterpret_cast<float2*>(out0 + p * split + ch);
                    if (acc0) {
                        const float2 old = *o;
                        *o = make_float2(old.x + v0, old.y + v1);
                    } else {
                        *o = make_float2(v0, v1);
                    }
                } else {
                    float2* o = reinterpret_cast<float2*>(out1 + p * (cout - split) + (ch - split));
                    if (acc1) {
                        const float2 old = *o;
                        *o = make_float2(old.x + v0, old.y + v1);
                    } else {
                        *o = make_float2(v0, v1);
                    }
                }
            }
        }
    }
    if (stats) {
        // per channel: each warp's MT / 4 pixels give a (mean, M2) pair by shuffles over g; the 4
        // pixel warps' pairs (equal counts) give the CTA's
        constexpr float kWarpPx = MT / 4;
#pragma unroll
        for (int nb = 0; nb < NB; ++nb) {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                float sm = 0.f;
#pragma unroll
                for (int m = 0; m < MB; ++m) sm += acc[m][nb][j] + acc[m][nb][j + 2];
#pragma unroll
                for (int o = 4; o < 32; o <<= 1) sm += __shfl_xor_sync(0xffffffffu, sm, o);
                const float mu = sm * (1.f / kWarpPx);
                float m2 = 0.f;
#pragma unroll
                for (int m = 0; m < MB; ++m) {
                    const float d0 = acc[m][nb][j] - mu, d1 = acc[m][nb][j + 2] - mu;
                    m2 += d0 * d0 + d1 * d1;
                }
#pragma unroll
                for (int o = 4; o < 32; o <<= 1) m2 += __shfl_xor_sync(0xffffffffu, m2, o);
                if (g == 0) wstat[wm][wn * (NT / 2) + nb * 8 + 2 * t + j] = make_float2(mu, m2);
            }
        }
        __syncthreads();
        if (tid < NT) {
            float mu = 0.f;
#pragma unroll
            for (int w = 0; w < 4; ++w) mu += wstat[w][tid].x;
            mu *= 0.25f;
            float m2 = 0.f;
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const float d = wstat[w][tid].x - mu;
                m2 += wstat[w][tid].y + kWarpPx * d * d;
            }
            stats[(size_t)blockIdx.x * cout + co0 + tid] = make_float2(mu, m2);
        }
    }
}

// ---------------------------------------------------------------------------------------------
// The flat-GEMM convolution on the 5th-generation tensor cores (tcgen05, accumulator in TMEM)
// ---------------------------------------------------------------------------------------------
//
// Same product, operands and ring as k_conv3x3_gemm<128, NT>: the im2col rows (pixel, item) and
// weight rows (output channel, item) land by cp.async in the canonical K-major, no-swizzle layout
// of tcgen05 -- a core matrix is 8 consecutive 16-byte rows, so [item][pixel][16 B] puts the 8-row
// groups 128 B apart (SBO) and the K-adjacent core matrices 128 * 16 B apart (LBO).  One thread
// issues tcgen05.mma (M = 128 pixels, N = NT channels, K = 16) for each K step of a chunk and
// commits it to the slot's mbarrier, which the producers wait on before refilling the slot; the
// accumulator lives in NT TMEM columns.  The epilogue reads TMEM with tcgen05.ld (warp w: lanes
// 32 (w % 4) .., columns (w / 4) NT / 2 ..), stores, and forms the statistics as k_conv3x3_gemm
// does.
//
// Every mbarrier wait is bounded.  A producer's wait for a slot (the MMAs of the chunk before have
// read it) gives up after `spin` non-blocking polls (host-settable, kTcSpin by default); the CTA
// then issues no
// further MMA, lets its cp.async copies land, and drains: it waits for the commit of the last
// chunk it issued, which covers every MMA it issued, for up to kTcDrain polls -- MMAs finish in
// microseconds, kTcDrain is seconds, so it runs out only when the GPU no longer makes progress.
// Only then does the CTA release its TMEM and exit: no MMA is in flight when its tensor memory
// or its shared-memory operands change hands.  A CTA that gave up counts itself in *timeouts and
// writes no output; the host turns the count into FMBYM_ERR_TIMEOUT.
__host__ __device__ constexpr size_t tc_conv_smem(int NT) { return kGStages * (size_t)(128 + NT) * kGK * 16; }
constexpr unsigned kTcSpin = 1u << 22;   // default polls before a producer's wait gives up
constexpr unsigned kTcDrain = 1u << 28;  // polls of the drain before the CTA releases its TMEM

__device__ __forceinline__ unsigned long long tc_desc(unsigned addr, unsigned lbo, unsigned sbo) {
    return (unsigned long long)((addr >> 4) & 0x3FFF) | ((unsigned long long)((lbo >> 4) & 0x3FFF) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Up to `limit` non-blocking tests of the barrier's phase (a producer's wait: the limit counts
// polls exactly, however short).
__device__ __forceinline__ bool mbar_poll(unsigned bar, unsigned parity, unsigned limit) {
    unsigned done = 0;
    for (unsigned it = 0; it < limit && !done; ++it)
        asm volatile("{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(bar), "r"(parity)
                     : "memory");
    return done != 0;
}

// Up to `limit` potentially blocking waits for the barrier's phase (the drain).
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, unsigned limit) {
    unsigned done = 0;
    for (unsigned it = 0; it < limit && !done; ++it)
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(bar), "r"(parity)
                     : "memory");
    return done != 0;
}

template <int NT>
__global__ void __launch_bounds__(256) k_conv3x3_tc(const bf16* __restrict__ in0, int c0, const bf16* __restrict__ in1,
                                                    int c1, const bf16* __restrict__ wt, int G, int cout,
                                                    float* __restrict__ out0, float* __restrict__ out1, int split,
                                                    int acc0, int acc1, float2* __restrict__ stats, int B, int H,
                                                    int W, unsigned* __restrict__ timeouts, unsigned spin) {
    constexpr int MT = 128;
    constexpr size_t SLOT = (size_t)(MT + NT) * kGK * 16;
    extern __shared__ __align__(1024) unsigned char smem_t[];
    __shared__ __align__(8) unsigned long long mbar[kGStages];
    __shared__ unsigned tmem_base;
    __shared__ int failed;
    __shared__ float2 wstat[4][NT];
    const int NI = 9 * G, nchunk = (NI + kGK - 1) / kGK, HW = H * W;
    const int p0 = blockIdx.x * MT, co0 = blockIdx.y * NT;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned sbase = (unsigned)__cvta_generic_to_shared(smem_t);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         (unsigned)__cvta_generic_to_shared(&tmem_base)),
                     "r"(NT));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        failed = 0;
        for (int s = 0; s < kGStages; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"((unsigned)__cvta_generic_to_shared(&mbar[s])));
        asm volatile("fence.mbarrier_init.release.cluster;\n");
    }
    const int gpx = tid % MT, gli = tid / MT;
    int gb, gy, gx;
    {
        const int p = p0 + gpx;
        gb = p / HW;
        const int r = p - gb * HW;
        gy = r / W;
        gx = r - gy * W;
    }
    auto stage = [&](int kc) {
        unsigned char* As = smem_t + (size_t)(kc % kGStages) * SLOT;
        unsigned char* Bs = As + (size_t)kGK * MT * 16;
        const int it0 = kc * kGK;
#pragma unroll
        for (int li = gli; li < kGK; li += 256 / MT) {
            const int item = it0 + li;
            const int tap = item < NI ? item / G : 0, grp = item - tap * G;
            const int yy = gy + tap / 3 - 1, xx = gx + tap % 3 - 1;
            const bool inside = item < NI && yy >= 0 && yy < H && xx >= 0 && xx < W;
            const size_t q = inside ? ((size_t)gb * H + yy) * W + xx : 0;
            const int ch = inside ? grp * 8 : 0;
            cp_async16(As + (size_t)(li * MT + gpx) * 16, ch < c0 ? in0 + q * c0 + ch : in1 + q * c1 + (ch - c0),
                       inside);
        }
        for (int e = tid; e < kGK * NT; e += 256) {
            const int li = e / NT, co = e - li * NT, item = it0 + li;
            const bool ok = item < NI;
            cp_async16(Bs + (size_t)e * 16, wt + ((size_t)(co0 + co) * NI + (ok ? item : 0)) * 8, ok);
        }
    };
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const unsigned tmem = tmem_base;
    // kind::f16: D f32, A and B bf16, both K-major, N = NT, M = 128
    const unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(NT >> 3) << 17) | ((unsigned)(MT >> 4) << 24);
    for (int k = 0; k < kGStages - 1; ++k) {
        if (k < nchunk) stage(k);
        cp_async_commit();
    }
    int issued = 0;   // chunks whose MMAs were committed (thread 0's count; others follow via failed)
    for (int kc = 0; kc < nchunk; ++kc) {
        const int nk = kc + kGStages - 1;
        if (nk < nchunk) {
            if (nk >= kGStages) {   // the slot's previous chunk (kc - 1) must have been consumed
                const unsigned bar = (unsigned)__cvta_generic_to_shared(&mbar[nk % kGStages]);
                if (!mbar_poll(bar, (unsigned)(((nk - kGStages) / kGStages) & 1), spin)) failed = 1;
            }
            __syncthreads();
            if (failed) break;
            stage(nk);
        }
        cp_async_commit();
        cp_async_wait_n(kGStages - 1);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        if (tid == 0) {
            const unsigned As = sbase + (unsigned)((kc % kGStages) * SLOT), Bs = As + kGK * MT * 16;
#pragma unroll
            for (int s = 0; s < kGK / 2; ++s) {
                const unsigned long long ad = tc_desc(As + s * 2 * MT * 16, MT * 16, 128);
                const unsigned long long bd = tc_desc(Bs + s * 2 * NT * 16, NT * 16, 128);
                const unsigned accum = (kc > 0 || s > 0) ? 1u : 0u;
                asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                             ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                (unsigned)__cvta_generic_to_shared(&mbar[kc % kGStages])));
        }
        issued = kc + 1;
    }
    cp_async_wait_n(0);
    // drain: the last committed chunk's barrier covers every MMA issued before it (after a
    // producer gave up too); the outcome is shared so that the whole CTA takes the same branch
    // around the warp-collective TMEM loads
    if (issued > 0) {
        const int last = issued - 1;
        const unsigned bar = (unsigned)__cvta_generic_to_shared(&mbar[last % kGStages]);
        if (!mbar_wait(bar, (unsigned)((last / kGStages) & 1), kTcDrain)) failed = 1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const bool ok = !failed && issued == nchunk;
    if (!ok && tid == 0) atomicAdd(timeouts, 1u);
    if (ok) {
        // epilogue: warp w holds pixels 32 (w % 4) + lane, channels (w / 4) NT / 2 + [0, NT / 2)
        const int wq = warp & 3, half = warp >> 2;
        const size_t p = (size_t)p0 + 32 * wq + lane;
#pragma unroll
        for (int cc = 0; cc < NT / 2; cc += 16) {
            const int cb = half * (NT / 2) + cc;
            unsigned r[16];
            const unsigned addr = tmem + ((unsigned)(32 * wq) << 16) + (unsigned)cb;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                           "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                         : "r"(addr));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n");
            float v[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
#pragma unroll
            for (int j = 0; j < 16; j += 2) {
                const int ch = co0 + cb + j;
                if (ch < split) {
                    float2* o = reinterpret_cast<float2*>(out0 + p * split + ch);
                    if (acc0) {
                        const float2 old = *o;
                        *o = make_float2(old.x + v[j], old.y + v[j + 1]);
                    } else {
                        *o = make_float2(v[j], v[j + 1]);
                    }
                } else {
                    float2* o = reinterpret_cast<float2*>(out1 + p * (cout - split) + (ch - split));
                    if (acc1) {
                        const float2 old = *o;
                        *o = make_float2(old.x + v[j], old.y + v[j + 1]);
                    } else {
                        *o = make_float2(v[j], v[j + 1]);
                    }
                }
            }
            if (stats) {
                // per channel: the warp's 32 pixels give a (mean, M2) pair by shuffles
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    float sm = v[j];
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) sm += __shfl_xor_sync(0xffffffffu, sm, o);
                    const float mu = sm * (1.f / 32.f), d = v[j] - mu;
                    float m2 = d * d;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) m2 += __shfl_xor_sync(0xffffffffu, m2, o);
                    if (lane == 0) wstat[wq][cb + j] = make_float2(mu, m2);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(NT));
    if (ok && stats && tid < NT) {
        float mu = 0.f;
#pragma unroll
        for (int w = 0; w < 4; ++w) mu += wstat[w][tid].x;
        mu *= 0.25f;
        float m2 = 0.f;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const float d = wstat[w][tid].x - mu;
            m2 += wstat[w][tid].y + 32.f * d * d;
        }
        stats[(size_t)blockIdx.x * cout + co0 + tid] = make_float2(mu, m2);
    }
}

// ---------------------------------------------------------------------------------------------
// BatchNorm
// ---------------------------------------------------------------------------------------------

// Combines the per-CTA (mean, M2) partials of one channel.  CTA k of the convolution's nparts
// covered n_k = ((ntiles - 1 - k) / nparts + 1) tiles of tile_px pixels; the batch mean is
// sum n_k mean_k / N and M2 = sum M2_k + sum n_k (mean_k - mean)^2 (two passes; each thread adds a
// fixed stride of partials in float32, the block adds the threads in a fixed-order float64 tree).
// Updates the running statistics (momentum 0.1, unbiased variance) and writes
// bn[c] = (mean, 1/sqrt(var + eps)) for the batch statistics.  One block per channel.
__global__ void __launch_bounds__(256) k_bn_finalize(const float2* __restrict__ stats, int nparts, int C,
                                                     int ntiles, float tile_px, float* __restrict__ run_mean,
                                                     float* __restrict__ run_var, float2* __restrict__ bn) {
    __shared__ double r[256];
    const int c = blockIdx.x;
    auto block_sum = [&](double v) {
        r[threadIdx.x] = v;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) r[threadIdx.x] += r[threadIdx.x + o];
            __syncthreads();
        }
        const double tot = r[0];
        __syncthreads();
        return tot;
    };
    auto count = [&](int k) { return (float)((ntiles - 1 - k) / nparts + 1) * tile_px; };
    float s = 0.f;
    for (int k = threadIdx.x; k < nparts; k += 256) s = fmaf(count(k), stats[(size_t)k * C + c].x, s);
    const double N = (double)ntiles * tile_px;
    const double mean = block_sum(s) / N;
    const float mf = (float)mean;
    float q = 0.f, e = 0.f;
    for (int k = threadIdx.x; k < nparts; k += 256) {
        const float2 v = stats[(size_t)k * C + c];
        const float d = v.x - mf;
        q += v.y;
        e = fmaf(count(k) * d, d, e);
    }
    const double m2 = block_sum(q) + block_sum(e);
    if (threadIdx.x == 0) {
        const double var = m2 / N;
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
// slab of pixel_per_cta pixels of dpre = da [pre > 0] and dpre xhat per channel.  A thread takes
// four channels (float4) of every (256 / (C / 4))-th pixel; the CTA adds its rows in order.
// C in {8, 16, 32, 64}; pix_per_cta a multiple of 256 / (C / 4).
__global__ void __launch_bounds__(256) k_bn_bwd_reduce(const float* __restrict__ y, const float* __restrict__ da,
                                                       const float2* __restrict__ bn,
                                                       const float* __restrict__ gamma,
                                                       const float* __restrict__ beta, long long npix, int C,
                                                       int pix_per_cta, float2* __restrict__ part) {
    __shared__ float4 s1[256], s2[256];
    const int q = C / 4, rows = 256 / q;
    const int cq = threadIdx.x % q, r = threadIdx.x / q;
    float4 a1 = make_float4(0.f, 0.f, 0.f, 0.f), a2 = a1;
    float mu[4], is[4], gm[4], bt[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float2 st = bn[4 * cq + j];
        mu[j] = st.x;
        is[j] = st.y;
        gm[j] = gamma[4 * cq + j];
        bt[j] = beta[4 * cq + j];
    }
    const long long p0 = (long long)blockIdx.x * pix_per_cta;
    const long long p1 = min(p0 + pix_per_cta, npix);
    const float4* y4 = reinterpret_cast<const float4*>(y);
    const float4* d4 = reinterpret_cast<const float4*>(da);
#pragma unroll 4
    for (long long p = p0 + r; p < p1; p += rows) {
        const float4 yv = y4[p * q + cq], dv = d4[p * q + cq];
        const float yy[4] = {yv.x, yv.y, yv.z, yv.w}, dd[4] = {dv.x, dv.y, dv.z, dv.w};
        float o1[4], o2[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float xh = (yy[j] - mu[j]) * is[j];
            const float dp = fmaf(xh, gm[j], bt[j]) > 0.f ? dd[j] : 0.f;
            o1[j] = dp;
            o2[j] = dp * xh;
        }
        a1.x += o1[0]; a1.y += o1[1]; a1.z += o1[2]; a1.w += o1[3];
        a2.x += o2[0]; a2.y += o2[1]; a2.z += o2[2]; a2.w += o2[3];
    }
    s1[threadIdx.x] = a1;
    s2[threadIdx.x] = a2;
    __syncthreads();
    if ((int)threadIdx.x < C) {
        const int c = threadIdx.x, qq = c / 4, j = c % 4;
        const float* f1 = reinterpret_cast<const float*>(s1);
        const float* f2 = reinterpret_cast<const float*>(s2);
        float t1 = 0.f, t2 = 0.f;
        for (int k = 0; k < rows; ++k) {
            t1 += f1[(k * q + qq) * 4 + j];
            t2 += f2[(k * q + qq) * 4 + j];
        }
        part[(size_t)blockIdx.x * C + c] = make_float2(t1, t2);
    }
}

// Part 2, one block per channel: the partials summed in a fixed order -> d beta = sum dpre,
// d gamma = sum dpre xhat (written to the gradient array) and the means used by the dy kernel,
// sums[c] = (mean dpre, mean dpre xhat).
__global__ void __launch_bounds__(256) k_bn_bwd_finalize(const float2* __restrict__ part, int nparts, int C,
                                                         float inv_n, float* __restrict__ dgamma,
                                                         float* __restrict__ dbeta, float2* __restrict__ sums) {
    __shared__ double r1[256], r2[256];
    const int c = blockIdx.x;
    double t1 = 0.0, t2 = 0.0;
    for (int i = threadIdx.x; i < nparts; i += 256) {
        const float2 v = part[(size_t)i * C + c];
        t1 += v.x;
        t2 += v.y;
    }
    r1[threadIdx.x] = t1;
    r2[threadIdx.x] = t2;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            r1[threadIdx.x] += r1[threadIdx.x + o];
            r2[threadIdx.x] += r2[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        dbeta[c] = (float)r1[0];
        dgamma[c] = (float)r2[0];
        sums[c] = make_float2((float)(r1[0] * inv_n), (float)(r2[0] * inv_n));
    }
}

// Part 3: dy = gamma invstd (dpre - mean dpre - xhat mean(dpre xhat)), rounded to bf16 for the
// tensor-core dgrad and wgrad.  Four channels per thread; n4 = pixels * C / 4.
__global__ void k_bn_bwd_dy(const float* __restrict__ y, const float* __restrict__ da, const float2* __restrict__ bn,
                            const float* __restrict__ gamma, const float* __restrict__ beta,
                            const float2* __restrict__ sums, bf16* __restrict__ dy, long long n4, int C) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n4) return;
    const int c0 = (int)((i * 4) % C);
    const float4 yv = reinterpret_cast<const float4*>(y)[i], dv = reinterpret_cast<const float4*>(da)[i];
    const float yy[4] = {yv.x, yv.y, yv.z, yv.w}, dd[4] = {dv.x, dv.y, dv.z, dv.w};
    bf16 o[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int c = c0 + j;
        const float2 s = bn[c];
        const float gm = gamma[c];
        const float xh = (yy[j] - s.x) * s.y;
        const float dp = fmaf(xh, gm, beta[c]) > 0.f ? dd[j] : 0.f;
        const float2 m = sums[c];
        o[j] = __float2bfloat16_rn(gm * s.y * (dp - m.x - xh * m.y));
    }
    reinterpret_cast<uint2*>(dy)[i] = make_uint2(pack2(o[0], o[1]), pack2(o[2], o[3]));
}

// ---------------------------------------------------------------------------------------------
// max-pool 2x2 and bilinear x2 (align_corners = False) with their adjoints
// ---------------------------------------------------------------------------------------------

// Pooling and upsampling kernels run on a 2-D grid: blockIdx.y walks image rows (b, y) with a
// stride of gridDim.y, blockIdx.x / threadIdx.x the pixels x channel vectors of one row, so that
// all index arithmetic is 32-bit.  Channel counts are multiples of 8.

// 2x2 max-pool, eight channels (16 bytes) per thread, flat 32-bit index over B * H/2 * W/2 * C/8.
__global__ void k_maxpool(const bf16* __restrict__ a, bf16* __restrict__ p, int B, int H, int W, int C) {
    const int Ho = H / 2, Wo = W / 2, q = C / 8;
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (unsigned)B * Ho * Wo * q) return;
    const int c = (int)(i % q) * 8;
    unsigned r = i / q;
    const int x = (int)(r % Wo);
    r /= Wo;
    const int y = (int)(r % Ho), b = (int)(r / Ho);
    const bf16* base = a + (((size_t)b * H + 2 * y) * W + 2 * x) * C + c;
    const uint4 v[4] = {*reinterpret_cast<const uint4*>(base), *reinterpret_cast<const uint4*>(base + C),
                        *reinterpret_cast<const uint4*>(base + (size_t)W * C),
                        *reinterpret_cast<const uint4*>(base + (size_t)W * C + C)};
    uint32_t o[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t w[4] = {(&v[0].x)[k], (&v[1].x)[k], (&v[2].x)[k], (&v[3].x)[k]};
        float lo = __uint_as_float(w[0] << 16), hi = __uint_as_float(w[0] & 0xffff0000u);
#pragma unroll
        for (int t = 1; t < 4; ++t) {
            lo = fmaxf(lo, __uint_as_float(w[t] << 16));
            hi = fmaxf(hi, __uint_as_float(w[t] & 0xffff0000u));
        }
        o[k] = pack2(__float2bfloat16_rn(lo), __float2bfloat16_rn(hi));   // exact: both are bf16 values
    }
    *reinterpret_cast<uint4*>(p + (((size_t)b * Ho + y) * Wo + x) * C + c) = make_uint4(o[0], o[1], o[2], o[3]);
}

// Routes d p to the first maximum of its window in row-major order (strict >), added to da.
// Four channels per thread (each window's da is touched by this thread only), flat 32-bit index
// over B * H/2 * W/2 * C/4.
__global__ void k_maxpool_bwd(const bf16* __restrict__ a, const float* __restrict__ dp, float* __restrict__ da,
                              int B, int H, int W, int C) {
    const int Ho = H / 2, Wo = W / 2, q = C / 4;
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (unsigned)B * Ho * Wo * q) return;
    const int c = (int)(i % q) * 4;
    unsigned r = i / q;
    const int x = (int)(r % Wo);
    r /= Wo;
    const int y = (int)(r % Ho), b = (int)(r / Ho);
    const size_t off[4] = {0, (size_t)C, (size_t)W * C, (size_t)W * C + C};
    const size_t base = (((size_t)b * H + 2 * y) * W + 2 * x) * C + c;
    float m[4];
    int best[4] = {0, 0, 0, 0};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const uint2 v = *reinterpret_cast<const uint2*>(a + base + off[t]);
        const float e[4] = {__uint_as_float(v.x << 16), __uint_as_float(v.x & 0xffff0000u),
                            __uint_as_float(v.y << 16), __uint_as_float(v.y & 0xffff0000u)};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (t == 0) m[k] = e[k];
            else if (e[k] > m[k]) {
                m[k] = e[k];
                best[k] = t;
            }
        }
    }
    const float4 g = *reinterpret_cast<const float4*>(dp + (((size_t)b * Ho + y) * Wo + x) * C + c);
    const float gv[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        if (best[0] != t && best[1] != t && best[2] != t && best[3] != t) continue;
        float4* dst = reinterpret_cast<float4*>(da + base + off[t]);
        float4 d = *dst;
        if (best[0] == t) d.x += gv[0];
        if (best[1] == t) d.y += gv[1];
        if (best[2] == t) d.z += gv[2];
        if (best[3] == t) d.w += gv[3];
        *dst = d;
    }
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

// Eight channels (16 bytes) of one input pixel (y, x) per thread, which writes its 2 x 2 output
// pixels (2y + dy, 2x + dx): with align_corners = False at scale 2 each of them is the bilinear
// mix of rows y - 1 + dy, y + dy and columns x - 1 + dx, x + dx with weights (1/4, 3/4) for
// d = 0 and (3/4, 1/4) for d = 1, and the edge clamping of the source index is the clamping of
// those rows and columns to the image (up_src gives the same weights, and the same arithmetic
// order is kept).  rows = B * h.
__global__ void k_upsample(const bf16* __restrict__ a, bf16* __restrict__ u, int B, int h, int w, int C) {
    const int H = 2 * h, W = 2 * w, q = C / 8;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= w * q) return;
    const int c = (j % q) * 8, x = j / q;
    const int xs[3] = {max(x - 1, 0), x, min(x + 1, w - 1)};
    for (int row = blockIdx.y; row < B * h; row += gridDim.y) {
        const int b = row / h, y = row % h;
        const int ys[3] = {max(y - 1, 0), y, min(y + 1, h - 1)};
        const bf16* base = a + (size_t)b * h * w * C + c;
        uint4 v[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int k = 0; k < 3; ++k) v[i][k] = *reinterpret_cast<const uint4*>(base + ((size_t)ys[i] * w + xs[k]) * C);
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const float ly0 = dy ? 0.75f : 0.25f, ly1 = 1.f - ly0;
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                const float lx0 = dx ? 0.75f : 0.25f, lx1 = 1.f - lx0;
                const uint32_t* p00 = &v[dy][dx].x;
                const uint32_t* p01 = &v[dy][dx + 1].x;
                const uint32_t* p10 = &v[dy + 1][dx].x;
                const uint32_t* p11 = &v[dy + 1][dx + 1].x;
                uint32_t o[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    float res[2];
#pragma unroll
                    for (int hlf = 0; hlf < 2; ++hlf) {
                        auto f = [&](uint32_t wd) { return __uint_as_float(hlf ? (wd & 0xffff0000u) : (wd << 16)); };
                        res[hlf] = ly0 * (lx0 * f(p00[k]) + lx1 * f(p01[k])) + ly1 * (lx0 * f(p10[k]) + lx1 * f(p11[k]));
                    }
                    o[k] = pack2(__float2bfloat16_rn(res[0]), __float2bfloat16_rn(res[1]));
                }
                *reinterpret_cast<uint4*>(u + (((size_t)b * H + 2 * y + dy) * W + 2 * x + dx) * C + c) =
                    make_uint4(o[0], o[1], o[2], o[3]);
            }
        }
    }
}

// Weight that the forward assigns from input index k to output index o (both taps if clamped).
__device__ __forceinline__ float up_w(int o, int k, int n) {
    int i0, i1;
    float l0, l1;
    up_src(o, n, i0, i1, l0, l1);
    return (i0 == k ? l0 : 0.f) + (i1 == k ? l1 : 0.f);
}

// Transpose of the upsampling in gather form: d a[k] = sum over the outputs o in [2k-1, 2k+2] (the
// only ones whose two taps can reach k) of the forward weights times d u[o]; written (not added)
// to da.  A thread takes a 2 x 2 block of input pixels (y0, y0 + 1) x (x0, x0 + 1) and four
// channels: their outputs are the 6 x 6 window of rows 2 y0 - 1 .. 2 y0 + 4 and columns
// 2 x0 - 1 .. 2 x0 + 4, each read once.  h and w even; rows = B * h / 2.
__global__ void k_upsample_bwd(const float* __restrict__ du, float* __restrict__ da, int B, int h, int w, int C) {
    const int H = 2 * h, W = 2 * w, q = C / 4;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= (w / 2) * q) return;
    const int c = (j % q) * 4, x0 = 2 * (j / q);
    // wx[i][k]: weight of output column 2 x0 - 1 + k on input column x0 + i (zero outside)
    float wx[2][6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const int X = 2 * x0 - 1 + k;
        wx[0][k] = (k < 4 && X >= 0 && X < W) ? up_w(X, x0, w) : 0.f;
        wx[1][k] = (k >= 2 && X < W) ? up_w(X, x0 + 1, w) : 0.f;
    }
    for (int row = blockIdx.y; row < B * (h / 2); row += gridDim.y) {
        const int b = row / (h / 2), y0 = 2 * (row % (h / 2));
        float4 s[2][2];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int k = 0; k < 2; ++k) s[i][k] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            const int Y = 2 * y0 - 1 + r;
            if (Y < 0 || Y >= H) continue;
            const float wy0 = r < 4 ? up_w(Y, y0, h) : 0.f, wy1 = r >= 2 ? up_w(Y, y0 + 1, h) : 0.f;
            const float* rowp = du + ((size_t)b * H + Y) * W * C + c;
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const int X = 2 * x0 - 1 + k;
                if (X < 0 || X >= W) continue;
                const float4 v = *reinterpret_cast<const float4*>(rowp + (size_t)X * C);
#pragma unroll
                for (int iy = 0; iy < 2; ++iy) {
                    const float wy = iy ? wy1 : wy0;
#pragma unroll
                    for (int ix = 0; ix < 2; ++ix) {
                        const float wt = wy * wx[ix][k];
                        s[iy][ix].x += wt * v.x;
                        s[iy][ix].y += wt * v.y;
                        s[iy][ix].z += wt * v.z;
                        s[iy][ix].w += wt * v.w;
                    }
                }
            }
        }
#pragma unroll
        for (int iy = 0; iy < 2; ++iy)
#pragma unroll
            for (int ix = 0; ix < 2; ++ix)
                *reinterpret_cast<float4*>(da + (((size_t)b * h + y0 + iy) * w + x0 + ix) * C + c) = s[iy][ix];
    }
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
// d W[o][c] = sum d z_o a[c] and d b[o] = sum d z_o (2 C + 2 values, fixed order).  Grid-stride
// over pixels, so the number of partials is the grid size.
template <int C>
__global__ void __launch_bounds__(256) k_head_bwd(const bf16* __restrict__ a, const float* __restrict__ hw,
                                                  const float* __restrict__ hb, const float* __restrict__ f,
                                                  const float* __restrict__ g, const float* __restrict__ dfo,
                                                  const float* __restrict__ dgo, float* __restrict__ da,
                                                  float* __restrict__ part, long long npix) {
    __shared__ float red[8][2 * C + 2];
    __shared__ float w0[C], w1[C];   // the bf16-rounded head weights
    float loc[2 * C + 2];
#pragma unroll
    for (int k = 0; k < 2 * C + 2; ++k) loc[k] = 0.f;
    if ((int)threadIdx.x < C) {
        w0[threadIdx.x] = __bfloat162float(__float2bfloat16_rn(hw[threadIdx.x]));
        w1[threadIdx.x] = __bfloat162float(__float2bfloat16_rn(hw[C + threadIdx.x]));
    }
    __syncthreads();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < npix;
         i += (long long)gridDim.x * blockDim.x) {
        float av[C];
        float z0 = hb[0], z1 = hb[1];
#pragma unroll
        for (int c = 0; c < C; c += 8) {
            const uint4 v = *reinterpret_cast<const uint4*>(a + i * C + c);
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                av[c + 2 * k] = __uint_as_float(w[k] << 16);
                av[c + 2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
            }
        }
#pragma unroll
        for (int c = 0; c < C; ++c) {
            z0 = fmaf(w0[c], av[c], z0);
            z1 = fmaf(w1[c], av[c], z1);
        }
        const float m0 = 1.f / (1.f + expf(-z0)), m1 = 1.f / (1.f + expf(-z1));
        const float d0 = dfo[i] * f[i] * m0 * (1.f - m0), d1 = dgo[i] * g[i] * m1 * (1.f - m1);
#pragma unroll
        for (int c = 0; c < C; c += 4)
            *reinterpret_cast<float4*>(da + i * C + c) =
                make_float4(w0[c] * d0 + w1[c] * d1, w0[c + 1] * d0 + w1[c + 1] * d1, w0[c + 2] * d0 + w1[c + 2] * d1,
                            w0[c + 3] * d0 + w1[c + 3] * d1);
#pragma unroll
        for (int c = 0; c < C; ++c) {
            loc[c] = fmaf(d0, av[c], loc[c]);
            loc[C + c] = fmaf(d1, av[c], loc[C + c]);
        }
        loc[2 * C] += d0;
        loc[2 * C + 1] += d1;
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

// Sums per-block partials column by column into out, one block per column: every thread adds a
// fixed stride of partials, then a fixed-order tree.
__global__ void __launch_bounds__(256) k_sum_parts(const float* __restrict__ part, int nparts, int width,
                                                   float* __restrict__ out) {
    __shared__ double r[256];
    const int k = blockIdx.x;
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += 256) s += part[(size_t)i * width + k];
    r[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) r[threadIdx.x] += r[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = (float)r[0];
}

// ---------------------------------------------------------------------------------------------
// weight gradient of a 3x3 convolution
// ---------------------------------------------------------------------------------------------
//
// dW[co][tap][ci] = sum over pixels p of dy[p][co] in[p + tap][ci]: an implicit GEMM with
// M = 16 output channels, N = 8 input channels, K = 16 pixels of one tile row, on
// mma.sync.m16n8k16.  A CTA owns 16 output channels and CIB input channels (CIB divides the
// layer's input channels) and walks a chunk of 8 R x 32 pixel tiles.  Both operands are staged
// pixel-major, one 16-byte row per pixel and group of 8 channels -- exactly the NHWC bytes -- by
// cp.async through a ring of `nstage` slots (zero-filled outside the image), and ldmatrix.trans
// turns those rows into the channel-by-pixel fragments, so a 3x3 tap is only a shifted row
// address.  Warps split into CIB / 8 channel groups times 64 / CIB row groups; the row groups'
// partial sums are added in a fixed order at the end and the CTA's dW goes to part[chunk], which
// k_wgrad_reduce sums over chunks in order (bitwise deterministic).  blockIdx.x = chunk * gz + z
// for the gz input-channel blocks, so the blocks of one chunk run together and share dy in L2.
// Requires cout and every input channel count to be multiples of 8 (the planes of the first
// layer are staged by plain loads instead).

template <int CIB>
__host__ __device__ inline size_t wgrad_buf_bytes(int R) {
    return (size_t)(2 * kTilePx * R + (CIB / 8) * (8 * R + 2) * kTileW) * 16;
}
template <int CIB>
__host__ __device__ inline size_t wgrad_smem(int R, int nstage) {   // the ring, or the row-group sums
    return nstage * wgrad_buf_bytes<CIB>(R) > (size_t)8 * 36 * 32 * 4 ? nstage * wgrad_buf_bytes<CIB>(R)
                                                                         : (size_t)8 * 36 * 32 * 4;
}

template <int CIB, bool PLANES>
__global__ void __launch_bounds__(256) k_wgrad(const bf16* __restrict__ dy, int cout, const bf16* __restrict__ in0,
                                               int c0, const bf16* __restrict__ in1, int c1,
                                               const float* __restrict__ pf, const float* __restrict__ pg, int B,
                                               int H, int W, int R, int gz, int tiles_per_chunk, int nstage,
                                               float* __restrict__ part) {
    constexpr int NG = CIB / 8, NRG = 8 / NG;
    const size_t BUF = wgrad_buf_bytes<CIB>(R);
    const int TH = 8 * R, TPX = kTilePx * R, HALO = (TH + 2) * kTileW;
    extern __shared__ __align__(128) unsigned char smem_w[];
    const int cin = PLANES ? 2 : c0 + c1;
    const int chunk = blockIdx.x / gz, co0 = blockIdx.y * 16, ci_base = (blockIdx.x % gz) * CIB;
    const int ngr = PLANES ? 1 : min(NG, (cin - ci_base) / 8);   // channel groups present
    const int cog = min(2, (cout - co0) / 8);                     // output groups present (1 or 2)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    const int wc = warp % NG, wr = warp / NG;
    const int tiles_x = W / kTW, tiles_img = tiles_x * (H / TH), ntiles = B * tiles_img;
    const int first = chunk * tiles_per_chunk, n = min(tiles_per_chunk, ntiles - first);

    if (cog == 1)  // the upper 8 rows of the A operand stay zero in every ring slot
        for (int i = tid; i < TPX; i += 256)
            for (int bsel = 0; bsel < nstage; ++bsel)
                *reinterpret_cast<uint4*>(smem_w + bsel * BUF + (size_t)(TPX + i) * 16) = make_uint4(0, 0, 0, 0);

    auto stage = [&](int k) {   // the k-th tile of this CTA's chunk into ring slot k % nstage
        const int tile = first + k;
        unsigned char* buf = smem_w + (k % nstage) * BUF;
        const int b = tile / tiles_img, rem = tile - b * tiles_img, ty = rem / tiles_x;
        const int ty0 = ty * TH, tx0 = (rem - ty * tiles_x) * kTW;
#pragma unroll 2
        for (int i = tid; i < cog * TPX; i += 256) {
            const int grp = i >= TPX, pix = i - grp * TPX;
            const size_t p = ((size_t)b * H + ty0 + pix / kTW) * W + tx0 + pix % kTW;
            cp_async16(buf + (size_t)(grp * TPX + pix) * 16, dy + p * cout + co0 + grp * 8, true);
        }
        unsigned char* ins = buf + (size_t)2 * TPX * 16;
#pragma unroll 2
        for (int pix = tid; pix < HALO; pix += 256) {
            const int hy = pix / kTileW;
            const int y = ty0 + hy - 1, x = tx0 + (pix - hy * kTileW) - 1;
            const bool inside = y >= 0 && y < H && x >= 0 && x < W;
            const size_t p = inside ? ((size_t)b * H + y) * W + x : 0;
            if constexpr (PLANES) {
                uint4 v = make_uint4(0, 0, 0, 0);
                if (inside) v.x = pack2(__float2bfloat16_rn(pf[p]), __float2bfloat16_rn(pg[p]));
                *reinterpret_cast<uint4*>(ins + (size_t)pix * 16) = v;
            } else {
                const bf16* s0 = in0 + p * c0;
                const bf16* s1 = in1 + p * c1 - c0;
#pragma unroll 1
                for (int grp = 0; grp < ngr; ++grp) {
                    const int c = ci_base + grp * 8;
                    cp_async16(ins + (size_t)(grp * HALO + pix) * 16, c < c0 ? s0 + c : s1 + c, inside);
                }
            }
        }
    };

    float acc[9][4];
#pragma unroll
    for (int k = 0; k < 9; ++k)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[k][j] = 0.f;

    // ldmatrix row addresses: A matrices (out group lane/8 & 1, pixels + 8 (lane/8 >> 1)); B: pixel lane
    const int a_row = ((lane >> 3) & 1) * TPX + ((lane >> 4) << 3) + (lane & 7);
    for (int k = 0; k < nstage - 1; ++k) {
        if (k < n) stage(k);
        cp_async_commit();
    }
    for (int it = 0; it < n; ++it) {
        if (it + nstage - 1 < n) stage(it + nstage - 1);
        cp_async_commit();
        cp_async_wait_n(nstage - 1);
        __syncthreads();
        const unsigned char* buf = smem_w + (it % nstage) * BUF;
        const unsigned char* ins = buf + (size_t)2 * TPX * 16 + (size_t)wc * HALO * 16;
        if (wc < ngr) {
#pragma unroll 1
            for (int row = wr; row < TH; row += NRG) {
                uint32_t a0[4], a1[4];
                ldsm_x4_trans(a0, buf + (size_t)(a_row + row * kTW) * 16);
                ldsm_x4_trans(a1, buf + (size_t)(a_row + row * kTW + 16) * 16);
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) {
                    const int ky = tap / 3, kx = tap % 3;
                    uint32_t bb[4];
                    ldsm_x4_trans(bb, ins + (size_t)((row + ky) * kTileW + kx + lane) * 16);
                    mma16816(acc[tap], a0, bb);
                    mma16816(acc[tap], a1, bb + 2);
                }
            }
        }
        __syncthreads();
    }
    // acc[tap][2 h + j]: output channel co0 + g + 8 h, input channel ci0 + 2 t + j.  With several
    // row groups, their accumulators meet in shared memory and are added in row-group order.
    float* o = part + (size_t)chunk * cout * 9 * cin;
    if constexpr (NRG == 1) {
        if (wc < ngr) {
            const int ci0 = ci_base + wc * 8;
#pragma unroll
            for (int tap = 0; tap < 9; ++tap)
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int co = co0 + g + 8 * (k >> 1), ci = ci0 + 2 * t + (k & 1);
                    if (co < cout && ci < cin) o[((size_t)co * 9 + tap) * cin + ci] = acc[tap][k];
                }
        }
    } else {
        float* red = reinterpret_cast<float*>(smem_w);
#pragma unroll
        for (int k = 0; k < 36; ++k) red[(warp * 36 + k) * 32 + lane] = acc[k / 4][k % 4];
        __syncthreads();
        for (int e = tid; e < ngr * 36 * 32; e += 256) {
            const int gi = e / (36 * 32), k = (e / 32) % 36, ln = e % 32;
            float sum = 0.f;
            for (int r = 0; r < NRG; ++r) sum += red[((r * NG + gi) * 36 + k) * 32 + ln];
            const int co = co0 + (ln >> 2) + 8 * ((k & 3) >> 1), ci = ci_base + gi * 8 + 2 * (ln & 3) + (k & 1);
            if (co < cout && ci < cin) o[((size_t)co * 9 + (k >> 2)) * cin + ci] = sum;
        }
    }
}

// Weight gradient as a flat GEMM over pixels (the layers k_conv3x3_gemm serves): dW[co][k] =
// sum_p dy[p][co] A[p][k], A the im2col of the layer input.  M = 16 output channels, N = 8 k (one
// item), K = 16 pixels.  A CTA owns kWM output channels (blockIdx.y), kWI items (blockIdx.z) and a
// chunk of kWP-pixel tiles (blockIdx.x); per tile, dy (kWP pixels x kWM channels) and the im2col
// block (kWI items x kWP pixels) arrive by cp.async through a ring of kWStages slots, and
// ldmatrix.trans gives the channel-by-pixel fragments.  Warps: 2 along output channels x 4 along
// items (4 items each).  The CTA's sums go to part[chunk] in the layout of k_wgrad, which
// k_wgrad_reduce adds in chunk order.  Requires B H W to be a multiple of kWP and cout of kWM.
constexpr int kWM = 32, kWI = 16, kWP = 64, kWStages = 3;
constexpr size_t kGemmWgradSlot = (size_t)(kWM / 8 + kWI) * kWP * 16;
constexpr size_t kGemmWgradSmem = kWStages * kGemmWgradSlot;

__global__ void __launch_bounds__(256) k_wgrad_gemm(const bf16* __restrict__ dy, int cout,
                                                    const bf16* __restrict__ in0, int c0,
                                                    const bf16* __restrict__ in1, int c1, int B, int H, int W,
                                                    int tiles_per_chunk, float* __restrict__ part) {
    extern __shared__ __align__(128) unsigned char smem_gw[];
    const int cin = c0 + c1, G = cin / 8, NI = 9 * G, HW = H * W, ntiles = B * HW / kWP;
    const int co0 = blockIdx.y * kWM, it0 = blockIdx.z * kWI;
    const int first = blockIdx.x * tiles_per_chunk, n = min(tiles_per_chunk, ntiles - first);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    const int wm = warp & 1, wi = warp >> 1;

    auto stage = [&](int k) {   // the k-th tile of this CTA's chunk into ring slot k % kWStages
        unsigned char* Ds = smem_gw + (size_t)(k % kWStages) * kGemmWgradSlot;   // [co group][px][16 B]
        unsigned char* As = Ds + (size_t)(kWM / 8) * kWP * 16;                    // [item][px][16 B]
        const int p0 = (first + k) * kWP;
        for (int e = tid; e < (kWM / 8) * kWP; e += 256) {
            const int cg = e / kWP, px = e - cg * kWP;
            cp_async16(Ds + (size_t)e * 16, dy + (size_t)(p0 + px) * cout + co0 + cg * 8, true);
        }
        // each thread gathers for one pixel (decoded once per tile) and every (256 / kWP)-th item
        const int px = tid % kWP, p = p0 + px, b = p / HW, r = p - b * HW, y = r / W, x = r - y * W;
#pragma unroll
        for (int li = tid / kWP; li < kWI; li += 256 / kWP) {
            const int item = it0 + li;
            const int tap = item < NI ? item / G : 0, grp = item - tap * G;
            const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
            const bool inside = item < NI && yy >= 0 && yy < H && xx >= 0 && xx < W;
            const size_t q = inside ? ((size_t)b * H + yy) * W + xx : 0;
            const int ch = inside ? grp * 8 : 0;
            cp_async16(As + (size_t)(li * kWP + px) * 16, ch < c0 ? in0 + q * c0 + ch : in1 + q * c1 + (ch - c0),
                       inside);
        }
    };

    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    const int mi = lane >> 3, r8 = lane & 7;
    // A (dy^T): matrices (channels 0-7 | 8-15) x (pixels 0-7 | 8-15); B: (pixels 0-7 | 8-15) x (item a | a+1)
    const int a_off = (wm * 2 + (mi & 1)) * kWP + (mi >> 1) * 8 + r8;
    const int b_off = (4 * wi + (mi >> 1)) * kWP + (mi & 1) * 8 + r8;
    for (int k = 0; k < kWStages - 1; ++k) {
        if (k < n) stage(k);
        cp_async_commit();
    }
    for (int it = 0; it < n; ++it) {
        if (it + kWStages - 1 < n) stage(it + kWStages - 1);
        cp_async_commit();
        cp_async_wait_n(kWStages - 1);
        __syncthreads();
        const unsigned char* Ds = smem_gw + (size_t)(it % kWStages) * kGemmWgradSlot;
        const unsigned char* As = Ds + (size_t)(kWM / 8) * kWP * 16;
#pragma unroll
        for (int s = 0; s < kWP / 16; ++s) {
            uint32_t a[4], b01[4], b23[4];
            ldsm_x4_trans(a, Ds + (size_t)(a_off + 16 * s) * 16);
            ldsm_x4_trans(b01, As + (size_t)(b_off + 16 * s) * 16);
            ldsm_x4_trans(b23, As + (size_t)(b_off + 2 * kWP + 16 * s) * 16);
            mma16816(acc[0], a, b01);
            mma16816(acc[1], a, b01 + 2);
            mma16816(acc[2], a, b23);
            mma16816(acc[3], a, b23 + 2);
        }
        __syncthreads();
    }
    // acc[i][j]: output channel co0 + 16 wm + g (+8 for j >= 2), item it0 + 4 wi + i, channel
    // 2 t + (j & 1) of that item's group
    float* o = part + (size_t)blockIdx.x * cout * 9 * cin;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int item = it0 + 4 * wi + i;
        if (item >= NI) continue;
        const int tap = item / G, ci0 = (item - tap * G) * 8;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int co = co0 + wm * 16 + g + 8 * (j >> 1), ci = ci0 + 2 * t + (j & 1);
            o[((size_t)co * 9 + tap) * cin + ci] = acc[i][j];
        }
    }
}

// dW (PyTorch layout [co][ci][3][3]) = sum over chunks of part[chunk][co][tap][ci] in chunk order.
// A block covers 32 consecutive entries; its 8 warps take every 8th chunk and are added in order.
__global__ void __launch_bounds__(256) k_wgrad_reduce(const float* __restrict__ part, int nchunks, int cout,
                                                      int cin, float* __restrict__ dw) {
    __shared__ float red[8][33];
    const int total = cout * 9 * cin;
    const int k = blockIdx.x * 32 + (threadIdx.x & 31), s = threadIdx.x >> 5;
    float acc = 0.f;
    if (k < total)
        for (int i = s; i < nchunks; i += 8) acc += part[(size_t)i * total + k];
    red[s][threadIdx.x & 31] = acc;
    __syncthreads();
    if (threadIdx.x < 32 && k < total) {
        float r = 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w) r += red[w][threadIdx.x];
        const int ci = k % cin, tap = (k / cin) % 9, co = k / (9 * cin);
        dw[((size_t)co * cin + ci) * 9 + tap] = r;
    }
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
