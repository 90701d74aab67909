// Forward kernels of the decoupled Fourier pose search (Alg. 1) for sm_103a.
//
// Per size group of B pairs the search is eight launches on one stream:
//   k_s1_rows   Hann window + real row FFTs of f and g (two real rows per complex FFT)
//   k_s1_cols   column FFTs, band-pass and |.|                       -> magnitudes [u][v]
//   k_angle     bilinear Cart2Pol of both magnitudes + FFT along angle, summed over radii
//   k_theta     inverse FFT along angle -> c_theta, z-score, softmax, expectation -> theta
//   k_s2_rows   bilinear Rotate of f by theta (on load) + ZeroPad + real row FFTs of f' and g
//   k_s2_cols   column FFTs of f' and g, conj(F') G, inverse column FFT, keep the N lag rows
//   k_s2_c2r    inverse real row FFTs, keep the N lag columns -> c_xy + block statistics
//   k_sxy       z-score, softmax and expectation over c_xy -> (t_x, t_y)
// Every FFT runs in shared memory (fft.cuh); HBM sees each spectrum once per pass.
#include <cfloat>
#include <cstdint>

#include "common.cuh"
#include "dev_util.cuh"

namespace fmbym {

// ---------------------------------------------------------------------------------------------
// stage 1
// ---------------------------------------------------------------------------------------------

// Hann-windowed real row FFTs of f (z = 0) and g (z = 1).  Rows 2k and 2k+1 share one complex
// FFT; the output row keeps u in [0, N/2) with the real DC and Nyquist values packed in u = 0.
// The first pass takes the windowed samples straight from global memory.
template <int N>
__global__ void __launch_bounds__(kThreads) k_s1_rows(DevPlan p, const long long* __restrict__ tab,
                                                      const float* __restrict__ f, const float* __restrict__ g,
                                                      float2* __restrict__ s1, int B) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    constexpr int T = FftPlan<N>::T, FPC = kThreads / T, SL = spad(N), W = N / 2;
    extern __shared__ float2 sm[];
    const int q = blockIdx.y, s = blockIdx.z, r0 = blockIdx.x * FPC * 2;
    const int k = threadIdx.x / T, j = threadIdx.x % T, r = r0 + 2 * k;
    const float* __restrict__ rp = (s ? g : f) + tab[3 * q] + (size_t)r * N;
    const float wa = p.window ? __ldg(&p.win[r]) : 1.f, wb = p.window ? __ldg(&p.win[r + 1]) : 1.f;
    first_pass_global<N>(sm + k * SL, 1, j, [&](int x) {
        const float wx = p.window ? __ldg(&p.win[x]) : 1.f;
        return make_float2(__ldg(rp + x) * (wa * wx), __ldg(rp + N + x) * (wb * wx));
    });
    __syncthreads();
    fft_passes_from<N, -1, 2>(sm + k * SL, 1, j, p.tw_n);
    float2* out = s1 + (size_t)(s * B + q) * N * W;
    for (int idx = threadIdx.x; idx < FPC * W; idx += kThreads) {
        const int kk = idx / W, u = idx % W, row = r0 + 2 * kk;
        const float2* Z = sm + kk * SL;
        const float2 zu = Z[spad(u)], zm = Z[spad(u == 0 ? W : N - u)];
        out[(size_t)row * W + u] = unpack_half(zu, zm, u == 0, false);
        out[(size_t)(row + 1) * W + u] = unpack_half(zu, zm, u == 0, true);
    }
}

// Column FFTs of the packed row spectra, band-pass and magnitude.  Column 0 holds the DC and
// Nyquist columns as one complex sequence; they are separated after the transform.  Output is
// the u-major half plane m[u][v], u in [0, N/2], v in [0, N), with the magnitudes of f and g of a
// pair interleaved (float2 per element) for the Cart2Pol gather.  With ph non-NULL the band-limited
// unit phasors F/|F| (0 outside the band or where F = 0) are kept for the adjoint, same layout.
template <int N>
__global__ void __launch_bounds__(kThreads) k_s1_cols(DevPlan p, const float2* __restrict__ s1,
                                                      float* __restrict__ mt, float2* __restrict__ ph, int B) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    constexpr int T = FftPlan<N>::T, C = kThreads / T, ES = C + 1, W = N / 2;
    extern __shared__ float2 sm[];
    const int q = blockIdx.y, s = blockIdx.z, u0 = blockIdx.x * C;
    const float2* in = s1 + (size_t)(s * B + q) * N * W;
    for (int idx = threadIdx.x; idx < N * C; idx += kThreads) {
        const int v = idx / C, c = idx % C;
        cp_async8(&sm[spad(v) * ES + c], &in[(size_t)v * W + u0 + c]);
    }
    cp_async_wait_all();
    __syncthreads();
    fft<N, -1>(sm + threadIdx.x / T, ES, threadIdx.x % T, true, p.tw_n);
    float* out = mt + (size_t)q * (W + 1) * N * 2 + s;   // (f, g) pairs: this scan's half of each
    float2* pho = ph ? ph + (size_t)(s * B + q) * (W + 1) * N : nullptr;
    // |z| within the band (else 0), and the phasor z / |z| there
    auto mag = [&](float2 z, int m2, size_t at) {
        const bool in_band = m2 >= p.m_lo && m2 <= p.m_hi;
        const float a = in_band ? sqrtf(fmaf(z.x, z.x, z.y * z.y)) : 0.f;
        out[2 * at] = a;
        if (pho) pho[at] = a > 0.f ? make_float2(z.x / a, z.y / a) : make_float2(0.f, 0.f);
    };
    for (int idx = threadIdx.x; idx < C * N; idx += kThreads) {
        const int cc = idx / N, v = idx % N;
        const int vs = v <= W ? v : v - N;
        const float2 z = sm[spad(v) * ES + cc];
        if (u0 + cc == 0) {
            const float2 zm = sm[spad((N - v) & (N - 1)) * ES + cc];
            mag(make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y)), vs * vs, v);
            mag(make_float2(0.5f * (z.y + zm.y), -0.5f * (z.x - zm.x)), vs * vs + W * W, (size_t)W * N + v);
        } else {
            const int u = u0 + cc;
            mag(z, vs * vs + u * u, (size_t)u * N + v);
        }
    }
}

// ---------------------------------------------------------------------------------------------
// stage 1 for the odd sides 127, 255, 511 (Sec. IV-B resolutions): the N-point DFTs by Bluestein
// ---------------------------------------------------------------------------------------------

// Hann-windowed row DFTs of an odd-sided scan (f for z = 0, g for z = 1), two real rows per complex
// DFT: Z = DFT_N(x_r + i x_{r+1}) gives X_r[u] = (Z[u] + conj Z[N - u]) / 2 and
// X_{r+1}[u] = (Z[u] - conj Z[N - u]) / 2i for u in [0, (N - 1)/2]; an odd N has no Nyquist
// column, so the packed rows hold (N + 1)/2 complex values, u = 0 the real DC value.  The last
// pair of rows has no second row (it reads as zero).
template <int N, int M>
__global__ void __launch_bounds__(kThreads) k_s1_rows_odd(DevPlan p, const long long* __restrict__ tab,
                                                          const float* __restrict__ f, const float* __restrict__ g,
                                                          float2* __restrict__ s1, int B) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    constexpr int T = FftPlan<M>::T, FPC = kThreads / T, SL = spad(M), W = (N + 1) / 2;
    extern __shared__ float2 sm[];
    const int q = blockIdx.y, s = blockIdx.z, r0 = blockIdx.x * FPC * 2;
    const int k = threadIdx.x / T, j = threadIdx.x % T, r = r0 + 2 * k;
    const bool oka = r < N, okb = r + 1 < N;
    const float* __restrict__ rp = (s ? g : f) + tab[3 * q] + (size_t)r * N;
    const float wa = oka ? (p.window ? __ldg(&p.win[r]) : 1.f) : 0.f;
    const float wb = okb ? (p.window ? __ldg(&p.win[r + 1]) : 1.f) : 0.f;
    bluestein<M>(sm + k * SL, 1, j, N, p, [&](int x) {
        const float wx = p.window ? __ldg(&p.win[x]) : 1.f;
        return make_float2(oka ? __ldg(rp + x) * (wa * wx) : 0.f, okb ? __ldg(rp + N + x) * (wb * wx) : 0.f);
    });
    float2* out = s1 + (size_t)(s * B + q) * N * W;
    for (int idx = threadIdx.x; idx < FPC * W; idx += kThreads) {
        const int kk = idx / W, u = idx % W, row = r0 + 2 * kk, um = u == 0 ? 0 : N - u;
        const float2* Z = sm + kk * SL;
        const float2 zu = c_cjmul(__ldg(&p.chirp[u]), Z[spad(u)]);
        const float2 zm = c_cjmul(__ldg(&p.chirp[um]), Z[spad(um)]);
        if (row < N)
            out[(size_t)row * W + u] = u == 0 ? make_float2(zu.x, 0.f)
                                              : make_float2(0.5f * (zu.x + zm.x), 0.5f * (zu.y - zm.y));
        if (row + 1 < N)
            out[(size_t)(row + 1) * W + u] = u == 0 ? make_float2(zu.y, 0.f)
                                                    : make_float2(0.5f * (zu.y + zm.y), -0.5f * (zu.x - zm.x));
    }
}

// Column DFTs of the packed row spectra of an odd side (every column u in [0, (N - 1)/2] is an
// ordinary complex column), band-pass, magnitude and, with ph non-NULL, the unit phasors kept for
// the adjoint: the layout of k_s1_cols, u-major [(N + 1)/2][N] with (f, g) interleaved.
template <int N, int M>
__global__ void __launch_bounds__(kThreads) k_s1_cols_odd(DevPlan p, const float2* __restrict__ s1,
                                                          float* __restrict__ mt, float2* __restrict__ ph, int B) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    constexpr int T = FftPlan<M>::T, C = kThreads / T, ES = C + 1, W = (N + 1) / 2;
    extern __shared__ float2 sm[];
    const int q = blockIdx.y, s = blockIdx.z, u0 = blockIdx.x * C;
    const int c = threadIdx.x % C, j = threadIdx.x / C, u = u0 + c;
    const float2* in = s1 + (size_t)(s * B + q) * N * W;
    bluestein<M>(sm + c, ES, j, N, p, [&](int v) {
        return u < W ? __ldg(&in[(size_t)v * W + u]) : make_float2(0.f, 0.f);
    });
    float* out = mt + (size_t)q * W * N * 2 + s;   // (f, g) pairs: this scan's half of each
    float2* pho = ph ? ph + (size_t)(s * B + q) * W * N : nullptr;
    for (int idx = threadIdx.x; idx < C * N; idx += kThreads) {
        const int cc = idx / N, v = idx % N, uu = u0 + cc;
        if (uu >= W) continue;
        const float2 z = c_cjmul(__ldg(&p.chirp[v]), sm[spad(v) * ES + cc]);
        const int vs = v <= N / 2 ? v : v - N, m2 = vs * vs + uu * uu;
        const bool in_band = m2 >= p.m_lo && m2 <= p.m_hi;
        const float a = in_band ? sqrtf(fmaf(z.x, z.x, z.y * z.y)) : 0.f;
        const size_t at = (size_t)uu * N + v;
        out[2 * at] = a;
        if (pho) pho[at] = a > 0.f ? make_float2(z.x / a, z.y / a) : make_float2(0.f, 0.f);
    }
}

// Cart2Pol of both magnitudes for RC radii, packed as z[a] = A_f[a] + i A_g[a], FFT along
// angle, then S[k] = sum_r conj(A^_f[k, r]) A^_g[k, r] for this chunk of radii.  The inverse FFT of
// S summed over chunks is the circular correlation along angle summed over radius (Eq. 7).
// Threads are radius-fastest (rr = tid mod RC): the polar table reads are contiguous, the first FFT
// pass takes the bilinear samples straight from the gather, and the sum over radii is a shuffle
// reduction over the RC lanes that hold one k.
template <int NT, int RC>
__global__ void __launch_bounds__(FftPlan<NT>::T * RC) k_angle(DevPlan p, const float* __restrict__ mt,
                                                                       float2* __restrict__ sp,
                                                                       float2* __restrict__ ahat, int B) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    constexpr int T = FftPlan<NT>::T, ES = RC;
    static_assert(RC == 8 || RC == 16, "the shuffle sum runs over aligned groups of RC lanes");
    extern __shared__ float2 sm[];
    const int q = blockIdx.y, ch = blockIdx.x, n = p.n, W = n / 2;
    const int rr = threadIdx.x % RC, j = threadIdx.x / RC, r = ch * RC + rr;
    const float2* m2 = reinterpret_cast<const float2*>(mt) + (size_t)q * (W + 1) * n;   // (f, g) pairs
    const bool live = r < p.nr;
    first_pass_global<NT>(sm + rr, ES, j, [&](int a) {
        float2 z = make_float2(0.f, 0.f);
        if (live) {
            const PolarSample ps = p.polar[a * p.nr + r];
            const float w00 = (1.f - ps.fy) * (1.f - ps.fx), w01 = (1.f - ps.fy) * ps.fx;
            const float w10 = ps.fy * (1.f - ps.fx), w11 = ps.fy * ps.fx;
            const float2 v00 = mag2_at(m2, n, ps.y0, ps.x0), v01 = mag2_at(m2, n, ps.y0, ps.x0 + 1);
            const float2 v10 = mag2_at(m2, n, ps.y0 + 1, ps.x0), v11 = mag2_at(m2, n, ps.y0 + 1, ps.x0 + 1);
            z.x = w00 * v00.x + w01 * v01.x + w10 * v10.x + w11 * v11.x;
            z.y = w00 * v00.y + w01 * v01.y + w10 * v10.y + w11 * v11.y;
        }
        return z;
    });
    __syncthreads();
    fft_passes_from<NT, -1, 2>(sm + rr, ES, j, p.tw_t);
    float2* out = sp + ((size_t)q * gridDim.x + ch) * NT;
    const unsigned grp = ((1u << RC) - 1u) << (threadIdx.x & (32 - RC));   // the RC lanes of this thread's k
    if (p.angle_score == 1) {
        // radial-mean score: the transform is linear, so the chunk's share of the transform of the
        // radial sums is the sum of its columns' transforms
#pragma unroll 4
        for (int m = 0; m < 16; ++m) {
            const int k = j + T * m;
            float2 z = sm[spad(k) * ES + rr];
#pragma unroll
            for (int o = RC / 2; o > 0; o >>= 1) {
                z.x += __shfl_xor_sync(grp, z.x, o);
                z.y += __shfl_xor_sync(grp, z.y, o);
            }
            if (rr == 0) out[k] = z;
        }
        return;
    }
#pragma unroll 4
    for (int m = 0; m < 16; ++m) {
        const int k = j + T * m, km = k == 0 ? 0 : NT - k;
        const float2 z = sm[spad(k) * ES + rr], zm = sm[spad(km) * ES + rr];
        if (ahat && live) ahat[((size_t)q * NT + k) * p.nr + r] = z;   // kept for the adjoint
        const float ax = 0.5f * (z.x + zm.x), ay = 0.5f * (z.y - zm.y);
        const float bx = 0.5f * (z.y + zm.y), by = -0.5f * (z.x - zm.x);
        float sx = ax * bx + ay * by, sy = ax * by - ay * bx;
#pragma unroll
        for (int o = RC / 2; o > 0; o >>= 1) {
            sx += __shfl_xor_sync(grp, sx, o);
            sy += __shfl_xor_sync(grp, sy, o);
        }
        if (rr == 0) out[k] = make_float2(sx, sy);
    }
}

// Sum the chunk spectra, inverse FFT along angle -> c_theta (lag order), then the soft-argmax of
// Alg. 1 over the angle candidates k delta_theta, delta_theta = pi / n_theta.
template <int NT>
__global__ void __launch_bounds__(256) k_theta(DevPlan p, const float2* __restrict__ sp, int nch,
                                               const long long* __restrict__ tab, float* __restrict__ th,
                                               float* __restrict__ pose, float* __restrict__ c_theta,
                                               float* __restrict__ ct, float2* __restrict__ ahat) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    constexpr int T = FftPlan<NT>::T;
    __shared__ float2 z[spad(NT)];
    __shared__ float c[NT];
    __shared__ float red[32], red2[64];
    const int q = blockIdx.x;
    // one CTA per pair reads all nch chunk spectra: 16 loads in flight per thread and bin (the
    // sum keeps the chunk order)
    for (int k = threadIdx.x; k < NT; k += blockDim.x) {
        float sx = 0.f, sy = 0.f;
        for (int h0 = 0; h0 < nch; h0 += 16) {
            float2 v[16];
#pragma unroll
            for (int u = 0; u < 16; ++u)
                if (h0 + u < nch) v[u] = sp[((size_t)q * nch + h0 + u) * NT + k];
#pragma unroll
            for (int u = 0; u < 16; ++u)
                if (h0 + u < nch) {
                    sx += v[u].x;
                    sy += v[u].y;
                }
        }
        z[spad(k)] = make_float2(sx, sy);
    }
    __syncthreads();
    if (p.angle_score == 1) {
        // z holds Z = M^_f + i M^_g, the transform of the radial sums of A_f + i A_g: keep it for the
        // adjoint, separate the two with the mirror k <-> n - k and form conj(M^_f) M^_g / n_r
        float2 sk[(NT + 255) / 256];
#pragma unroll
        for (int m = 0; m < (NT + 255) / 256; ++m) {
            const int k = threadIdx.x + 256 * m;
            if (k < NT) {
                const float2 a = z[spad(k)], b = z[spad(k == 0 ? 0 : NT - k)];
                if (ahat) ahat[((size_t)q * NT + k) * p.nr] = a;
                const float ax = 0.5f * (a.x + b.x), ay = 0.5f * (a.y - b.y);
                const float bx = 0.5f * (a.y + b.y), by = -0.5f * (a.x - b.x);
                const float inr = 1.f / (float)p.nr;
                sk[m] = make_float2((ax * bx + ay * by) * inr, (ax * by - ay * bx) * inr);
            }
        }
        __syncthreads();
#pragma unroll
        for (int m = 0; m < (NT + 255) / 256; ++m) {
            const int k = threadIdx.x + 256 * m;
            if (k < NT) z[spad(k)] = sk[m];
        }
        __syncthreads();
    }
    fft<NT, +1>(z, 1, threadIdx.x, threadIdx.x < T, p.tw_t);
    float lsum = 0.f, lmax = -FLT_MAX;
    for (int i = threadIdx.x; i < NT; i += blockDim.x) {
        const float v = z[spad((i - NT / 2 + NT) % NT)].x * (1.f / NT);
        c[i] = v;
        lsum += v;
        lmax = fmaxf(lmax, v);
    }
    // sum and maximum in one block reduction
    {
        lsum = warp_sum(lsum);
        lmax = warp_max(lmax);
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
        if (lane == 0) {
            red[wid] = lsum;
            red2[wid] = lmax;
        }
        __syncthreads();
        if (wid == 0) {
            float a = lane < nw ? red[lane] : 0.f, b = lane < nw ? red2[lane] : -FLT_MAX;
            a = warp_sum(a);
            b = warp_max(b);
            if (lane == 0) {
                red[0] = a;
                red2[0] = b;
            }
        }
        __syncthreads();
        lsum = red[0];
        lmax = red2[0];
        __syncthreads();
    }
    const float mean = lsum * (1.f / NT);
    const float cmax = lmax;
    float lvar = 0.f;
    for (int i = threadIdx.x; i < NT; i += blockDim.x) lvar += (c[i] - mean) * (c[i] - mean);
    const float sd = sqrtf(block_reduce<false>(lvar, red) * (1.f / NT));
    const float inv = p.score_norm == 1 ? 1.f / p.temp_theta : (sd > 0.f ? 1.f / (sd * p.temp_theta) : 0.f);
    float le = 0.f, lek = 0.f;
    for (int i = threadIdx.x; i < NT; i += blockDim.x) {
        const float e = expf((c[i] - cmax) * inv);
        le += e;
        lek += e * (float)(i - NT / 2);
    }
    float sums[2] = {le, lek};
    block_sum_n<2>(sums, red2);
    const float se = sums[0], sek = sums[1];
    for (int i = threadIdx.x; i < NT; i += blockDim.x) ct[(size_t)q * NT + i] = c[i];
    if (c_theta) {
        float* out = c_theta + tab[3 * q + 1];
        for (int i = threadIdx.x; i < NT; i += blockDim.x) out[i] = c[i];
    }
    if (threadIdx.x == 0) {
        const float theta = (float)((double)sek / (double)se * (3.14159265358979323846 / NT));
        pose[3 * tab[3 * q + 2]] = theta;
        double sd_, cd_;
        sincos((double)theta, &sd_, &cd_);
        const float ch = (float)cd_, sh = (float)sd_;
        float* t = th + 8 * q;
        t[0] = theta;
        t[1] = ch;
        t[2] = (float)(cd_ - (double)ch);
        t[3] = sh;
        t[4] = (float)(sd_ - (double)sh);
    }
}

// ---------------------------------------------------------------------------------------------
// stage 2
// ---------------------------------------------------------------------------------------------

// Rows of the rotated source f' (z = 0, rotation on load) and of g (z = 1), zero-padded to P,
// real row FFTs packed two rows per complex FFT, output u in [0, P/2) (DC/Nyquist packed in 0).
// Under Alg. 1's own stage 2 (rotate_target 1) f is read as it is and g is turned back by theta.
// The first pass takes its inputs straight from the gather (no staging in shared memory).
// ODD: the scan side is N - 1 (odd) inside this kernel's frame N: the scan's rows and columns are
// read with stride N - 1, its last frame row and column are zero, and Rotate turns about (N - 1)/2.
template <int N, int P, bool ODD>
__global__ void __launch_bounds__(tpb_for(P), P == 768 ? 6 : 65536 / (tpb_for(P) * 64)) k_s2_rows(DevPlan p, const long long* __restrict__ tab,
                                                        const float* __restrict__ f, const float* __restrict__ g,
                                                        const float* __restrict__ th, float2* __restrict__ s2, int B) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    constexpr int T = FftPlan<P>::T, TPB = tpb_for(P), FPC = TPB / T, SL = spad(P), W = P / 2;
    constexpr int NI = ODD ? N - 1 : N;   // the scan side
    extern __shared__ float2 sm[];
    const int q = blockIdx.y, s = blockIdx.z, r0 = blockIdx.x * FPC * 2;
    const int k = threadIdx.x / T, j = threadIdx.x % T;
    const int r = r0 + 2 * k;                                 // rows r and r + 1
    const bool okb = !ODD || r + 1 < NI;                      // row r + 1 lies in the scan
    const float* __restrict__ src = (s ? g : f) + tab[3 * q];
    if (s == p.rotate_target) {
        const float* t = th + 8 * q;
        const float sg = p.rotate_target ? -1.f : 1.f;   // g turns by -theta
        const RotFixed rf = rot_fixed(t[1], t[2], sg * t[3], sg * t[4], NI);
        // rows r and r + 1: (Y - c) steps add S to px and C to py
        const long long pxr = rf.px0 + rf.S * r, pyr = rf.py0 + rf.C * r;
        first_pass_global<P>(sm + k * SL, 1, j, [&](int x) {
            if (x >= NI) return make_float2(0.f, 0.f);
            const long long px = pxr + rf.C * x, py = pyr - rf.S * x;
            return make_float2(rotated_sample_fixed(src, NI, px, py),
                               okb ? rotated_sample_fixed(src, NI, px + rf.S, py + rf.C) : 0.f);
        });
    } else {
        const float* rp = src + (size_t)r * NI;
        first_pass_global<P>(sm + k * SL, 1, j, [&](int x) {
            return x < NI ? make_float2(__ldg(rp + x), okb ? __ldg(rp + NI + x) : 0.f) : make_float2(0.f, 0.f);
        });
    }
    __syncthreads();
    fft_passes_from<P, -1, 2>(sm + k * SL, 1, j, p.tw_p);
    float2* out = s2 + (size_t)(s * B + q) * N * W;
    for (int idx = threadIdx.x; idx < FPC * W; idx += TPB) {
        const int kk = idx / W, u = idx % W, row = r0 + 2 * kk;
        const float2* Z = sm + kk * SL;
        const float2 zu = Z[spad(u)], zm = Z[spad(u == 0 ? W : P - u)];
        out[(size_t)row * W + u] = unpack_half(zu, zm, u == 0, false);
        out[(size_t)(row + 1) * W + u] = unpack_half(zu, zm, u == 0, true);
    }
}

// Column pass of the correlation: FFT the columns of F' and G (rows >= N are the zero pad),
// multiply conj(F') G (A1), inverse FFT, keep the N lag rows s_y in [-N/2, N/2).  Column 0 holds
// the DC and Nyquist columns packed; their products are formed after separating them.
//
// Shared traffic is cut to what the middle passes need: the forward's first radix-16 pass reads
// its inputs straight from global memory, the forward's last pass, the product and the inverse's
// first pass (the inverse runs the radices in reverse order, so both touch the same butterfly
// positions) happen in registers, and the inverse's last radix-16 pass stores the kept rows
// straight to global memory.  Threads are column-fastest (c = tid mod C) over a tile of stride
// C, which makes every shared access phase free of bank conflicts and every global access a run
// of C consecutive columns.
// V: the radix order (FftPlan<P, V>).
template <int N, int P, int C, int V>
__global__ void __launch_bounds__(C * FftPlan<P>::T, col_min_blocks(P, C)) k_s2_cols(DevPlan p, const float2* __restrict__ s2,
                                                      float2* __restrict__ s3, float2* __restrict__ s2hat, int B) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    using PL = FftPlan<P, V>;
    constexpr int T = PL::T, TPB = C * T, ES = C, W = P / 2, TILE = spad(P) * ES;
    constexpr int RL = last_radix<P, V>(), NBL = P / RL;
    extern __shared__ float2 sm[];
    float2* tf = sm;
    float2* tg = sm + TILE;
    const int q = blockIdx.y, u0 = blockIdx.x * C;
    const int c = threadIdx.x % C, j = threadIdx.x / C;
    const float2* __restrict__ tw = p.tw_p;
    const float2* inf = s2 + (size_t)q * N * W + u0 + c;
    const float2* ing = s2 + (size_t)(B + q) * N * W + u0 + c;
    // forward first pass from global memory (rows >= N are the zero pad)
    first_pass_global2<P>(
        tf + c, tg + c, ES, j,
        [&](int v) { return v < N ? __ldg(inf + (size_t)v * W) : make_float2(0.f, 0.f); },
        [&](int v) { return v < N ? __ldg(ing + (size_t)v * W) : make_float2(0.f, 0.f); });
    __syncthreads();
    // the middle pass of both images: in one pair of barriers when a thread holds one butterfly of
    // it, else one image after the other (fewer live registers)
    if constexpr (PL::NP == 3) {
        if constexpr (P / PL::R2 <= T) {
            fft_pass2<P, T, PL::R2, 16, -1>(tf + c, tg + c, ES, j, tw);
        } else {
            fft_pass<P, T, PL::R2, 16, -1>(tf + c, ES, j, true, tw);
            fft_pass<P, T, PL::R2, 16, -1>(tg + c, ES, j, true, tw);
        }
    }
    // with s2hat the two transforms are kept for the adjoint ([2][B][P/2][P], column-major: the
    // adjoint's column pass reads each column's P positions in runs)
    float2* kf = s2hat ? s2hat + (size_t)q * P * W : nullptr;
    float2* kg = s2hat ? s2hat + (size_t)(B + q) * P * W : nullptr;
    if (blockIdx.x != 0) {
        fused_turn<P, 0, V>(tf + c, tg + c, ES, j, tw, [](float2 F, float2 G) { return c_cjmul(F, G); },
                         [&](int pos, float2 F, float2 G) {
                             if (kf) {
                                 kf[(size_t)(u0 + c) * P + pos] = F;
                                 kg[(size_t)(u0 + c) * P + pos] = G;
                             }
                         });
    } else {
        // the tile holding column 0: last forward pass in shared memory, then the products with
        // the DC / Nyquist split (which pairs v with P - v), then the inverse's first pass
        fft_pass2<P, T, RL, NBL, -1>(tf + c, tg + c, ES, j, tw);
        if (kf) {
            for (int idx = threadIdx.x; idx < P * C; idx += TPB) {
                const int v = idx % P, cc = idx / P;
                kf[(size_t)(u0 + cc) * P + v] = tf[spad(v) * ES + cc];
                kg[(size_t)(u0 + cc) * P + v] = tg[spad(v) * ES + cc];
            }
        }
        constexpr int PER = P * C / TPB;
        float2 qv[PER];
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            const int idx = threadIdx.x + m * TPB, v = idx / C, cc = idx % C;
            const float2 F = tf[spad(v) * ES + cc], G = tg[spad(v) * ES + cc];
            if (cc == 0) {
                const int vm = (v == 0 ? 0 : P - v);
                const float2 Fm = tf[spad(vm) * ES + cc], Gm = tg[spad(vm) * ES + cc];
                const float2 af = make_float2(0.5f * (F.x + Fm.x), 0.5f * (F.y - Fm.y));
                const float2 bf = make_float2(0.5f * (F.y + Fm.y), -0.5f * (F.x - Fm.x));
                const float2 ag = make_float2(0.5f * (G.x + Gm.x), 0.5f * (G.y - Gm.y));
                const float2 bg = make_float2(0.5f * (G.y + Gm.y), -0.5f * (G.x - Gm.x));
                const float2 p0 = c_cjmul(af, ag), pn = c_cjmul(bf, bg);
                qv[m] = make_float2(p0.x - pn.y, p0.y + pn.x);
            } else {
                qv[m] = c_cjmul(F, G);
            }
        }
        __syncthreads();
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            const int idx = threadIdx.x + m * TPB, v = idx / C, cc = idx % C;
            tg[spad(v) * ES + cc] = qv[m];
        }
        __syncthreads();
        fft_pass<P, T, RL, 1, +1>(tg + c, ES, j, true, tw);
    }
    // inverse middle and last passes; P-position pos holds lag s_y = pos (pos < P/2) or pos - P,
    // kept as lag row i = s_y + N/2 when 0 <= i < N
    float2* out = s3 + (size_t)q * N * W + u0 + c;
    inverse_rest_global<P, V>(tg + c, ES, j, tw, [&](int pos, float2 v) {
        const int i = pos < P / 2 ? pos + N / 2 : pos - P + N / 2;
        if (i >= 0 && i < N) out[(size_t)i * W] = v;
    });
}

// Inverse real row FFTs (two lag rows per complex FFT, Hermitian extension of the packed half
// rows), keep the N lag columns s_x in [-N/2, N/2), scale by 1/P^2 -> c_xy.  Each block also
// writes the mean, sum of squared deviations and maximum of its scores for the z-score.  The
// first pass builds its inputs from global memory and the last pass stores the kept columns
// straight to global memory (and to the tile, for the second statistics pass).
// ODD: the scan side is N - 1 inside this kernel's frame N; frame lag index 0 (lag -N/2, not a
// candidate of an odd side) is left out of c_xy (layout [N - 1][N - 1]) and of the statistics.
template <int N, int P, bool ODD>
__global__ void __launch_bounds__(kThreads) k_s2_c2r(DevPlan p, const long long* __restrict__ tab,
                                                     const float2* __restrict__ s3, float* __restrict__ cxy_ws,
                                                     float* __restrict__ cxy_out, float* __restrict__ st, int B) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    constexpr int T = FftPlan<P>::T, TPB = tpb_for(P), FPC = TPB / T, SL = spad(P), W = P / 2;
    constexpr int NI = ODD ? N - 1 : N, LO = ODD ? 1 : 0;   // candidates per axis; first kept frame index
    extern __shared__ float2 sm[];
    __shared__ float red[32];
    const int q = blockIdx.y, i0 = blockIdx.x * FPC * 2;
    const int k = threadIdx.x / T, j = threadIdx.x % T, i = i0 + 2 * k;
    const float2* ra = s3 + ((size_t)q * N + i) * W;
    float2* buf = sm + k * SL;
    first_pass_global<P, +1>(buf, 1, j, [&](int x) { return pack_inverse(ra, ra + W, x, P); });
    __syncthreads();
    const float scale = 1.f / ((float)P * (float)P);
    const bool oka = i >= LO;   // frame lag row i holds a candidate (row i + 1 always does)
    float* out = (cxy_out ? cxy_out + tab[3 * q] : cxy_ws + (size_t)q * NI * NI) + (size_t)(i - LO) * NI - LO;
    float lsum = 0.f, lmax = -FLT_MAX;
    // P-position pos holds lag s_x = pos (pos < P/2) or pos - P; column jj = s_x + N/2
    rest_global<P, +1>(buf, 1, j, p.tw_p, [&](int pos, float2 z) {
        if (pos < N / 2 || pos >= P - N / 2) {
            const int jj = pos < N / 2 ? pos + N / 2 : pos - P + N / 2;
            const float va = z.x * scale, vb = z.y * scale;
            if (jj >= LO) {
                if (oka) {
                    out[jj] = va;
                    lsum += va;
                    lmax = fmaxf(lmax, va);
                }
                out[NI + jj] = vb;
                lsum += vb;
                lmax = fmaxf(lmax, vb);
            }
            buf[spad(pos)] = make_float2(va, vb);   // same position the last pass read: no race
        }
    });
    const float cnt = (float)((FPC * 2 - (ODD && blockIdx.x == 0 ? 1 : 0)) * NI);
    const float mean = block_reduce<false>(lsum, red) * (1.f / cnt);
    const float bmax = block_reduce<true>(lmax, red);
    float lm2 = 0.f;
    for (int idx = threadIdx.x; idx < FPC * N; idx += TPB) {
        const int kk = idx / N, jj = idx % N, nn = (jj - N / 2 + P) % P;
        if (jj < LO) continue;
        const float2 z = sm[kk * SL + spad(nn)];
        const float da = z.x - mean, db = z.y - mean;
        lm2 += (i0 + 2 * kk >= LO ? da * da : 0.f) + db * db;
    }
    const float m2 = block_reduce<false>(lm2, red);
    if (threadIdx.x == 0) {
        float* o = st + ((size_t)q * gridDim.x + blockIdx.x) * 4;
        o[0] = mean;
        o[1] = m2;
        o[2] = bmax;
        o[3] = cnt;
    }
}

// Soft-argmax over the translation candidates (Alg. 1 stage 2): the blocks of a pair first
// combine the per-block statistics of k_s2_c2r into the mean, population std and maximum, then
// each sums e = exp((c - max) / (std T)) and its first moments over a slab of rows; the last block
// of the pair adds the slabs in order and writes (t_x, t_y) = delta_xy E[s].  It also keeps, for
// the adjoint, the statistics and the sums of e z, e z s_x and e z s_y with z = (c - mean) / std:
// with them the z-score adjoint needs no second pass over the scores (see k_b_rows).
// ODD: the scan side is N - 1 inside the frame N; the scores are the (N - 1)^2 candidates of an odd
// side, c_xy [N - 1][N - 1] at frame lags 1 .. N - 1 (lag = frame index - N/2), read one by one.
template <int N, bool ODD>
__global__ void __launch_bounds__(kThreads) k_sxy(DevPlan p, const long long* __restrict__ tab,
                                                  const float* __restrict__ cxy_ws, const float* __restrict__ cxy_out,
                                                  const float* __restrict__ st, int nblk, float* __restrict__ sx,
                                                  unsigned* __restrict__ cnt, float* __restrict__ pose,
                                                  float* __restrict__ xm, const float* __restrict__ th) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    __shared__ float red[32 * 6];
    __shared__ float stat[4];
    __shared__ bool last;
    const int q = blockIdx.y;
    constexpr int NI = ODD ? N - 1 : N;
    constexpr int ROWS = N / kSplitXY, TOT = ROWS * (N / 4), PER = (TOT + kThreads - 1) / kThreads;
    const int y0 = blockIdx.x * ROWS;
    const float* c = cxy_out ? cxy_out + tab[3 * q] : cxy_ws + (size_t)q * NI * NI;
    // the scores first (they do not depend on the statistics), so their loads overlap the
    // statistics' reduction below
    float4 vv[PER];
    if constexpr (!ODD) {
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            const int idx = threadIdx.x + m * kThreads;
            if (TOT % kThreads == 0 || idx < TOT)
                vv[m] = *reinterpret_cast<const float4*>(c + (size_t)(y0 + idx / (N / 4)) * N + (idx % (N / 4)) * 4);
        }
    }
    if (threadIdx.x < 32) {
        float mu, sd, cmax;
        xy_stats_warp(st + (size_t)q * nblk * 4, nblk, (float)NI * (float)NI, mu, sd, cmax, ODD);
        if (threadIdx.x == 0) {
            stat[0] = cmax;
            stat[1] = p.score_norm == 1 ? 1.f / p.temp_xy : (sd > 0.f ? 1.f / (sd * p.temp_xy) : 0.f);
            stat[2] = mu;
            stat[3] = sd;
        }
    }
    __syncthreads();
    const float cmax = stat[0], inv = stat[1], mu = stat[2], sd = stat[3];
    const float isd = sd > 0.f ? 1.f / sd : 0.f;
    float le = 0.f, lx = 0.f, ly = 0.f, lz = 0.f, lzx = 0.f, lzy = 0.f;
    if constexpr (ODD) {
        for (int idx = threadIdx.x; idx < ROWS * N; idx += kThreads) {
            const int yy = y0 + idx / N, xx = idx % N;
            if (yy < 1 || xx < 1) continue;
            const float v = __ldg(c + (size_t)(yy - 1) * NI + (xx - 1));
            const float e = expf((v - cmax) * inv), z = (v - mu) * isd;
            const float sxv = (float)(xx - N / 2), syv = (float)(yy - N / 2);
            le += e;
            lx += e * sxv;
            ly += e * syv;
            lz += e * z;
            lzx += e * z * sxv;
            lzy += e * z * syv;
        }
    } else {
#pragma unroll
    for (int m = 0; m < PER; ++m) {
        const int idx = threadIdx.x + m * kThreads;
        if (TOT % kThreads != 0 && idx >= TOT) break;
        const int yy = y0 + idx / (N / 4), x4 = (idx % (N / 4)) * 4;
        const float4 v = vv[m];
        const float e0 = expf((v.x - cmax) * inv), e1 = expf((v.y - cmax) * inv);
        const float e2 = expf((v.z - cmax) * inv), e3 = expf((v.w - cmax) * inv);
        const float es = (e0 + e1) + (e2 + e3);
        const float sx0 = (float)(x4 - N / 2), sy = (float)(yy - N / 2);
        const float ex = e1 + 2.f * e2 + 3.f * e3;
        le += es;
        lx += es * sx0 + ex;
        ly += es * sy;
        const float z0 = (v.x - mu) * isd, z1 = (v.y - mu) * isd, z2 = (v.z - mu) * isd, z3 = (v.w - mu) * isd;
        const float ez = (e0 * z0 + e1 * z1) + (e2 * z2 + e3 * z3);
        lz += ez;
        lzx += ez * sx0 + (e1 * z1 + 2.f * e2 * z2 + 3.f * e3 * z3);
        lzy += ez * sy;
    }
    }
    float sums[6] = {le, lx, ly, lz, lzx, lzy};
    block_sum_n<6>(sums, red);
    if (threadIdx.x == 0) {
        float* o = sx + ((size_t)q * kSplitXY + blockIdx.x) * 8;
#pragma unroll
        for (int k = 0; k < 6; ++k) o[k] = sums[k];
        __threadfence();
        last = atomicAdd(&cnt[q], 1u) == kSplitXY - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const volatile float* o = sx + (size_t)q * kSplitXY * 8;
        float a = 0.f, bx = 0.f, by = 0.f, z = 0.f, zx = 0.f, zy = 0.f;
        for (int i = 0; i < kSplitXY; ++i) {
            a += o[8 * i];
            bx += o[8 * i + 1];
            by += o[8 * i + 2];
            z += o[8 * i + 3];
            zx += o[8 * i + 4];
            zy += o[8 * i + 5];
        }
        const long long pr = tab[3 * q + 2];
        const float tpx = p.delta_xy * (bx / a), tpy = p.delta_xy * (by / a);
        if (p.rotate_target) {   // BuildSO2 / MatMul of Alg. 1: t = R(theta) t'
            const float* t = th + 8 * q;
            const float ct = t[1] + t[2], sn = t[3] + t[4];
            pose[3 * pr + 1] = ct * tpx - sn * tpy;
            pose[3 * pr + 2] = sn * tpx + ct * tpy;
        } else {
            pose[3 * pr + 1] = tpx;
            pose[3 * pr + 2] = tpy;
        }
        float* m = xm + (size_t)q * 8;
        m[0] = mu;
        m[1] = sd;
        m[2] = cmax;
        m[3] = inv;
        m[4] = a;
        m[5] = z;
        m[6] = zx;
        m[7] = zy;
        cnt[q] = 0u;
    }
}

// ---------------------------------------------------------------------------------------------
// full-circle heading (the extension of Sec. V): stage 2 at theta and at theta + pi
// ---------------------------------------------------------------------------------------------

// Keeps stage 1's heading splits and turns every pair's heading by pi: theta' = theta + pi for
// theta < 0, theta - pi otherwise (in (-pi, pi]); its cosine and sine are the negated splits.
__global__ void k_fc_flip(float* __restrict__ th, float* __restrict__ fc, int B) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= B) return;
    float* t = th + 8 * q;
    float* k = fc + 8 * q;
    const float pi = 3.14159265358979323846f;
    for (int i = 0; i < 5; ++i) k[i] = t[i];
    t[0] = t[0] < 0.f ? t[0] + pi : t[0] - pi;
    for (int i = 1; i < 5; ++i) t[i] = -t[i];
}

// The highest translation score of each pair (the maximum of the block maxima of k_s2_c2r).
__device__ __forceinline__ float fc_peak(const float* __restrict__ st, int nblk, int q) {
    float m = -FLT_MAX;
    for (int b = 0; b < nblk; ++b) m = fmaxf(m, st[((size_t)q * nblk + b) * 4 + 2]);
    return m;
}

// After the theta + pi pass: records its peak and puts stage 1's heading back.
__global__ void k_fc_restore(const float* __restrict__ st, int nblk, float* __restrict__ th, float* __restrict__ fc,
                             int B) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= B) return;
    float* k = fc + 8 * q;
    k[5] = fc_peak(st, nblk, q);
    for (int i = 0; i < 5; ++i) th[8 * q + i] = k[i];
}

// After the theta pass: where the theta + pi peak is higher (strictly), the heading turns by pi
// (th and the pose's theta); the last stage-2 pass then runs at every pair's winner.
__global__ void k_fc_select(const long long* __restrict__ tab, const float* __restrict__ st, int nblk,
                            float* __restrict__ th, const float* __restrict__ fc, float* __restrict__ pose, int B) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= B) return;
    const float* k = fc + 8 * q;
    if (k[5] > fc_peak(st, nblk, q)) {
        float* t = th + 8 * q;
        const float pi = 3.14159265358979323846f;
        t[0] = k[0] < 0.f ? k[0] + pi : k[0] - pi;
        for (int i = 1; i < 5; ++i) t[i] = -k[i];
        pose[3 * tab[3 * q + 2]] = t[0];
    }
}

// ---------------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------------

template <int L> constexpr size_t smem_rows() { return (size_t)(tpb_for(L) / FftPlan<L>::T) * spad(L) * sizeof(float2); }
template <int N> constexpr size_t smem_cols1() {
    return (size_t)spad(N) * (kThreads / FftPlan<N>::T + 1) * sizeof(float2);
}
template <int P, int C> constexpr size_t smem_cols2() { return 2 * (size_t)spad(P) * C * sizeof(float2); }
template <int NT, int RC> constexpr size_t smem_angle() { return (size_t)spad(NT) * RC * sizeof(float2); }

template <int N, int P, bool ODD>
static cudaError_t launch_stage2(const DevPlan& p, const Ws& w, int B, const long long* tab, const float* f,
                                 const float* g, float* pose, float* c_xy, cudaStream_t st);

template <int NT>
static cudaError_t launch_stage1_angle(const DevPlan& p, const Ws& w, int B, const long long* tab, float* pose,
                                       float* c_theta, cudaStream_t st) {
    const int nch = angle_chunks(p);
    w.tr->before(K_ANGLE, st);
    if (p.angle_rc == 8)
        launch_pdl(k_angle<NT, 8>, dim3(nch, B), FftPlan<NT>::T * 8, smem_angle<NT, 8>(), st, p, w.mt, w.sp, w.ahat, B);
    else
        launch_pdl(k_angle<NT, 16>, dim3(nch, B), FftPlan<NT>::T * 16, smem_angle<NT, 16>(), st, p, w.mt, w.sp, w.ahat, B);
    w.tr->before(K_THETA, st);
    launch_pdl(k_theta<NT>, B, 256, 0, st, p, w.sp, nch, tab, w.th, pose, c_theta, w.ct, w.ahat);
    return cudaGetLastError();
}

// Stage 1 of a scan side N: the power-of-two FFTs, or (M > 0) the Bluestein DFTs of an odd N.
template <int N, int M>
static void launch_stage1_spectra(const DevPlan& p, const Ws& w, int B, const long long* tab, const float* f,
                                  const float* g, cudaStream_t st) {
    if constexpr (M == 0) {
        constexpr int T1 = FftPlan<N>::T;
        w.tr->before(K_S1_ROWS, st);
        launch_pdl(k_s1_rows<N>, dim3((N / 2) / (kThreads / T1), B, 2), kThreads, smem_rows<N>(), st, p, tab, f, g, w.s1, B);
        w.tr->before(K_S1_COLS, st);
        launch_pdl(k_s1_cols<N>, dim3((N / 2) / (kThreads / T1), B, 2), kThreads, smem_cols1<N>(), st, p, w.s1, w.mt, w.phs,
                   B);
    } else {
        constexpr int TM = FftPlan<M>::T, FPC = kThreads / TM, W = (N + 1) / 2;
        static_assert(W % FPC == 0 && W % (kThreads / TM) == 0, "row pairs and columns fill whole CTAs");
        w.tr->before(K_S1_ROWS, st);
        launch_pdl(k_s1_rows_odd<N, M>, dim3(W / FPC, B, 2), kThreads, (size_t)FPC * spad(M) * sizeof(float2), st, p, tab,
                   f, g, w.s1, B);
        w.tr->before(K_S1_COLS, st);
        launch_pdl(k_s1_cols_odd<N, M>, dim3(W / (kThreads / TM), B, 2), kThreads, smem_cols1<M>(), st, p, w.s1, w.mt,
                   w.phs, B);
    }
}

// N: the scan side; NE: stage 2's frame (N, or N + 1 for odd N); M: Bluestein length (0: none).
template <int N, int NE, int M, int P>
static cudaError_t launch_np(const DevPlan& p, const Ws& w, int B, const long long* tab, const float* f,
                             const float* g, float* pose, float* c_theta, float* c_xy, cudaStream_t st) {
    constexpr bool ODD = (N & 1) != 0;
    StageRange range("fmbym forward");
    launch_stage1_spectra<N, M>(p, w, B, tab, f, g, st);
    cudaError_t e;
    if (p.nt == 128) e = launch_stage1_angle<128>(p, w, B, tab, pose, c_theta, st);
    else if (p.nt == 256) e = launch_stage1_angle<256>(p, w, B, tab, pose, c_theta, st);
    else if (p.nt == 400) e = launch_stage1_angle<400>(p, w, B, tab, pose, c_theta, st);
    else e = launch_stage1_direct(p, w, B, tab, pose, c_theta, st);   // no FFT plan: direct sums
    if (e != cudaSuccess) return e;
    if (!p.full_circle) return launch_stage2<NE, P, ODD>(p, w, B, tab, f, g, pose, c_xy, st);
    // full circle: the two candidate passes keep nothing for the adjoint and write no scores for
    // the caller; the third pass runs at each pair's winner
    Ws wc = w;
    wc.s2hat = nullptr;
    const int nb = (B + 127) / 128, nblk = c2r_blocks(p);
    launch_pdl(k_fc_flip, nb, 128, 0, st, w.th, w.fc, B);
    if ((e = launch_stage2<NE, P, ODD>(p, wc, B, tab, f, g, w.fcpose, nullptr, st)) != cudaSuccess) return e;
    launch_pdl(k_fc_restore, nb, 128, 0, st, (const float*)w.st, nblk, w.th, w.fc, B);
    if ((e = launch_stage2<NE, P, ODD>(p, wc, B, tab, f, g, pose, nullptr, st)) != cudaSuccess) return e;
    launch_pdl(k_fc_select, nb, 128, 0, st, tab, (const float*)w.st, nblk, w.th, (const float*)w.fc, pose, B);
    return launch_stage2<NE, P, ODD>(p, w, B, tab, f, g, pose, c_xy, st);
}

// The stage-2 column pass in radix order V with the size's column tile.
template <int N, int P, int V>
static void launch_s2_cols(const DevPlan& p, const Ws& w, int B, cudaStream_t st) {
    constexpr int T2 = FftPlan<P>::T, C0 = tpb_for(P) / T2;   // the default tile; the 3 * 2^k lengths
    if constexpr (P % 3 == 0) {                                  // also have half and double
        if (p.col_tile == C0 / 2)
            launch_pdl(k_s2_cols<N, P, C0 / 2, V>, dim3((P / 2) / (C0 / 2), B), (C0 / 2) * T2, smem_cols2<P, C0 / 2>(), st,
                       p, w.s2, w.s3, w.s2hat, B);
        else if (p.col_tile == 2 * C0)
            launch_pdl(k_s2_cols<N, P, 2 * C0, V>, dim3((P / 2) / (2 * C0), B), 2 * C0 * T2, smem_cols2<P, 2 * C0>(), st,
                       p, w.s2, w.s3, w.s2hat, B);
        else
            launch_pdl(k_s2_cols<N, P, C0, V>, dim3((P / 2) / C0, B), C0 * T2, smem_cols2<P, C0>(), st, p, w.s2, w.s3,
                       w.s2hat, B);
    } else {
        launch_pdl(k_s2_cols<N, P, C0, V>, dim3((P / 2) / C0, B), C0 * T2, smem_cols2<P, C0>(), st, p, w.s2, w.s3, w.s2hat,
                   B);
    }
}

// Stage 2 of Alg. 1 for the headings in w.th: Rotate, the padded correlation and the translation
// soft-argmax -> pose[.][1..2], block statistics of c_xy in w.st.  N is the frame (ODD: the scan
// side is N - 1).
template <int N, int P, bool ODD>
static cudaError_t launch_stage2(const DevPlan& p, const Ws& w, int B, const long long* tab, const float* f,
                                 const float* g, float* pose, float* c_xy, cudaStream_t st) {
    constexpr int T2 = FftPlan<P>::T, TB2 = tpb_for(P);
    w.tr->before(K_S2_ROWS, st);
    launch_pdl(k_s2_rows<N, P, ODD>, dim3((N / 2) / (TB2 / T2), B, 2), TB2, smem_rows<P>(), st, p, tab, f, g, w.th, w.s2,
               B);
    w.tr->before(K_S2_COLS, st);
    if constexpr (P % 3 == 0) {
        if (p.col_plan == 1) launch_s2_cols<N, P, 1>(p, w, B, st);
        else launch_s2_cols<N, P, 0>(p, w, B, st);
    } else {
        launch_s2_cols<N, P, 0>(p, w, B, st);
    }
    const int nblk = (N / 2) / (TB2 / T2);
    w.tr->before(K_S2_C2R, st);
    launch_pdl(k_s2_c2r<N, P, ODD>, dim3(nblk, B), TB2, smem_rows<P>(), st, p, tab, w.s3, w.cxy, c_xy, w.st, B);
    w.tr->before(K_SXY, st);
    launch_pdl(k_sxy<N, ODD>, dim3(kSplitXY, B), kThreads, 0, st, p, tab, w.cxy, c_xy, w.st, nblk, w.sx, w.cnt, pose, w.xm,
               w.th);
    w.tr->close(st);
    return cudaGetLastError();
}

cudaError_t launch_forward(const DevPlan& p, const Ws& w, int B, const long long* tab, const float* f,
                           const float* g, float* pose, float* c_theta, float* c_xy, cudaStream_t st) {
    if (B <= 0) return cudaSuccess;
    switch (p.n) {
        case 127: return launch_np<127, 128, 256, 192>(p, w, B, tab, f, g, pose, c_theta, c_xy, st);
        case 255: return launch_np<255, 256, 512, 384>(p, w, B, tab, f, g, pose, c_theta, c_xy, st);
        case 511: return launch_np<511, 512, 1024, 768>(p, w, B, tab, f, g, pose, c_theta, c_xy, st);
        case 128: return p.p == 192 ? launch_np<128, 128, 0, 192>(p, w, B, tab, f, g, pose, c_theta, c_xy, st)
                                    : launch_np<128, 128, 0, 128>(p, w, B, tab, f, g, pose, c_theta, c_xy, st);
        case 256: return p.p == 384 ? launch_np<256, 256, 0, 384>(p, w, B, tab, f, g, pose, c_theta, c_xy, st)
                                    : launch_np<256, 256, 0, 256>(p, w, B, tab, f, g, pose, c_theta, c_xy, st);
        default: return p.p == 768 ? launch_np<512, 512, 0, 768>(p, w, B, tab, f, g, pose, c_theta, c_xy, st)
                                   : launch_np<512, 512, 0, 512>(p, w, B, tab, f, g, pose, c_theta, c_xy, st);
    }
}

cudaError_t launch_forward_stage2(const DevPlan& p, const Ws& w, int B, const long long* tab, const float* f,
                                  const float* g, float* pose, float* c_xy, cudaStream_t st) {
    if (B <= 0) return cudaSuccess;
    switch (p.n) {
        case 127: return launch_stage2<128, 192, true>(p, w, B, tab, f, g, pose, c_xy, st);
        case 255: return launch_stage2<256, 384, true>(p, w, B, tab, f, g, pose, c_xy, st);
        case 511: return launch_stage2<512, 768, true>(p, w, B, tab, f, g, pose, c_xy, st);
        case 128: return p.p == 192 ? launch_stage2<128, 192, false>(p, w, B, tab, f, g, pose, c_xy, st)
                                    : launch_stage2<128, 128, false>(p, w, B, tab, f, g, pose, c_xy, st);
        case 256: return p.p == 384 ? launch_stage2<256, 384, false>(p, w, B, tab, f, g, pose, c_xy, st)
                                    : launch_stage2<256, 256, false>(p, w, B, tab, f, g, pose, c_xy, st);
        default: return p.p == 768 ? launch_stage2<512, 768, false>(p, w, B, tab, f, g, pose, c_xy, st)
                                   : launch_stage2<512, 512, false>(p, w, B, tab, f, g, pose, c_xy, st);
    }
}

template <typename K>
static cudaError_t allow_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int N, int P, bool ODD>
static cudaError_t prepare_np() {
    cudaError_t e;
    if constexpr (!ODD) {
        if ((e = allow_smem(k_s1_rows<N>, smem_rows<N>())) != cudaSuccess) return e;
        if ((e = allow_smem(k_s1_cols<N>, smem_cols1<N>())) != cudaSuccess) return e;
    }
    if ((e = allow_smem(k_s2_rows<N, P, ODD>, smem_rows<P>())) != cudaSuccess) return e;
    constexpr int C0 = tpb_for(P) / FftPlan<P>::T;
    if ((e = allow_smem(k_s2_cols<N, P, C0, 0>, smem_cols2<P, C0>())) != cudaSuccess) return e;
    if constexpr (P % 3 == 0) {
        if ((e = allow_smem(k_s2_cols<N, P, C0 / 2, 0>, smem_cols2<P, C0 / 2>())) != cudaSuccess) return e;
        if ((e = allow_smem(k_s2_cols<N, P, 2 * C0, 0>, smem_cols2<P, 2 * C0>())) != cudaSuccess) return e;
        if ((e = allow_smem(k_s2_cols<N, P, C0, 1>, smem_cols2<P, C0>())) != cudaSuccess) return e;
        if ((e = allow_smem(k_s2_cols<N, P, C0 / 2, 1>, smem_cols2<P, C0 / 2>())) != cudaSuccess) return e;
        if ((e = allow_smem(k_s2_cols<N, P, 2 * C0, 1>, smem_cols2<P, 2 * C0>())) != cudaSuccess) return e;
    }
    return allow_smem(k_s2_c2r<N, P, ODD>, smem_rows<P>());
}

template <int N, int M>
static cudaError_t prepare_odd() {
    cudaError_t e;
    constexpr int FPC = kThreads / FftPlan<M>::T;
    if ((e = allow_smem(k_s1_rows_odd<N, M>, (size_t)FPC * spad(M) * sizeof(float2))) != cudaSuccess) return e;
    return allow_smem(k_s1_cols_odd<N, M>, smem_cols1<M>());
}

const char* const kKindNames[K_COUNT] = {
    "s1_rows", "s1_cols", "angle", "theta", "s2_rows", "s2_cols", "s2_c2r", "sxy",
    "b_sxy", "b_cols", "b_rows", "b_rot", "b_theta", "b_angle", "b_s1cols", "b_s1rows", "b_c2r", "b_polT",
    "loss"};

cudaError_t prepare_forward_kernels() {
    cudaError_t e;
    if ((e = prepare_np<128, 192, false>()) != cudaSuccess) return e;
    if ((e = prepare_np<128, 128, false>()) != cudaSuccess) return e;
    if ((e = prepare_np<256, 384, false>()) != cudaSuccess) return e;
    if ((e = prepare_np<256, 256, false>()) != cudaSuccess) return e;
    if ((e = prepare_np<512, 768, false>()) != cudaSuccess) return e;
    if ((e = prepare_np<512, 512, false>()) != cudaSuccess) return e;
    if ((e = prepare_np<128, 192, true>()) != cudaSuccess) return e;
    if ((e = prepare_np<256, 384, true>()) != cudaSuccess) return e;
    if ((e = prepare_np<512, 768, true>()) != cudaSuccess) return e;
    if ((e = prepare_odd<127, 256>()) != cudaSuccess) return e;
    if ((e = prepare_odd<255, 512>()) != cudaSuccess) return e;
    if ((e = prepare_odd<511, 1024>()) != cudaSuccess) return e;
    if ((e = allow_smem(k_angle<128, 8>, smem_angle<128, 8>())) != cudaSuccess) return e;
    if ((e = allow_smem(k_angle<256, 8>, smem_angle<256, 8>())) != cudaSuccess) return e;
    if ((e = allow_smem(k_angle<400, 8>, smem_angle<400, 8>())) != cudaSuccess) return e;
    if ((e = allow_smem(k_angle<128, 16>, smem_angle<128, 16>())) != cudaSuccess) return e;
    if ((e = allow_smem(k_angle<256, 16>, smem_angle<256, 16>())) != cudaSuccess) return e;
    return allow_smem(k_angle<400, 16>, smem_angle<400, 16>());
}

}  // namespace fmbym
