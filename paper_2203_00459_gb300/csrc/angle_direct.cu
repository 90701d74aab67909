// The angle stage of Alg. 1 for angle counts without an FFT plan -- Alg. 1's own n_theta = 733
// among them: the same Cart2Pol samples, angle scores (Eq. 7, or the radial mean that Alg. 1
// prints), soft-argmax and their adjoint as the FFT route of fwd.cu / bwd.cu, with the circular
// correlation along angle evaluated as its direct sum.  Per pair n_theta^2 n_r multiply-adds
// (6.9e7 at 733 x 128), twice that in the adjoint, spread over chunks of 8 radii.
//
//   k_polar_direct  bilinear Cart2Pol of |F_f| and |F_g| -> pol[q][r][a] = (A_f, A_g)
//   k_angle_direct  c partials per chunk of radii: sum_r sum_a A_f[a,r] A_g[(a + l) mod n, r],
//                   four lags per thread over a shifted copy of A_g (register-blocked sums)
//   k_theta_direct  chunk sum, z-score, softmax, expectation -> theta (as k_theta)
//   k_b_theta_direct  soft-argmax adjoint -> d c (as k_b_theta, without the transform)
//   k_b_angle_direct  d A_f[a,r] = sum_l dc_l A_g[a + l, r], d A_g[b,r] = sum_l dc_l A_f[b - l, r]
#include <cfloat>

#include "common.cuh"
#include "dev_util.cuh"

namespace fmbym {

constexpr int kDirectMaxNT = 1024;   // largest angle count: one CTA holds every lag, four per thread
constexpr int kDirectRadii = 8;      // radii per CTA of the per-radius score

bool fft_angle_count(int nt) { return nt == 128 || nt == 256 || nt == 400; }

int angle_direct_chunks(const DevPlan& p) { return p.angle_score == 1 ? 1 : (p.nr + kDirectRadii - 1) / kDirectRadii; }

// Cart2Pol of both magnitude spectra (the gather of k_angle), radius-major: pol[q][r][a].  A CTA
// takes a tile of 32 angles x 32 radii: the sample table (angle-major, a n_r + r) is read along
// radius, the bilinear values go through shared memory, and the output is written along angle.
constexpr int kPolTile = 32;
__global__ void __launch_bounds__(256) k_polar_direct(DevPlan p, const float* __restrict__ mt,
                                                      float2* __restrict__ pol, int B) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    __shared__ float2 tile[kPolTile][kPolTile + 1];
    const int q = blockIdx.z, n = p.n, W = n / 2, nt = p.nt, nr = p.nr;
    const int a0 = blockIdx.x * kPolTile, r0 = blockIdx.y * kPolTile;
    const int lane = threadIdx.x & 31, row = threadIdx.x >> 5;   // 8 rows of 32
    const float2* m2 = reinterpret_cast<const float2*>(mt) + (size_t)q * (W + 1) * n;
#pragma unroll
    for (int k = 0; k < kPolTile / 8; ++k) {
        const int al = row + 8 * k, a = a0 + al, r = r0 + lane;
        float2 val = make_float2(0.f, 0.f);
        if (a < nt && r < nr) {
            const PolarSample ps = p.polar[a * nr + r];
            const float w00 = (1.f - ps.fy) * (1.f - ps.fx), w01 = (1.f - ps.fy) * ps.fx;
            const float w10 = ps.fy * (1.f - ps.fx), w11 = ps.fy * ps.fx;
            const float2 v00 = mag2_at(m2, n, ps.y0, ps.x0), v01 = mag2_at(m2, n, ps.y0, ps.x0 + 1);
            const float2 v10 = mag2_at(m2, n, ps.y0 + 1, ps.x0), v11 = mag2_at(m2, n, ps.y0 + 1, ps.x0 + 1);
            val = make_float2(w00 * v00.x + w01 * v01.x + w10 * v10.x + w11 * v11.x,
                              w00 * v00.y + w01 * v01.y + w10 * v10.y + w11 * v11.y);
        }
        tile[al][lane] = val;
    }
    __syncthreads();
    float2* out = pol + (size_t)q * nt * nr;
#pragma unroll
    for (int k = 0; k < kPolTile / 8; ++k) {
        const int rl = row + 8 * k, r = r0 + rl, a = a0 + lane;
        if (a < nt && r < nr) out[(size_t)r * nt + a] = tile[lane][rl];
    }
}

// 16 multiply-adds of one step: o[j] += u[4k + kk] v[x0 + 4k + kk + j], the window of v in (a, b).
__device__ __forceinline__ void circ_step(const float4 uu, const float4 a, const float4 b, float o[4]) {
    const float uv[4] = {uu.x, uu.y, uu.z, uu.w};
    const float wv[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
#pragma unroll
        for (int j = 0; j < 4; ++j) o[j] = fmaf(uv[kk], wv[kk + j], o[j]);
}

// out[x] = sum_k u[k] v[x + k] for the four outputs x = x0 .. x0 + 3 of this thread (x0 a multiple
// of 4): u zero-padded to ntp (a multiple of 4), v long enough for x0 + ntp + 3.  Each step takes
// four u at once (one broadcast float4) and slides a window of v by one float4, so 16 multiply-adds
// cost two shared loads; two steps per iteration keep the window in place (no register moves).
__device__ __forceinline__ void circ_sum4(const float* __restrict__ u, const float* __restrict__ v, int ntp,
                                          int x0, float o[4]) {
    const float4* u4 = reinterpret_cast<const float4*>(u);
    const float4* v4 = reinterpret_cast<const float4*>(v + x0);
    const int K = ntp / 4;
    float4 w0 = v4[0];
    o[0] = o[1] = o[2] = o[3] = 0.f;
    int k = 0;
#pragma unroll 1
    for (; k + 1 < K; k += 2) {
        const float4 u0 = u4[k], u1 = u4[k + 1], w1 = v4[k + 1], w2 = v4[k + 2];
        circ_step(u0, w0, w1, o);
        circ_step(u1, w1, w2, o);
        w0 = w2;
    }
    if (k < K) circ_step(u4[k], w0, v4[k + 1], o);
}

__host__ __device__ constexpr int direct_pad(int nt) { return (nt + 3) & ~3; }
inline int direct_threads(int nt) { return ((direct_pad(nt) / 4 + 31) / 32) * 32; }

// c[i] = sum_r sum_a A_f[a, r] A_g[(a + l_i) mod n, r], l_i = i - n/2, as sum_a u[a] v[a + i] with
// u = A_f (zero-padded) and v[m] = A_g[(m - n/2) mod n] over 2 ntp entries.  Thread t holds lags
// 4t .. 4t + 3.  Per-radius score: CTA x takes radii [8x, 8x + 8); radial mean: one CTA
// correlates the radial sums and scales by 1/n_r.
__global__ void __launch_bounds__(kDirectMaxNT / 4) k_angle_direct(DevPlan p, const float2* __restrict__ pol,
                                                                   float* __restrict__ part, int B) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    __shared__ __align__(16) float u[kDirectMaxNT], v[2 * kDirectMaxNT], mg[kDirectMaxNT];
    const int q = blockIdx.y, nt = p.nt, ntp = direct_pad(nt), tid = threadIdx.x, T = blockDim.x;
    const int sh = nt - nt / 2, x0 = 4 * tid;
    const float2* P = pol + (size_t)q * nt * p.nr;
    float acc[4] = {0.f, 0.f, 0.f, 0.f}, o[4];
    auto correlate = [&]() {
        __syncthreads();
        if (x0 < ntp) {
            circ_sum4(u, v, ntp, x0, o);
            for (int j = 0; j < 4; ++j) acc[j] += o[j];
        }
        __syncthreads();
    };
    if (p.angle_score == 1) {
        for (int a = tid; a < ntp; a += T) {
            float mf = 0.f, m = 0.f;
            if (a < nt)
                for (int r = 0; r < p.nr; ++r) {
                    const float2 w = P[(size_t)r * nt + a];
                    mf += w.x;
                    m += w.y;
                }
            u[a] = mf;
            mg[a] = m;
        }
        __syncthreads();
        for (int m = tid; m < 2 * ntp; m += T) v[m] = mg[(m + sh) % nt];
        correlate();
        for (int j = 0; j < 4; ++j) acc[j] *= 1.f / (float)p.nr;
    } else {
        // the next radius is fetched into registers while the current one is summed
        const int r0 = blockIdx.x * kDirectRadii, r1 = min(r0 + kDirectRadii, p.nr);
        const int tm = T % nt, i0 = (tid + sh) % nt;
        float pu[4], pv[8];
        auto fetch = [&](int r) {
            const float2* row = P + (size_t)r * nt;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int a = tid + i * T;
                pu[i] = a < nt ? row[a].x : 0.f;
            }
            int idx = i0;   // (m + n - n/2) mod n for m = tid + i T
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                pv[i] = tid + i * T < 2 * ntp ? row[idx].y : 0.f;
                idx += tm;
                if (idx >= nt) idx -= nt;
            }
        };
        if (r0 < r1) fetch(r0);
        for (int r = r0; r < r1; ++r) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (tid + i * T < ntp) u[tid + i * T] = pu[i];
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (tid + i * T < 2 * ntp) v[tid + i * T] = pv[i];
            __syncthreads();
            if (r + 1 < r1) fetch(r + 1);
            if (x0 < ntp) {
                circ_sum4(u, v, ntp, x0, o);
                for (int j = 0; j < 4; ++j) acc[j] += o[j];
            }
            __syncthreads();
        }
    }
    float* out = part + ((size_t)q * gridDim.x + blockIdx.x) * nt;
    for (int j = 0; j < 4; ++j)
        if (x0 + j < nt) out[x0 + j] = acc[j];
}

__device__ __forceinline__ void block_sum_max(float& s, float& m, float* red) {   // red: 64 floats
    s = warp_sum(s);
    m = warp_max(m);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) {
        red[wid] = s;
        red[32 + wid] = m;
    }
    __syncthreads();
    if (wid == 0) {
        float a = lane < nw ? red[lane] : 0.f, b = lane < nw ? red[32 + lane] : -FLT_MAX;
        a = warp_sum(a);
        b = warp_max(b);
        if (lane == 0) {
            red[0] = a;
            red[32] = b;
        }
    }
    __syncthreads();
    s = red[0];
    m = red[32];
    __syncthreads();
}

// Sum of the chunk partials -> c_theta (lag order), then the soft-argmax of Alg. 1 over the angle
// candidates k delta_theta, delta_theta = pi / n_theta (the tail of k_theta).  One CTA per pair.
__global__ void __launch_bounds__(kDirectMaxNT) k_theta_direct(DevPlan p, const float* __restrict__ part, int nch,
                                                               const long long* __restrict__ tab, float* __restrict__ th,
                                                               float* __restrict__ pose, float* __restrict__ c_theta,
                                                               float* __restrict__ ct) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    __shared__ float red[64];
    const int q = blockIdx.x, nt = p.nt, i = threadIdx.x;
    float v = 0.f;
    if (i < nt)
        for (int h = 0; h < nch; ++h) v += part[((size_t)q * nch + h) * nt + i];
    float s = i < nt ? v : 0.f, m = i < nt ? v : -FLT_MAX;
    block_sum_max(s, m, red);
    const float mean = s / nt, cmax = m;
    const float sd = sqrtf(block_reduce<false>(i < nt ? (v - mean) * (v - mean) : 0.f, red) / nt);
    const float inv = p.score_norm == 1 ? 1.f / p.temp_theta : (sd > 0.f ? 1.f / (sd * p.temp_theta) : 0.f);
    const float e = i < nt ? expf((v - cmax) * inv) : 0.f;
    float sums[2] = {e, e * (float)(i - nt / 2)};
    block_sum_n<2>(sums, red);
    if (i < nt) {
        ct[(size_t)q * nt + i] = v;
        if (c_theta) c_theta[tab[3 * q + 1] + i] = v;
    }
    if (i == 0) {
        const float theta = (float)((double)sums[1] / (double)sums[0] * (3.14159265358979323846 / nt));
        pose[3 * tab[3 * q + 2]] = theta;
        double sd_, cd_;
        sincos((double)theta, &sd_, &cd_);
        const float chh = (float)cd_, shh = (float)sd_;
        float* t = th + 8 * q;
        t[0] = theta;
        t[1] = chh;
        t[2] = (float)(cd_ - (double)chh);
        t[3] = shh;
        t[4] = (float)(sd_ - (double)shh);
    }
}

// Angle soft-argmax adjoint (the math of k_b_theta): d c_theta in lag order, from dL/dtheta in
// bsc[q][8] and the scores kept in ct.
__global__ void __launch_bounds__(kDirectMaxNT) k_b_theta_direct(DevPlan p, const float* __restrict__ ct,
                                                                 const float* __restrict__ bsc,
                                                                 float* __restrict__ dcout) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    __shared__ float red[64];
    const int q = blockIdx.x, nt = p.nt, i = threadIdx.x;
    const float c = i < nt ? ct[(size_t)q * nt + i] : 0.f;
    float s = i < nt ? c : 0.f, m = i < nt ? c : -FLT_MAX;
    block_sum_max(s, m, red);
    const float mean = s / nt, cmax = m;
    const float sd = sqrtf(block_reduce<false>(i < nt ? (c - mean) * (c - mean) : 0.f, red) / nt);
    const float inv = p.score_norm == 1 ? 1.f / p.temp_theta : (sd > 0.f ? 1.f / (sd * p.temp_theta) : 0.f);
    const float e = i < nt ? expf((c - cmax) * inv) : 0.f;
    const float se = block_reduce<false>(e, red);
    const float dth = bsc[(size_t)q * 16 + 8];
    const float dl = 3.14159265358979323846f / nt;
    const float pp = e / se, qk = dth * (float)(i - nt / 2) * dl;
    const float pq = block_reduce<false>(i < nt ? pp * qk : 0.f, red);
    const float dz = i < nt ? pp * (qk - pq) / p.temp_theta : 0.f;
    const float z = sd > 0.f ? (c - mean) / sd : 0.f;
    float sums[2] = {dz, dz * z};
    block_sum_n<2>(sums, red);
    const float m1 = sums[0] / nt, m2 = sums[1] / nt;
    if (i < nt) {
        float dc = dz;
        if (p.score_norm != 1) dc = sd > 0.f ? (dz - m1 - z * m2) / sd : 0.f;
        dcout[(size_t)q * nt + i] = dc;
    }
}

// Correlation adjoint for each radius of the CTA's chunk:
//   d A_f[a] = sum_i dc_i A_g[(a + l_i) mod n] = sum_i dc[i] v[a + i],    v[m] = A_g[(m - n/2) mod n]
//   d A_g[b] = sum_i dc_i A_f[(b - l_i) mod n] = sum_i' dcr[i'] w[b + i'], dcr[i'] = dc[n - 1 - i'],
//                                                                        w[m] = A_f[(m + n/2 + 1) mod n]
// (both the sums of circ_sum4); with the radial mean, d M / n_r goes to every radius.  gpol[q][a][r]
// as the FFT route leaves it for k_b_polT.
__global__ void __launch_bounds__(kDirectMaxNT / 4) k_b_angle_direct(DevPlan p, const float2* __restrict__ pol,
                                                                     const float* __restrict__ dc,
                                                                     float2* __restrict__ gpol, int B) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    __shared__ __align__(16) float dcs[kDirectMaxNT], dcr[kDirectMaxNT], v[2 * kDirectMaxNT], w[2 * kDirectMaxNT];
    const int q = blockIdx.y, nt = p.nt, ntp = direct_pad(nt), tid = threadIdx.x, T = blockDim.x;
    const int shg = nt - nt / 2, shf = nt / 2 + 1, x0 = 4 * tid;
    const float2* P = pol + (size_t)q * nt * p.nr;
    float2* G = gpol + (size_t)q * nt * p.nr;
    for (int i = tid; i < ntp; i += T) {
        dcs[i] = i < nt ? dc[(size_t)q * nt + i] : 0.f;
        dcr[i] = i < nt ? dc[(size_t)q * nt + nt - 1 - i] : 0.f;
    }
    float dfa[4], dga[4];
    auto adjoint = [&]() {
        __syncthreads();
        if (x0 < ntp) {
            circ_sum4(dcs, v, ntp, x0, dfa);
            circ_sum4(dcr, w, ntp, x0, dga);
        }
        __syncthreads();
    };
    if (p.angle_score == 1) {
        __shared__ float mfs[kDirectMaxNT], mgs[kDirectMaxNT];   // radial sums M_f, M_g
        for (int a = tid; a < nt; a += T) {
            float mf = 0.f, mg = 0.f;
            for (int r = 0; r < p.nr; ++r) {
                const float2 x = P[(size_t)r * nt + a];
                mf += x.x;
                mg += x.y;
            }
            mfs[a] = mf;
            mgs[a] = mg;
        }
        __syncthreads();
        for (int m = tid; m < 2 * ntp; m += T) {
            v[m] = mgs[(m + shg) % nt];
            w[m] = mfs[(m + shf) % nt];
        }
        adjoint();
        const float s = 1.f / (float)p.nr;
        for (int j = 0; j < 4; ++j)
            if (x0 + j < nt)
                for (int r = 0; r < p.nr; ++r) G[(size_t)(x0 + j) * p.nr + r] = make_float2(dfa[j] * s, dga[j] * s);
    } else {
        // the next radius is fetched into registers while the current one is summed
        const int r0 = blockIdx.x * kDirectRadii, r1 = min(r0 + kDirectRadii, p.nr);
        const int tm = T % nt, ig = (tid + shg) % nt, jf = (tid + shf) % nt;
        float pv[8], pw[8];
        auto fetch = [&](int r) {
            const float2* row = P + (size_t)r * nt;
            int a = ig, b = jf;   // (m + shg) mod n and (m + shf) mod n for m = tid + i T
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const bool in = tid + i * T < 2 * ntp;
                pv[i] = in ? row[a].y : 0.f;
                pw[i] = in ? row[b].x : 0.f;
                a += tm;
                if (a >= nt) a -= nt;
                b += tm;
                if (b >= nt) b -= nt;
            }
        };
        if (r0 < r1) fetch(r0);
        for (int r = r0; r < r1; ++r) {
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (tid + i * T < 2 * ntp) {
                    v[tid + i * T] = pv[i];
                    w[tid + i * T] = pw[i];
                }
            __syncthreads();
            if (r + 1 < r1) fetch(r + 1);
            if (x0 < ntp) {
                circ_sum4(dcs, v, ntp, x0, dfa);
                circ_sum4(dcr, w, ntp, x0, dga);
            }
            __syncthreads();
            for (int j = 0; j < 4; ++j)
                if (x0 + j < nt) G[(size_t)(x0 + j) * p.nr + r] = make_float2(dfa[j], dga[j]);
        }
    }
}

cudaError_t launch_stage1_direct(const DevPlan& p, const Ws& w, int B, const long long* tab, float* pose,
                                 float* c_theta, cudaStream_t st) {
    const int nch = angle_direct_chunks(p);
    float* part = reinterpret_cast<float*>(w.sp);
    // the samples stay in ahat for the adjoint; a plain forward keeps nothing and borrows the
    // adjoint's polar-gradient buffer (same size)
    float2* pol = w.ahat ? w.ahat : w.gpol;
    w.tr->before(K_ANGLE, st);
    launch_pdl(k_polar_direct, dim3((p.nt + kPolTile - 1) / kPolTile, (p.nr + kPolTile - 1) / kPolTile, B), 256, 0, st,
               p, w.mt, pol, B);
    launch_pdl(k_angle_direct, dim3(nch, B), direct_threads(p.nt), 0, st, p, (const float2*)pol, part, B);
    w.tr->before(K_THETA, st);
    launch_pdl(k_theta_direct, B, kDirectMaxNT, 0, st, p, (const float*)part, nch, tab, w.th, pose, c_theta, w.ct);
    return cudaGetLastError();
}

void launch_stage1_adjoint_direct(const DevPlan& p, const Ws& w, int B, cudaStream_t st) {
    float* dc = reinterpret_cast<float*>(w.bdc);
    w.tr->before(K_B_THETA, st);
    launch_pdl(k_b_theta_direct, B, kDirectMaxNT, 0, st, p, (const float*)w.ct, (const float*)w.bsc, dc);
    w.tr->before(K_B_ANGLE, st);
    launch_pdl(k_b_angle_direct, dim3(angle_direct_chunks(p), B), direct_threads(p.nt), 0, st, p, (const float2*)w.ahat,
               (const float*)dc, w.gpol, B);
}

}  // namespace fmbym
