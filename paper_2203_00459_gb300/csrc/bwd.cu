// Adjoint of the decoupled Fourier pose search (the end-to-end differentiability of Sec. III-C,
// through which the masking network of Sec. III-D is trained by Eq. 13).
//
// Given dL/d(theta, t_x, t_y) per pair, the kernels below produce dL/df and dL/dg.  The forward
// intermediates are recomputed first (launch_forward into the workspace), or, in a training call,
// are still in the workspace from that call's own forward; nothing is kept between calls.  Order
// of the adjoint, last forward step first:
//   k_b_rows     translation soft-argmax adjoint d c_xy (from the moments the forward kept),
//                embedded in the P x P lag grid, real row FFTs
//   k_b_cols     column FFTs of D, F' and G; conj(D) G (-> d f') and D F' (-> d g); inverse
//   k_b_c2r      inverse row FFTs, keep x in [0, N): d f' and the stage-2 part of d g
//   k_b_rot      Rotate adjoint: d f (transpose of the bilinear gather, in gather form) and
//                d theta through the rotated source, reduced per pair
//   k_b_theta    angle soft-argmax adjoint -> d c_theta, then its FFT along angle
//   k_b_angle    angle-correlation adjoint in frequency: d A_f, d A_g
//   k_b_polT     transpose of the bilinear Cart2Pol gather (precomputed CSR, no atomics)
//   k_b_s1cols   |z| adjoint z/|z| with the band-pass, inverse column FFTs of the half plane
//   k_b_s1rows   inverse row FFTs of the half plane, window -> stage-1 parts of d f and d g
// Every reduction has a fixed order, so repeated calls give identical bits.
#include <cfloat>

#include "common.cuh"
#include "dev_util.cuh"

namespace fmbym {

// ---------------------------------------------------------------------------------------------
// translation soft-argmax adjoint
// ---------------------------------------------------------------------------------------------

// With p = softmax(y), y = (c - mean)/(std T), t = delta E_p[s]: dL/dy = p (q - <p, q>) with
// q_s = delta (dtx s_x + dty s_y) and <p, q> = dtx t_x + dty t_y; dz = dL/dy / T.  The z-score
// adjoint needs mean(dz) and mean(dz z) over the n = N^2 lags.  Since sum p = 1 and
// sum p q = <p, q>, mean(dz) = 0, and mean(dz z) = (delta (dtx S_zx + dty S_zy) - <p, q> S_z) /
// (n T S) with S = sum e, S_z = sum e z, S_zx = sum e z s_x, S_zy = sum e z s_y, the sums the
// forward's soft-argmax keeps (xm).  r receives (mean dz, mean dz z, mean, std, max, 1/(std T),
// S, <p, q>, 1/S, 1/T, 1/std).
__device__ __forceinline__ void xy_adjoint_scalars(const DevPlan& p, const float* __restrict__ m, float tx,
                                                   float ty, float dtx, float dty, int n, float* r) {
    const float pq = dtx * tx + dty * ty;
    r[0] = 0.f;
    r[1] = (p.delta_xy * (dtx * m[6] + dty * m[7]) - pq * m[5]) / ((float)n * (float)n * p.temp_xy * m[4]);
    r[2] = m[0];
    r[3] = m[1];
    r[4] = m[2];
    r[5] = m[3];
    r[6] = m[4];
    r[7] = pq;
    r[8] = 1.f / m[4];
    r[9] = 1.f / p.temp_xy;
    r[10] = m[1] > 0.f ? 1.f / m[1] : 0.f;
}

// d c_xy at lag (i, j) from the scores and the per-pair scalars of xy_adjoint_scalars.
__device__ __forceinline__ float dcxy(const DevPlan& p, const float* r, float cv, int i, int j, int n, float dtx,
                                      float dty) {
    const float pp = expf((cv - r[4]) * r[5]) * r[8];
    const float qq = p.delta_xy * (dtx * (float)(j - n / 2) + dty * (float)(i - n / 2));
    const float dz = pp * (qq - r[7]) * r[9];
    if (p.score_norm == 1) return dz;
    if (!(r[3] > 0.f)) return 0.f;
    const float z = (cv - r[2]) * r[10];
    return (dz - r[0] - z * r[1]) * r[10];
}

// ---------------------------------------------------------------------------------------------
// padded correlation adjoint: d f'(x) = sum_s D(s) g(x + s), d g(y) = sum_s D(s) f'(y - s)
// ---------------------------------------------------------------------------------------------

// Lag rows of D (row i holds s_y = i - N/2; column j sits at P-position (j - N/2) mod P), two
// rows per complex FFT of length P, packed real-FFT output rows [N][P/2].  The first pass forms
// d c_xy straight from global memory.
// ODD: the scan side is N - 1 inside the frame N; c_xy is [N - 1][N - 1] at frame lags 1 .. N - 1, and
// D is zero at frame lag index 0 (lag -N/2, not a candidate of an odd side).
template <int N, int P, bool ODD>
__global__ void __launch_bounds__(kThreads) k_b_rows(DevPlan p, const long long* __restrict__ tab,
                                                     const float* __restrict__ cxy, const float* __restrict__ xm,
                                                     const float* __restrict__ fwd_pose,
                                                     const float* __restrict__ dpose, float2* __restrict__ b1, int B) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    constexpr int T = FftPlan<P>::T, TPB = tpb_for(P), FPC = TPB / T, SL = spad(P), W = P / 2;
    extern __shared__ float2 sm[];
    __shared__ float r[11];
    const int q = blockIdx.y, i0 = blockIdx.x * FPC * 2;
    const int k = threadIdx.x / T, jt = threadIdx.x % T, i = i0 + 2 * k;
    const long long pr = tab[3 * q + 2];
    float dtx = dpose[3 * pr + 1], dty = dpose[3 * pr + 2];
    float tx = fwd_pose[3 * pr + 1], ty = fwd_pose[3 * pr + 2];
    if (p.rotate_target) {   // t = R(theta) t': the soft-argmax sees t' and dt' = R(theta)^T dt
        float sn, cs;
        sincosf(fwd_pose[3 * pr], &sn, &cs);
        const float a = cs * dtx + sn * dty, b = -sn * dtx + cs * dty;
        const float c = cs * tx + sn * ty, d = -sn * tx + cs * ty;
        dtx = a;
        dty = b;
        tx = c;
        ty = d;
    }
    constexpr int NI = ODD ? N - 1 : N, LO = ODD ? 1 : 0;
    if (threadIdx.x == 0) xy_adjoint_scalars(p, xm + (size_t)q * 8, tx, ty, dtx, dty, NI, r);
    __syncthreads();
    float rv[11];   // the pair's scalars in registers: each of the thread's 32 lags reads them
#pragma unroll
    for (int t = 0; t < 11; ++t) rv[t] = r[t];
    const float* c = cxy + (size_t)q * NI * NI + (size_t)(i - LO) * NI - LO;
    const bool oka = i >= LO;
    first_pass_global<P>(sm + k * SL, 1, jt, [&](int x) {
        const int j = x + N / 2 < P ? x + N / 2 : x + N / 2 - P;   // lag column at P-position x
        float2 v = make_float2(0.f, 0.f);
        if (j < N && j >= LO) {
            if (oka) v.x = dcxy(p, rv, __ldg(c + j), i, j, N, dtx, dty);
            v.y = dcxy(p, rv, __ldg(c + NI + j), i + 1, j, N, dtx, dty);
        }
        return v;
    });
    __syncthreads();
    fft_passes_from<P, -1, 2>(sm + k * SL, 1, jt, p.tw_p);
    float2* out = b1 + (size_t)q * N * W;
    for (int idx = threadIdx.x; idx < FPC * W; idx += TPB) {
        const int kk = idx / W, u = idx % W, row = i0 + 2 * kk;
        const float2* Z = sm + kk * SL;
        const float2 zu = Z[spad(u)], zm = Z[spad(u == 0 ? W : P - u)];
        out[(size_t)row * W + u] = unpack_half(zu, zm, u == 0, false);
        out[(size_t)(row + 1) * W + u] = unpack_half(zu, zm, u == 0, true);
    }
}

// Separates the packed column 0 of an FFT'd tile into the DC column (A) and Nyquist column (B).
__device__ __forceinline__ void split0(float2 z, float2 zm, float2& a, float2& b) {
    a = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
    b = make_float2(0.5f * (z.y + zm.y), -0.5f * (z.x - zm.x));
}

// Column pass of the correlation adjoint: FFT the columns of D (lag rows placed at their P-rows),
// Q1 = conj(D) G^ (-> d f') and Q2 = D F'^ (-> d g) with the column spectra F'^, G^ that the
// forward kept (s2hat), inverse FFT both, keep the spatial rows y < N.  The packed column 0
// multiplies its DC and Nyquist parts separately.  D's first pass reads global memory; its last
// pass, both products and both inverses' first passes run in registers (the inverse in the
// reverse radix order); both inverses' last passes store to global memory.
// V: the radix order (FftPlan<P, V>).
template <int N, int P, int C, int V>
__global__ void __launch_bounds__(C * FftPlan<P>::T, col_min_blocks(P, C)) k_b_cols(DevPlan p, const float2* __restrict__ b1,
                                                                       const float2* __restrict__ s2hat,
                                                                       float2* __restrict__ b2, int B) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    using PL = FftPlan<P, V>;
    constexpr int T = PL::T, TPB = C * T, ES = C, W = P / 2, TILE = spad(P) * ES;
    constexpr int RL = last_radix<P, V>(), NBL = P / RL, BPL = (NBL + T - 1) / T, PER = P * C / TPB;
    extern __shared__ float2 sm[];
    float2* tD = sm;
    float2* tX = sm + TILE;
    const int q = blockIdx.y, u0 = blockIdx.x * C;
    const int c = threadIdx.x % C, j = threadIdx.x / C;
    const float2* __restrict__ tw = p.tw_p;
    const float2* inD = b1 + (size_t)q * N * W + u0 + c;
    const float2* hF = s2hat + (size_t)q * P * W;          // F'^ [W][P], column-major
    const float2* hG = s2hat + (size_t)(B + q) * P * W;    // G^  [W][P]
    const float2 zero = make_float2(0.f, 0.f);
    // the tile's columns of F'^ and G^ (C runs of P positions each) are read only after D's first
    // two passes: start bringing them into L2 now
    if (threadIdx.x < 2 * C)
        prefetch_l2((threadIdx.x < C ? hF : hG) + (size_t)(u0 + threadIdx.x % C) * P, P * sizeof(float2));
    // P-row v of D holds lag row i = (v + N/2) mod P (zero when i >= N)
    first_pass_global<P>(tD + c, ES, j, [&](int v) {
        const int i = v + N / 2 < P ? v + N / 2 : v + N / 2 - P;
        return i < N ? __ldg(inD + (size_t)i * W) : zero;
    });
    __syncthreads();
    if constexpr (PL::NP == 3) fft_pass<P, T, PL::R2, 16, -1>(tD + c, ES, j, true, tw);
    if (blockIdx.x != 0) {
        const int u = u0 + c;
        // D's last forward pass, then Q1 = conj(D) G^ and its inverse first pass straight into tX,
        // which nothing reads here.  Q2 = D F'^ and its inverse first pass are held in registers
        // until every thread has read its D, then written over tD.  With one butterfly per thread
        // (BPL = 1) Q2 is formed from the D values in registers; with several, D's final values go
        // back in place (same thread, same positions) and Q2 is formed after the Q1 loop, which
        // keeps fewer values live while the loads of G^ are in flight (measured faster there).
        constexpr bool KEEP_D = BPL > 1;
        float2 o2[BPL][RL];
#pragma unroll
        for (int m = 0; m < BPL; ++m) {
            const int b = j + m * T;
            if (NBL % T == 0 || b < NBL) {
                float2 d[RL], o[RL];
#pragma unroll
                for (int t = 0; t < RL; ++t) d[t] = tD[spad(b + t * NBL) * ES + c];
                twiddle<P, RL, NBL, -1>(d, b, tw);
                dft<RL, -1>(d);
#pragma unroll
                for (int t = 0; t < RL; ++t) {
                    if constexpr (KEEP_D) tD[spad(b + t * NBL) * ES + c] = d[t];
                    o[t] = c_cjmul(d[t], __ldg(hG + (size_t)u * P + b + t * NBL));
                }
                dft<RL, +1>(o);
#pragma unroll
                for (int t = 0; t < RL; ++t) tX[spad(RL * b + t) * ES + c] = o[t];
                if constexpr (!KEEP_D) {
                    // F'^ is loaded only now (the fence keeps the compiler from hoisting the loads
                    // above Q1), so that G^, F'^ and D are not all live at once
                    asm volatile("" ::: "memory");
#pragma unroll
                    for (int t = 0; t < RL; ++t) o2[m][t] = c_mul(d[t], __ldg(hF + (size_t)u * P + b + t * NBL));
                    dft<RL, +1>(o2[m]);
                }
            }
        }
        if constexpr (KEEP_D) {
#pragma unroll
            for (int m = 0; m < BPL; ++m) {
                const int b = j + m * T;
                if (NBL % T == 0 || b < NBL) {
#pragma unroll
                    for (int t = 0; t < RL; ++t)
                        o2[m][t] = c_mul(tD[spad(b + t * NBL) * ES + c], __ldg(hF + (size_t)u * P + b + t * NBL));
                    dft<RL, +1>(o2[m]);
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int m = 0; m < BPL; ++m) {
            const int b = j + m * T;
            if (NBL % T == 0 || b < NBL) {
#pragma unroll
                for (int t = 0; t < RL; ++t) tD[spad(RL * b + t) * ES + c] = o2[m][t];
            }
        }
        __syncthreads();
    } else {
        // the tile holding column 0: D's last pass in shared memory, the products with the DC /
        // Nyquist split (pairs v with P - v), then both inverses' first passes
        fft_pass<P, T, RL, NBL, -1>(tD + c, ES, j, true, tw);
        float2 q1[PER], q2[PER];
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            const int idx = threadIdx.x + m * TPB, v = idx / C, cc = idx % C, u = u0 + cc;
            const float2 D = tD[spad(v) * ES + cc];
            const float2 G = __ldg(hG + (size_t)u * P + v), F = __ldg(hF + (size_t)u * P + v);
            if (cc == 0) {
                const int vm = v == 0 ? 0 : P - v;
                float2 ad, bd, ag, bg, af, bf;
                split0(D, tD[spad(vm) * ES + cc], ad, bd);
                split0(G, __ldg(hG + (size_t)u * P + vm), ag, bg);
                split0(F, __ldg(hF + (size_t)u * P + vm), af, bf);
                const float2 g0 = c_cjmul(ad, ag), gn = c_cjmul(bd, bg);
                const float2 f0 = c_mul(ad, af), fn = c_mul(bd, bf);
                q1[m] = make_float2(g0.x - gn.y, g0.y + gn.x);
                q2[m] = make_float2(f0.x - fn.y, f0.y + fn.x);
            } else {
                q1[m] = c_cjmul(D, G);
                q2[m] = c_mul(D, F);
            }
        }
        __syncthreads();
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            const int idx = threadIdx.x + m * TPB, v = idx / C, cc = idx % C;
            tX[spad(v) * ES + cc] = q1[m];
            tD[spad(v) * ES + cc] = q2[m];
        }
        __syncthreads();
        fft_pass2<P, T, RL, 1, +1>(tX + c, tD + c, ES, j, tw);
    }
    float2* o1 = b2 + (size_t)q * N * W + u0 + c;
    float2* o2 = b2 + (size_t)(B + q) * N * W + u0 + c;
    inverse_rest_global2<P, V>(
        tX + c, tD + c, ES, j, tw, [&](int y, float2 v) { if (y < N) o1[(size_t)y * W] = v; },
        [&](int y, float2 v) { if (y < N) o2[(size_t)y * W] = v; });
}

// Inverse row FFTs of the two adjoint spectra, keep x in [0, N), scale 1/P^2:
// z = 0 -> d f' (workspace), z = 1 -> d g (stage-2 part, written to the caller's buffer); under
// rotate_target 1, z = 0 -> d f (caller) and z = 1 -> d g' (workspace).  The
// first pass builds its inputs from global memory and the last pass stores straight to it.
// ODD: the scan side is N - 1 inside the frame N: rows and columns below N - 1 are kept, with stride
// N - 1 (the frame's last row and column belong to no pixel).
template <int N, int P, bool ODD>
__global__ void __launch_bounds__(kThreads) k_b_c2r(DevPlan p, const long long* __restrict__ tab,
                                                    const float2* __restrict__ b2, float* __restrict__ gfr,
                                                    float* __restrict__ df, float* __restrict__ dg, int B) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    constexpr int T = FftPlan<P>::T, TPB = tpb_for(P), FPC = TPB / T, SL = spad(P), W = P / 2;
    constexpr int NI = ODD ? N - 1 : N;
    extern __shared__ float2 sm[];
    const int q = blockIdx.y, s = blockIdx.z, i0 = blockIdx.x * FPC * 2;
    const int k = threadIdx.x / T, j = threadIdx.x % T, y = i0 + 2 * k;
    const float2* ra = b2 + ((size_t)(s * B + q) * N + y) * W;
    first_pass_global<P, +1>(sm + k * SL, 1, j, [&](int x) { return pack_inverse(ra, ra + W, x, P); });
    __syncthreads();
    const float scale = 1.f / ((float)P * (float)P);
    // the rotated operand's gradient goes to the workspace for the Rotate adjoint, the other one
    // straight to the caller (f' and g by default; f and g' under rotate_target 1)
    float* out = (s == p.rotate_target ? gfr + (size_t)q * NI * NI : (s == 0 ? df : dg) + tab[3 * q]) + (size_t)y * NI;
    const bool okb = !ODD || y + 1 < NI;
    rest_global<P, +1>(sm + k * SL, 1, j, p.tw_p, [&](int x, float2 z) {
        if (x < NI) {
            out[x] = z.x * scale;
            if (okb) out[NI + x] = z.y * scale;
        }
    });
}

// ---------------------------------------------------------------------------------------------
// Rotate adjoint
// ---------------------------------------------------------------------------------------------

// One thread per pixel (PX pixels per thread), which plays two roles:
//  (a) output pixel X of f': its d theta term d f'(X) (dv/dpx (py - c) - dv/dpy (px - c)), since
//      d px / d theta = py - c and d py / d theta = -(px - c);
//  (b) source pixel y of f: d f(y) = sum over the output pixels X whose bilinear sample reads y of
//      weight * d f'(X).  Such X lie within sqrt 2 of X0 = c + R(theta)(y - c), i.e. in the 3 x 3
//      box around its rounded position, and the bilinear weight of y in X's sample is the tent
//      (1 - |dx|)(1 - |dy|) of the offset R(-theta)(X - X0) of that sample from y.
// The adjoint's coordinates are two fused multiply-adds (error ~ 1e-4 px at N = 512, which moves a
// bilinear weight by as much; the forward's error-free coordinates decide the scores, these only
// their gradient).  d theta is reduced per pair (last block adds the block sums in order) into
// bsc[q][8] together with the direct term dL/dtheta.
// Under rotate_target 1 the rotated scan is g, turned by -theta: f and df here are g and dg, the
// sine changes sign, d theta takes the rotation term with the opposite sign, and the translation
// t = R(theta) t' adds dt . (dR/dtheta) t' = t_x dt_y - t_y dt_x (fwd_pose holds t).
// ODD: the scan side is N - 1 inside the frame N: the pixels of the frame's last row and column are
// skipped, strides and bounds are N - 1 and the centre (N - 1)/2.
template <int N, int PX, bool ODD>
__global__ void __launch_bounds__(kThreads) k_b_rot(DevPlan p, const long long* __restrict__ tab,
                                                    const float* __restrict__ f, const float* __restrict__ th,
                                                    const float* __restrict__ gfr, const float* __restrict__ dpose,
                                                    float* __restrict__ df, float* __restrict__ gpart,
                                                    unsigned* __restrict__ cnt, float* __restrict__ bsc,
                                                    const float* __restrict__ fwd_pose) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    __shared__ float red[32];
    __shared__ bool last;
    constexpr int NB = N * N / (kThreads * PX), NI = ODD ? N - 1 : N;
    const int q = blockIdx.y;
    const float* t = th + 8 * q;
    const float sg = p.rotate_target ? -1.f : 1.f;
    const float ct = t[1] + t[2], stn = sg * (t[3] + t[4]);
    const float c = 0.5f * NI;
    const float* src = f + tab[3 * q];
    const float* d = gfr + (size_t)q * NI * NI;
    float contrib = 0.f;
#pragma unroll
    for (int m = 0; m < PX; ++m) {
        const int fidx = (blockIdx.x * PX + m) * kThreads + threadIdx.x;
        const int Y = fidx / N, X = fidx % N;
        if (ODD && (X >= NI || Y >= NI)) continue;
        const int idx = Y * NI + X;
        const float dX = (float)X - c, dY = (float)Y - c;
        // (a) d theta at output pixel X, sampled at c + R(-theta)(X - c)
        {
            const float px = fmaf(ct, dX, fmaf(stn, dY, c)), py = fmaf(ct, dY, fmaf(-stn, dX, c));
            const float fx0 = floorf(px), fy0 = floorf(py);
            const int x0 = (int)fx0, y0 = (int)fy0;
            const float fx = px - fx0, fy = py - fy0;
            auto at = [&](int yy, int xx) {
                return ((unsigned)yy < (unsigned)NI && (unsigned)xx < (unsigned)NI) ? __ldg(src + (size_t)yy * NI + xx)
                                                                                    : 0.f;
            };
            float v00, v01, v10, v11;
            if ((unsigned)x0 < (unsigned)(NI - 1) && (unsigned)y0 < (unsigned)(NI - 1)) {   // all four taps inside
                const float* s0 = src + (size_t)y0 * NI + x0;
                v00 = __ldg(s0);
                v01 = __ldg(s0 + 1);
                v10 = __ldg(s0 + NI);
                v11 = __ldg(s0 + NI + 1);
            } else {
                v00 = at(y0, x0);
                v01 = at(y0, x0 + 1);
                v10 = at(y0 + 1, x0);
                v11 = at(y0 + 1, x0 + 1);
            }
            const float dvx = (1.f - fy) * (v01 - v00) + fy * (v11 - v10);
            const float dvy = (1.f - fx) * (v10 - v00) + fx * (v11 - v01);
            contrib += __ldg(d + idx) * (dvx * (py - c) - dvy * (px - c));
        }
        // (b) d f at source pixel (X, Y): X0 = c + R(theta)(y - c); a candidate output pixel M
        // samples at y + R(-theta)(M - X0), so its bilinear weight on y is the tent of
        // (dx, dy) = R(-theta)(M - X0); the taps of the 3 x 3 box differ by constant steps
        {
            const float qx = fmaf(ct, dX, fmaf(-stn, dY, c)), qy = fmaf(stn, dX, fmaf(ct, dY, c));
            const int mx0 = (int)floorf(qx + 0.5f) - 1, my0 = (int)floorf(qy + 0.5f) - 1;
            const float ex0 = (float)mx0 - qx, ey0 = (float)my0 - qy;
            const float dx0 = fmaf(ct, ex0, stn * ey0), dy0 = fmaf(ct, ey0, -stn * ex0);
            float acc = 0.f;
            if ((unsigned)mx0 < (unsigned)(NI - 2) && (unsigned)my0 < (unsigned)(NI - 2)) {
                // the whole box inside: no bounds tests, and a tap outside the tent adds 0 * d
                // (clamped weights), which leaves the sum bitwise as skipping it would
                const float* dm = d + (size_t)my0 * NI + mx0;
#pragma unroll
                for (int oy = 0; oy < 3; ++oy) {
                    const float dxr = fmaf(stn, (float)oy, dx0), dyr = fmaf(ct, (float)oy, dy0);
#pragma unroll
                    for (int ox = 0; ox < 3; ++ox) {
                        const float wx = fmaxf(1.f - fabsf(fmaf(ct, (float)ox, dxr)), 0.f);
                        const float wy = fmaxf(1.f - fabsf(fmaf(-stn, (float)ox, dyr)), 0.f);
                        acc = fmaf(wy * wx, __ldg(dm + oy * NI + ox), acc);
                    }
                }
            } else {
#pragma unroll
                for (int oy = 0; oy < 3; ++oy) {
                    const int my = my0 + oy;
                    const float dxr = fmaf(stn, (float)oy, dx0), dyr = fmaf(ct, (float)oy, dy0);
#pragma unroll
                    for (int ox = 0; ox < 3; ++ox) {
                        const int mx = mx0 + ox;
                        const float wx = 1.f - fabsf(fmaf(ct, (float)ox, dxr)), wy = 1.f - fabsf(fmaf(-stn, (float)ox, dyr));
                        if (wx > 0.f && wy > 0.f && (unsigned)my < (unsigned)NI && (unsigned)mx < (unsigned)NI)
                            acc = fmaf(wy * wx, __ldg(d + (size_t)my * NI + mx), acc);
                    }
                }
            }
            df[tab[3 * q] + idx] = acc;
        }
    }
    const float bs = block_reduce<false>(contrib, red);
    if (threadIdx.x == 0) {
        gpart[(size_t)q * NB + blockIdx.x] = bs;
        __threadfence();
        last = atomicAdd(&cnt[q], 1u) == NB - 1;
    }
    __syncthreads();
    if (last) {
        __threadfence();
        const volatile float* g = gpart + (size_t)q * NB;
        float s = 0.f;
        for (int i = threadIdx.x; i < NB; i += kThreads) s += g[i];
        s = block_reduce<false>(s, red);
        if (threadIdx.x == 0) {
            const long long pr = tab[3 * q + 2];
            float dth = dpose[3 * pr] + sg * s;
            if (p.rotate_target)
                dth += fwd_pose[3 * pr + 1] * dpose[3 * pr + 2] - fwd_pose[3 * pr + 2] * dpose[3 * pr + 1];
            bsc[(size_t)q * 16 + 8] = dth;
            cnt[q] = 0u;
        }
    }
}

// ---------------------------------------------------------------------------------------------
// stage-1 adjoint
// ---------------------------------------------------------------------------------------------

// Angle soft-argmax adjoint (as for the translation, with q_k = dtheta k delta_theta), z-score
// adjoint, then the FFT along angle of d c_theta laid out circularly (lag k at index k mod n).
template <int NT>
__global__ void __launch_bounds__(256) k_b_theta(DevPlan p, const float* __restrict__ ct,
                                                 const float* __restrict__ bsc, float2* __restrict__ bdc) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    constexpr int T = FftPlan<NT>::T;
    __shared__ float2 z[spad(NT)];
    __shared__ float c[NT];
    __shared__ float red[32];
    const int q = blockIdx.x;
    float lsum = 0.f, lmax = -FLT_MAX;
    for (int i = threadIdx.x; i < NT; i += blockDim.x) {
        const float v = ct[(size_t)q * NT + i];
        c[i] = v;
        lsum += v;
        lmax = fmaxf(lmax, v);
    }
    const float mean = block_reduce<false>(lsum, red) * (1.f / NT);
    const float cmax = block_reduce<true>(lmax, red);
    float lvar = 0.f;
    for (int i = threadIdx.x; i < NT; i += blockDim.x) lvar += (c[i] - mean) * (c[i] - mean);
    const float sd = sqrtf(block_reduce<false>(lvar, red) * (1.f / NT));
    const float inv = p.score_norm == 1 ? 1.f / p.temp_theta : (sd > 0.f ? 1.f / (sd * p.temp_theta) : 0.f);
    float le = 0.f;
    for (int i = threadIdx.x; i < NT; i += blockDim.x) le += expf((c[i] - cmax) * inv);
    const float se = block_reduce<false>(le, red);
    const float dth = bsc[(size_t)q * 16 + 8];
    const float dl = 3.14159265358979323846f / NT;
    float lpq = 0.f;
    for (int i = threadIdx.x; i < NT; i += blockDim.x)
        lpq += expf((c[i] - cmax) * inv) / se * (dth * (float)(i - NT / 2) * dl);
    const float pq = block_reduce<false>(lpq, red);
    float l1 = 0.f, l2 = 0.f;
    float dz[(NT + 255) / 256];
#pragma unroll
    for (int m = 0; m < (NT + 255) / 256; ++m) {
        const int i = threadIdx.x + 256 * m;
        dz[m] = 0.f;
        if (i < NT) {
            const float pp = expf((c[i] - cmax) * inv) / se;
            dz[m] = pp * (dth * (float)(i - NT / 2) * dl - pq) / p.temp_theta;
            l1 += dz[m];
            l2 += dz[m] * (sd > 0.f ? (c[i] - mean) / sd : 0.f);
        }
    }
    const float m1 = block_reduce<false>(l1, red) * (1.f / NT);
    const float m2 = block_reduce<false>(l2, red) * (1.f / NT);
#pragma unroll
    for (int m = 0; m < (NT + 255) / 256; ++m) {
        const int i = threadIdx.x + 256 * m;
        if (i < NT) {
            float dc = dz[m];
            if (p.score_norm != 1) dc = sd > 0.f ? (dz[m] - m1 - (c[i] - mean) / sd * m2) / sd : 0.f;
            z[spad((i - NT / 2 + NT) % NT)] = make_float2(dc, 0.f);
        }
    }
    __syncthreads();
    fft<NT, -1>(z, 1, threadIdx.x, threadIdx.x < T, p.tw_t);
    for (int k = threadIdx.x; k < NT; k += blockDim.x) bdc[(size_t)q * NT + k] = z[spad(k)];
}

// Angle-correlation adjoint for a chunk of radii: from the forward's Z = FFT along angle of
// A_f + i A_g (kept in ahat), d A_f = iFFT(conj(DC) A^_g) / n and d A_g = iFFT(DC A^_f) / n, both
// real, packed as one inverse FFT of U_f + i U_g.  With the radial-mean score the same holds for
// the radial sums M (their transform kept at radius 0), and every radius receives d M / n_r.  Threads are radius-fastest; the first pass
// forms U_f + i U_g straight from global memory (A^_f, A^_g from Z[k] and Z[n - k]) and the last
// pass stores d A straight to global memory.
template <int NT, int RC>
__global__ void __launch_bounds__(FftPlan<NT>::T * RC) k_b_angle(DevPlan p, const float2* __restrict__ ahat,
                                                                         const float2* __restrict__ bdc,
                                                                         float2* __restrict__ gpol, int B) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    constexpr int T = FftPlan<NT>::T, ES = RC;
    extern __shared__ float2 sm[];
    const int q = blockIdx.y, ch = blockIdx.x;
    const int rr = threadIdx.x % RC, j = threadIdx.x / RC, r = ch * RC + rr;
    const bool live = r < p.nr;
    // per-radius score: this radius' transform; radial-mean score: the transform of the radial sums
    // (kept at radius 0), the same for every radius
    const bool marginal = p.angle_score == 1;
    const float2* Z = ahat + (size_t)q * NT * p.nr + (marginal ? 0 : r);
    const float2* DC = bdc + (size_t)q * NT;
    first_pass_global<NT, +1>(sm + rr, ES, j, [&](int k) {
        if (!live) return make_float2(0.f, 0.f);
        const int km = k == 0 ? 0 : NT - k;
        float2 af, ag;
        split0(__ldg(Z + (size_t)k * p.nr), __ldg(Z + (size_t)km * p.nr), af, ag);
        const float2 dc = __ldg(&DC[k]);
        const float2 uf = c_cjmul(dc, ag), ug = c_mul(dc, af);
        return make_float2(uf.x - ug.y, uf.y + ug.x);
    });
    __syncthreads();
    const float sc = marginal ? 1.f / ((float)NT * (float)p.nr) : 1.f / NT;
    float2* o = gpol + (size_t)q * NT * p.nr + r;
    rest_global<NT, +1>(sm + rr, ES, j, p.tw_t, [&](int a, float2 v) {
        if (live) o[(size_t)a * p.nr] = make_float2(v.x * sc, v.y * sc);
    });
}


// Transpose of the Cart2Pol gather: d a[e] = sum over the samples that read element e of the
// half plane, with the forward's bilinear weights (precomputed CSR on the host).  Blocks below
// `light_blocks` give each element a thread and skip the heavy rows; the blocks after them give
// each heavy row a warp (lane-strided taps, fixed-order warp sum).  The f and g gradients of a
// sample sit side by side, so one gathered sector serves both scans.
__global__ void __launch_bounds__(kThreads) k_b_polT(DevPlan p, const float2* __restrict__ gpol,
                                                     float2* __restrict__ gmt, int B, int light_blocks) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    const int n = p.n, E = (n / 2 + 1) * n;
    const int q = blockIdx.y;
    const float2* da = gpol + (size_t)q * p.nt * p.nr;   // (d A_f, d A_g) of each sample
    float2* o = gmt + (size_t)q * E;   // (d a_f, d a_g) pairs
    if ((int)blockIdx.x < light_blocks) {
        const int e = blockIdx.x * kThreads + threadIdx.x;
        if (e >= E) return;
        const int k0 = __ldg(&p.csr_ptr[e]), k1 = __ldg(&p.csr_ptr[e + 1]);
        if (k1 - k0 > kHeavyRow) return;
        float af = 0.f, ag = 0.f;
#pragma unroll 4
        for (int k = k0; k < k1; ++k) {
            const float w = __ldg(&p.csr_w[k]);
            const float2 v = __ldg(&da[__ldg(&p.csr_col[k])]);
            af += w * v.x;
            ag += w * v.y;
        }
        o[e] = make_float2(af, ag);
        return;
    }
    const int hw = ((int)blockIdx.x - light_blocks) * (kThreads / 32) + (threadIdx.x >> 5);
    if (hw >= p.n_heavy) return;
    const int e = __ldg(&p.heavy[hw]), lane = threadIdx.x & 31;
    const int k0 = __ldg(&p.csr_ptr[e]), k1 = __ldg(&p.csr_ptr[e + 1]);
    float af = 0.f, ag = 0.f;
#pragma unroll 4
    for (int k = k0 + lane; k < k1; k += 32) {
        const float w = __ldg(&p.csr_w[k]);
        const float2 v = __ldg(&da[__ldg(&p.csr_col[k])]);
        af += w * v.x;
        ag += w * v.y;
    }
    af = warp_sum(af);
    ag = warp_sum(ag);
    if (lane == 0) o[e] = make_float2(af, ag);
}

// |z| adjoint with the band-pass, then the column part of the half-plane DFT adjoint:
// dF = d a band F/|F| with the forward's kept phasors.  The DFT adjoint is
// d x[y,x] = Re sum_{v, u <= N/2} dF[v,u] exp(+2 pi i (v y + u x)/N): here the inverse column
// transform, with interior columns halved (a real row transform counts them twice) and the
// DC/Nyquist columns made Hermitian (only the real part of their row sums counts) so that they
// can share the packed column 0.  The first pass forms dF straight from global memory.
// The inputs are u-major (a column's N values are contiguous): with one warp per column (N = 512)
// a warp reads 32 consecutive positions, and the transposed result leaves through the tile (each
// column's sequence at a stride of 2 mod 16 float2 apart, so the row-wise read-back is free of
// bank conflicts) as runs of C columns; the smaller sides are column-fastest (c = tid mod C) and
// store straight from the last pass.
template <int N> __host__ __device__ constexpr bool s1cols_warp() { return FftPlan<N>::T == 32; }
template <int N> __host__ __device__ constexpr int s1cols_stride() { return (spad(N) + 15) / 16 * 16 + 2; }
template <int N>
__global__ void __launch_bounds__(kThreads) k_b_s1cols(DevPlan p, const float2* __restrict__ phs,
                                                       const float2* __restrict__ gmt, float2* __restrict__ gs1,
                                                       int B) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    constexpr bool WARP = s1cols_warp<N>();
    constexpr int T = FftPlan<N>::T, C = kThreads / T, ES = WARP ? 1 : C, W = N / 2, SC = s1cols_stride<N>();
    extern __shared__ float2 sm[];
    const int q = blockIdx.y, s = blockIdx.z, u0 = blockIdx.x * C;
    const int c = WARP ? threadIdx.x / T : threadIdx.x % C, j = WARP ? threadIdx.x % T : threadIdx.x / C, u = u0 + c;
    float2* seq = WARP ? sm + c * SC : sm + c;
    const float* dm = reinterpret_cast<const float*>(gmt + (size_t)q * (W + 1) * N) + s;   // stride 2
    const float2* ph = phs + (size_t)(s * B + q) * (W + 1) * N;
    first_pass_global<N, +1>(seq, ES, j, [&](int v) {
        if (u != 0) return c_scale(__ldg(ph + (size_t)u * N + v), 0.5f * __ldg(dm + 2 * ((size_t)u * N + v)));
        // packed DC (u = 0) and Nyquist (u = N/2) columns, each made Hermitian
        const int vm = (N - v) & (N - 1);
        const float2 a = c_scale(__ldg(ph + v), __ldg(dm + 2 * v));
        const float2 am = c_scale(__ldg(ph + vm), __ldg(dm + 2 * vm));
        const float2 b = c_scale(__ldg(ph + (size_t)W * N + v), __ldg(dm + 2 * ((size_t)W * N + v)));
        const float2 bm = c_scale(__ldg(ph + (size_t)W * N + vm), __ldg(dm + 2 * ((size_t)W * N + vm)));
        const float2 sa = make_float2(0.5f * (a.x + am.x), 0.5f * (a.y - am.y));
        const float2 sb = make_float2(0.5f * (b.x + bm.x), 0.5f * (b.y - bm.y));
        return make_float2(sa.x - sb.y, sa.y + sb.x);
    });
    __syncthreads();
    if constexpr (WARP) {
        // the last pass writes its outputs back to the positions it read (same thread), then the
        // tile leaves row by row
        rest_global<N, +1>(seq, 1, j, p.tw_n, [&](int y, float2 v) { seq[spad(y)] = v; });
        __syncthreads();
        float2* out = gs1 + (size_t)(s * B + q) * N * W + u0;
        for (int idx = threadIdx.x; idx < C * N; idx += kThreads) {
            const int cc = idx % C, y = idx / C;
            out[(size_t)y * W + cc] = sm[cc * SC + spad(y)];
        }
    } else {
        float2* out = gs1 + (size_t)(s * B + q) * N * W + u;
        rest_global<N, +1>(seq, ES, j, p.tw_n, [&](int y, float2 v) { out[(size_t)y * W] = v; });
    }
}

// Row part of the half-plane DFT adjoint (a real inverse FFT of each row, two rows per complex
// FFT), times the window; added to d f (z = 0) or d g (z = 1).
template <int N>
__global__ void __launch_bounds__(kThreads) k_b_s1rows(DevPlan p, const long long* __restrict__ tab,
                                                       const float2* __restrict__ gs1, float* __restrict__ df,
                                                       float* __restrict__ dg, int B) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    constexpr int T = FftPlan<N>::T, FPC = kThreads / T, SL = spad(N), W = N / 2;
    extern __shared__ float2 sm[];
    const int q = blockIdx.y, s = blockIdx.z, r0 = blockIdx.x * FPC * 2;
    const int k = threadIdx.x / T, j = threadIdx.x % T, y = r0 + 2 * k;
    const float2* ra = gs1 + ((size_t)(s * B + q) * N + y) * W;
    first_pass_global<N, +1>(sm + k * SL, 1, j, [&](int x) { return pack_inverse(ra, ra + W, x, N); });
    __syncthreads();
    float* out = (s ? dg : df) + tab[3 * q] + (size_t)y * N;
    const float wa = p.window ? __ldg(&p.win[y]) : 1.f, wb = p.window ? __ldg(&p.win[y + 1]) : 1.f;
    rest_global<N, +1>(sm + k * SL, 1, j, p.tw_n, [&](int x, float2 z) {
        float va = z.x, vb = z.y;
        if (p.window) {
            const float wx = __ldg(&p.win[x]);
            va *= wa * wx;
            vb *= wb * wx;
        }
        out[x] += va;
        out[N + x] += vb;
    });
}

// The same two steps for an odd side, whose N-point inverse DFTs run as Bluestein convolutions:
// the inverse DFT is conj(DFT(conj x)).  The half plane of an odd N has no Nyquist column; the
// interior columns u in [1, (N - 1)/2] are halved and the DC column is not.
template <int N, int M>
__global__ void __launch_bounds__(kThreads) k_b_s1cols_odd(DevPlan p, const float2* __restrict__ phs,
                                                           const float2* __restrict__ gmt, float2* __restrict__ gs1,
                                                           int B) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    constexpr int T = FftPlan<M>::T, C = kThreads / T, ES = C, W = (N + 1) / 2;
    extern __shared__ float2 sm[];
    const int q = blockIdx.y, s = blockIdx.z, u0 = blockIdx.x * C;
    const int c = threadIdx.x % C, j = threadIdx.x / C, u = u0 + c;
    const float* dm = reinterpret_cast<const float*>(gmt + (size_t)q * W * N) + s;   // stride 2
    const float2* ph = phs + (size_t)(s * B + q) * W * N;
    bluestein<M>(sm + c, ES, j, N, p, [&](int v) {
        if (u >= W) return make_float2(0.f, 0.f);
        const float sc = u == 0 ? 1.f : 0.5f;
        return c_conj(c_scale(__ldg(ph + (size_t)u * N + v), sc * __ldg(dm + 2 * ((size_t)u * N + v))));
    });
    float2* out = gs1 + (size_t)(s * B + q) * N * W + u0;
    for (int idx = threadIdx.x; idx < C * N; idx += kThreads) {
        const int cc = idx % C, y = idx / C;
        if (u0 + cc < W) out[(size_t)y * W + cc] = c_conj(c_cjmul(__ldg(&p.chirp[y]), sm[spad(y) * ES + cc]));
    }
}

// Row part for an odd side: rows y and y + 1 of the column-transformed half plane H, extended
// Hermitian (G[0] = Re H[0], G[u] = H[u], G[N - u] = conj H[u]) and packed as G_y + i G_{y+1}; the
// inverse N-point DFT gives row y in the real part and row y + 1 in the imaginary part.
template <int N, int M>
__global__ void __launch_bounds__(kThreads) k_b_s1rows_odd(DevPlan p, const long long* __restrict__ tab,
                                                           const float2* __restrict__ gs1, float* __restrict__ df,
                                                           float* __restrict__ dg, int B) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    constexpr int T = FftPlan<M>::T, FPC = kThreads / T, SL = spad(M), W = (N + 1) / 2;
    extern __shared__ float2 sm[];
    const int q = blockIdx.y, s = blockIdx.z, r0 = blockIdx.x * FPC * 2;
    const int k = threadIdx.x / T, j = threadIdx.x % T, y = r0 + 2 * k;
    const bool oka = y < N, okb = y + 1 < N;
    const float2* ra = gs1 + ((size_t)(s * B + q) * N + y) * W;
    const float2* rb = ra + W;
    bluestein<M>(sm + k * SL, 1, j, N, p, [&](int x) {
        float2 a = make_float2(0.f, 0.f), b = a;
        const int u = x <= N / 2 ? x : N - x;
        if (oka) a = __ldg(ra + u);
        if (okb) b = __ldg(rb + u);
        float2 z;
        if (x == 0) z = make_float2(a.x, b.x);
        else if (x <= N / 2) z = make_float2(a.x - b.y, a.y + b.x);
        else z = make_float2(a.x + b.y, b.x - a.y);
        return c_conj(z);
    });
    float* out = (s ? dg : df) + tab[3 * q] + (size_t)y * N;
    const float wa = p.window && oka ? __ldg(&p.win[y]) : 1.f, wb = p.window && okb ? __ldg(&p.win[y + 1]) : 1.f;
    for (int x = j; x < N; x += T) {
        const float2 z = c_conj(c_cjmul(__ldg(&p.chirp[x]), sm[k * SL + spad(x)]));
        float va = z.x, vb = z.y;
        if (p.window) {
            const float wx = __ldg(&p.win[x]);
            va *= wa * wx;
            vb *= wb * wx;
        }
        if (oka) out[x] += va;
        if (okb) out[N + x] += vb;
    }
}

// ---------------------------------------------------------------------------------------------
// pose loss (Eq. 13) and its gradient
// ---------------------------------------------------------------------------------------------

// L = mean over pairs of sum over (theta, t_x, t_y) of |pose - gt| (kind 1, Eq. 13) or
// (pose - gt)^2 (kind 2); dpose = dL/dpose.  One block; fixed-order reduction.  The mean is over
// norm_pairs pairs (n_pairs, or the whole call when these pairs are one chunk of it).
__global__ void __launch_bounds__(256) k_pose_loss(int n_pairs, int norm_pairs, const float* __restrict__ pose,
                                                   const float* __restrict__ gt, int kind, float* __restrict__ loss,
                                                   float* __restrict__ dpose) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    __shared__ float red[32];
    const float inv = 1.f / (float)norm_pairs;
    float acc = 0.f;
    for (int i = threadIdx.x; i < 3 * n_pairs; i += blockDim.x) {
        const float d = pose[i] - gt[i];
        float l, gr;
        if (kind == 1) {
            l = fabsf(d);
            gr = d > 0.f ? inv : (d < 0.f ? -inv : 0.f);
        } else {
            l = d * d;
            gr = 2.f * d * inv;
        }
        acc += l;
        if (dpose) dpose[i] = gr;
    }
    acc = block_reduce<false>(acc, red);
    if (threadIdx.x == 0 && loss) loss[0] = acc * inv;
}

cudaError_t launch_pose_loss(int n_pairs, const float* pose, const float* gt, int kind, float* loss, float* dpose,
                             Tracer* tr, cudaStream_t st, int norm_pairs) {
    tr->before(K_LOSS, st);
    launch_pdl(k_pose_loss, 1, 256, 0, st, n_pairs, norm_pairs > 0 ? norm_pairs : n_pairs, pose, gt, kind, loss, dpose);
    tr->close(st);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------------

template <int L> constexpr size_t b_smem_rows() { return (size_t)(tpb_for(L) / FftPlan<L>::T) * spad(L) * sizeof(float2); }
template <int P, int C> constexpr size_t b_smem_cols() { return 2 * (size_t)spad(P) * C * sizeof(float2); }
template <int N> constexpr size_t b_smem_s1cols() {
    return (size_t)(s1cols_warp<N>() ? s1cols_stride<N>() : spad(N)) * (kThreads / FftPlan<N>::T) * sizeof(float2);
}
template <int NT, int RC> constexpr size_t b_smem_angle() { return (size_t)spad(NT) * RC * sizeof(float2); }

template <int NT>
static void launch_stage1_adjoint(const DevPlan& p, const Ws& w, int B, cudaStream_t st) {
    w.tr->before(K_B_THETA, st);
    launch_pdl(k_b_theta<NT>, B, 256, 0, st, p, w.ct, w.bsc, w.bdc);
    w.tr->before(K_B_ANGLE, st);
    if (p.angle_rc == 8)
        launch_pdl(k_b_angle<NT, 8>, dim3(angle_chunks(p), B), FftPlan<NT>::T * 8, b_smem_angle<NT, 8>(), st, p, w.ahat, w.bdc,
                                                                                                     w.gpol, B);
    else
        launch_pdl(k_b_angle<NT, 16>, dim3(angle_chunks(p), B), FftPlan<NT>::T * 16, b_smem_angle<NT, 16>(), st, 
            p, w.ahat, w.bdc, w.gpol, B);
}

template <int N, int PX, bool ODD>
static void launch_b_rot(const DevPlan& p, const Ws& w, int B, const long long* tab, const float* f,
                         const float* dpose, float* df, cudaStream_t st, const float* fwd_pose) {
    launch_pdl(k_b_rot<N, PX, ODD>, dim3(N * N / (kThreads * PX), B), kThreads, 0, st, p, tab, f, w.th, w.gfr, dpose, df,
               w.gpart, w.cnt, w.bsc, fwd_pose);
}

// N: the scan side; NE: stage 2's frame (N, or N + 1 for odd N); M: Bluestein length (0: none).
// The adjoint's column pass in radix order V with the size's column tile.
template <int N, int P, int V>
static void launch_b_cols(const DevPlan& p, const Ws& w, int B, cudaStream_t st) {
    constexpr int T2 = FftPlan<P>::T, C0 = tpb_for(P) / T2;   // the default tile; the 3 * 2^k lengths
    if constexpr (P % 3 == 0) {                                  // also have half and double
        if (p.col_tile == C0 / 2)
            launch_pdl(k_b_cols<N, P, C0 / 2, V>, dim3((P / 2) / (C0 / 2), B), (C0 / 2) * T2, b_smem_cols<P, C0 / 2>(), st,
                       p, w.b1, w.s2hat, w.b2, B);
        else if (p.col_tile == 2 * C0)
            launch_pdl(k_b_cols<N, P, 2 * C0, V>, dim3((P / 2) / (2 * C0), B), 2 * C0 * T2, b_smem_cols<P, 2 * C0>(), st,
                       p, w.b1, w.s2hat, w.b2, B);
        else
            launch_pdl(k_b_cols<N, P, C0, V>, dim3((P / 2) / C0, B), C0 * T2, b_smem_cols<P, C0>(), st, p, w.b1, w.s2hat,
                       w.b2, B);
    } else {
        launch_pdl(k_b_cols<N, P, C0, V>, dim3((P / 2) / C0, B), C0 * T2, b_smem_cols<P, C0>(), st, p, w.b1, w.s2hat,
                   w.b2, B);
    }
}

template <int N, int NE, int M, int P>
static cudaError_t launch_b(const DevPlan& p, const Ws& w, int B, const long long* tab, const float* f,
                            const float* g, const float* dpose, float* df, float* dg, cudaStream_t st,
                            const float* fwd_pose) {
    constexpr bool ODD = (N & 1) != 0;
    StageRange range("fmbym adjoint");
    if (!fwd_pose) {
        cudaError_t e = launch_forward(p, w, B, tab, f, g, w.bpose, nullptr, nullptr, st);
        if (e != cudaSuccess) return e;
        fwd_pose = w.bpose;
    }
    constexpr int T2 = FftPlan<P>::T, TB2 = tpb_for(P);
    w.tr->before(K_B_ROWS, st);
    launch_pdl(k_b_rows<NE, P, ODD>, dim3((NE / 2) / (TB2 / T2), B), TB2, b_smem_rows<P>(), st, p, tab, w.cxy, w.xm,
               fwd_pose, dpose, w.b1, B);
    w.tr->before(K_B_COLS, st);
    if constexpr (P % 3 == 0) {
        if (p.col_plan == 1) launch_b_cols<NE, P, 1>(p, w, B, st);
        else launch_b_cols<NE, P, 0>(p, w, B, st);
    } else {
        launch_b_cols<NE, P, 0>(p, w, B, st);
    }
    w.tr->before(K_B_C2R, st);
    launch_pdl(k_b_c2r<NE, P, ODD>, dim3((NE / 2) / (TB2 / T2), B, 2), TB2, b_smem_rows<P>(), st, p, tab, w.b2, w.gfr, df,
               dg, B);
    w.tr->before(K_B_ROT, st);
    const float* rsrc = p.rotate_target ? g : f;
    float* rdst = p.rotate_target ? dg : df;
    switch (p.rot_px) {
        case 1: launch_b_rot<NE, 1, ODD>(p, w, B, tab, rsrc, dpose, rdst, st, fwd_pose); break;
        case 2: launch_b_rot<NE, 2, ODD>(p, w, B, tab, rsrc, dpose, rdst, st, fwd_pose); break;
        case 8: launch_b_rot<NE, 8, ODD>(p, w, B, tab, rsrc, dpose, rdst, st, fwd_pose); break;
        default: launch_b_rot<NE, 4, ODD>(p, w, B, tab, rsrc, dpose, rdst, st, fwd_pose); break;
    }
    if (p.nt == 128) launch_stage1_adjoint<128>(p, w, B, st);
    else if (p.nt == 256) launch_stage1_adjoint<256>(p, w, B, st);
    else if (p.nt == 400) launch_stage1_adjoint<400>(p, w, B, st);
    else launch_stage1_adjoint_direct(p, w, B, st);   // no FFT plan: direct sums
    w.tr->before(K_B_POLT, st);
    const int E = (N / 2 + 1) * N, lb = (E + kThreads - 1) / kThreads;
    const int hb = (p.n_heavy + kThreads / 32 - 1) / (kThreads / 32);
    launch_pdl(k_b_polT, dim3(lb + hb, B), kThreads, 0, st, p, w.gpol, w.gmt, B, lb);
    if constexpr (M == 0) {
        constexpr int T1 = FftPlan<N>::T;
        w.tr->before(K_B_S1COLS, st);
        launch_pdl(k_b_s1cols<N>, dim3((N / 2) / (kThreads / T1), B, 2), kThreads, b_smem_s1cols<N>(), st, p, w.phs,
                   w.gmt, w.gs1, B);
        w.tr->before(K_B_S1ROWS, st);
        launch_pdl(k_b_s1rows<N>, dim3((N / 2) / (kThreads / T1), B, 2), kThreads, b_smem_rows<N>(), st, p, tab, w.gs1,
                   df, dg, B);
    } else {
        constexpr int TM = FftPlan<M>::T, W = (N + 1) / 2;
        w.tr->before(K_B_S1COLS, st);
        launch_pdl(k_b_s1cols_odd<N, M>, dim3(W / (kThreads / TM), B, 2), kThreads, b_smem_s1cols<M>(), st, p, w.phs,
                   w.gmt, w.gs1, B);
        w.tr->before(K_B_S1ROWS, st);
        launch_pdl(k_b_s1rows_odd<N, M>, dim3(W / (kThreads / TM), B, 2), kThreads, b_smem_rows<M>(), st, p, tab, w.gs1,
                   df, dg, B);
    }
    w.tr->close(st);
    return cudaGetLastError();
}

cudaError_t launch_backward(const DevPlan& p, const Ws& w, int B, const long long* tab, const float* f,
                            const float* g, const float* dpose, float* df, float* dg, cudaStream_t st,
                            const float* fwd_pose) {
    if (B <= 0) return cudaSuccess;
    switch (p.n) {
        case 127: return launch_b<127, 128, 256, 192>(p, w, B, tab, f, g, dpose, df, dg, st, fwd_pose);
        case 255: return launch_b<255, 256, 512, 384>(p, w, B, tab, f, g, dpose, df, dg, st, fwd_pose);
        case 511: return launch_b<511, 512, 1024, 768>(p, w, B, tab, f, g, dpose, df, dg, st, fwd_pose);
        case 128: return p.p == 192 ? launch_b<128, 128, 0, 192>(p, w, B, tab, f, g, dpose, df, dg, st, fwd_pose)
                                    : launch_b<128, 128, 0, 128>(p, w, B, tab, f, g, dpose, df, dg, st, fwd_pose);
        case 256: return p.p == 384 ? launch_b<256, 256, 0, 384>(p, w, B, tab, f, g, dpose, df, dg, st, fwd_pose)
                                    : launch_b<256, 256, 0, 256>(p, w, B, tab, f, g, dpose, df, dg, st, fwd_pose);
        default: return p.p == 768 ? launch_b<512, 512, 0, 768>(p, w, B, tab, f, g, dpose, df, dg, st, fwd_pose)
                                   : launch_b<512, 512, 0, 512>(p, w, B, tab, f, g, dpose, df, dg, st, fwd_pose);
    }
}

template <typename K>
static cudaError_t allow(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int N, int P, bool ODD>
static cudaError_t prepare_b() {
    cudaError_t e;
    if ((e = allow(k_b_rows<N, P, ODD>, b_smem_rows<P>())) != cudaSuccess) return e;
    constexpr int C0 = tpb_for(P) / FftPlan<P>::T;
    if ((e = allow(k_b_cols<N, P, C0, 0>, b_smem_cols<P, C0>())) != cudaSuccess) return e;
    if constexpr (P % 3 == 0) {
        if ((e = allow(k_b_cols<N, P, C0 / 2, 0>, b_smem_cols<P, C0 / 2>())) != cudaSuccess) return e;
        if ((e = allow(k_b_cols<N, P, 2 * C0, 0>, b_smem_cols<P, 2 * C0>())) != cudaSuccess) return e;
        if ((e = allow(k_b_cols<N, P, C0, 1>, b_smem_cols<P, C0>())) != cudaSuccess) return e;
        if ((e = allow(k_b_cols<N, P, C0 / 2, 1>, b_smem_cols<P, C0 / 2>())) != cudaSuccess) return e;
        if ((e = allow(k_b_cols<N, P, 2 * C0, 1>, b_smem_cols<P, 2 * C0>())) != cudaSuccess) return e;
    }
    if ((e = allow(k_b_c2r<N, P, ODD>, b_smem_rows<P>())) != cudaSuccess) return e;
    if constexpr (ODD) {
        constexpr int M = 2 * N;   // the Bluestein length of the odd side N - 1
        if ((e = allow(k_b_s1cols_odd<N - 1, M>, b_smem_s1cols<M>())) != cudaSuccess) return e;
        return allow(k_b_s1rows_odd<N - 1, M>, b_smem_rows<M>());
    } else {
        if ((e = allow(k_b_s1cols<N>, b_smem_s1cols<N>())) != cudaSuccess) return e;
        return allow(k_b_s1rows<N>, b_smem_rows<N>());
    }
}

cudaError_t prepare_backward_kernels() {
    cudaError_t e;
    if ((e = prepare_b<128, 192, false>()) != cudaSuccess) return e;
    if ((e = prepare_b<128, 128, false>()) != cudaSuccess) return e;
    if ((e = prepare_b<256, 384, false>()) != cudaSuccess) return e;
    if ((e = prepare_b<256, 256, false>()) != cudaSuccess) return e;
    if ((e = prepare_b<512, 768, false>()) != cudaSuccess) return e;
    if ((e = prepare_b<512, 512, false>()) != cudaSuccess) return e;
    if ((e = prepare_b<128, 192, true>()) != cudaSuccess) return e;
    if ((e = prepare_b<256, 384, true>()) != cudaSuccess) return e;
    if ((e = prepare_b<512, 768, true>()) != cudaSuccess) return e;
    if ((e = allow(k_b_angle<128, 8>, b_smem_angle<128, 8>())) != cudaSuccess) return e;
    if ((e = allow(k_b_angle<256, 8>, b_smem_angle<256, 8>())) != cudaSuccess) return e;
    if ((e = allow(k_b_angle<400, 8>, b_smem_angle<400, 8>())) != cudaSuccess) return e;
    if ((e = allow(k_b_angle<128, 16>, b_smem_angle<128, 16>())) != cudaSuccess) return e;
    if ((e = allow(k_b_angle<256, 16>, b_smem_angle<256, 16>())) != cudaSuccess) return e;
    return allow(k_b_angle<400, 16>, b_smem_angle<400, 16>());
}

}  // namespace fmbym
