// Shared-memory FFT engine for sm_103a.
//
// A group of T threads transforms one complex sequence of length L that lives in shared
// memory.  The transform is a Stockham autosort FFT (natural order in, natural order out): each
// pass p of radix R reads the butterfly inputs x[b + t L/R] (t < R) of butterfly b into
// registers, multiplies them by the twiddles W_{Ns R}^{(b mod Ns) t} (Ns = product of the
// radices of the earlier passes), does the radix-R DFT in registers and writes the outputs to
// x[(b / Ns) Ns R + (b mod Ns) + t Ns].  All reads of a pass finish before its writes start
// (one __syncthreads between them), so a single buffer suffices.
//
// Element i of a sequence sits at base + spad(i) * es, with spad(i) = i + i/16: the padding
// word every 16 elements makes the radix-16 scatter of the first pass bank-conflict free, and
// an element stride es > 1 interleaves several sequences (column tiles).
//
// Twiddles come from a table tw[k] = exp(-2 pi i k / L), k < L, computed in double precision on
// the host and rounded to float; the inverse transform uses their conjugates.  A butterfly loads
// one base twiddle (two for radix 16) and forms the other powers by at most three complex
// products, which keeps the table loads (divergent across a warp) off the L1 critical path.  Forward is the
// unnormalised DFT X[k] = sum_n x[n] exp(-2 pi i n k / L); inverse has the + sign and no 1/L.
#pragma once
#include <cuda_runtime.h>

namespace fmbym {

__host__ __device__ __forceinline__ constexpr int spad(int i) { return i + (i >> 4); }

// Asynchronous 8-byte global -> shared copy (cp.async); many can be in flight per thread.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
// Waits for every cp.async this thread issued (a __syncthreads must follow before others read).
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// Hint that brings [p, p + bytes) of global memory into L2 (one bulk prefetch; p and bytes
// multiples of 16).  No value is read into the SM, so a later load of the range hits L2.
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}

__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ float2 c_cjmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ float2 c_scale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 c_conj(float2 a) { return make_float2(a.x, -a.y); }
// a * (S i): S = -1 (forward) gives a * (-i), S = +1 gives a * i
template <int S> __device__ __forceinline__ float2 c_rot(float2 a) {
    return S < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

// ---------------------------------------------------------------------------------------------
// small DFTs in registers, y[k] = sum_n x[n] exp(S 2 pi i n k / R), in place, natural order
// ---------------------------------------------------------------------------------------------

template <int S> __device__ __forceinline__ void dft2(float2* v) {
    float2 a = v[0];
    v[0] = c_add(a, v[1]);
    v[1] = c_sub(a, v[1]);
}

template <int S> __device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
    float2 a = c_add(x0, x2), b = c_sub(x0, x2), c = c_add(x1, x3), d = c_rot<S>(c_sub(x1, x3));
    x0 = c_add(a, c);
    x2 = c_sub(a, c);
    x1 = c_add(b, d);
    x3 = c_sub(b, d);
}

template <int S> __device__ __forceinline__ void dft4(float2* v) { dft4<S>(v[0], v[1], v[2], v[3]); }

constexpr float kSqrtHalf = 0.70710678118654752440f;
constexpr float kCos8 = 0.92387953251128675613f;  // cos(pi/8)
constexpr float kSin8 = 0.38268343236508977173f;  // sin(pi/8)

template <int S> __device__ __forceinline__ void dft8(float2* v) {
    float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<S>(e0, e1, e2, e3);
    dft4<S>(o0, o1, o2, o3);
    // W8^1 = (1 + S i)/sqrt2, W8^2 = S i, W8^3 = (-1 + S i)/sqrt2
    o1 = make_float2((o1.x - S * o1.y) * kSqrtHalf, (o1.y + S * o1.x) * kSqrtHalf);
    o2 = c_rot<S>(o2);
    o3 = make_float2((-o3.x - S * o3.y) * kSqrtHalf, (-o3.y + S * o3.x) * kSqrtHalf);
    v[0] = c_add(e0, o0); v[4] = c_sub(e0, o0);
    v[1] = c_add(e1, o1); v[5] = c_sub(e1, o1);
    v[2] = c_add(e2, o2); v[6] = c_sub(e2, o2);
    v[3] = c_add(e3, o3); v[7] = c_sub(e3, o3);
}

// W16^m = exp(S 2 pi i m / 16) for the products m = n2 k1 that the 4 x 4 split needs
template <int S, int M> __device__ __forceinline__ float2 tw16(float2 a) {
    constexpr int m = M & 15;
    if constexpr (m == 0) return a;
    else if constexpr (m == 4) return c_rot<S>(a);
    else if constexpr (m == 8) return make_float2(-a.x, -a.y);
    else {
        constexpr float cs[16] = {1.f, kCos8, kSqrtHalf, kSin8, 0.f, -kSin8, -kSqrtHalf, -kCos8,
                                  -1.f, -kCos8, -kSqrtHalf, -kSin8, 0.f, kSin8, kSqrtHalf, kCos8};
        constexpr float sn[16] = {0.f, kSin8, kSqrtHalf, kCos8, 1.f, kCos8, kSqrtHalf, kSin8,
                                  0.f, -kSin8, -kSqrtHalf, -kCos8, -1.f, -kCos8, -kSqrtHalf, -kSin8};
        return c_mul(a, make_float2(cs[m], S * sn[m]));
    }
}

// 16-point DFT as 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2.
template <int S> __device__ __forceinline__ void dft16(float2* v) {
    // step 1: length-4 DFTs over n1 for each n2 (results A[n2][k1] stored at v[4 k1 + n2])
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<S>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
    // step 2: twiddles W16^{n2 k1}
    v[5] = tw16<S, 1>(v[5]);   v[6] = tw16<S, 2>(v[6]);   v[7] = tw16<S, 3>(v[7]);
    v[9] = tw16<S, 2>(v[9]);   v[10] = tw16<S, 4>(v[10]); v[11] = tw16<S, 6>(v[11]);
    v[13] = tw16<S, 3>(v[13]); v[14] = tw16<S, 6>(v[14]); v[15] = tw16<S, 9>(v[15]);
    // step 3: length-4 DFTs over n2 for each k1; output k1 + 4 k2
    float2 y[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        float2 a0 = v[4 * k1], a1 = v[4 * k1 + 1], a2 = v[4 * k1 + 2], a3 = v[4 * k1 + 3];
        dft4<S>(a0, a1, a2, a3);
        y[k1] = a0; y[k1 + 4] = a1; y[k1 + 8] = a2; y[k1 + 12] = a3;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = y[i];
}

// 3-point DFT: y1 = x0 - (x1 + x2)/2 + S i (sqrt3/2)(x1 - x2), y2 the conjugate combination
template <int S> __device__ __forceinline__ void dft3(float2* v) {
    constexpr float h = 0.86602540378443864676f;  // sqrt(3)/2
    const float2 t = c_add(v[1], v[2]);
    const float2 d = c_rot<S>(c_sub(v[1], v[2]));
    const float2 m = make_float2(v[0].x - 0.5f * t.x, v[0].y - 0.5f * t.y);
    v[0] = c_add(v[0], t);
    v[1] = make_float2(m.x + h * d.x, m.y + h * d.y);
    v[2] = make_float2(m.x - h * d.x, m.y - h * d.y);
}

// 5-point DFT from cos/sin of 2 pi/5 and 4 pi/5
template <int S> __device__ __forceinline__ void dft5(float2* v) {
    constexpr float c1 = 0.30901699437494742410f;   // cos(2 pi / 5)
    constexpr float c2 = -0.80901699437494742410f;  // cos(4 pi / 5)
    constexpr float s1 = 0.95105651629515357212f;   // sin(2 pi / 5)
    constexpr float s2 = 0.58778525229247312917f;   // sin(4 pi / 5)
    float2 x0 = v[0];
    float2 t1 = c_add(v[1], v[4]), t2 = c_add(v[2], v[3]);
    float2 t3 = c_sub(v[1], v[4]), t4 = c_sub(v[2], v[3]);
    float2 a1 = make_float2(x0.x + c1 * t1.x + c2 * t2.x, x0.y + c1 * t1.y + c2 * t2.y);
    float2 a2 = make_float2(x0.x + c2 * t1.x + c1 * t2.x, x0.y + c2 * t1.y + c1 * t2.y);
    float2 b1 = make_float2(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y);
    float2 b2 = make_float2(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y);
    v[0] = make_float2(x0.x + t1.x + t2.x, x0.y + t1.y + t2.y);
    // y1 = a1 + S i b1, y4 = a1 - S i b1, y2 = a2 + S i b2, y3 = a2 - S i b2
    float2 ib1 = c_rot<S>(b1), ib2 = c_rot<S>(b2);
    v[1] = c_add(a1, ib1);
    v[4] = c_sub(a1, ib1);
    v[2] = c_add(a2, ib2);
    v[3] = c_sub(a2, ib2);
}

template <int R, int S> __device__ __forceinline__ void dft(float2* v) {
    if constexpr (R == 2) dft2<S>(v);
    else if constexpr (R == 3) dft3<S>(v);
    else if constexpr (R == 4) dft4<S>(v);
    else if constexpr (R == 5) dft5<S>(v);
    else if constexpr (R == 8) dft8<S>(v);
    else if constexpr (R == 16) dft16<S>(v);
    else static_assert(R == 2, "unsupported radix");
}

// ---------------------------------------------------------------------------------------------
// one Stockham pass; every thread of the CTA must call it (it contains __syncthreads)
// ---------------------------------------------------------------------------------------------

// Twiddles W_{NS R}^{(b mod NS) t} of butterfly b applied to its inputs v[1..R-1] (no-op for NS = 1):
// one table load of W^bm (and of W^(4 bm) for radix 16); the other powers by complex products at
// most three deep.
template <int L, int R, int NS, int S>
__device__ __forceinline__ void twiddle(float2* v, int b, const float2* __restrict__ tw) {
    if constexpr (NS > 1) {
        constexpr int STEP = L / (NS * R);
        const int bm = b % NS;
        float2 w[R];
        w[1] = __ldg(&tw[bm * STEP]);
        if constexpr (S > 0) w[1].y = -w[1].y;
        if constexpr (R >= 16) {
            w[4] = __ldg(&tw[4 * bm * STEP]);
            if constexpr (S > 0) w[4].y = -w[4].y;
            w[2] = c_mul(w[1], w[1]);
            w[3] = c_mul(w[2], w[1]);
            w[8] = c_mul(w[4], w[4]);
            w[12] = c_mul(w[8], w[4]);
#pragma unroll
            for (int t = 5; t < R; ++t)
                if ((t & 3) != 0) w[t] = c_mul(w[t & ~3], w[t & 3]);
        } else {
#pragma unroll
            for (int t = 2; t < R; ++t) w[t] = (t & 1) ? c_mul(w[t - 1], w[1]) : c_mul(w[t / 2], w[t / 2]);
        }
#pragma unroll
        for (int t = 1; t < R; ++t) v[t] = c_mul(v[t], w[t]);
    }
}

// Position of output t of butterfly b in a pass of radix R after passes of product NS.
template <int R, int NS> __device__ __forceinline__ int pass_out(int b, int t) {
    return (b / NS) * NS * R + (b % NS) + t * NS;
}

template <int L, int T, int R, int NS, int S>
__device__ __forceinline__ void fft_pass(float2* buf, int es, int j, bool active, const float2* __restrict__ tw) {
    constexpr int NB = L / R;                // butterflies in the pass
    constexpr int BPT = (NB + T - 1) / T;    // butterflies per thread
    static_assert(L % R == 0, "radix must divide the length");
    float2 v[BPT][R];
#pragma unroll
    for (int m = 0; m < BPT; ++m) {
        const int b = j + m * T;
        if (active && (NB % T == 0 || b < NB)) {
#pragma unroll
            for (int t = 0; t < R; ++t) v[m][t] = buf[spad(b + t * NB) * es];
            twiddle<L, R, NS, S>(v[m], b, tw);
            dft<R, S>(v[m]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < BPT; ++m) {
        const int b = j + m * T;
        if (active && (NB % T == 0 || b < NB)) {
#pragma unroll
            for (int t = 0; t < R; ++t) buf[spad(pass_out<R, NS>(b, t)) * es] = v[m][t];
        }
    }
    __syncthreads();
}

// The same pass on two sequences at once (one pair of barriers for both).
template <int L, int T, int R, int NS, int S>
__device__ __forceinline__ void fft_pass2(float2* b0, float2* b1, int es, int j, const float2* __restrict__ tw) {
    constexpr int NB = L / R;
    constexpr int BPT = (NB + T - 1) / T;
    float2 v[BPT][R], w[BPT][R];
#pragma unroll
    for (int m = 0; m < BPT; ++m) {
        const int b = j + m * T;
        if (NB % T == 0 || b < NB) {
#pragma unroll
            for (int t = 0; t < R; ++t) {
                v[m][t] = b0[spad(b + t * NB) * es];
                w[m][t] = b1[spad(b + t * NB) * es];
            }
            twiddle<L, R, NS, S>(v[m], b, tw);
            dft<R, S>(v[m]);
            twiddle<L, R, NS, S>(w[m], b, tw);
            dft<R, S>(w[m]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < BPT; ++m) {
        const int b = j + m * T;
        if (NB % T == 0 || b < NB) {
#pragma unroll
            for (int t = 0; t < R; ++t) {
                b0[spad(pass_out<R, NS>(b, t)) * es] = v[m][t];
                b1[spad(pass_out<R, NS>(b, t)) * es] = w[m][t];
            }
        }
    }
    __syncthreads();
}

template <int L, int T, int S, int NS, int R, int... Rest>
__device__ __forceinline__ void fft_passes(float2* buf, int es, int j, bool active, const float2* __restrict__ tw) {
    fft_pass<L, T, R, NS, S>(buf, es, j, active, tw);
    if constexpr (sizeof...(Rest) > 0) fft_passes<L, T, S, NS * R, Rest...>(buf, es, j, active, tw);
}

// Radix plans: every length uses radix 16 first; T = L/16 threads per sequence.  NP passes of
// radices R1 = 16, R2 (, R3).  The column kernels that chain a forward transform, a pointwise
// product and an inverse run the inverse in the reverse radix order: the forward's last pass and
// the inverse's first pass then read and write the same butterfly positions, so the product
// happens in registers between them.
//
// V = 1 is the other valid order of the 3 * 2^k lengths, the middle and last radices swapped
// (16, 3, R): its last pass has L / R = 48 butterflies for every such length, one per thread at
// 768, so the fused turn of a column pass has no ragged tail, at the cost of holding R points per
// butterfly.  The autotuner picks the order of the stage-2 column passes per size.
template <int L, int V = 0> struct FftPlan;
template <> struct FftPlan<128> { static constexpr int T = 8, NP = 2, R2 = 8, R3 = 1; };
template <> struct FftPlan<192> { static constexpr int T = 12, NP = 3, R2 = 4, R3 = 3; };
template <> struct FftPlan<256> { static constexpr int T = 16, NP = 2, R2 = 16, R3 = 1; };
template <> struct FftPlan<384> { static constexpr int T = 24, NP = 3, R2 = 8, R3 = 3; };
template <> struct FftPlan<400> { static constexpr int T = 25, NP = 3, R2 = 5, R3 = 5; };
template <> struct FftPlan<512> { static constexpr int T = 32, NP = 3, R2 = 16, R3 = 2; };
template <> struct FftPlan<768> { static constexpr int T = 48, NP = 3, R2 = 16, R3 = 3; };
template <> struct FftPlan<1024> { static constexpr int T = 64, NP = 3, R2 = 16, R3 = 4; };
template <> struct FftPlan<192, 1> { static constexpr int T = 12, NP = 3, R2 = 3, R3 = 4; };
template <> struct FftPlan<384, 1> { static constexpr int T = 24, NP = 3, R2 = 3, R3 = 8; };
template <> struct FftPlan<768, 1> { static constexpr int T = 48, NP = 3, R2 = 3, R3 = 16; };

// In-place FFT of one sequence (element i at buf[spad(i) * es]) by thread j < T of its group.
// S = -1 forward, +1 inverse.  Threads with active = false only take part in the barriers.
template <int L, int S>
__device__ __forceinline__ void fft(float2* buf, int es, int j, bool active, const float2* __restrict__ tw) {
    using PL = FftPlan<L>;
    if constexpr (PL::NP == 2) fft_passes<L, PL::T, S, 1, 16, PL::R2>(buf, es, j, active, tw);
    else fft_passes<L, PL::T, S, 1, 16, PL::R2, PL::R3>(buf, es, j, active, tw);
}

// ---------------------------------------------------------------------------------------------
// column transforms fed from and stored to global memory
// ---------------------------------------------------------------------------------------------
//
// A tile holds C columns interleaved element by element (element i of column c at
// buf[spad(i) * C + c]); thread (c, j) of the tile is column c's thread j < T.

// The forward first pass (radix 16, no twiddles) of two columns whose inputs come from global
// memory: thread j loads x[j + t T], t < 16, through load0(pos) and load1(pos) (all 32 loads in
// flight before the first use) and writes the outputs to the tiles.
template <int L, int S = -1, class Load0, class Load1>
__device__ __forceinline__ void first_pass_global2(float2* b0, float2* b1, int es, int j, Load0 load0, Load1 load1) {
    constexpr int T = FftPlan<L>::T;
    float2 v[16], w[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) {
        v[t] = load0(j + t * T);
        w[t] = load1(j + t * T);
    }
    dft16<S>(v);
    dft16<S>(w);
#pragma unroll
    for (int t = 0; t < 16; ++t) {
        b0[spad(16 * j + t) * es] = v[t];
        b1[spad(16 * j + t) * es] = w[t];
    }
}

template <int L, int S = -1, class Load>
__device__ __forceinline__ void first_pass_global(float2* b0, int es, int j, Load load) {
    constexpr int T = FftPlan<L>::T;
    float2 v[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) v[t] = load(j + t * T);
    dft16<S>(v);
#pragma unroll
    for (int t = 0; t < 16; ++t) b0[spad(16 * j + t) * es] = v[t];
}

// The forward transform's last pass of two columns, their pointwise product and the inverse
// transform's first pass, in registers.  With the inverse in the reverse radix order, the forward's
// last pass (radix RL, stride L / RL) writes exactly the positions b + t L/RL that it reads, and
// the inverse's first pass (radix RL, no twiddles) reads them: one thread owns a butterfly from
// the forward through the product to the inverse.  MODE_A = 0: a is transformed here; 1: a is
// transformed here and its final values are stored back in place (same thread, same positions,
// no barrier needed); 2: a already holds its final values.  prod(A, X) gives the product; the
// inverse first pass's outputs go to tb.  keep(pos, A, X) sees both transformed values at each
// position (to store them for a later pass).  Every thread of the CTA must call it.
template <int L, int MODE_A, int V, class Prod, class Keep>
__device__ __forceinline__ void fused_turn(float2* ta, float2* tb, int es, int j, const float2* __restrict__ tw,
                                           Prod prod, Keep keep) {
    using PL = FftPlan<L, V>;
    constexpr int T = PL::T, RL = PL::NP == 3 ? PL::R3 : PL::R2, NBL = L / RL, BPL = (NBL + T - 1) / T;
    float2 o[BPL][RL];
#pragma unroll
    for (int m = 0; m < BPL; ++m) {
        const int b = j + m * T;
        if (NBL % T == 0 || b < NBL) {
            float2 a[RL], x[RL];
#pragma unroll
            for (int t = 0; t < RL; ++t) {
                a[t] = ta[spad(b + t * NBL) * es];
                x[t] = tb[spad(b + t * NBL) * es];
            }
            if constexpr (MODE_A != 2) {
                twiddle<L, RL, NBL, -1>(a, b, tw);
                dft<RL, -1>(a);
                if constexpr (MODE_A == 1) {
#pragma unroll
                    for (int t = 0; t < RL; ++t) ta[spad(b + t * NBL) * es] = a[t];
                }
            }
            twiddle<L, RL, NBL, -1>(x, b, tw);
            dft<RL, -1>(x);
#pragma unroll
            for (int t = 0; t < RL; ++t) {
                keep(b + t * NBL, a[t], x[t]);
                o[m][t] = prod(a[t], x[t]);
            }
            dft<RL, +1>(o[m]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < BPL; ++m) {
        const int b = j + m * T;
        if (NBL % T == 0 || b < NBL) {
#pragma unroll
            for (int t = 0; t < RL; ++t) tb[spad(RL * b + t) * es] = o[m][t];
        }
    }
    __syncthreads();
}

// fused_turn without keeping the transformed values.
template <int L, int MODE_A, int V, class Prod>
__device__ __forceinline__ void fused_turn(float2* ta, float2* tb, int es, int j, const float2* __restrict__ tw,
                                           Prod prod) {
    fused_turn<L, MODE_A, V>(ta, tb, es, j, tw, prod, [](int, float2, float2) {});
}

// The inverse transform's remaining passes after fused_turn (or after its first pass): the middle
// pass (three-pass plans), then the last pass (radix 16, stride T) with its outputs handed to
// store(pos, value) instead of the tile.
template <int L, int V, class Store>
__device__ __forceinline__ void inverse_rest_global(float2* buf, int es, int j, const float2* __restrict__ tw,
                                                    Store store) {
    using PL = FftPlan<L, V>;
    constexpr int T = PL::T, RL = PL::NP == 3 ? PL::R3 : PL::R2;
    if constexpr (PL::NP == 3) fft_pass<L, T, PL::R2, RL, +1>(buf, es, j, true, tw);
    float2 v[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) v[t] = buf[spad(j + t * T) * es];
    twiddle<L, 16, T, +1>(v, j, tw);
    dft16<+1>(v);
#pragma unroll
    for (int t = 0; t < 16; ++t) store(j + t * T, v[t]);
}

// inverse_rest_global of two sequences: one middle pass over both (one pair of barriers) when a
// thread holds one butterfly of it, else one middle pass after the other (fewer live registers),
// then each last pass.
template <int L, int V, class Store0, class Store1>
__device__ __forceinline__ void inverse_rest_global2(float2* b0, float2* b1, int es, int j,
                                                     const float2* __restrict__ tw, Store0 store0, Store1 store1) {
    using PL = FftPlan<L, V>;
    constexpr int T = PL::T, RL = PL::NP == 3 ? PL::R3 : PL::R2;
    if constexpr (PL::NP == 3) {
        if constexpr (L / PL::R2 <= T) {
            fft_pass2<L, T, PL::R2, RL, +1>(b0, b1, es, j, tw);
        } else {
            fft_pass<L, T, PL::R2, RL, +1>(b0, es, j, true, tw);
            fft_pass<L, T, PL::R2, RL, +1>(b1, es, j, true, tw);
        }
    }
    float2 v[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) v[t] = b0[spad(j + t * T) * es];
    twiddle<L, 16, T, +1>(v, j, tw);
    dft16<+1>(v);
#pragma unroll
    for (int t = 0; t < 16; ++t) store0(j + t * T, v[t]);
#pragma unroll
    for (int t = 0; t < 16; ++t) v[t] = b1[spad(j + t * T) * es];
    twiddle<L, 16, T, +1>(v, j, tw);
    dft16<+1>(v);
#pragma unroll
    for (int t = 0; t < 16; ++t) store1(j + t * T, v[t]);
}

// The passes after the first (FIRST = 2), in the plan's own radix order, in shared memory.
template <int L, int S, int FIRST>
__device__ __forceinline__ void fft_passes_from(float2* buf, int es, int j, const float2* __restrict__ tw) {
    using PL = FftPlan<L>;
    static_assert(FIRST == 2, "only the passes after the first");
    if constexpr (PL::NP == 2) fft_pass<L, PL::T, PL::R2, 16, S>(buf, es, j, true, tw);
    else fft_passes<L, PL::T, S, 16, PL::R2, PL::R3>(buf, es, j, true, tw);
}

// The middle pass (three-pass plans) and the last pass of a transform in the plan's own radix
// order after first_pass_global; the last pass (radix RL, stride L / RL) hands its outputs to
// store(pos, value), pos in natural order.
template <int L, int S, class Store>
__device__ __forceinline__ void rest_global(float2* buf, int es, int j, const float2* __restrict__ tw, Store store) {
    using PL = FftPlan<L>;
    constexpr int T = PL::T, RL = PL::NP == 3 ? PL::R3 : PL::R2, NBL = L / RL, BPL = (NBL + T - 1) / T;
    if constexpr (PL::NP == 3) fft_pass<L, T, PL::R2, 16, S>(buf, es, j, true, tw);
#pragma unroll
    for (int m = 0; m < BPL; ++m) {
        const int b = j + m * T;
        if (NBL % T == 0 || b < NBL) {
            float2 v[RL];
#pragma unroll
            for (int t = 0; t < RL; ++t) v[t] = buf[spad(b + t * NBL) * es];
            twiddle<L, RL, NBL, S>(v, b, tw);
            dft<RL, S>(v);
#pragma unroll
            for (int t = 0; t < RL; ++t) store(b + t * NBL, v[t]);
        }
    }
}

// A packed pair of real rows, Z = FFT(x_a + i x_b) of length L, gives the half spectra
// X_a[u] = (Z[u] + conj Z[L-u]) / 2 and X_b[u] = (Z[u] - conj Z[L-u]) / 2i.  Column u = 0 of the
// half spectra packs the real DC and Nyquist values (X[0], X[L/2]) as one complex number.
// zu = Z[u], zm = Z[u == 0 ? L/2 : L - u]; odd selects X_b.
__device__ __forceinline__ float2 unpack_half(float2 zu, float2 zm, bool u0, bool odd) {
    if (u0) return odd ? make_float2(zu.y, zm.y) : make_float2(zu.x, zm.x);
    return odd ? make_float2(0.5f * (zu.y + zm.y), -0.5f * (zu.x - zm.x))
               : make_float2(0.5f * (zu.x + zm.x), 0.5f * (zu.y - zm.y));
}

// Z[x] of the packed inverse transform of two half spectra A (row ra) and B (row rb), columns
// u in [0, L/2) with column 0 holding (DC, Nyquist): Z[x] = A[x] + i B[x] under the Hermitian
// extension A[L - u] = conj A[u], so that the inverse of Z is a + i b for the real rows a, b.
__device__ __forceinline__ float2 pack_inverse(const float2* __restrict__ ra, const float2* __restrict__ rb, int x,
                                               int L) {
    const int W = L / 2;
    if (x == 0 || x == W) {
        const float2 a = __ldg(ra), b = __ldg(rb);
        return x == 0 ? make_float2(a.x, b.x) : make_float2(a.y, b.y);
    }
    if (x < W) {
        const float2 a = __ldg(ra + x), b = __ldg(rb + x);
        return make_float2(a.x - b.y, a.y + b.x);
    }
    const float2 a = __ldg(ra + (L - x)), b = __ldg(rb + (L - x));
    return make_float2(a.x + b.y, b.x - a.y);
}

// Last radix of the forward plan and the stride of its pass.
template <int L, int V = 0> __host__ __device__ constexpr int last_radix() {
    return FftPlan<L, V>::NP == 3 ? FftPlan<L, V>::R3 : FftPlan<L, V>::R2;
}

// Threads of a CTA that runs several length-L sequences side by side: a multiple of both the
// group size and 32 (192 for the 3 * 2^k lengths, 256 otherwise).
__host__ __device__ constexpr int tpb_for(int L) { return (L % 3 == 0) ? 192 : 256; }

// Minimum resident CTAs asked of the compiler for a column pass of length L with C columns per
// CTA: the 3 * 2^k lengths keep 576 threads per SM (96 registers a thread), the others 512.
__host__ __device__ constexpr int col_min_blocks(int L, int C) {
    return (L % 3 == 0 ? 576 : 512) / (C * (L / 16)) > 0 ? (L % 3 == 0 ? 576 : 512) / (C * (L / 16)) : 1;
}

}  // namespace fmbym
