// Shared declarations of the CUDA library: per-size device plans, the workspace layout of one
// size group, and the launchers of the forward and backward kernel sequences.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <vector>

#include "fft.cuh"

namespace fmbym {

constexpr int kThreads = 256;   // threads of the FFT kernels
// Device side of a programmatic dependent launch: waits until the kernel launched before this one
// on the stream has completed and its writes are visible (returns at once without such a
// predecessor).  Every kernel of the search calls it before its first global memory access.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// Launches a kernel that may be scheduled while its predecessor on the stream drains (programmatic
// stream serialization).  Because the kernel's grid_dep_wait() orders all of its reads and writes
// after the predecessor's completion, only the launch and the scheduling of its blocks overlap.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// An NVTX range over the launches of one stage (visible to Nsight tools on the host timeline;
// costs nothing measurable without a tool attached).
struct StageRange {
    explicit StageRange(const char* name) { nvtxRangePushA(name); }
    ~StageRange() { nvtxRangePop(); }
};

// Launch schedules with more than one compiled variant; each size's DevPlan names the variant its
// launches use (the defaults below, or the autotuner's measured choice).
constexpr int kAngleRadiiMin = 8;   // radii per CTA of the angle correlation and its adjoint: 8 or 16
constexpr int kAngleRadii = 16;
constexpr int kRotPixels = 4;       // pixels per thread of the Rotate adjoint: 1, 2, 4 or 8
constexpr int kSplitXY = 32;    // CTAs per pair of the translation soft-argmax

// One bilinear Cart2Pol sample: floor of the (u, v) frequency and the fractions.
struct PolarSample {
    int x0, y0;
    float fx, fy;
};

// Device-side plan of one scan size (tables built on the host in double precision).
struct DevPlan {
    int n, p, nt, nr;      // scan side, padded side (2N or N), angle bins, radii
    int m_lo, m_hi;        // band-pass: keep integer rho^2 in [m_lo, m_hi]
    int window, score_norm, angle_score, full_circle, rotate_target;
    float temp_theta, temp_xy, delta_xy;
    const float* win;      // [N] periodic Hann
    const float2* tw_n;    // [N]  exp(-2 pi i k / N)
    const float2* tw_p;    // [P]  exp(-2 pi i k / P)
    const float2* tw_t;    // [n_theta] exp(-2 pi i k / n_theta)
    const PolarSample* polar;  // [n_theta][n_r]
    // odd N only (the paper's 127, 255, 511): the N-point DFTs of stage 1 run as Bluestein
    // convolutions through M-point FFTs, M = 2 (N + 1) >= 2N - 1
    int m;                 // M (0 for even N)
    const float2* tw_m;    // [M]  exp(-2 pi i k / M)
    const float2* chirp;   // [N]  w[n] = exp(+i pi n^2 / N), exponent reduced mod 2N in integers
    const float2* bh;      // [M]  FFT_M of the chirp filter b (b[m] = w[|m|] for |m| < N), times 1/M
    // transpose of the bilinear polar gather onto the u-major half plane [N/2+1][N]: the
    // samples that read element e are csr_col[csr_ptr[e] .. csr_ptr[e+1]) with weights csr_w
    const int* csr_ptr;
    const int* csr_col;
    const float* csr_w;
    // elements whose CSR row has more than kHeavyRow taps (near the DC bin every angle samples the
    // same few elements); the adjoint gives each of them a warp instead of a thread
    const int* heavy;
    int n_heavy;
    // launch schedules: columns per CTA of the stage-2 column passes (half, the default, or twice
    // tpb_for(P) / T), radii per CTA of the angle kernels, pixels per thread of the Rotate adjoint,
    // radix order of the stage-2 column passes (FftPlan<P, col_plan>; 1 only for P = 3 * 2^k)
    int col_tile, angle_rc, rot_px, col_plan;
};

constexpr int kHeavyRow = 32;

// Stage 2 of an odd scan side N runs in the even frame N + 1 (one zero row and column; the lag
// set of the frame has one extra lag, -(N + 1)/2, that the kernels leave out).
__host__ __device__ constexpr int frame_n(int n) { return n + (n & 1); }

inline int angle_chunks(const DevPlan& p) { return (p.nr + p.angle_rc - 1) / p.angle_rc; }
inline int angle_chunks_max(const DevPlan& p) { return (p.nr + kAngleRadiiMin - 1) / kAngleRadiiMin; }
inline int fft_threads(int L) { return L / 16 == 25 ? 25 : L / 16; }
inline int c2r_blocks(const DevPlan& p) { return (frame_n(p.n) / 2) / (tpb_for(p.p) / fft_threads(p.p)); }

// Kernel kinds, for the launch tracer.
enum Kind {
    K_S1_ROWS, K_S1_COLS, K_ANGLE, K_THETA, K_S2_ROWS, K_S2_COLS, K_S2_C2R, K_SXY,
    K_B_SXY, K_B_COLS, K_B_ROWS, K_B_ROT, K_B_THETA, K_B_ANGLE, K_B_S1COLS, K_B_S1ROWS, K_B_C2R, K_B_POLT,
    K_LOSS, K_COUNT
};
extern const char* const kKindNames[K_COUNT];

// Launch tracer: counts launches and, when on, records one CUDA event before every launch and one
// after the last launch of a call on the launching stream, so kernel i lasts from its event to the
// next one.  Events come from a fixed pool; recording stops when the pool is used up.
struct Tracer {
    bool on = false;
    std::vector<cudaEvent_t> ev;
    std::vector<int> kind;
    size_t used = 0;
    long long launches = 0;
    void before(int k, cudaStream_t st) {
        ++launches;
        if (!on || used >= ev.size()) return;
        cudaEventRecord(ev[used], st);
        kind[used++] = k;
    }
    void close(cudaStream_t st) {
        if (!on || used >= ev.size()) return;
        cudaEventRecord(ev[used], st);
        kind[used++] = -1;
    }
};

// Workspace of one size group of B pairs (pointers into the handle's workspace).
struct Ws {
    float2* s1;   // [2][B][N][N/2]   stage-1 row spectra (packed real FFT rows)
    float* mt;    // [B][N/2+1][N][2] stage-1 band-passed magnitudes of (f, g), u-major, interleaved
    float2* sp;   // [B][chunks][n_theta] per-chunk sums of conj(A_f) A_g along angle
    float* th;    // [B][8] theta, cos hi/lo, sin hi/lo
    float2* s2;   // [2][B][N][P/2]   stage-2 row spectra of the rotated source and the target
    float2* s3;   // [B][N][P/2]      product after the inverse column pass, lag rows
    float* cxy;   // [B][N][N]        translation scores when the caller does not keep them
    float* st;    // [B][c2r blocks][4] per-block mean, M2, max of the translation scores
    float* sx;    // [B][kSplitXY][8] soft-argmax partial sums
    float* xm;    // [B][8]           translation soft-argmax statistics and moments kept for the adjoint
    float* fc;    // [B][8]           full circle: stage 1's heading splits, the theta + pi peak
    float* fcpose;  // [pairs][3]     full circle: the theta + pi candidate's translation, by pair index
    unsigned* cnt;  // [B] completion counters of the last-block reductions: a handle-wide array that
                    // is zero between launches (the last block of a pair resets its counter)
    float* ct;    // [B][n_theta]     angle scores in lag order (kept for the adjoint)
    float2* ahat; // [B][n_theta][n_r] FFT along angle of A_f + i A_g, kept by the forward for the
                  //                  adjoint (NULL: not kept)
    float2* phs;  // [2][B][N/2+1][N] band-limited unit phasors F/|F| of stage 1, kept likewise
    float2* s2hat;  // [2][B][P/2][P] column spectra of f' and g (both 2D transforms), column-major,
                    //                kept likewise
    // adjoint
    float* bpose; // [pairs][3]       recomputed pose, indexed by pair (handle-wide)
    float* bsc;   // [B][16]          per-pair scalars of the adjoint (d theta at 8)
    float* gpart; // [B][N*N/256]     per-block partial sums of d theta through Rotate
    float2* b1;   // [B][N][P/2]      row spectra of the embedded d c_xy (lag rows)
    float2* b2;   // [2][B][N][P/2]   inverse column pass of conj(D) G and D F'
    float* gfr;   // [B][N][N]        d rotated source
    float2* bdc;  // [B][n_theta]     FFT of d c_theta along angle
    float2* gpol; // [B][n_theta][n_r] d polar arrays of (f, g)
    float2* gmt;  // [B][N/2+1][N]    d magnitudes of (f, g)
    float2* gs1;  // [2][B][N][N/2]   inverse column pass of the stage-1 adjoint
    Tracer* tr;   // launch tracer of the handle
};

size_t ws_bytes(const DevPlan& p, int B, bool backward);
Ws ws_carve(const DevPlan& p, int B, void* base, bool backward);

// tab: device long long [B][3] = (scan offset, c_theta offset, pair index)
// Stage 2 only, for the headings already in w.th (the exhaustive search's inner step).
cudaError_t launch_forward_stage2(const DevPlan& p, const Ws& w, int B, const long long* tab, const float* f,
                                  const float* g, float* pose, float* c_xy, cudaStream_t st);
// Exhaustive rotate-then-correlate search over n_angles host headings (exhaustive.cu).
// The angle stage by direct circular sums, for angle counts without an FFT plan (angle_direct.cu).
bool fft_angle_count(int nt);
cudaError_t launch_stage1_direct(const DevPlan& p, const Ws& w, int B, const long long* tab, float* pose,
                                 float* c_theta, cudaStream_t st);
void launch_stage1_adjoint_direct(const DevPlan& p, const Ws& w, int B, cudaStream_t st);
cudaError_t launch_exhaustive(const DevPlan& p, const Ws& w, int B, const long long* tab, const float* f,
                              const float* g, int n_angles, const float* angles, float* cand, float4* best,
                              float* peaks, float* pose, cudaStream_t st);
cudaError_t launch_forward(const DevPlan& p, const Ws& w, int B, const long long* tab, const float* f,
                           const float* g, float* pose, float* c_theta, float* c_xy, cudaStream_t st);
// fwd_pose: NULL recomputes the forward into the workspace first (the stateless adjoint); otherwise
// the workspace still holds this call's forward intermediates and fwd_pose is its pose output.
cudaError_t launch_backward(const DevPlan& p, const Ws& w, int B, const long long* tab, const float* f,
                            const float* g, const float* dpose, float* df, float* dg, cudaStream_t st,
                            const float* fwd_pose);
// norm_pairs: the count the mean divides by (0: n_pairs)
cudaError_t launch_pose_loss(int n_pairs, const float* pose, const float* gt, int kind, float* loss, float* dpose,
                             Tracer* tr, cudaStream_t st, int norm_pairs = 0);
cudaError_t prepare_kernels();

}  // namespace fmbym
