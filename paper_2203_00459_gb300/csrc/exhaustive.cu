// Exhaustive rotate-then-correlate search: the brute-force method that the decoupled search
// replaces (the "raw" rows of Tab. IIIa; Sec. I and III describe it as trying every heading by
// rotating one scan and correlating it with the other).  For every candidate heading theta_k the
// source is rotated and correlated with the target by the decoupled search's own stage-2 kernels
// (Rotate, zero-padded correlation, soft-argmax), so the two methods differ only in how the
// heading is found.  The heading is the candidate whose correlation peak is highest (the first
// one on ties), the translation that candidate's stage-2 soft-argmax.
#include <cfloat>
#include <cmath>

#include "common.cuh"

namespace fmbym {

// The heading of every pair for this candidate: theta and the float splits of its cosine and sine.
__global__ void k_ex_theta(float* __restrict__ th, int B, float theta, float ch, float cl, float sh, float sl) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= B) return;
    float* t = th + 8 * q;
    t[0] = theta;
    t[1] = ch;
    t[2] = cl;
    t[3] = sh;
    t[4] = sl;
}

// Peak of each pair's correlation for candidate k (the maximum of the stage-2 block maxima) and
// the running best (peak, theta, t_x, t_y).
__global__ void k_ex_update(const long long* __restrict__ tab, const float* __restrict__ st, int nblk,
                            const float* __restrict__ cand, int B, int k, float theta, float4* __restrict__ best,
                            float* __restrict__ peaks, int n_angles) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= B) return;
    float m = -FLT_MAX;
    for (int b = 0; b < nblk; ++b) m = fmaxf(m, st[((size_t)q * nblk + b) * 4 + 2]);
    const long long pr = tab[3 * q + 2];
    if (peaks) peaks[pr * n_angles + k] = m;
    if (k == 0 || m > best[q].x) best[q] = make_float4(m, theta, cand[3 * pr + 1], cand[3 * pr + 2]);
}

__global__ void k_ex_write(const long long* __restrict__ tab, const float4* __restrict__ best, int B,
                           float* __restrict__ pose) {
    grid_dep_wait();   // the previous kernel on the stream has completed (PDL launch)
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= B) return;
    const long long pr = tab[3 * q + 2];
    pose[3 * pr] = best[q].y;
    pose[3 * pr + 1] = best[q].z;
    pose[3 * pr + 2] = best[q].w;
}

cudaError_t launch_exhaustive(const DevPlan& p, const Ws& w, int B, const long long* tab, const float* f,
                              const float* g, int n_angles, const float* angles, float* cand, float4* best,
                              float* peaks, float* pose, cudaStream_t st) {
    if (B <= 0) return cudaSuccess;
    const int nb = (B + 255) / 256;
    const int nblk = c2r_blocks(p);
    for (int k = 0; k < n_angles; ++k) {
        // the same splits the decoupled search forms for its own heading
        const float theta = angles[k];
        const double cd = std::cos((double)theta), sd = std::sin((double)theta);
        const float ch = (float)cd, sh = (float)sd;
        launch_pdl(k_ex_theta, nb, 256, 0, st, w.th, B, theta, ch, (float)(cd - (double)ch), sh, (float)(sd - (double)sh));
        cudaError_t e = launch_forward_stage2(p, w, B, tab, f, g, cand, nullptr, st);
        if (e != cudaSuccess) return e;
        launch_pdl(k_ex_update, nb, 256, 0, st, tab, w.st, nblk, cand, B, k, theta, best, peaks, n_angles);
    }
    launch_pdl(k_ex_write, nb, 256, 0, st, tab, best, B, pose);
    return cudaGetLastError();
}

}  // namespace fmbym
