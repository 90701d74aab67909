// fmbym_pose_noalloc: the forward search for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all: a plug-in running inside a host framework that
// owns every device allocation, or a real-time process whose memory budget is fixed at start-up.
// This entry point serves them.  It takes the caller's input and output buffers, as fmbym_pose
// does, but its scratch (the per-size twiddle/window/polar tables, the pair table, the
// completion counters and every intermediate of the search) lives in one file-scope
// `static __device__` array of kNoAllocBytes.  The driver reserves that array when it loads the
// library onto a device, and every device that loads the library keeps it until the process exits.
//
// The kernels are the ones fmbym_pose runs (launch_forward); only the memory they use differs.
#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/fmbym.h"
#include "common.cuh"

namespace fmbym {
cudaError_t prepare_kernels();
}

using namespace fmbym;

namespace {

// Size of the static scratch: enough for one 512x512 pair, or several smaller ones.
constexpr size_t kNoAllocBytes = size_t(16) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kNoAllocBytes];

// Per-device state.  In host code g_scratch names a host-side stand-in, not the device array,
// so the device address is looked up once per device with cudaGetSymbolAddress.
struct DeviceState {
    bool ready = false;
    unsigned char* base = nullptr;  // device address of g_scratch on this device
};
DeviceState g_dev[kMaxDevices];
std::mutex g_mutex;
thread_local std::string g_error;
thread_local Tracer g_tracer;       // counts launches; never records events

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

int fail(int code, const std::string& msg) {
    g_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(FMBYM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

struct Layout {
    size_t win, tw_n, tw_p, tw_t, polar, tab, cnt, work, total;
};

Layout layout(const DevPlan& p, int n_pairs) {
    Layout l{};
    size_t off = 0;
    l.win = off;   off += align256(sizeof(float) * p.n);
    l.tw_n = off;  off += align256(sizeof(float2) * p.n);
    l.tw_p = off;  off += align256(sizeof(float2) * p.p);
    l.tw_t = off;  off += align256(sizeof(float2) * p.nt);
    l.polar = off; off += align256(sizeof(PolarSample) * p.nt * p.nr);
    l.tab = off;   off += align256(sizeof(long long) * 3 * n_pairs);
    l.cnt = off;   off += align256(sizeof(unsigned) * n_pairs);
    l.work = off;  off += ws_bytes(p, n_pairs, false);
    l.total = off;
    return l;
}

// Writes every table of one call into the array on the GPU: the periodic Hann window, the
// twiddles of lengths N, P and n_theta, the bilinear Cart2Pol samples (all in double precision,
// rounded to float as the handle's host-built tables are), the pair table (packed pairs: scan
// offset i N^2, c_theta offset i n_theta, pair index i) and the zeroed completion counters.  No
// host memory is read, so nothing has to stay alive on the host after the call returns.
__global__ void k_noalloc_tables(int n, int pp, int nt, int nr, int n_pairs, float* __restrict__ win,
                                 float2* __restrict__ tw_n, float2* __restrict__ tw_p, float2* __restrict__ tw_t,
                                 PolarSample* __restrict__ polar, long long* __restrict__ tab,
                                 unsigned* __restrict__ cnt) {
    const long long n_pol = (long long)nt * nr;
    const long long total = n + n + pp + nt + n_pol + n_pairs;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        long long k = i;
        if (k < n) {   // w[k] = 0.5 - 0.5 cos(2 pi k / N)
            win[k] = (float)(0.5 - 0.5 * cospi(2.0 * (double)k / (double)n));
            continue;
        }
        k -= n;
        // tw[k] = exp(-2 pi i k / L) for L = N, P, n_theta
        if (k < n) {
            double sv, cv;
            sincospi(-2.0 * (double)k / (double)n, &sv, &cv);
            tw_n[k] = make_float2((float)cv, (float)sv);
            continue;
        }
        k -= n;
        if (k < pp) {
            double sv, cv;
            sincospi(-2.0 * (double)k / (double)pp, &sv, &cv);
            tw_p[k] = make_float2((float)cv, (float)sv);
            continue;
        }
        k -= pp;
        if (k < nt) {
            double sv, cv;
            sincospi(-2.0 * (double)k / (double)nt, &sv, &cv);
            tw_t[k] = make_float2((float)cv, (float)sv);
            continue;
        }
        k -= nt;
        if (k < n_pol) {   // alpha_a = a pi / n_theta, rho_r = r (N/2) / n_r
            const int a = (int)(k / nr), r = (int)(k % nr);
            double sa, ca;
            sincospi((double)a / (double)nt, &sa, &ca);
            const double rho = (double)r * (n / 2.0) / nr;
            const double u = rho * ca, v = rho * sa;
            const double x0 = floor(u), y0 = floor(v);
            polar[k] = PolarSample{(int)x0, (int)y0, (float)(u - x0), (float)(v - y0)};
            continue;
        }
        k -= n_pol;
        tab[3 * k] = k * n * n;
        tab[3 * k + 1] = k * nt;
        tab[3 * k + 2] = k;
        cnt[k] = 0u;   // the counters keep whatever the last call left: clear them
    }
}

std::string check_cfg(const fmbym_size_cfg& c) {
    if (c.n != 128 && c.n != 256 && c.n != 512) return "n must be 128, 256 or 512";
    if (c.n_theta != 128 && c.n_theta != 256 && c.n_theta != 400) return "n_theta must be 128, 256 or 400";
    if (c.n_r < 1 || c.n_r > c.n / 2) return "n_r must be in [1, n/2]";
    if (!(c.temp_theta > 0.f) || !(c.temp_xy > 0.f) || !(c.delta_xy > 0.f))
        return "temperatures and delta_xy must be positive";
    if ((c.window | c.pad_mode | c.score_norm | c.angle_score | c.full_circle | c.rotate_target) & ~1)
        return "window, pad_mode, score_norm, angle_score, full_circle and rotate_target must be 0 or 1";
    if (c.rotate_target == 1 && c.full_circle == 1) return "rotate_target 1 needs full_circle 0";
    if (!(c.band_lo >= 0.f) || !(c.band_hi >= c.band_lo)) return "need 0 <= band_lo <= band_hi";
    return "";
}

}  // namespace

extern "C" {

const char* fmbym_noalloc_last_error(void) { return g_error.c_str(); }

unsigned long long fmbym_noalloc_capacity(void) { return (unsigned long long)kNoAllocBytes; }

int fmbym_pose_noalloc(void* stream, const fmbym_size_cfg* cfg, int n_pairs, const float* f, const float* g,
                       float* pose, float* c_theta, float* c_xy) {
    g_error.clear();
    if (!cfg) return fail(FMBYM_ERR_INVALID_ARG, "cfg is NULL");
    const std::string bad = check_cfg(*cfg);
    if (!bad.empty()) {
        const bool size = (cfg->n != 128 && cfg->n != 256 && cfg->n != 512) ||
                          (cfg->n_theta != 128 && cfg->n_theta != 256 && cfg->n_theta != 400);
        return fail(size ? FMBYM_ERR_UNSUPPORTED_SIZE : FMBYM_ERR_INVALID_ARG, bad);
    }
    if (n_pairs < 0) return fail(FMBYM_ERR_INVALID_ARG, "n_pairs < 0");
    if (n_pairs == 0) return FMBYM_OK;
    if (!f || !g || !pose) return fail(FMBYM_ERR_INVALID_ARG, "f, g and pose must not be NULL");
    if (((uintptr_t)f | (uintptr_t)g | (uintptr_t)c_xy) & 15)
        return fail(FMBYM_ERR_INVALID_ARG, "f, g and c_xy must be 16-byte aligned");

    DevPlan p{};
    p.n = cfg->n;
    p.p = cfg->pad_mode == 1 ? cfg->n : 3 * cfg->n / 2;
    p.nt = cfg->n_theta;
    p.nr = cfg->n_r;
    p.window = cfg->window;
    p.score_norm = cfg->score_norm;
    p.angle_score = cfg->angle_score;
    p.full_circle = cfg->full_circle;
    p.rotate_target = cfg->rotate_target;
    p.temp_theta = cfg->temp_theta;
    p.temp_xy = cfg->temp_xy;
    p.delta_xy = cfg->delta_xy;
    p.col_tile = tpb_for(p.p) / fft_threads(p.p);   // the default launch schedules
    p.angle_rc = kAngleRadii;
    p.rot_px = kRotPixels;
    p.col_plan = 0;
    const int mmax = (cfg->n / 2) * (cfg->n / 2) * 2;
    p.m_lo = mmax + 1;
    p.m_hi = -1;
    for (int m = 0; m <= mmax; ++m) {
        const double r = std::sqrt((double)m);
        if (r >= cfg->band_lo && p.m_lo > mmax) p.m_lo = m;
        if (r <= cfg->band_hi) p.m_hi = m;
    }
    const Layout l = layout(p, n_pairs);
    if (l.total > kNoAllocBytes) {
        return fail(FMBYM_ERR_WORKSPACE, "n_pairs=" + std::to_string(n_pairs) + " at n=" + std::to_string(p.n) +
                                             " needs " + std::to_string(l.total) + " bytes of scratch; the static array holds " +
                                             std::to_string(kNoAllocBytes));
    }

    std::lock_guard<std::mutex> lock(g_mutex);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(FMBYM_ERR_INVALID_ARG, "device index out of range");
    DeviceState& ds = g_dev[dev];
    if (!ds.ready) {
        // once per device, with that device current
        if ((e = prepare_kernels()) != cudaSuccess) return cuda_fail(e, "kernel attributes");
        void* addr = nullptr;
        if ((e = cudaGetSymbolAddress(&addr, g_scratch)) != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
        ds.base = (unsigned char*)addr;
        ds.ready = true;
    }
    cudaStream_t st = (cudaStream_t)stream;
    float* d_win = (float*)(ds.base + l.win);
    float2* d_twn = (float2*)(ds.base + l.tw_n);
    float2* d_twp = (float2*)(ds.base + l.tw_p);
    float2* d_twt = (float2*)(ds.base + l.tw_t);
    PolarSample* d_pol = (PolarSample*)(ds.base + l.polar);
    long long* d_tab = (long long*)(ds.base + l.tab);
    unsigned* d_cnt = (unsigned*)(ds.base + l.cnt);
    k_noalloc_tables<<<152, 256, 0, st>>>(p.n, p.p, p.nt, p.nr, n_pairs, d_win, d_twn, d_twp, d_twt, d_pol, d_tab,
                                          d_cnt);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "table launch");
    p.win = d_win;
    p.tw_n = d_twn;
    p.tw_p = d_twp;
    p.tw_t = d_twt;
    p.polar = d_pol;
    Ws w = ws_carve(p, n_pairs, ds.base + l.work, false);
    w.tr = &g_tracer;
    w.cnt = d_cnt;
    if ((e = launch_forward(p, w, n_pairs, d_tab, f, g, pose, c_theta, c_xy, st)) != cudaSuccess)
        return cuda_fail(e, "forward launch");
    return FMBYM_OK;
}

}  // extern "C"
