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
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

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
    bool have_tables = false;
    fmbym_size_cfg tables_for{};    // configuration whose tables the array currently holds
};
DeviceState g_dev[kMaxDevices];
std::mutex g_mutex;
thread_local std::string g_error;
thread_local Tracer g_tracer;       // counts launches; never records events

constexpr double kPi = 3.14159265358979323846;

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

int fail(int code, const std::string& msg) {
    g_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(FMBYM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool same_cfg(const fmbym_size_cfg& a, const fmbym_size_cfg& b) { return std::memcmp(&a, &b, sizeof a) == 0; }

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

// Copies the per-size tables (double precision on the host, rounded to float) into the array.
cudaError_t upload_tables(const DevPlan& p, unsigned char* base, const Layout& l, cudaStream_t st) {
    std::vector<float> win(p.n);
    for (int i = 0; i < p.n; ++i) win[i] = (float)(0.5 - 0.5 * std::cos(2.0 * kPi * i / p.n));
    auto twiddles = [](int L) {
        std::vector<float2> t(L);
        for (int k = 0; k < L; ++k) {
            const double a = -2.0 * kPi * (double)k / (double)L;
            t[k] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
        return t;
    };
    const std::vector<float2> twn = twiddles(p.n), twp = twiddles(p.p), twt = twiddles(p.nt);
    std::vector<PolarSample> pol((size_t)p.nt * p.nr);
    for (int a = 0; a < p.nt; ++a) {
        const double alpha = (double)a * kPi / p.nt;
        for (int r = 0; r < p.nr; ++r) {
            const double rho = (double)r * (p.n / 2.0) / p.nr;
            const double u = rho * std::cos(alpha), v = rho * std::sin(alpha);
            const double x0 = std::floor(u), y0 = std::floor(v);
            pol[(size_t)a * p.nr + r] = PolarSample{(int)x0, (int)y0, (float)(u - x0), (float)(v - y0)};
        }
    }
    cudaError_t e;
    if ((e = cudaMemcpyAsync(base + l.win, win.data(), sizeof(float) * win.size(), cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(base + l.tw_n, twn.data(), sizeof(float2) * twn.size(), cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(base + l.tw_p, twp.data(), sizeof(float2) * twp.size(), cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(base + l.tw_t, twt.data(), sizeof(float2) * twt.size(), cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(base + l.polar, pol.data(), sizeof(PolarSample) * pol.size(), cudaMemcpyHostToDevice,
                             st)))
        return e;
    // copies from pageable host memory return once the source has been read, so the vectors
    // may be released here
    return cudaSuccess;
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
    if (!ds.have_tables || !same_cfg(ds.tables_for, *cfg)) {
        ds.have_tables = false;
        if ((e = upload_tables(p, ds.base, l, st)) != cudaSuccess) return cuda_fail(e, "table upload");
        ds.tables_for = *cfg;
        ds.have_tables = true;
    }
    p.win = (const float*)(ds.base + l.win);
    p.tw_n = (const float2*)(ds.base + l.tw_n);
    p.tw_p = (const float2*)(ds.base + l.tw_p);
    p.tw_t = (const float2*)(ds.base + l.tw_t);
    p.polar = (const PolarSample*)(ds.base + l.polar);

    // pair table: packed pairs, offset p N^2, c_theta offset p n_theta
    std::vector<long long> tab(3 * (size_t)n_pairs);
    for (int i = 0; i < n_pairs; ++i) {
        tab[3 * i] = (long long)i * p.n * p.n;
        tab[3 * i + 1] = (long long)i * p.nt;
        tab[3 * i + 2] = i;
    }
    long long* d_tab = (long long*)(ds.base + l.tab);
    unsigned* d_cnt = (unsigned*)(ds.base + l.cnt);
    if ((e = cudaMemcpyAsync(d_tab, tab.data(), sizeof(long long) * tab.size(), cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
        return cuda_fail(e, "pair table copy");
    // the counters keep whatever the last call left: clear them
    if ((e = cudaMemsetAsync(d_cnt, 0, sizeof(unsigned) * n_pairs, st)) != cudaSuccess)
        return cuda_fail(e, "counter clear");
    Ws w = ws_carve(p, n_pairs, ds.base + l.work, false);
    w.tr = &g_tracer;
    w.cnt = d_cnt;
    if ((e = launch_forward(p, w, n_pairs, d_tab, f, g, pose, c_theta, c_xy, st)) != cudaSuccess)
        return cuda_fail(e, "forward launch");
    return FMBYM_OK;
}

}  // extern "C"
