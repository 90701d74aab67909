// Host side of the C ABI (include/fmbym.h): handle, per-size plans, workspace, argument checks,
// grouping of mixed-size batches, and the host-buffer entry point.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/fmbym.h"
#include "common.cuh"

using namespace fmbym;

namespace {

constexpr double kPi = 3.14159265358979323846;

struct HostPlan {
    fmbym_size_cfg cfg;
    DevPlan dev;
    void* tables = nullptr;  // one allocation holding every table of the plan
};

thread_local std::string g_create_error;

// the power-of-two sides, and the paper's odd sides 127, 255, 511 (Sec. IV-B resolutions)
bool supported_n(int n) { return n == 128 || n == 256 || n == 512 || n == 127 || n == 255 || n == 511; }
// 128, 256 and 400 angles take the FFT route; any other count up to 1024 (Alg. 1's 733 among them)
// the direct sums of angle_direct.cu
bool supported_nt(int nt) { return nt >= 8 && nt <= 1024; }

}  // namespace

// One captured call layout: its CUDA graph and the device copy of its pair table.
struct GraphEntry {
    std::vector<long long> key;  // kind, pair count, buffer pointers, pair table
    cudaGraphExec_t exec = nullptr;
    long long* d_tab = nullptr;
    long long kernels = 0;
    unsigned long long last_use = 0;
};

struct fmbym_handle {
    int device = 0;
    int max_pairs = 0;
    int flags = 0;
    std::vector<HostPlan> plans;
    std::vector<void*> ws;        // one workspace region per size, for max_pairs pairs
    std::vector<size_t> ws_slot;  // byte offset of each size's second slot (half of max_pairs)
    size_t ws_size = 0;
    std::vector<cudaStream_t> side;   // streams of the size groups after the first
    cudaEvent_t ev_fork = nullptr;
    std::vector<cudaEvent_t> ev_join;
    cudaStream_t cap = nullptr;       // capture stream of the graph cache
    std::vector<GraphEntry> graphs;
    unsigned long long use_clock = 0;
    long long* d_tab = nullptr;   // [max_pairs][3]
    long long* d_tab2 = nullptr;  // [max_pairs][3] pair table of calls in workspace slot 1
    long long* h_tab = nullptr;   // pinned staging of the pair table
    cudaEvent_t tab_free = nullptr;
    float* d_stage_f = nullptr;   // host-buffer entry points' staging
    float* d_stage_g = nullptr;
    float* d_stage_pose = nullptr;
    float* d_stage_df = nullptr;  // [stage_elems] each: the training call's gradients
    float* d_stage_dg = nullptr;
    float* d_stage_small = nullptr;  // [max_pairs][3] gt, [max_pairs][3] dpose, [1] loss, [2] chunk losses
    cudaStream_t s_in = nullptr, s_out = nullptr;   // host-buffer training call: copy streams
    cudaStream_t s_alt = nullptr;                   // host-buffer training call: odd chunks' calls
    cudaEvent_t ev_start = nullptr, ev_in[4] = {}, ev_done[4] = {}, ev_alt = nullptr;
    unsigned* d_cnt = nullptr;    // [max_pairs] completion counters, zero between launches
    float* d_bpose = nullptr;     // [max_pairs][3] pose recomputed by the adjoint
    float4* d_best = nullptr;     // [max_pairs] running best of the exhaustive search
    float* d_fcpose = nullptr;    // [max_pairs][3] full-circle candidate translations
    long long stage_elems = 0;
    Tracer tracer;
    std::string err;
};

namespace fmbym {

// Workspace of one size group of B pairs; every region starts on a 256-byte boundary.
static size_t carve(const DevPlan& p, int B, char* base, Ws* w, bool backward) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        char* r = base ? base + off : nullptr;
        off += (bytes + 255) & ~size_t(255);
        return r;
    };
    // Wn: the packed row spectra's width (N/2 for even N, (N + 1)/2 for odd N); ne: stage 2's frame
    const size_t n = p.n, P = p.p, Wn = (n + 1) / 2, Wp = P / 2, b = (size_t)B, ne = frame_n(p.n);
    Ws t{};
    t.s1 = (float2*)take(2 * b * n * Wn * sizeof(float2));
    t.mt = (float*)take(2 * b * (n / 2 + 1) * n * sizeof(float));
    t.sp = (float2*)take(b * angle_chunks_max(p) * p.nt * sizeof(float2));
    t.th = (float*)take(b * 8 * sizeof(float));
    t.s2 = (float2*)take(2 * b * ne * Wp * sizeof(float2));
    t.s3 = (float2*)take(b * ne * Wp * sizeof(float2));
    t.cxy = (float*)take(b * n * n * sizeof(float));
    t.st = (float*)take(b * c2r_blocks(p) * 4 * sizeof(float));
    t.sx = (float*)take(b * kSplitXY * 8 * sizeof(float));
    t.xm = (float*)take(b * 8 * sizeof(float));
    t.fc = (float*)take(b * 8 * sizeof(float));
    t.fcpose = (float*)take(b * 3 * sizeof(float));
    t.ct = (float*)take(b * p.nt * sizeof(float));
    if (backward) {
        t.ahat = (float2*)take(b * p.nt * p.nr * sizeof(float2));
        t.phs = (float2*)take(2 * b * (n / 2 + 1) * n * sizeof(float2));
        t.s2hat = (float2*)take(2 * b * P * Wp * sizeof(float2));
        t.bsc = (float*)take(b * 16 * sizeof(float));
        t.gpart = (float*)take(b * (ne * ne / 256) * sizeof(float));
        t.b1 = (float2*)take(b * ne * Wp * sizeof(float2));
        t.b2 = (float2*)take(2 * b * ne * Wp * sizeof(float2));
        t.gfr = (float*)take(b * n * n * sizeof(float));
        t.bdc = (float2*)take(b * p.nt * sizeof(float2));
        t.gpol = (float2*)take(b * p.nt * p.nr * sizeof(float2));
        t.gmt = (float2*)take(b * (n / 2 + 1) * n * sizeof(float2));
        t.gs1 = (float2*)take(2 * b * n * Wn * sizeof(float2));
    }
    if (w) *w = t;
    return off;
}

size_t ws_bytes(const DevPlan& p, int B, bool backward) { return carve(p, B, nullptr, nullptr, backward); }
Ws ws_carve(const DevPlan& p, int B, void* base, bool backward) {
    Ws w;
    carve(p, B, (char*)base, &w, backward);
    return w;
}

cudaError_t prepare_forward_kernels();
cudaError_t prepare_backward_kernels();
cudaError_t prepare_kernels() {
    cudaError_t e = prepare_forward_kernels();
    if (e != cudaSuccess) return e;
    return prepare_backward_kernels();
}

}  // namespace fmbym

namespace {

int fail(fmbym_handle* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    else g_create_error = msg;
    return code;
}

int cuda_fail(fmbym_handle* h, cudaError_t e, const char* what) {
    return fail(h, FMBYM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

std::string validate(const fmbym_size_cfg& c) {
    char buf[256];
    if (!supported_n(c.n)) {
        snprintf(buf, sizeof buf, "n=%d not supported (127, 128, 255, 256, 511, 512)", c.n);
        return buf;
    }
    if (!supported_nt(c.n_theta)) {
        snprintf(buf, sizeof buf, "n_theta=%d not supported (8..1024)", c.n_theta);
        return buf;
    }
    if (c.n_r < 1 || c.n_r > c.n / 2) return "n_r must be in [1, n/2]";
    if (!(c.temp_theta > 0.f) || !(c.temp_xy > 0.f) || !(c.delta_xy > 0.f))
        return "temperatures and delta_xy must be positive";
    if (c.window != 0 && c.window != 1) return "window must be 0 or 1";
    if (c.pad_mode != 0 && c.pad_mode != 1) return "pad_mode must be 0 or 1";
    if (c.pad_mode == 1 && (c.n & 1)) return "pad_mode 1 (N-periodic) needs an even n";
    if (c.score_norm != 0 && c.score_norm != 1) return "score_norm must be 0 or 1";
    if (c.angle_score != 0 && c.angle_score != 1) return "angle_score must be 0 or 1";
    if (c.full_circle != 0 && c.full_circle != 1) return "full_circle must be 0 or 1";
    if (c.rotate_target != 0 && c.rotate_target != 1) return "rotate_target must be 0 or 1";
    if (c.rotate_target == 1 && c.full_circle == 1) return "rotate_target 1 needs full_circle 0";
    if (!(c.band_lo >= 0.f) || !(c.band_hi >= c.band_lo)) return "need 0 <= band_lo <= band_hi";
    return "";
}

// Builds the device tables of one size in double precision.
cudaError_t build_plan(HostPlan& hp) {
    const fmbym_size_cfg& c = hp.cfg;
    DevPlan& d = hp.dev;
    d.n = c.n;
    // zero pad to 1.5 N (1.5 (N + 1) for odd N): lags |s| <= N/2 never alias
    d.p = c.pad_mode == 1 ? c.n : 3 * frame_n(c.n) / 2;
    d.m = (c.n & 1) ? 2 * (c.n + 1) : 0;
    d.tw_m = d.chirp = d.bh = nullptr;
    d.col_tile = tpb_for(d.p) / fft_threads(d.p);
    d.angle_rc = kAngleRadii;
    d.rot_px = kRotPixels;
    d.col_plan = 0;
    d.nt = c.n_theta;
    d.nr = c.n_r;
    d.window = c.window;
    d.score_norm = c.score_norm;
    d.angle_score = c.angle_score;
    d.full_circle = c.full_circle;
    d.rotate_target = c.rotate_target;
    d.temp_theta = c.temp_theta;
    d.temp_xy = c.temp_xy;
    d.delta_xy = c.delta_xy;
    // band-pass on integer rho^2 = v^2 + u^2: keep band_lo <= sqrt(m) <= band_hi
    const int mmax = (c.n / 2) * (c.n / 2) * 2;
    d.m_lo = mmax + 1;
    d.m_hi = -1;
    for (int m = 0; m <= mmax; ++m) {
        const double r = std::sqrt((double)m);
        if (r >= c.band_lo && d.m_lo > mmax) d.m_lo = m;
        if (r <= c.band_hi) d.m_hi = m;
    }
    std::vector<float> win(c.n);
    for (int i = 0; i < c.n; ++i) win[i] = (float)(0.5 - 0.5 * std::cos(2.0 * kPi * i / c.n));
    auto twiddles = [](int L) {
        std::vector<float2> t(L);
        for (int k = 0; k < L; ++k) {
            const double a = -2.0 * kPi * (double)k / (double)L;
            t[k] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
        return t;
    };
    std::vector<float2> twn = twiddles(d.n), twp = twiddles(d.p), twt = twiddles(d.nt);
    // Bluestein tables of an odd N: N k = (n^2 + k^2 - (k - n)^2) / 2 turns the N-point DFT into
    // X[k] = conj(w[k]) sum_n (x[n] conj(w[n])) w[k - n] with w[n] = exp(i pi n^2 / N), a linear
    // convolution of length 2N - 1 <= M done by M-point FFTs: bh = FFT_M(b) / M of the circular
    // filter b[m] = w[m], b[M - m] = w[m] (0 < m < N).  n^2 is reduced modulo 2N in integers, and
    // bh is a direct DFT sum in double precision.
    std::vector<float2> twm, chirp, bh;
    if (d.m) {
        twm = twiddles(d.m);
        const int N = d.n, M = d.m;
        std::vector<double> wr(N), wi(N);
        for (int k = 0; k < N; ++k) {
            const long long e = ((long long)k * k) % (2LL * N);
            wr[k] = std::cos(kPi * (double)e / N);
            wi[k] = std::sin(kPi * (double)e / N);
        }
        chirp.resize(N);
        for (int k = 0; k < N; ++k) chirp[k] = make_float2((float)wr[k], (float)wi[k]);
        std::vector<double> br(M, 0.0), bi(M, 0.0);
        for (int k = 0; k < N; ++k) {
            br[k] = wr[k];
            bi[k] = wi[k];
            if (k > 0) {
                br[M - k] = wr[k];
                bi[M - k] = wi[k];
            }
        }
        bh.resize(M);
        for (int k = 0; k < M; ++k) {
            double sr = 0.0, si = 0.0;
            for (int j = 0; j < M; ++j) {
                const long long e = ((long long)j * k) % M;
                const double a = -2.0 * kPi * (double)e / M, ca = std::cos(a), sa = std::sin(a);
                sr += br[j] * ca - bi[j] * sa;
                si += br[j] * sa + bi[j] * ca;
            }
            bh[k] = make_float2((float)(sr / M), (float)(si / M));
        }
    }
    std::vector<PolarSample> pol((size_t)d.nt * d.nr);
    for (int a = 0; a < d.nt; ++a) {
        const double alpha = (double)a * kPi / d.nt;
        for (int r = 0; r < d.nr; ++r) {
            const double rho = (double)r * (d.n / 2.0) / d.nr;
            const double u = rho * std::cos(alpha), v = rho * std::sin(alpha);
            const double x0 = std::floor(u), y0 = std::floor(v);
            pol[(size_t)a * d.nr + r] = PolarSample{(int)x0, (int)y0, (float)(u - x0), (float)(v - y0)};
        }
    }
    // transpose of the gather: for each half-plane element, the samples (a n_r + r) that read it
    // and their bilinear weights, computed in float exactly as the gather kernel forms them
    const int ne = (d.n / 2 + 1) * d.n;
    std::vector<int> cnt(ne + 1, 0), col;
    std::vector<float> wt;
    {
        struct Tap { int e, s; float w; };
        std::vector<Tap> taps;
        taps.reserve((size_t)4 * pol.size());
        for (size_t sidx = 0; sidx < pol.size(); ++sidx) {
            const PolarSample& ps = pol[sidx];
            const float wy[2] = {1.f - ps.fy, ps.fy}, wx[2] = {1.f - ps.fx, ps.fx};
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                    int vi = ((ps.y0 + dy) % d.n + d.n) % d.n, ui = ((ps.x0 + dx) % d.n + d.n) % d.n;
                    if (ui > d.n / 2) {
                        vi = (d.n - vi) % d.n;
                        ui = d.n - ui;
                    }
                    taps.push_back(Tap{ui * d.n + vi, (int)sidx, wy[dy] * wx[dx]});
                }
        }
        for (const Tap& t : taps) cnt[t.e + 1]++;
        for (int i = 0; i < ne; ++i) cnt[i + 1] += cnt[i];
        col.resize(taps.size());
        wt.resize(taps.size());
        std::vector<int> fill(cnt.begin(), cnt.end() - 1);
        for (const Tap& t : taps) {
            col[fill[t.e]] = t.s;
            wt[fill[t.e]++] = t.w;
        }
    }
    std::vector<int> heavy;
    for (int i = 0; i < ne; ++i)
        if (cnt[i + 1] - cnt[i] > kHeavyRow) heavy.push_back(i);
    if (heavy.empty()) heavy.push_back(-1);  // keeps the allocation non-empty; n_heavy stays 0
    d.n_heavy = heavy[0] < 0 ? 0 : (int)heavy.size();
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t b_win = al(win.size() * 4), b_twn = al(twn.size() * 8), b_twp = al(twp.size() * 8),
                 b_twt = al(twt.size() * 8), b_pol = al(pol.size() * sizeof(PolarSample)),
                 b_ptr = al(cnt.size() * 4), b_col = al(col.size() * 4), b_wt = al(wt.size() * 4),
                 b_hv = al(heavy.size() * 4), b_twm = al(twm.size() * 8), b_chirp = al(chirp.size() * 8),
                 b_bh = al(bh.size() * 8);
    char* base = nullptr;
    cudaError_t e = cudaMalloc(&base, b_win + b_twn + b_twp + b_twt + b_pol + b_ptr + b_col + b_wt + b_hv + b_twm +
                                          b_chirp + b_bh);
    if (e != cudaSuccess) return e;
    hp.tables = base;
    char* cur = base;
    auto put = [&](const void* src, size_t bytes, size_t padded) {
        char* dst = cur;
        cudaError_t err = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
        cur += padded;
        return std::make_pair(dst, err);
    };
    auto r1 = put(win.data(), win.size() * 4, b_win);
    auto r2 = put(twn.data(), twn.size() * 8, b_twn);
    auto r3 = put(twp.data(), twp.size() * 8, b_twp);
    auto r4 = put(twt.data(), twt.size() * 8, b_twt);
    auto r5 = put(pol.data(), pol.size() * sizeof(PolarSample), b_pol);
    auto r6 = put(cnt.data(), cnt.size() * 4, b_ptr);
    auto r7 = put(col.data(), col.size() * 4, b_col);
    auto r8 = put(wt.data(), wt.size() * 4, b_wt);
    auto r9 = put(heavy.data(), heavy.size() * 4, b_hv);
    for (auto& r : {r1, r2, r3, r4, r5, r6, r7, r8, r9})
        if (r.second != cudaSuccess) return r.second;
    if (d.m) {
        auto r10 = put(twm.data(), twm.size() * 8, b_twm);
        auto r11 = put(chirp.data(), chirp.size() * 8, b_chirp);
        auto r12 = put(bh.data(), bh.size() * 8, b_bh);
        for (auto& r : {r10, r11, r12})
            if (r.second != cudaSuccess) return r.second;
        d.tw_m = (const float2*)r10.first;
        d.chirp = (const float2*)r11.first;
        d.bh = (const float2*)r12.first;
    }
    d.heavy = (const int*)r9.first;
    d.csr_ptr = (const int*)r6.first;
    d.csr_col = (const int*)r7.first;
    d.csr_w = (const float*)r8.first;
    d.win = (const float*)r1.first;
    d.tw_n = (const float2*)r2.first;
    d.tw_p = (const float2*)r3.first;
    d.tw_t = (const float2*)r4.first;
    d.polar = (const PolarSample*)r5.first;
    return cudaSuccess;
}

struct Group {
    int size_idx;
    int count;
    int first;  // first row of the group in the pair table
};

// Validates the per-call arguments and fills the pinned pair table grouped by size.
int make_table(fmbym_handle* h, int n_pairs, const int* size_idx, const long long* offsets,
               std::vector<Group>& groups, long long* total_elems) {
    if (n_pairs < 0) return fail(h, FMBYM_ERR_INVALID_ARG, "n_pairs < 0");
    if (n_pairs > h->max_pairs) return fail(h, FMBYM_ERR_WORKSPACE, "n_pairs exceeds max_pairs of the handle");
    const int ns = (int)h->plans.size();
    std::vector<long long> off(n_pairs), ct(n_pairs);
    long long acc = 0, acc_t = 0, end = 0;
    for (int i = 0; i < n_pairs; ++i) {
        const int s = size_idx ? size_idx[i] : 0;
        if (s < 0 || s >= ns) return fail(h, FMBYM_ERR_INVALID_ARG, "size_idx out of range");
        const long long nn = (long long)h->plans[s].cfg.n * h->plans[s].cfg.n;
        off[i] = offsets ? offsets[i] : acc;
        // the kernels of the power-of-two sides read scans, scores and gradients as float4 rows;
        // those of the odd sides read them element by element
        const bool odd = (h->plans[s].cfg.n & 1) != 0;
        if (off[i] < 0 || (!odd && (off[i] & 3)))
            return fail(h, FMBYM_ERR_INVALID_ARG, "offsets must be >= 0, and multiples of 4 for the even sides");
        acc += nn;
        ct[i] = acc_t;
        acc_t += h->plans[s].cfg.n_theta;
        end = std::max(end, off[i] + nn);
    }
    if (total_elems) *total_elems = end;
    // wait until the previous call's copy of the table has been consumed
    cudaError_t e = cudaEventSynchronize(h->tab_free);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventSynchronize");
    groups.clear();
    int row = 0;
    for (int s = 0; s < ns; ++s) {
        Group g{s, 0, row};
        for (int i = 0; i < n_pairs; ++i) {
            if ((size_idx ? size_idx[i] : 0) != s) continue;
            h->h_tab[3 * row] = off[i];
            h->h_tab[3 * row + 1] = ct[i];
            h->h_tab[3 * row + 2] = i;
            ++row;
            ++g.count;
        }
        if (g.count) groups.push_back(g);
    }
    return FMBYM_OK;
}

// Buffers of one forward (kind 0), backward (kind 1) or training (kind 2: forward, pose loss and
// the adjoint of the loss without recomputing the forward) call.
struct LaunchArgs {
    int kind;
    const float* f;
    const float* g;
    float* pose;
    float* c_theta;
    float* c_xy;
    const float* dpose;
    float* df;
    float* dg;
    const float* gt;      // kind 2: ground-truth poses
    int loss_kind;        // kind 2: 1 = L1 (Eq. 13), 2 = L2
    float* loss;          // kind 2: the loss (device scalar)
    float* dpose_out;     // kind 2: dL/dpose, written by the loss and read by the adjoint
    int norm_pairs;       // kind 2: the count the loss averages over (0: this call's pairs)
    int slot;             // workspace slot: 0 = the whole region; 1 = the second half (at most
                          // (max_pairs + 1) / 2 pairs), so that two calls can run concurrently
};

// phase 0 launches the forward of one size group, phase 1 its adjoint (after a forward recompute
// unless the call is a training call, whose forward left its intermediates in the workspace).
cudaError_t launch_group(fmbym_handle* h, const Group& gr, const long long* dtab, const LaunchArgs& a,
                         cudaStream_t s, int phase) {
    const DevPlan& p = h->plans[gr.size_idx].dev;
    const size_t half = a.slot ? (size_t)(h->max_pairs + 1) / 2 : 0;   // slot 1: the upper halves
    Ws w = ws_carve(p, gr.count, (char*)h->ws[gr.size_idx] + (a.slot ? h->ws_slot[gr.size_idx] : 0), true);
    w.tr = &h->tracer;
    w.cnt = h->d_cnt + (size_t)gr.size_idx * h->max_pairs + half;
    w.bpose = h->d_bpose + 3 * half;
    w.fcpose = h->d_fcpose + 3 * half;   // indexed by the call's pair index, which spans every group
    const long long* tab = dtab + 3 * gr.first;
    if (phase == 0) {
        const bool train = a.kind == 2;
        if (!train) {   // a plain forward keeps nothing for an adjoint
            w.ahat = nullptr;
            w.phs = nullptr;
            w.s2hat = nullptr;
        }
        return launch_forward(p, w, gr.count, tab, a.f, a.g, a.pose, train ? nullptr : a.c_theta,
                              train ? nullptr : a.c_xy, s);
    }
    if (a.kind == 2) return launch_backward(p, w, gr.count, tab, a.f, a.g, a.dpose_out, a.df, a.dg, s, a.pose);
    return launch_backward(p, w, gr.count, tab, a.f, a.g, a.dpose, a.df, a.dg, s, nullptr);
}

// Launches one phase of every size group: the first on the caller's stream, the others on the
// handle's side streams forked from it and joined back, so that groups of different sizes run
// concurrently.  With more than one group the tracer only counts launches (its events assume one
// stream).
cudaError_t enqueue_phase(fmbym_handle* h, cudaStream_t st, const std::vector<Group>& groups, const long long* dtab,
                          const LaunchArgs& a, int phase) {
    if (groups.size() == 1) return launch_group(h, groups[0], dtab, a, st, phase);
    const bool tracing = h->tracer.on;
    h->tracer.on = false;
    cudaError_t e = cudaEventRecord(h->ev_fork, st);
    for (size_t k = 1; k < groups.size() && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(h->side[k - 1], h->ev_fork, 0);
    for (size_t k = 0; k < groups.size() && e == cudaSuccess; ++k) {
        cudaStream_t s = k == 0 ? st : h->side[k - 1];
        e = launch_group(h, groups[k], dtab, a, s, phase);
        if (e == cudaSuccess && k > 0) e = cudaEventRecord(h->ev_join[k - 1], s);
        if (e == cudaSuccess && k > 0) e = cudaStreamWaitEvent(st, h->ev_join[k - 1], 0);
    }
    h->tracer.on = tracing;
    return e;
}

// A forward call is phase 0, a backward call phase 1; a training call runs phase 0, the loss over
// all pairs on the caller's stream (after every group's forward has joined it), then phase 1.
cudaError_t enqueue(fmbym_handle* h, cudaStream_t st, const std::vector<Group>& groups, const long long* dtab,
                    const LaunchArgs& a, int n_pairs) {
    if (a.kind != 2) return enqueue_phase(h, st, groups, dtab, a, a.kind);
    cudaError_t e = enqueue_phase(h, st, groups, dtab, a, 0);
    if (e == cudaSuccess)
        e = launch_pose_loss(n_pairs, a.pose, a.gt, a.loss_kind, a.loss, a.dpose_out, &h->tracer, st, a.norm_pairs);
    if (e == cudaSuccess) e = enqueue_phase(h, st, groups, dtab, a, 1);
    return e;
}

constexpr size_t kMaxGraphs = 16;

// Runs one call.  With FMBYM_FLAG_GRAPH (and tracing off) each distinct layout (kind, pairs,
// buffers, pair table) is captured once into a CUDA graph whose pair table lives in its own
// device buffer, and replayed with a single cudaGraphLaunch; the least recently used of more than
// kMaxGraphs graphs is released.  Otherwise the pair table is copied from pinned memory and the
// groups are launched directly.
int run_call(fmbym_handle* h, cudaStream_t st, int n_pairs, const std::vector<Group>& groups, const LaunchArgs& a) {
    cudaError_t e;
    if ((h->flags & FMBYM_FLAG_GRAPH) && !h->tracer.on) {
        std::vector<long long> key = {a.kind, n_pairs, (long long)(uintptr_t)a.f, (long long)(uintptr_t)a.g,
                                      (long long)(uintptr_t)a.pose, (long long)(uintptr_t)a.c_theta,
                                      (long long)(uintptr_t)a.c_xy, (long long)(uintptr_t)a.dpose,
                                      (long long)(uintptr_t)a.df, (long long)(uintptr_t)a.dg,
                                      (long long)(uintptr_t)a.gt, a.loss_kind, (long long)(uintptr_t)a.loss,
                                      (long long)(uintptr_t)a.dpose_out, a.norm_pairs, a.slot};
        key.insert(key.end(), h->h_tab, h->h_tab + 3 * (size_t)n_pairs);
        GraphEntry* ge = nullptr;
        for (auto& x : h->graphs)
            if (x.key == key) ge = &x;
        if (!ge) {
            if (h->graphs.size() >= kMaxGraphs) {
                auto lru = std::min_element(h->graphs.begin(), h->graphs.end(),
                                            [](const GraphEntry& x, const GraphEntry& y) { return x.last_use < y.last_use; });
                // the released graph may still run on this stream or on the second slot's
                if ((e = cudaStreamSynchronize(st)) != cudaSuccess || (e = cudaStreamSynchronize(h->s_alt)) != cudaSuccess)
                    return cuda_fail(h, e, "cudaStreamSynchronize");
                cudaGraphExecDestroy(lru->exec);
                cudaFree(lru->d_tab);
                h->graphs.erase(lru);
            }
            GraphEntry n;
            n.key = key;
            if ((e = cudaMalloc(&n.d_tab, sizeof(long long) * 3 * n_pairs)) != cudaSuccess ||
                (e = cudaMemcpy(n.d_tab, h->h_tab, sizeof(long long) * 3 * n_pairs, cudaMemcpyHostToDevice)) !=
                    cudaSuccess) {
                cudaFree(n.d_tab);
                return cuda_fail(h, e, "graph table");
            }
            const long long before = h->tracer.launches;
            cudaGraph_t graph = nullptr;
            if ((e = cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
                cudaFree(n.d_tab);
                return cuda_fail(h, e, "cudaStreamBeginCapture");
            }
            cudaError_t le = enqueue(h, h->cap, groups, n.d_tab, a, n_pairs);
            e = cudaStreamEndCapture(h->cap, &graph);
            n.kernels = h->tracer.launches - before;
            h->tracer.launches = before;
            if (le != cudaSuccess || e != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                cudaFree(n.d_tab);
                return cuda_fail(h, le != cudaSuccess ? le : e, "graph capture");
            }
            e = cudaGraphInstantiate(&n.exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                cudaFree(n.d_tab);
                return cuda_fail(h, e, "cudaGraphInstantiate");
            }
            h->graphs.push_back(std::move(n));
            ge = &h->graphs.back();
        }
        ge->last_use = ++h->use_clock;
        if ((e = cudaGraphLaunch(ge->exec, st)) != cudaSuccess) return cuda_fail(h, e, "cudaGraphLaunch");
        h->tracer.launches += ge->kernels;
        return FMBYM_OK;
    }
    long long* dtab = a.slot ? h->d_tab2 : h->d_tab;
    if ((e = cudaMemcpyAsync(dtab, h->h_tab, sizeof(long long) * 3 * n_pairs, cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
        return cuda_fail(h, e, "pair table copy");
    if ((e = cudaEventRecord(h->tab_free, st)) != cudaSuccess) return cuda_fail(h, e, "cudaEventRecord");
    if ((e = enqueue(h, st, groups, dtab, a, n_pairs)) != cudaSuccess)
        return cuda_fail(h, e, a.kind == 0 ? "forward launch" : a.kind == 1 ? "backward launch" : "training launch");
    return FMBYM_OK;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

// ---------------------------------------------------------------------------------------------
// launch-schedule autotuner
// ---------------------------------------------------------------------------------------------

// Candidate values of one launch schedule of a size; the first is the default.
std::vector<int> tune_candidates(const DevPlan& d, int knob) {
    const int c0 = tpb_for(d.p) / fft_threads(d.p);
    if (knob == FMBYM_TUNE_COL_TILE) return d.p % 3 == 0 ? std::vector<int>{c0, c0 / 2, 2 * c0} : std::vector<int>{c0};
    if (knob == FMBYM_TUNE_ANGLE_RADII) return {kAngleRadii, kAngleRadiiMin};
    if (knob == FMBYM_TUNE_COL_PLAN) return d.p % 3 == 0 ? std::vector<int>{0, 1} : std::vector<int>{0};
    return {kRotPixels, 1, 2, 8};
}

int& tune_field(DevPlan& d, int knob) {
    return knob == FMBYM_TUNE_COL_TILE      ? d.col_tile
           : knob == FMBYM_TUNE_ANGLE_RADII ? d.angle_rc
           : knob == FMBYM_TUNE_COL_PLAN    ? d.col_plan
                                            : d.rot_px;
}

void release_graphs(fmbym_handle* h) {
    for (auto& x : h->graphs) {
        cudaGraphExecDestroy(x.exec);
        cudaFree(x.d_tab);
    }
    h->graphs.clear();
}

// Scan-like test data for timing: a counter-based hash of (seed, index) mapped to [0, 1), cubed so
// that most pixels are dim and a few bright (the timings do not depend on the values).
__global__ void k_tune_fill(float* __restrict__ x, long long n, unsigned seed) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        unsigned h = (unsigned)i * 0x9E3779B1u ^ seed;
        h ^= h >> 16;
        h *= 0x85EBCA6Bu;
        h ^= h >> 13;
        h *= 0xC2B2AE35u;
        h ^= h >> 16;
        const float u = (float)(h >> 8) * (1.f / 16777216.f);
        x[i] = u * u * u;
    }
}

// Times a training call of max_pairs pairs of each size under every candidate of every schedule
// (coordinate descent, one pass in knob order) and keeps the fastest.
int autotune(fmbym_handle* h) {
    const int saved_flags = h->flags;
    h->flags &= ~FMBYM_FLAG_GRAPH;
    cudaStream_t st = h->cap;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    int rc = e == cudaSuccess ? FMBYM_OK : FMBYM_ERR_CUDA;
    for (size_t s = 0; s < h->plans.size() && rc == FMBYM_OK; ++s) {
        const int n = h->plans[s].cfg.n, B = h->max_pairs;
        const long long elems = (long long)B * n * n;
        float *f = nullptr, *g = nullptr, *df = nullptr, *dg = nullptr, *small = nullptr;
        if ((e = cudaMalloc(&f, sizeof(float) * elems)) != cudaSuccess || (e = cudaMalloc(&g, sizeof(float) * elems)) != cudaSuccess ||
            (e = cudaMalloc(&df, sizeof(float) * elems)) != cudaSuccess || (e = cudaMalloc(&dg, sizeof(float) * elems)) != cudaSuccess ||
            (e = cudaMalloc(&small, sizeof(float) * (9 * (size_t)B + 1))) != cudaSuccess ||
            (e = cudaMemsetAsync(small, 0, sizeof(float) * (9 * (size_t)B + 1), st)) != cudaSuccess) {
            rc = FMBYM_ERR_CUDA;
        } else {
            k_tune_fill<<<1024, 256, 0, st>>>(f, elems, 12345u + (unsigned)s);
            k_tune_fill<<<1024, 256, 0, st>>>(g, elems, 67890u + (unsigned)s);
            const std::vector<int> si((size_t)B, (int)s);
            float *gt = small, *pose = small + 3 * B, *dpose = small + 6 * B, *loss = small + 9 * B;
            auto timed = [&](float& ms) -> int {
                float best = 1e30f;
                for (int rep = 0; rep < 4 && rc == FMBYM_OK; ++rep) {
                    if ((e = cudaEventRecord(a, st)) != cudaSuccess) return FMBYM_ERR_CUDA;
                    const int r = fmbym_pose_train(h, st, B, si.data(), nullptr, f, g, gt, 2, pose, loss, dpose, df, dg);
                    if (r != FMBYM_OK) return r;
                    if ((e = cudaEventRecord(b, st)) != cudaSuccess || (e = cudaEventSynchronize(b)) != cudaSuccess)
                        return FMBYM_ERR_CUDA;
                    float t = 0.f;
                    cudaEventElapsedTime(&t, a, b);
                    if (rep > 0) best = std::min(best, t);   // the first call warms up
                }
                ms = best;
                return FMBYM_OK;
            };
            DevPlan& d = h->plans[s].dev;
            for (int knob = 0; knob < FMBYM_TUNE_COUNT && rc == FMBYM_OK; ++knob) {
                const std::vector<int> cand = tune_candidates(d, knob);
                int best_v = tune_field(d, knob);
                float best_ms = 1e30f;
                for (int v : cand) {
                    tune_field(d, knob) = v;
                    float ms = 0.f;
                    if ((rc = timed(ms)) != FMBYM_OK) break;
                    if (ms < best_ms) {
                        best_ms = ms;
                        best_v = v;
                    }
                }
                tune_field(d, knob) = best_v;
            }
        }
        cudaStreamSynchronize(st);
        cudaFree(f);
        cudaFree(g);
        cudaFree(df);
        cudaFree(dg);
        cudaFree(small);
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    h->flags = saved_flags;
    if (rc != FMBYM_OK && h->err.empty()) h->err = std::string("autotune: ") + cudaGetErrorString(e);
    return rc;
}

}  // namespace

extern "C" {

int fmbym_version(void) { return 10000; }

const char* fmbym_last_error(const fmbym_handle* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

unsigned long long fmbym_workspace_bytes(const fmbym_handle* h) { return h ? h->ws_size : 0ull; }

void fmbym_destroy(fmbym_handle* h) {
    if (!h) return;
    cudaDeviceSynchronize();
    for (auto& p : h->plans) cudaFree(p.tables);
    for (void* w : h->ws) cudaFree(w);
    for (auto& ge : h->graphs) {
        if (ge.exec) cudaGraphExecDestroy(ge.exec);
        cudaFree(ge.d_tab);
    }
    for (cudaStream_t st : h->side) cudaStreamDestroy(st);
    for (cudaEvent_t ev : h->ev_join) cudaEventDestroy(ev);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->cap) cudaStreamDestroy(h->cap);
    cudaFree(h->d_tab);
    cudaFree(h->d_tab2);
    cudaFree(h->d_stage_f);
    cudaFree(h->d_stage_g);
    cudaFree(h->d_stage_pose);
    cudaFree(h->d_stage_df);
    cudaFree(h->d_stage_dg);
    cudaFree(h->d_stage_small);
    if (h->s_in) cudaStreamDestroy(h->s_in);
    if (h->s_out) cudaStreamDestroy(h->s_out);
    if (h->s_alt) cudaStreamDestroy(h->s_alt);
    if (h->ev_alt) cudaEventDestroy(h->ev_alt);
    if (h->ev_start) cudaEventDestroy(h->ev_start);
    for (int c = 0; c < 4; ++c) {
        if (h->ev_in[c]) cudaEventDestroy(h->ev_in[c]);
        if (h->ev_done[c]) cudaEventDestroy(h->ev_done[c]);
    }
    cudaFree(h->d_cnt);
    cudaFree(h->d_bpose);
    cudaFree(h->d_best);
    cudaFree(h->d_fcpose);
    if (h->h_tab) cudaFreeHost(h->h_tab);
    for (cudaEvent_t e : h->tracer.ev) cudaEventDestroy(e);
    if (h->tab_free) cudaEventDestroy(h->tab_free);
    delete h;
}

int fmbym_create(fmbym_handle** out, const fmbym_config* cfg) {
    g_create_error.clear();
    if (!out) return fail(nullptr, FMBYM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!cfg || cfg->n_sizes < 1 || !cfg->sizes) return fail(nullptr, FMBYM_ERR_INVALID_ARG, "need at least one size");
    if (cfg->max_pairs < 1) return fail(nullptr, FMBYM_ERR_INVALID_ARG, "max_pairs must be >= 1");
    for (int i = 0; i < cfg->n_sizes; ++i) {
        const std::string v = validate(cfg->sizes[i]);
        if (!v.empty()) {
            const bool size = !supported_n(cfg->sizes[i].n) || !supported_nt(cfg->sizes[i].n_theta) ||
                              (cfg->sizes[i].pad_mode == 1 && (cfg->sizes[i].n & 1));
            return fail(nullptr, size ? FMBYM_ERR_UNSUPPORTED_SIZE : FMBYM_ERR_INVALID_ARG,
                        "size " + std::to_string(i) + ": " + v);
        }
    }
    fmbym_handle* h = new fmbym_handle();
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(nullptr, e, "cudaGetDevice");
    }
    h->max_pairs = cfg->max_pairs;
    static bool prepared = false;
    if (!prepared) {
        e = prepare_kernels();
        if (e != cudaSuccess) {
            delete h;
            return cuda_fail(nullptr, e, "kernel attributes");
        }
        prepared = true;
    }
    h->flags = cfg->flags;
    int nmax = 0;
    for (int i = 0; i < cfg->n_sizes; ++i) {
        HostPlan hp;
        hp.cfg = cfg->sizes[i];
        e = build_plan(hp);
        h->plans.push_back(hp);
        if (e != cudaSuccess) {
            fmbym_destroy(h);
            return cuda_fail(nullptr, e, "plan tables");
        }
        // the region holds max_pairs pairs, or two slots of (max_pairs + 1) / 2 pairs each
        const size_t off = (ws_bytes(hp.dev, (cfg->max_pairs + 1) / 2, true) + 255) & ~(size_t)255;
        const size_t b = std::max(ws_bytes(hp.dev, cfg->max_pairs, true), 2 * off);
        void* w = nullptr;
        if ((e = cudaMalloc(&w, b)) != cudaSuccess || (e = cudaMemset(w, 0, b)) != cudaSuccess) {
            fmbym_destroy(h);
            return cuda_fail(nullptr, e, "workspace allocation");
        }
        h->ws.push_back(w);
        h->ws_slot.push_back(off);
        h->ws_size += b;
        nmax = std::max(nmax, hp.cfg.n);
    }
    for (int i = 1; i < cfg->n_sizes; ++i) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) break;
        h->side.push_back(st);
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) break;
        h->ev_join.push_back(ev);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess ||
        (e = cudaMalloc(&h->d_tab, sizeof(long long) * 3 * cfg->max_pairs)) != cudaSuccess ||
        (e = cudaMalloc(&h->d_tab2, sizeof(long long) * 3 * cfg->max_pairs)) != cudaSuccess ||
        (e = cudaMallocHost(&h->h_tab, sizeof(long long) * 3 * cfg->max_pairs)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&h->tab_free, cudaEventDisableTiming)) != cudaSuccess) {
        fmbym_destroy(h);
        return cuda_fail(nullptr, e, "stream, event or table allocation");
    }
    h->stage_elems = (long long)cfg->max_pairs * nmax * nmax;
    if ((e = cudaMalloc(&h->d_stage_f, sizeof(float) * h->stage_elems)) != cudaSuccess ||
        (e = cudaMalloc(&h->d_stage_g, sizeof(float) * h->stage_elems)) != cudaSuccess ||
        (e = cudaMalloc(&h->d_stage_pose, sizeof(float) * 3 * cfg->max_pairs)) != cudaSuccess ||
        (e = cudaMalloc(&h->d_stage_df, sizeof(float) * h->stage_elems)) != cudaSuccess ||
        (e = cudaMalloc(&h->d_stage_dg, sizeof(float) * h->stage_elems)) != cudaSuccess ||
        (e = cudaMalloc(&h->d_stage_small, sizeof(float) * (6 * (size_t)cfg->max_pairs + 3))) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&h->s_in, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&h->s_out, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&h->s_alt, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&h->ev_alt, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&h->ev_start, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaMalloc(&h->d_cnt, sizeof(unsigned) * cfg->max_pairs * cfg->n_sizes)) != cudaSuccess ||
        (e = cudaMemset(h->d_cnt, 0, sizeof(unsigned) * cfg->max_pairs * cfg->n_sizes)) != cudaSuccess ||
        (e = cudaMalloc(&h->d_bpose, sizeof(float) * 3 * cfg->max_pairs)) != cudaSuccess ||
        (e = cudaMalloc(&h->d_best, sizeof(float4) * cfg->max_pairs)) != cudaSuccess ||
        (e = cudaMalloc(&h->d_fcpose, sizeof(float) * 3 * cfg->max_pairs)) != cudaSuccess) {
        fmbym_destroy(h);
        return cuda_fail(nullptr, e, "staging allocation");
    }
    for (int c = 0; c < 4 && e == cudaSuccess; ++c) {
        if ((e = cudaEventCreateWithFlags(&h->ev_in[c], cudaEventDisableTiming)) == cudaSuccess)
            e = cudaEventCreateWithFlags(&h->ev_done[c], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        fmbym_destroy(h);
        return cuda_fail(nullptr, e, "copy events");
    }
    if (cfg->flags & FMBYM_FLAG_AUTOTUNE) {
        const int rc = autotune(h);
        if (rc != FMBYM_OK) {
            g_create_error = h->err;
            fmbym_destroy(h);
            return rc;
        }
    }
    *out = h;
    return FMBYM_OK;
}

int fmbym_get_tuning(const fmbym_handle* h, int size, int* values) {
    if (!h || !values) return fail(nullptr, FMBYM_ERR_INVALID_ARG, "handle or values is NULL");
    if (size < 0 || size >= (int)h->plans.size()) return FMBYM_ERR_INVALID_ARG;
    const DevPlan& d = h->plans[size].dev;
    values[FMBYM_TUNE_COL_TILE] = d.col_tile;
    values[FMBYM_TUNE_ANGLE_RADII] = d.angle_rc;
    values[FMBYM_TUNE_ROT_PIXELS] = d.rot_px;
    values[FMBYM_TUNE_COL_PLAN] = d.col_plan;
    return FMBYM_OK;
}

int fmbym_set_tuning(fmbym_handle* h, int size, const int* values) {
    if (!h || !values) return fail(nullptr, FMBYM_ERR_INVALID_ARG, "handle or values is NULL");
    h->err.clear();
    if (size < 0 || size >= (int)h->plans.size()) return fail(h, FMBYM_ERR_INVALID_ARG, "size index out of range");
    DevPlan& d = h->plans[size].dev;
    for (int knob = 0; knob < FMBYM_TUNE_COUNT; ++knob) {
        const std::vector<int> cand = tune_candidates(d, knob);
        if (std::find(cand.begin(), cand.end(), values[knob]) == cand.end())
            return fail(h, FMBYM_ERR_INVALID_ARG, "schedule value " + std::to_string(values[knob]) + " of knob " +
                                                      std::to_string(knob) + " is not a candidate");
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaDeviceSynchronize");
    release_graphs(h);
    for (int knob = 0; knob < FMBYM_TUNE_COUNT; ++knob) tune_field(d, knob) = values[knob];
    return FMBYM_OK;
}

// A packed call of one size and 16 or more pairs runs as two halves on two streams (the caller's
// and an internal one) in the workspace's two slots, so that each half's kernels overlap the
// other's ramps, tails and one-CTA-per-pair kernels.  Per pair the results are those of one call:
// in a training call each half's loss gradient is normalised by the whole call's pair count, and
// the call's loss is taken over all pairs once both halves are done.
bool halves_apply(const fmbym_handle* h, const long long* offsets, const std::vector<Group>& groups, int n_pairs) {
    return !offsets && groups.size() == 1 && n_pairs >= 16 && !h->tracer.on;
}

int run_halves(fmbym_handle* h, cudaStream_t st, int n_pairs, const int* size_idx, const LaunchArgs& a) {
    cudaError_t e;
    if ((e = cudaEventRecord(h->ev_start, st)) != cudaSuccess || (e = cudaStreamWaitEvent(h->s_alt, h->ev_start, 0)) != cudaSuccess)
        return cuda_fail(h, e, "stream fork");
    const fmbym_size_cfg& c = h->plans[size_idx ? size_idx[0] : 0].cfg;
    const long long nn = (long long)c.n * c.n;
    for (int k = 0; k < 2; ++k) {
        const int i0 = k ? n_pairs / 2 : 0, i1 = k ? n_pairs : n_pairs / 2;
        std::vector<long long> off(i1 - i0);
        for (int i = i0; i < i1; ++i) off[i - i0] = (long long)i * nn;
        std::vector<Group> cg;
        int rc = make_table(h, i1 - i0, size_idx ? size_idx + i0 : nullptr, off.data(), cg, nullptr);
        if (rc != FMBYM_OK) return rc;
        LaunchArgs ak = a;   // per-pair outputs and inputs indexed by the pair: shifted to the half
        if (ak.pose) ak.pose += 3 * (size_t)i0;
        if (ak.c_theta) ak.c_theta += (size_t)i0 * c.n_theta;
        if (ak.dpose) ak.dpose += 3 * (size_t)i0;
        if (a.kind == 2) {
            ak.gt += 3 * (size_t)i0;
            ak.dpose_out += 3 * (size_t)i0;
            ak.loss = h->d_stage_small + 6 * (size_t)h->max_pairs + 1 + k;   // the halves' partial losses
            ak.norm_pairs = n_pairs;
        }
        ak.slot = k;
        if ((rc = run_call(h, k ? h->s_alt : st, i1 - i0, cg, ak)) != FMBYM_OK) return rc;
    }
    if ((e = cudaEventRecord(h->ev_alt, h->s_alt)) != cudaSuccess || (e = cudaStreamWaitEvent(st, h->ev_alt, 0)) != cudaSuccess)
        return cuda_fail(h, e, "stream join");
    if (a.kind == 2 && (e = launch_pose_loss(n_pairs, a.pose, a.gt, a.loss_kind, a.loss, nullptr, &h->tracer, st)) != cudaSuccess)
        return cuda_fail(h, e, "loss");
    return FMBYM_OK;
}

int fmbym_pose(fmbym_handle* h, void* stream, int n_pairs, const int* size_idx, const long long* offsets,
               const float* f, const float* g, float* pose, float* c_theta, float* c_xy) {
    if (!h) return fail(nullptr, FMBYM_ERR_INVALID_ARG, "handle is NULL");
    h->err.clear();
    if (n_pairs == 0) return FMBYM_OK;
    if (!f || !g || !pose) return fail(h, FMBYM_ERR_INVALID_ARG, "f, g and pose must not be NULL");
    if (!aligned16(f) || !aligned16(g) || (c_xy && !aligned16(c_xy)))
        return fail(h, FMBYM_ERR_INVALID_ARG, "f, g and c_xy must be 16-byte aligned");
    std::vector<Group> groups;
    int rc = make_table(h, n_pairs, size_idx, offsets, groups, nullptr);
    if (rc != FMBYM_OK) return rc;
    LaunchArgs a{};
    a.kind = 0;
    a.f = f;
    a.g = g;
    a.pose = pose;
    a.c_theta = c_theta;
    a.c_xy = c_xy;
    if (!halves_apply(h, offsets, groups, n_pairs)) return run_call(h, (cudaStream_t)stream, n_pairs, groups, a);
    return run_halves(h, (cudaStream_t)stream, n_pairs, size_idx, a);
}

int fmbym_pose_backward(fmbym_handle* h, void* stream, int n_pairs, const int* size_idx, const long long* offsets,
                        const float* f, const float* g, const float* dpose, float* df, float* dg) {
    if (!h) return fail(nullptr, FMBYM_ERR_INVALID_ARG, "handle is NULL");
    h->err.clear();
    if (n_pairs == 0) return FMBYM_OK;
    if (!f || !g || !dpose || !df || !dg) return fail(h, FMBYM_ERR_INVALID_ARG, "NULL buffer");
    if (!aligned16(f) || !aligned16(g) || !aligned16(df) || !aligned16(dg))
        return fail(h, FMBYM_ERR_INVALID_ARG, "f, g, df and dg must be 16-byte aligned");
    std::vector<Group> groups;
    int rc = make_table(h, n_pairs, size_idx, offsets, groups, nullptr);
    if (rc != FMBYM_OK) return rc;
    LaunchArgs a{};
    a.kind = 1;
    a.f = f;
    a.g = g;
    a.dpose = dpose;
    a.df = df;
    a.dg = dg;
    if (!halves_apply(h, offsets, groups, n_pairs)) return run_call(h, (cudaStream_t)stream, n_pairs, groups, a);
    return run_halves(h, (cudaStream_t)stream, n_pairs, size_idx, a);
}

int fmbym_pose_train(fmbym_handle* h, void* stream, int n_pairs, const int* size_idx, const long long* offsets,
                     const float* f, const float* g, const float* gt, int loss_kind, float* pose, float* loss,
                     float* dpose, float* df, float* dg) {
    if (!h) return fail(nullptr, FMBYM_ERR_INVALID_ARG, "handle is NULL");
    h->err.clear();
    if (n_pairs == 0) return FMBYM_OK;
    if (loss_kind != 1 && loss_kind != 2) return fail(h, FMBYM_ERR_INVALID_ARG, "loss_kind not 1/2");
    if (!f || !g || !gt || !pose || !loss || !dpose || !df || !dg) return fail(h, FMBYM_ERR_INVALID_ARG, "NULL buffer");
    if (!aligned16(f) || !aligned16(g) || !aligned16(df) || !aligned16(dg))
        return fail(h, FMBYM_ERR_INVALID_ARG, "f, g, df and dg must be 16-byte aligned");
    std::vector<Group> groups;
    int rc = make_table(h, n_pairs, size_idx, offsets, groups, nullptr);
    if (rc != FMBYM_OK) return rc;
    LaunchArgs a{};
    a.kind = 2;
    a.f = f;
    a.g = g;
    a.pose = pose;
    a.gt = gt;
    a.loss_kind = loss_kind;
    a.loss = loss;
    a.dpose_out = dpose;
    a.df = df;
    a.dg = dg;
    cudaStream_t st = (cudaStream_t)stream;
    if (!halves_apply(h, offsets, groups, n_pairs)) return run_call(h, st, n_pairs, groups, a);
    return run_halves(h, st, n_pairs, size_idx, a);
}

int fmbym_pose_exhaustive(fmbym_handle* h, void* stream, int n_pairs, int size, const long long* offsets,
                          const float* f, const float* g, int n_angles, const float* angles, float* pose,
                          float* peaks) {
    if (!h) return fail(nullptr, FMBYM_ERR_INVALID_ARG, "handle is NULL");
    h->err.clear();
    if (n_pairs == 0) return FMBYM_OK;
    if (size < 0 || size >= (int)h->plans.size()) return fail(h, FMBYM_ERR_INVALID_ARG, "size index out of range");
    if (n_angles < 1 || !angles) return fail(h, FMBYM_ERR_INVALID_ARG, "need n_angles >= 1 host angles");
    if (h->plans[size].cfg.rotate_target != 0)
        return fail(h, FMBYM_ERR_INVALID_ARG, "the exhaustive search rotates the source (rotate_target 0)");
    if (!f || !g || !pose) return fail(h, FMBYM_ERR_INVALID_ARG, "f, g and pose must not be NULL");
    if (!aligned16(f) || !aligned16(g)) return fail(h, FMBYM_ERR_INVALID_ARG, "f and g must be 16-byte aligned");
    if (n_pairs < 0 || n_pairs > h->max_pairs) return fail(h, FMBYM_ERR_WORKSPACE, "n_pairs exceeds max_pairs");
    std::vector<int> si((size_t)n_pairs, size);
    std::vector<Group> groups;
    int rc = make_table(h, n_pairs, si.data(), offsets, groups, nullptr);
    if (rc != FMBYM_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(h->d_tab, h->h_tab, sizeof(long long) * 3 * n_pairs, cudaMemcpyHostToDevice, st)) !=
            cudaSuccess ||
        (e = cudaEventRecord(h->tab_free, st)) != cudaSuccess)
        return cuda_fail(h, e, "pair table copy");
    const Group& gr = groups[0];
    const DevPlan& p = h->plans[size].dev;
    Ws w = ws_carve(p, gr.count, h->ws[size], true);
    w.tr = &h->tracer;
    w.cnt = h->d_cnt + (size_t)size * h->max_pairs;
    w.bpose = h->d_bpose;
    w.s2hat = nullptr;   // nothing is kept for an adjoint
    if ((e = launch_exhaustive(p, w, gr.count, h->d_tab, f, g, n_angles, angles, h->d_bpose, h->d_best, peaks, pose,
                               st)) != cudaSuccess)
        return cuda_fail(h, e, "exhaustive search launch");
    return FMBYM_OK;
}

int fmbym_pose_host(fmbym_handle* h, void* stream, int n_pairs, const int* size_idx, const long long* offsets,
                    long long total_elems, const float* f_host, const float* g_host, float* pose_host) {
    if (!h) return fail(nullptr, FMBYM_ERR_INVALID_ARG, "handle is NULL");
    h->err.clear();
    if (n_pairs == 0) return FMBYM_OK;
    if (!f_host || !g_host || !pose_host) return fail(h, FMBYM_ERR_INVALID_ARG, "NULL buffer");
    if (total_elems < 0 || total_elems > h->stage_elems)
        return fail(h, FMBYM_ERR_WORKSPACE, "total_elems exceeds the staging area");
    std::vector<Group> groups;
    long long need = 0;
    int rc = make_table(h, n_pairs, size_idx, offsets, groups, &need);
    if (rc != FMBYM_OK) return rc;
    if (need > total_elems) return fail(h, FMBYM_ERR_INVALID_ARG, "offsets reach beyond total_elems");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(h->d_stage_f, f_host, sizeof(float) * total_elems, cudaMemcpyHostToDevice, st)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(h->d_stage_g, g_host, sizeof(float) * total_elems, cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
        return cuda_fail(h, e, "host-to-device copy");
    LaunchArgs a{};
    a.kind = 0;
    a.f = h->d_stage_f;
    a.g = h->d_stage_g;
    a.pose = h->d_stage_pose;
    rc = run_call(h, st, n_pairs, groups, a);
    if (rc != FMBYM_OK) return rc;
    if ((e = cudaMemcpyAsync(pose_host, h->d_stage_pose, sizeof(float) * 3 * n_pairs, cudaMemcpyDeviceToHost, st)) !=
        cudaSuccess)
        return cuda_fail(h, e, "device-to-host copy");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
    return FMBYM_OK;
}

int fmbym_pose_train_host(fmbym_handle* h, void* stream, int n_pairs, const int* size_idx, const long long* offsets,
                          long long total_elems, const float* f_host, const float* g_host, const float* gt_host,
                          int loss_kind, float* pose_host, float* loss_host, float* df_host, float* dg_host) {
    if (!h) return fail(nullptr, FMBYM_ERR_INVALID_ARG, "handle is NULL");
    h->err.clear();
    if (n_pairs == 0) return FMBYM_OK;
    if (loss_kind != 1 && loss_kind != 2) return fail(h, FMBYM_ERR_INVALID_ARG, "loss_kind not 1/2");
    if (!f_host || !g_host || !gt_host || !pose_host || !loss_host || !df_host || !dg_host)
        return fail(h, FMBYM_ERR_INVALID_ARG, "NULL buffer");
    if (total_elems < 0 || total_elems > h->stage_elems)
        return fail(h, FMBYM_ERR_WORKSPACE, "total_elems exceeds the staging area");
    std::vector<Group> groups;
    long long need = 0;
    int rc = make_table(h, n_pairs, size_idx, offsets, groups, &need);
    if (rc != FMBYM_OK) return rc;
    if (need > total_elems) return fail(h, FMBYM_ERR_INVALID_ARG, "offsets reach beyond total_elems");
    cudaStream_t st = (cudaStream_t)stream;
    float* d_gt = h->d_stage_small;
    float* d_dpose = h->d_stage_small + 3 * (size_t)h->max_pairs;
    float* d_loss = h->d_stage_small + 6 * (size_t)h->max_pairs;
    float* d_chunk_loss = d_loss + 1;
    cudaError_t e;
    LaunchArgs a{};
    a.kind = 2;
    a.f = h->d_stage_f;
    a.g = h->d_stage_g;
    a.gt = d_gt;
    a.loss_kind = loss_kind;
    a.df = h->d_stage_df;
    a.dg = h->d_stage_dg;
    // Packed pairs (offsets NULL) of 16 or more run as a pipeline of 4 chunks of pairs: chunk c's
    // copies in (stream s_in) overlap chunk c - 1's training call (the caller's stream), and chunk
    // c - 1's gradients go back (stream s_out) while chunk c computes.  The first and last chunks
    // hold an eighth of the pairs each and the middle two three eighths: only the first chunk's
    // copy in and the last one's copy out are not hidden behind a training call, while every
    // chunk adds the fixed cost of a call.  Each chunk's loss is normalised by the whole call's pair
    // count, so dpose, pose, df and dg are those of the one-piece call; the call's loss is then
    // taken over all pairs at the end.  When every pair has one size, the odd chunks run on a
    // second stream in the workspace's second slot, so that a chunk's first kernels overlap the
    // previous chunk's last ones (each call ends in kernels of one CTA per pair).
    const int chunks = (!offsets && n_pairs >= 16) ? 4 : 1;
    const double bound[5] = {0.0, 0.125, 0.5, 0.875, 1.0};
    if (chunks == 1) {
        const size_t bytes = sizeof(float) * (size_t)total_elems;
        if ((e = cudaMemcpyAsync(h->d_stage_f, f_host, bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(h->d_stage_g, g_host, bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(d_gt, gt_host, sizeof(float) * 3 * n_pairs, cudaMemcpyHostToDevice, st)) !=
                cudaSuccess)
            return cuda_fail(h, e, "host-to-device copy");
        a.pose = h->d_stage_pose;
        a.loss = d_loss;
        a.dpose_out = d_dpose;
        rc = run_call(h, st, n_pairs, groups, a);
        if (rc != FMBYM_OK) return rc;
        if ((e = cudaMemcpyAsync(pose_host, h->d_stage_pose, sizeof(float) * 3 * n_pairs, cudaMemcpyDeviceToHost,
                                 st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(loss_host, d_loss, sizeof(float), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(df_host, h->d_stage_df, bytes, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(dg_host, h->d_stage_dg, bytes, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return cuda_fail(h, e, "device-to-host copy");
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
        return FMBYM_OK;
    }
    // element offset of every pair in the packed layout, and the chunk boundaries
    std::vector<long long> off(n_pairs + 1, 0);
    for (int i = 0; i < n_pairs; ++i) {
        const long long nn = (long long)h->plans[size_idx ? size_idx[i] : 0].cfg.n;
        off[i + 1] = off[i] + nn * nn;
    }
    const bool two = groups.size() == 1;
    if ((e = cudaEventRecord(h->ev_start, st)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(h->s_in, h->ev_start, 0)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(h->s_out, h->ev_start, 0)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(h->s_alt, h->ev_start, 0)) != cudaSuccess)
        return cuda_fail(h, e, "copy stream fork");
    for (int c = 0; c < chunks; ++c) {
        const int slot = two ? (c & 1) : 0;
        cudaStream_t cs = slot ? h->s_alt : st;
        const int i0 = (int)std::lround(n_pairs * bound[c]), i1 = (int)std::lround(n_pairs * bound[c + 1]);
        const size_t e0 = (size_t)off[i0], ne = (size_t)(off[i1] - off[i0]);
        if ((e = cudaMemcpyAsync(h->d_stage_f + e0, f_host + e0, sizeof(float) * ne, cudaMemcpyHostToDevice, h->s_in)) !=
                cudaSuccess ||
            (e = cudaMemcpyAsync(h->d_stage_g + e0, g_host + e0, sizeof(float) * ne, cudaMemcpyHostToDevice, h->s_in)) !=
                cudaSuccess ||
            (e = cudaMemcpyAsync(d_gt + 3 * (size_t)i0, gt_host + 3 * (size_t)i0, sizeof(float) * 3 * (i1 - i0),
                                 cudaMemcpyHostToDevice, h->s_in)) != cudaSuccess ||
            (e = cudaEventRecord(h->ev_in[c], h->s_in)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(cs, h->ev_in[c], 0)) != cudaSuccess)
            return cuda_fail(h, e, "host-to-device copy");
        std::vector<Group> cg;
        rc = make_table(h, i1 - i0, size_idx ? size_idx + i0 : nullptr, off.data() + i0, cg, nullptr);
        if (rc != FMBYM_OK) return rc;
        LaunchArgs ac = a;
        ac.gt = d_gt + 3 * (size_t)i0;
        ac.pose = h->d_stage_pose + 3 * (size_t)i0;
        ac.dpose_out = d_dpose + 3 * (size_t)i0;
        ac.loss = d_chunk_loss + slot;
        ac.norm_pairs = n_pairs;
        ac.slot = slot;
        rc = run_call(h, cs, i1 - i0, cg, ac);
        if (rc != FMBYM_OK) return rc;
        if ((e = cudaEventRecord(h->ev_done[c], cs)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(h->s_out, h->ev_done[c], 0)) != cudaSuccess ||
            (e = cudaMemcpyAsync(df_host + e0, h->d_stage_df + e0, sizeof(float) * ne, cudaMemcpyDeviceToHost,
                                 h->s_out)) != cudaSuccess ||
            (e = cudaMemcpyAsync(dg_host + e0, h->d_stage_dg + e0, sizeof(float) * ne, cudaMemcpyDeviceToHost,
                                 h->s_out)) != cudaSuccess)
            return cuda_fail(h, e, "device-to-host copy");
    }
    // the call's loss over every pair (the chunks' losses were partial), after both streams' chunks
    if ((e = cudaEventRecord(h->ev_alt, h->s_alt)) != cudaSuccess || (e = cudaStreamWaitEvent(st, h->ev_alt, 0)) != cudaSuccess)
        return cuda_fail(h, e, "stream join");
    if ((e = launch_pose_loss(n_pairs, h->d_stage_pose, d_gt, loss_kind, d_loss, nullptr, &h->tracer, st)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(pose_host, h->d_stage_pose, sizeof(float) * 3 * n_pairs, cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(loss_host, d_loss, sizeof(float), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(h, e, "device-to-host copy");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess || (e = cudaStreamSynchronize(h->s_out)) != cudaSuccess ||
        (e = cudaStreamSynchronize(h->s_in)) != cudaSuccess)
        return cuda_fail(h, e, "cudaStreamSynchronize");
    return FMBYM_OK;
}

int fmbym_pose_loss(fmbym_handle* h, void* stream, int n_pairs, const float* pose, const float* gt, int kind,
                    float* loss, float* dpose) {
    if (!h) return fail(nullptr, FMBYM_ERR_INVALID_ARG, "handle is NULL");
    h->err.clear();
    if (n_pairs < 0 || (kind != 1 && kind != 2)) return fail(h, FMBYM_ERR_INVALID_ARG, "n_pairs < 0 or kind not 1/2");
    if (n_pairs == 0) return FMBYM_OK;
    if (!pose || !gt) return fail(h, FMBYM_ERR_INVALID_ARG, "pose and gt must not be NULL");
    cudaError_t e = launch_pose_loss(n_pairs, pose, gt, kind, loss, dpose, &h->tracer, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "loss launch");
    return FMBYM_OK;
}

int fmbym_set_tracing(fmbym_handle* h, int on) {
    if (!h) return fail(nullptr, FMBYM_ERR_INVALID_ARG, "handle is NULL");
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaDeviceSynchronize");
    if (on && h->tracer.ev.empty()) {
        const size_t n = 1 << 14;
        h->tracer.ev.resize(n);
        h->tracer.kind.resize(n);
        for (size_t i = 0; i < n; ++i)
            if ((e = cudaEventCreate(&h->tracer.ev[i])) != cudaSuccess) return cuda_fail(h, e, "cudaEventCreate");
    }
    h->tracer.on = on != 0;
    h->tracer.used = 0;
    return FMBYM_OK;
}

int fmbym_trace_summary(fmbym_handle* h, int cap, double* total_ms, long long* count, int* n_kinds) {
    if (!h || !total_ms || !count || cap < 1) return fail(h, FMBYM_ERR_INVALID_ARG, "bad arguments");
    const int nk = std::min(cap, (int)K_COUNT);
    for (int k = 0; k < nk; ++k) {
        total_ms[k] = 0.0;
        count[k] = 0;
    }
    if (n_kinds) *n_kinds = (int)K_COUNT;
    Tracer& t = h->tracer;
    if (t.used == 0) return FMBYM_OK;
    cudaError_t e = cudaEventSynchronize(t.ev[t.used - 1]);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventSynchronize");
    for (size_t i = 0; i + 1 < t.used; ++i) {
        const int k = t.kind[i];
        if (k < 0 || k >= nk) continue;
        float ms = 0.f;
        if ((e = cudaEventElapsedTime(&ms, t.ev[i], t.ev[i + 1])) != cudaSuccess)
            return cuda_fail(h, e, "cudaEventElapsedTime");
        total_ms[k] += ms;
        count[k] += 1;
    }
    return FMBYM_OK;
}

const char* fmbym_trace_kind_name(int kind) { return (kind >= 0 && kind < K_COUNT) ? kKindNames[kind] : ""; }

long long fmbym_launch_count(const fmbym_handle* h) { return h ? h->tracer.launches : 0; }

}  // extern "C"
