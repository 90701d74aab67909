// Host side of the masking network h_alpha (Sec. III-D): the layer graph of a U-Net with L levels
// (two 3x3 conv + BN + ReLU per level, max-pool down, bilinear x2 up concatenated before the skip,
// 1x1 sigmoid head), its buffers, and the forward, backward and Adam entry points of
// include/fmbym.h.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/fmbym.h"
#include "unet_kernels.cuh"

using namespace fmbym::unet;

namespace {

int round8(int c) { return (c + 7) / 8 * 8; }

// One 3x3 conv + BN + ReLU layer and its buffers.
struct Layer {
    std::string name;
    int cin, cout, H, W;       // input channels, output channels, resolution
    int cinp, coutp;           // channels rounded up to 8
    int ns_f = 0, ns_d = 0;    // cp.async ring depth of the forward and dgrad convolutions
    int R_f = 1, R_d = 1;      // their rows per warp (CTA tile 8 R x 32)
    int wg_cib = 8, wg_R = 1, wg_ns = 2, wg_slots = 0;   // the weight gradient's plan
    bool gemm_f = false, gemm_d = false, gemm_w = false;  // forward / dgrad / wgrad on the flat-GEMM kernels
    int slots_f = 0, slots_d = 0;   // their resident CTAs on the device
    long long w_off, g_off, b_off, rs_off;  // offsets in the parameter and running-stat arrays
    bf16* wf = nullptr;        // forward weights [cout][9][cinp]
    bf16* wd = nullptr;        // dgrad weights [cin][9][coutp]
    float* y = nullptr;        // pre-BN output, float32 NHWC
    bf16* a = nullptr;         // post-ReLU output, bf16 NHWC
    float* da = nullptr;       // gradient of a
    bf16* dy = nullptr;        // gradient of y (bf16, tensor-core operand)
    float2* bn = nullptr;      // (mean, invstd) used by the last forward
    float2* bsums = nullptr;   // adjoint means
    // input: planes (first layer), or [in0 (c0), in1 (c1)]
    bool planes = false;
    const bf16* in0 = nullptr;
    int c0 = 0;
    const bf16* in1 = nullptr;
    int c1 = 0;
};

}  // namespace

struct fmbym_unet {
    int levels = 0, ch[8] = {0}, H = 0, W = 0, max_batch = 0;
    std::vector<Layer> layers;          // enc0a, enc0b, ..., enc{L-1}b, dec{L-2}a, ..., dec0b
    std::vector<bf16*> pooled;          // pooled[i] = maxpool(a of enc{i-1}b), level i >= 1
    std::vector<bf16*> upped;           // upped[i] = upsample(deeper) at level i < L-1
    std::vector<float*> dpool, dup;     // gradients of pooled and upped
    long long n_params = 0, n_running = 0, head_w = 0, head_b = 0;
    float* params = nullptr;            // float32 master parameters
    float* grads = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    float* running = nullptr;           // running mean / var of every BN channel
    float2* stats = nullptr;            // per-CTA conv statistics
    float2* bnpart = nullptr;           // BN adjoint partials
    float* wpart = nullptr;             // wgrad partials
    float* hpart = nullptr;             // head partials
    size_t stats_cap = 0, bnpart_cap = 0, wpart_cap = 0, hpart_cap = 0;
    int nsm = 0;
    int gw_slots = 0;                   // resident CTAs of the flat-GEMM weight gradient
    int conv_path = 0;                  // flat-GEMM convolutions: 0 mma.sync, 1 tcgen05
    unsigned* tc_timeouts = nullptr;    // device counter of tcgen05 CTAs whose wait gave up
    unsigned tc_spin = kTcSpin;         // polls before a tcgen05 producer's wait gives up
    unsigned tc_seen = 0;               // counter value the calls have already reported
    bool tc_ran = false;                // this call launched a tcgen05 convolution
    std::vector<void*> allocs;
    long long launches = 0;
    int last_batch = -1;
    std::string err;
};

namespace {

thread_local std::string g_unet_create_error;

// After a call that ran tcgen05 convolutions: waits for the stream and reports a CTA that gave up
// a bounded wait (its outputs are incomplete) as FMBYM_ERR_TIMEOUT.  Calls on the mma.sync path
// stay asynchronous.
int tc_status(fmbym_unet* u, cudaStream_t st, const char* what) {
    if (!u->tc_ran) return FMBYM_OK;
    u->tc_ran = false;
    unsigned v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, u->tc_timeouts, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        u->err = std::string(what) + ": " + cudaGetErrorString(e);
        return FMBYM_ERR_CUDA;
    }
    if (v != u->tc_seen) {
        u->err = std::string(what) + ": " + std::to_string(v - u->tc_seen) +
                 " tcgen05 convolution CTA(s) gave up a bounded wait; their outputs are incomplete";
        u->tc_seen = v;
        return FMBYM_ERR_TIMEOUT;
    }
    return FMBYM_OK;
}

int ufail(fmbym_unet* u, int code, const std::string& m) {
    if (u) u->err = m;
    else g_unet_create_error = m;
    return code;
}

int ucuda(fmbym_unet* u, cudaError_t e, const char* what) {
    return ufail(u, FMBYM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <typename T>
cudaError_t ualloc(fmbym_unet* u, T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T) + 16);
    if (e == cudaSuccess) {
        u->allocs.push_back(q);
        *p = (T*)q;
    }
    return e;
}

const int kBlock = 256;
inline unsigned blocks(long long n) { return (unsigned)((n + kBlock - 1) / kBlock); }
// 2-D grid of the row kernels: threads over one row's work items, blocks in y over the rows
inline dim3 row_grid(int per_row, int rows) { return dim3(blocks(per_row), (unsigned)std::min(rows, 65535)); }

// Ring depth and resident CTAs of a convolution with COUT outputs, G input groups and R-row warps:
// three tile buffers while the CTA stays under 64 KB of shared memory, else two, else one; 0 if
// even one does not fit.
template <int COUT, int R>
cudaError_t conv_plan_t(const fmbym_unet* u, int G, int& ns, int& slots) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k_conv3x3<COUT, R>);
    if (e != cudaSuccess) return e;
    int dev = 0, optin = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const size_t cap = (size_t)optin - fa.sharedSizeBytes, wb = conv_weight_bytes(COUT, G),
                 tb = conv_tile_bytes(G, R);
    ns = wb + 3 * tb <= 64 * 1024 ? 3 : wb + 2 * tb <= cap ? 2 : wb + tb <= cap ? 1 : 0;
    slots = 0;
    if (!ns) return cudaSuccess;
    e = cudaFuncSetAttribute(k_conv3x3<COUT, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
    int occ = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_conv3x3<COUT, R>, 256, wb + ns * tb);
    slots = std::max(1, occ) * u->nsm;
    return e;
}

// Tile height of a convolution: narrow outputs (8, 16, 24 channels) take the tallest CTA tile
// (R = 4, 2, 1 rows per warp) that divides the image height and keeps two input tiles and the
// weights within 64 KB; everything else R = 1.
cudaError_t conv_plan(const fmbym_unet* u, int cout, int G, int H, int& R, int& ns, int& slots) {
    ns = 0;
    slots = 0;
    if (cout == 8 || cout == 16 || cout == 24) {
        for (R = 4; R > 1; R /= 2) {
            if (H % (8 * R) || conv_weight_bytes(cout, G) + 2 * conv_tile_bytes(G, R) > 64 * 1024) continue;
            cudaError_t e;
            if (R == 4) e = cout == 8 ? conv_plan_t<8, 4>(u, G, ns, slots) : cout == 16 ? conv_plan_t<16, 4>(u, G, ns, slots)
                                                                                       : conv_plan_t<24, 4>(u, G, ns, slots);
            else e = cout == 8 ? conv_plan_t<8, 2>(u, G, ns, slots) : cout == 16 ? conv_plan_t<16, 2>(u, G, ns, slots)
                                                                                 : conv_plan_t<24, 2>(u, G, ns, slots);
            return e;
        }
    }
    R = 1;
    switch (cout) {
        case 8: return conv_plan_t<8, 1>(u, G, ns, slots);
        case 16: return conv_plan_t<16, 1>(u, G, ns, slots);
        case 24: return conv_plan_t<24, 1>(u, G, ns, slots);
        case 32: return conv_plan_t<32, 1>(u, G, ns, slots);
        case 48: return conv_plan_t<48, 1>(u, G, ns, slots);
        case 64: return conv_plan_t<64, 1>(u, G, ns, slots);
        case 96: return conv_plan_t<96, 1>(u, G, ns, slots);
        case 128: return conv_plan_t<128, 1>(u, G, ns, slots);
        default: return cudaSuccess;
    }
}

template <int COUT, int R>
cudaError_t conv_launch(fmbym_unet* u, const Layer& L, int B, bool dgrad, cudaStream_t st, float* out0,
                        float* out1, int split, int acc0, int acc1, float2* stats) {
    const int G = (dgrad ? L.coutp : L.cinp) / 8, ns = dgrad ? L.ns_d : L.ns_f;
    const bf16* w = dgrad ? L.wd : L.wf;
    const size_t smem = conv_weight_bytes(COUT, G) + ns * conv_tile_bytes(G, R);
    const int ntiles = B * (L.H / (8 * R)) * (L.W / kTW);
    const int grid = std::min(ntiles, dgrad ? L.slots_d : L.slots_f);
    ++u->launches;
    if (dgrad)
        k_conv3x3<COUT, R><<<grid, 256, smem, st>>>(L.dy, L.cout, nullptr, 0, nullptr, nullptr, w, G, ns, out0,
                                                    out1, split, acc0, acc1, nullptr, B, L.H, L.W);
    else
        k_conv3x3<COUT, R><<<grid, 256, smem, st>>>(L.in0, L.c0, L.in1, L.c1,
                                                    L.planes ? (const float*)L.in0 : nullptr,
                                                    L.planes ? (const float*)L.in1 : nullptr, w, G, ns, out0, out1,
                                                    split, acc0, acc1, stats, B, L.H, L.W);
    return cudaGetLastError();
}

// Flat-GEMM convolution tile: 128 pixels x 64 output channels while that still gives a CTA per SM,
// else 64 x 32; on the tcgen05 path always 128 pixels.
bool gemm_big(const fmbym_unet* u, int co, long long npix) {
    return co % 64 == 0 && npix % 128 == 0 && (u->conv_path == 1 || (npix / 128) * (co / 64) >= u->nsm);
}

template <int NT>
cudaError_t tc_conv_launch(fmbym_unet* u, const Layer& L, int B, bool dgrad, cudaStream_t st, float* out0,
                           float* out1, int split, int acc0, int acc1, float2* stats) {
    const int co = dgrad ? L.cin : L.cout, G = (dgrad ? L.coutp : L.cinp) / 8;
    const dim3 grid((unsigned)((long long)B * L.H * L.W / 128), (unsigned)(co / NT));
    ++u->launches;
    u->tc_ran = true;
    if (dgrad)
        k_conv3x3_tc<NT><<<grid, 256, tc_conv_smem(NT), st>>>(L.dy, L.cout, nullptr, 0, L.wd, G, co, out0, out1,
                                                              split, acc0, acc1, nullptr, B, L.H, L.W,
                                                              u->tc_timeouts, u->tc_spin);
    else
        k_conv3x3_tc<NT><<<grid, 256, tc_conv_smem(NT), st>>>(L.in0, L.c0, L.in1, L.c1, L.wf, G, co, out0, out1,
                                                              split, acc0, acc1, stats, B, L.H, L.W,
                                                              u->tc_timeouts, u->tc_spin);
    return cudaGetLastError();
}

template <int MT, int NT>
cudaError_t gemm_conv_launch(fmbym_unet* u, const Layer& L, int B, bool dgrad, cudaStream_t st, float* out0,
                             float* out1, int split, int acc0, int acc1, float2* stats) {
    const int co = dgrad ? L.cin : L.cout, G = (dgrad ? L.coutp : L.cinp) / 8;
    const dim3 grid((unsigned)((long long)B * L.H * L.W / MT), (unsigned)(co / NT));
    const size_t smem = gemm_conv_smem(MT, NT);
    ++u->launches;
    if (dgrad)
        k_conv3x3_gemm<MT, NT><<<grid, 256, smem, st>>>(L.dy, L.cout, nullptr, 0, nullptr, nullptr, L.wd, G, co, out0,
                                                         out1, split, acc0, acc1, nullptr, B, L.H, L.W);
    else
        k_conv3x3_gemm<MT, NT><<<grid, 256, smem, st>>>(L.in0, L.c0, L.in1, L.c1,
                                                         L.planes ? (const float*)L.in0 : nullptr,
                                                         L.planes ? (const float*)L.in1 : nullptr, L.wf, G, co, out0,
                                                         out1, split, acc0, acc1, stats, B, L.H, L.W);
    return cudaGetLastError();
}

cudaError_t conv_dispatch(fmbym_unet* u, const Layer& L, int B, bool dgrad, cudaStream_t st, float* out0,
                          float* out1, int split, int acc0, int acc1, float2* stats) {
    const int co = dgrad ? L.cin : L.cout, R = dgrad ? L.R_d : L.R_f;
    if (dgrad ? L.gemm_d : L.gemm_f) {
        const long long npix = (long long)B * L.H * L.W;
        if (u->conv_path == 1 && !L.planes && gemm_big(u, co, npix))
            return co % 128 == 0 && (npix / 128) * (co / 128) >= u->nsm
                       ? tc_conv_launch<128>(u, L, B, dgrad, st, out0, out1, split, acc0, acc1, stats)
                       : tc_conv_launch<64>(u, L, B, dgrad, st, out0, out1, split, acc0, acc1, stats);
        return gemm_big(u, co, npix) ? gemm_conv_launch<128, 64>(u, L, B, dgrad, st, out0, out1, split, acc0, acc1, stats)
                                     : gemm_conv_launch<64, 32>(u, L, B, dgrad, st, out0, out1, split, acc0, acc1, stats);
    }
#define FMBYM_CONV(C, RR) \
    if (co == C && R == RR) return conv_launch<C, RR>(u, L, B, dgrad, st, out0, out1, split, acc0, acc1, stats);
    FMBYM_CONV(8, 4) FMBYM_CONV(16, 4) FMBYM_CONV(24, 4) FMBYM_CONV(8, 2) FMBYM_CONV(16, 2) FMBYM_CONV(24, 2)
    FMBYM_CONV(8, 1) FMBYM_CONV(16, 1) FMBYM_CONV(24, 1) FMBYM_CONV(32, 1) FMBYM_CONV(48, 1) FMBYM_CONV(64, 1)
    FMBYM_CONV(96, 1) FMBYM_CONV(128, 1)
#undef FMBYM_CONV
    return cudaErrorInvalidValue;
}

// BN adjoint slabs: about four CTAs per SM, each a whole number of the reduce kernel's pixel rows.
int bn_pix_per_cta(const fmbym_unet* u, long long px, int C) {
    const long long rows = 256 / (C / 4), target = 4LL * u->nsm;
    const long long per = (px + target - 1) / target;
    return (int)std::max(rows, (per + rows - 1) / rows * rows);
}

// Partials of the head adjoint: a grid of eight CTAs per SM, grid-stride over the pixels.
int head_grid(const fmbym_unet* u) { return 8 * u->nsm; }

// Weight-gradient plan of a layer: CIB input channels per CTA (the largest of 64, 32, 16, 8 that
// divides the input channels, so that no warp idles), CTA tiles of 8 R x 32 pixels (R up to 2 for
// CIB 8 and 16, dividing the height, else 1), a ring of three slots while they stay under 60 KB of
// shared memory, else two, and the resident CTAs of that configuration.
template <int CIB, bool PLANES>
cudaError_t wgrad_plan_t(const fmbym_unet* u, Layer& l) {
    const int rmax = PLANES ? 1 : CIB <= 16 ? 2 : 1;
    l.wg_R = 1;
    for (int r = rmax; r > 1; r /= 2)
        if (l.H % (8 * r) == 0) {
            l.wg_R = r;
            break;
        }
    l.wg_ns = 3 * wgrad_buf_bytes<CIB>(l.wg_R) <= 60 * 1024 ? 3 : 2;
    const size_t smem = wgrad_smem<CIB>(l.wg_R, l.wg_ns);
    cudaError_t e = cudaFuncSetAttribute(k_wgrad<CIB, PLANES>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_wgrad<CIB, PLANES>, 256, smem);
    l.wg_slots = std::max(1, occ) * u->nsm;
    return e;
}

cudaError_t wgrad_plan(const fmbym_unet* u, Layer& l) {
    if (l.planes) {
        l.wg_cib = 8;
        return wgrad_plan_t<8, true>(u, l);
    }
    l.wg_cib = l.cin % 64 == 0 ? 64 : l.cin % 32 == 0 ? 32 : l.cin % 16 == 0 ? 16 : 8;
    switch (l.wg_cib) {
        case 64: return wgrad_plan_t<64, false>(u, l);
        case 32: return wgrad_plan_t<32, false>(u, l);
        case 16: return wgrad_plan_t<16, false>(u, l);
        default: return wgrad_plan_t<8, false>(u, l);
    }
}

// Channel blocks gy (16 outputs) x gz (CIB inputs), and the pixel tiles cut into one wave of
// chunks over the resident CTAs.
struct WgradGeom {
    int gy, gz, chunks, tpc, used;
};

WgradGeom wgrad_geom(const Layer& l, int B) {
    WgradGeom w;
    w.gy = (l.cout + 15) / 16;
    w.gz = l.planes ? 1 : l.cin / l.wg_cib;
    const int ntiles = B * (l.H / (8 * l.wg_R)) * (l.W / kTW);
    w.chunks = std::max(1, std::min(ntiles, l.wg_slots / (w.gy * w.gz)));
    w.tpc = (ntiles + w.chunks - 1) / w.chunks;
    w.used = (ntiles + w.tpc - 1) / w.tpc;
    return w;
}

template <int CIB, bool PLANES>
void wgrad_run(const Layer& l, const WgradGeom& w, int n, const float* f, const float* g, float* part,
               cudaStream_t st) {
    k_wgrad<CIB, PLANES><<<dim3(w.used * w.gz, w.gy), 256, wgrad_smem<CIB>(l.wg_R, l.wg_ns), st>>>(
        l.dy, l.cout, PLANES ? nullptr : l.in0, PLANES ? 0 : l.c0, l.in1, l.c1, f, g, n, l.H, l.W, l.wg_R, w.gz,
        w.tpc, l.wg_ns, part);
}

// Flat-GEMM weight gradient: kWM output channels x kWI items per CTA, pixel tiles of kWP cut
// into one wave of chunks over the resident CTAs.
WgradGeom gemm_wgrad_geom(const fmbym_unet* u, const Layer& l, int B) {
    WgradGeom w;
    w.gy = l.cout / kWM;
    w.gz = (9 * (l.cin / 8) + kWI - 1) / kWI;
    const int ntiles = (int)((long long)B * l.H * l.W / kWP);
    w.chunks = std::max(1, std::min(ntiles, u->gw_slots / (w.gy * w.gz)));
    w.tpc = (ntiles + w.chunks - 1) / w.chunks;
    w.used = (ntiles + w.tpc - 1) / w.tpc;
    return w;
}

// Inputs of layer k for a batch of B (planes for the first layer are set per call).
void wire_inputs(fmbym_unet* u) {
    const int L = u->levels;
    for (int i = 0; i < L; ++i) {
        Layer& a = u->layers[2 * i];
        Layer& b = u->layers[2 * i + 1];
        if (i > 0) {
            a.in0 = u->pooled[i];
            a.c0 = u->ch[i - 1];
        }
        b.in0 = a.a;
        b.c0 = a.cout;
    }
    for (int j = 0; j < L - 1; ++j) {
        const int i = L - 2 - j;  // level of this decoder pair
        Layer& a = u->layers[2 * L + 2 * j];
        Layer& b = u->layers[2 * L + 2 * j + 1];
        a.in0 = u->upped[i];
        a.c0 = u->ch[i + 1];
        a.in1 = u->layers[2 * i + 1].a;  // skip: a of enc{i}b
        a.c1 = u->ch[i];
        b.in0 = a.a;
        b.c0 = a.cout;
    }
}

}  // namespace

extern "C" {

const char* fmbym_unet_last_error(const fmbym_unet* u) { return u ? u->err.c_str() : g_unet_create_error.c_str(); }

void fmbym_unet_destroy(fmbym_unet* u) {
    if (!u) return;
    cudaDeviceSynchronize();
    for (void* p : u->allocs) cudaFree(p);
    delete u;
}

int fmbym_unet_create(fmbym_unet** out, const fmbym_unet_config* cfg) {
    g_unet_create_error.clear();
    if (!out || !cfg) return ufail(nullptr, FMBYM_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    const int L = cfg->levels;
    if (L < 2 || L > 8) return ufail(nullptr, FMBYM_ERR_INVALID_ARG, "levels must be in [2, 8]");
    for (int i = 0; i < L; ++i) {
        const int c = cfg->channels[i];
        if (c != 8 && c != 16 && c != 32 && c != 64 && c != 128 && c != 256)
            return ufail(nullptr, FMBYM_ERR_UNSUPPORTED_SIZE, "channels must be 8, 16, 32, 64, 128 or 256");
        if (i > 0 && c < cfg->channels[i - 1]) return ufail(nullptr, FMBYM_ERR_INVALID_ARG, "channels must not decrease");
    }
    if (cfg->channels[0] > 64) return ufail(nullptr, FMBYM_ERR_UNSUPPORTED_SIZE, "the first level has at most 64 channels");
    if (cfg->max_batch < 1) return ufail(nullptr, FMBYM_ERR_INVALID_ARG, "max_batch must be >= 1");
    const int H = cfg->height, W = cfg->width;
    if (H <= 0 || W <= 0 || H % (8 << (L - 1)) || W % (8 << (L - 1)) || W % kTW)
        return ufail(nullptr, FMBYM_ERR_UNSUPPORTED_SIZE,
                     "height and width must be multiples of 8*2^(L-1), and width of 32");
    if ((long long)cfg->max_batch * H * W * cfg->channels[L - 1] / 4 >= (1LL << 31))
        return ufail(nullptr, FMBYM_ERR_UNSUPPORTED_SIZE, "max_batch * height * width * channels too large");
    fmbym_unet* u = new fmbym_unet();
    u->levels = L;
    for (int i = 0; i < L; ++i) u->ch[i] = cfg->channels[i];
    u->H = H;
    u->W = W;
    u->max_batch = cfg->max_batch;
    const int B = cfg->max_batch;
    // layer list and parameter offsets (the order of the flat parameter array)
    long long off = 0, roff = 0;
    auto add = [&](const std::string& nm, int cin, int cout, int lvl) {
        Layer l;
        l.name = nm;
        l.cin = cin;
        l.cout = cout;
        l.H = H >> lvl;
        l.W = W >> lvl;
        l.cinp = round8(cin);
        l.coutp = round8(cout);
        l.w_off = off;
        off += (long long)cout * cin * 9;
        l.g_off = off;
        off += cout;
        l.b_off = off;
        off += cout;
        l.rs_off = roff;
        roff += 2 * cout;
        u->layers.push_back(l);
    };
    int cprev = 2;
    for (int i = 0; i < L; ++i) {
        add("enc" + std::to_string(i) + "a", cprev, u->ch[i], i);
        add("enc" + std::to_string(i) + "b", u->ch[i], u->ch[i], i);
        cprev = u->ch[i];
    }
    int deeper = u->ch[L - 1];
    for (int i = L - 2; i >= 0; --i) {
        add("dec" + std::to_string(i) + "a", deeper + u->ch[i], u->ch[i], i);
        add("dec" + std::to_string(i) + "b", u->ch[i], u->ch[i], i);
        deeper = u->ch[i];
    }
    u->head_w = off;
    off += 2 * u->ch[0];
    u->head_b = off;
    off += 2;
    u->n_params = off;
    u->n_running = roff;
    u->layers[0].planes = true;
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) {
        if (e == cudaSuccess) e = x;
    };
    chk(ualloc(u, &u->params, off));
    chk(ualloc(u, &u->grads, off));
    chk(ualloc(u, &u->adam_m, off));
    chk(ualloc(u, &u->adam_v, off));
    chk(ualloc(u, &u->running, roff));
    int dev = 0;
    chk(cudaGetDevice(&dev));
    chk(cudaDeviceGetAttribute(&u->nsm, cudaDevAttrMultiProcessorCount, dev));
    {
        int occ = 0;
        chk(cudaFuncSetAttribute(k_wgrad_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmWgradSmem));
        chk(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_wgrad_gemm, 256, kGemmWgradSmem));
        u->gw_slots = std::max(1, occ) * u->nsm;
        chk(cudaFuncSetAttribute(k_conv3x3_gemm<64, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)gemm_conv_smem(64, 32)));
        chk(cudaFuncSetAttribute(k_conv3x3_gemm<128, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)gemm_conv_smem(128, 64)));
        chk(cudaFuncSetAttribute(k_conv3x3_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_conv_smem(64)));
        chk(cudaFuncSetAttribute(k_conv3x3_tc<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tc_conv_smem(128)));
        chk(ualloc(u, &u->tc_timeouts, 1));
        chk(cudaMemset(u->tc_timeouts, 0, sizeof(unsigned)));
    }
    size_t stats_cap = 0, bn_cap = 0, w_cap = 0;
    bool too_big = false;
    for (Layer& l : u->layers) {
        const size_t px = (size_t)B * l.H * l.W;
        chk(ualloc(u, &l.wf, (size_t)l.cout * 9 * l.cinp));
        chk(ualloc(u, &l.wd, (size_t)l.cin * 9 * l.coutp));
        chk(ualloc(u, &l.y, px * l.cout));
        chk(ualloc(u, &l.a, px * l.cout));
        chk(ualloc(u, &l.da, px * l.cout));
        chk(ualloc(u, &l.dy, px * l.cout));
        chk(ualloc(u, &l.bn, l.cout));
        chk(ualloc(u, &l.bsums, l.cout));
        stats_cap = std::max(stats_cap, px / kTilePx * l.cout);
        bn_cap = std::max(bn_cap, (size_t)4 * u->nsm * l.cout);   // bn_pix_per_cta keeps the slabs at most 4 per SM
        // tile kernels where the image is at least a tile wide and the weights fit in shared memory,
        // the flat-GEMM kernels otherwise
        const bool wide = l.W % kTW == 0;
        if (wide) {
            chk(wgrad_plan(u, l));
            w_cap = std::max(w_cap, (size_t)wgrad_geom(l, B).chunks * l.cout * 9 * l.cin);
            chk(conv_plan(u, l.cout, l.cinp / 8, l.H, l.R_f, l.ns_f, l.slots_f));
            if (!l.planes) chk(conv_plan(u, l.cin, l.coutp / 8, l.H, l.R_d, l.ns_d, l.slots_d));
        }
        l.gemm_w = !wide;
        l.gemm_f = !wide || !l.ns_f;
        l.gemm_d = !l.planes && (!wide || !l.ns_d);
        if (l.gemm_w) w_cap = std::max(w_cap, (size_t)gemm_wgrad_geom(u, l, B).chunks * l.cout * 9 * l.cin);
        if (l.gemm_f) stats_cap = std::max(stats_cap, px / 64 * l.cout);
        if ((l.gemm_f && l.cout % 32) || (l.gemm_d && l.cin % 32) || (l.gemm_w && (l.planes || l.cout % kWM)))
            too_big = true;
    }
    u->pooled.assign(L, nullptr);
    u->upped.assign(L, nullptr);
    u->dpool.assign(L, nullptr);
    u->dup.assign(L, nullptr);
    for (int i = 1; i < L; ++i) {
        const size_t px = (size_t)B * (H >> i) * (W >> i);
        chk(ualloc(u, &u->pooled[i], px * u->ch[i - 1]));
        chk(ualloc(u, &u->dpool[i], px * u->ch[i - 1]));
    }
    for (int i = 0; i + 1 < L; ++i) {
        const size_t px = (size_t)B * (H >> i) * (W >> i);
        chk(ualloc(u, &u->upped[i], px * u->ch[i + 1]));
        chk(ualloc(u, &u->dup[i], px * u->ch[i + 1]));
    }
    u->stats_cap = stats_cap;
    u->bnpart_cap = bn_cap;
    u->wpart_cap = w_cap;
    u->hpart_cap = (size_t)head_grid(u) * (2 * u->ch[0] + 2);
    chk(ualloc(u, &u->stats, stats_cap));
    chk(ualloc(u, &u->bnpart, bn_cap));
    chk(ualloc(u, &u->wpart, w_cap));
    chk(ualloc(u, &u->hpart, u->hpart_cap));
    if (e == cudaSuccess) {
        // running statistics start at mean 0, variance 1
        std::vector<float> rs(roff);
        for (const Layer& l : u->layers)
            for (int c = 0; c < l.cout; ++c) {
                rs[l.rs_off + c] = 0.f;
                rs[l.rs_off + l.cout + c] = 1.f;
            }
        chk(cudaMemcpy(u->running, rs.data(), rs.size() * 4, cudaMemcpyHostToDevice));
        chk(cudaMemset(u->params, 0, off * 4));
        chk(cudaMemset(u->grads, 0, off * 4));
        chk(cudaMemset(u->adam_m, 0, off * 4));
        chk(cudaMemset(u->adam_v, 0, off * 4));
    }
    if (e != cudaSuccess) {
        fmbym_unet_destroy(u);
        return ucuda(nullptr, e, "U-Net allocation");
    }
    if (too_big) {
        fmbym_unet_destroy(u);
        return ufail(nullptr, FMBYM_ERR_UNSUPPORTED_SIZE, "a layer fits neither the tile nor the flat-GEMM convolution");
    }
    wire_inputs(u);
    *out = u;
    return FMBYM_OK;
}

long long fmbym_unet_param_count(const fmbym_unet* u) { return u ? u->n_params : 0; }
long long fmbym_unet_running_count(const fmbym_unet* u) { return u ? u->n_running : 0; }
float* fmbym_unet_params(fmbym_unet* u) { return u ? u->params : nullptr; }
float* fmbym_unet_grads(fmbym_unet* u) { return u ? u->grads : nullptr; }
float* fmbym_unet_running(fmbym_unet* u) { return u ? u->running : nullptr; }
long long fmbym_unet_launch_count(const fmbym_unet* u) { return u ? u->launches : 0; }

int fmbym_unet_set_conv_path(fmbym_unet* u, int path) {
    if (!u) return ufail(nullptr, FMBYM_ERR_INVALID_ARG, "handle is NULL");
    if (path != 0 && path != 1) return ufail(u, FMBYM_ERR_INVALID_ARG, "conv path must be 0 (mma.sync) or 1 (tcgen05)");
    u->conv_path = path;
    return FMBYM_OK;
}

int fmbym_unet_set_tc_wait_limit(fmbym_unet* u, unsigned polls) {
    if (!u) return ufail(nullptr, FMBYM_ERR_INVALID_ARG, "handle is NULL");
    u->tc_spin = polls == 0 ? kTcSpin : polls;
    return FMBYM_OK;
}

long long fmbym_unet_tc_timeouts(fmbym_unet* u) {
    if (!u || !u->tc_timeouts) return 0;
    unsigned v = 0;
    if (cudaMemcpy(&v, u->tc_timeouts, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    return (long long)v;
}

int fmbym_unet_layer_tensor(fmbym_unet* u, void* stream, int layer, int which, int n, float* dst) {
    if (!u || layer < 0 || layer >= (int)u->layers.size() || which < 0 || which > 3 || !dst || n < 1 ||
        n > u->max_batch)
        return ufail(u, FMBYM_ERR_INVALID_ARG, "bad layer tensor request");
    const Layer& l = u->layers[layer];
    const long long cnt = (long long)n * l.H * l.W * l.cout;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (which == 0) e = cudaMemcpyAsync(dst, l.y, cnt * 4, cudaMemcpyDeviceToDevice, st);
    else if (which == 2) e = cudaMemcpyAsync(dst, l.da, cnt * 4, cudaMemcpyDeviceToDevice, st);
    else {
        // bf16 -> float32 widening through the upsample-free path: copy raw and widen on the host side
        std::vector<uint16_t> tmp(cnt);
        e = cudaMemcpyAsync(tmp.data(), which == 1 ? (const void*)l.a : (const void*)l.dy, cnt * 2,
                            cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        std::vector<float> wide(cnt);
        for (long long i = 0; i < cnt; ++i) {
            const uint32_t bits = (uint32_t)tmp[i] << 16;
            memcpy(&wide[i], &bits, 4);
        }
        if (e == cudaSuccess) e = cudaMemcpy(dst, wide.data(), cnt * 4, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) return ucuda(u, e, "layer tensor");
    return FMBYM_OK;
}

int fmbym_unet_load(fmbym_unet* u, void* stream, const float* params, const float* running) {
    if (!u) return ufail(nullptr, FMBYM_ERR_INVALID_ARG, "handle is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (params) e = cudaMemcpyAsync(u->params, params, u->n_params * 4, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && running)
        e = cudaMemcpyAsync(u->running, running, u->n_running * 4, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && params) {
        cudaMemsetAsync(u->adam_m, 0, u->n_params * 4, st);
        e = cudaMemsetAsync(u->adam_v, 0, u->n_params * 4, st);
    }
    if (e != cudaSuccess) return ucuda(u, e, "load");
    return FMBYM_OK;
}

int fmbym_unet_store(fmbym_unet* u, void* stream, float* params, float* running, float* grads) {
    if (!u) return ufail(nullptr, FMBYM_ERR_INVALID_ARG, "handle is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (params) e = cudaMemcpyAsync(params, u->params, u->n_params * 4, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && running)
        e = cudaMemcpyAsync(running, u->running, u->n_running * 4, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && grads) e = cudaMemcpyAsync(grads, u->grads, u->n_params * 4, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return ucuda(u, e, "store");
    return FMBYM_OK;
}

int fmbym_unet_store_adam(fmbym_unet* u, void* stream, float* m, float* v) {
    if (!u) return ufail(nullptr, FMBYM_ERR_INVALID_ARG, "handle is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (m) e = cudaMemcpyAsync(m, u->adam_m, u->n_params * 4, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && v) e = cudaMemcpyAsync(v, u->adam_v, u->n_params * 4, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return ucuda(u, e, "store_adam");
    return FMBYM_OK;
}

int fmbym_unet_load_adam(fmbym_unet* u, void* stream, const float* m, const float* v) {
    if (!u) return ufail(nullptr, FMBYM_ERR_INVALID_ARG, "handle is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (m) e = cudaMemcpyAsync(u->adam_m, m, u->n_params * 4, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && v) e = cudaMemcpyAsync(u->adam_v, v, u->n_params * 4, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return ucuda(u, e, "load_adam");
    return FMBYM_OK;
}

int fmbym_unet_forward(fmbym_unet* u, void* stream, int n, const float* f, const float* g, int training,
                       float* f_out, float* g_out, float* masks) {
    if (!u) return ufail(nullptr, FMBYM_ERR_INVALID_ARG, "handle is NULL");
    u->err.clear();
    if (n < 0 || n > u->max_batch) return ufail(u, FMBYM_ERR_WORKSPACE, "batch exceeds max_batch");
    if (n == 0) return FMBYM_OK;
    if (!f || !g) return ufail(u, FMBYM_ERR_INVALID_ARG, "f and g must not be NULL");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    const int L = u->levels;
    Layer& first = u->layers[0];
    first.in0 = (const bf16*)f;  // planes: read as float inside the conv kernel
    first.in1 = (const bf16*)g;
    // weights for this step
    for (Layer& l : u->layers) {
        const int nf = l.cout * 9 * l.cinp, nd = l.cin * 9 * l.coutp;
        ++u->launches;
        k_prep_weights<<<blocks(std::max(nf, nd)), kBlock, 0, st>>>(u->params + l.w_off, l.cout, l.cin, l.cinp,
                                                                  l.coutp, l.wf, l.wd);
    }
    auto conv_bn = [&](Layer& l) -> cudaError_t {
        const long long px = (long long)n * l.H * l.W;
        const int tile_px = l.gemm_f ? (gemm_big(u, l.cout, px) ? 128 : 64) : kTilePx * l.R_f;
        const int ntiles = (int)(px / tile_px);
        const int nparts = l.gemm_f ? ntiles : std::min(ntiles, l.slots_f);   // the conv's grid
        cudaError_t r = conv_dispatch(u, l, n, false, st, l.y, nullptr, l.cout, 0, 0, training ? u->stats : nullptr);
        if (r != cudaSuccess) return r;
        ++u->launches;
        if (training)
            k_bn_finalize<<<l.cout, 256, 0, st>>>(u->stats, nparts, l.cout, ntiles, (float)tile_px,
                                                  u->running + l.rs_off, u->running + l.rs_off + l.cout, l.bn);
        else
            k_bn_eval<<<(l.cout + 127) / 128, 128, 0, st>>>(u->running + l.rs_off, u->running + l.rs_off + l.cout, l.cout, l.bn);
        ++u->launches;
        k_bn_relu<<<blocks(px * l.cout / 8), kBlock, 0, st>>>(l.y, l.bn, u->params + l.g_off, u->params + l.b_off,
                                                              l.a, px * l.cout / 8, l.cout);
        return cudaGetLastError();
    };
    for (int i = 0; i < L && e == cudaSuccess; ++i) {
        if (i > 0) {
            const Layer& prev = u->layers[2 * i - 1];
            ++u->launches;
            k_maxpool<<<blocks((long long)n * (prev.H / 2) * (prev.W / 2) * (prev.cout / 8)), kBlock, 0, st>>>(
                prev.a, u->pooled[i], n, prev.H, prev.W, prev.cout);
        }
        e = conv_bn(u->layers[2 * i]);
        if (e == cudaSuccess) e = conv_bn(u->layers[2 * i + 1]);
    }
    for (int j = 0; j < L - 1 && e == cudaSuccess; ++j) {
        const int i = L - 2 - j;
        const Layer& deep = (j == 0) ? u->layers[2 * L - 1] : u->layers[2 * L + 2 * (j - 1) + 1];
        ++u->launches;
        k_upsample<<<row_grid(deep.W * (deep.cout / 8), n * deep.H), kBlock, 0, st>>>(
            deep.a, u->upped[i], n, deep.H, deep.W, deep.cout);
        e = conv_bn(u->layers[2 * L + 2 * j]);
        if (e == cudaSuccess) e = conv_bn(u->layers[2 * L + 2 * j + 1]);
    }
    if (e == cudaSuccess) {
        const Layer& last = u->layers.back();
        const long long npix = (long long)n * u->H * u->W;
        ++u->launches;
        switch (u->ch[0]) {
            case 8: k_head<8><<<blocks(npix), kBlock, 0, st>>>(last.a, u->params + u->head_w, u->params + u->head_b, f, g, f_out, g_out, masks, npix, u->H * u->W); break;
            case 16: k_head<16><<<blocks(npix), kBlock, 0, st>>>(last.a, u->params + u->head_w, u->params + u->head_b, f, g, f_out, g_out, masks, npix, u->H * u->W); break;
            case 32: k_head<32><<<blocks(npix), kBlock, 0, st>>>(last.a, u->params + u->head_w, u->params + u->head_b, f, g, f_out, g_out, masks, npix, u->H * u->W); break;
            default: k_head<64><<<blocks(npix), kBlock, 0, st>>>(last.a, u->params + u->head_w, u->params + u->head_b, f, g, f_out, g_out, masks, npix, u->H * u->W); break;
        }
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return ucuda(u, e, "U-Net forward");
    u->last_batch = training ? n : -1;
    return tc_status(u, st, "U-Net forward");
}

int fmbym_unet_backward(fmbym_unet* u, void* stream, int n, const float* f, const float* g, const float* df_out,
                        const float* dg_out) {
    if (!u) return ufail(nullptr, FMBYM_ERR_INVALID_ARG, "handle is NULL");
    u->err.clear();
    if (n != u->last_batch) return ufail(u, FMBYM_ERR_INVALID_ARG, "backward needs a training forward of the same batch");
    if (!f || !g || !df_out || !dg_out) return ufail(u, FMBYM_ERR_INVALID_ARG, "NULL buffer");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    const int L = u->levels, C0 = u->ch[0];
    const long long npix = (long long)n * u->H * u->W;
    // head
    {
        const Layer& last = u->layers.back();
        const int nb = (int)std::min<long long>(blocks(npix), head_grid(u)), width = 2 * C0 + 2;
        ++u->launches;
        switch (C0) {
            case 8: k_head_bwd<8><<<nb, kBlock, 0, st>>>(last.a, u->params + u->head_w, u->params + u->head_b, f, g, df_out, dg_out, last.da, u->hpart, npix); break;
            case 16: k_head_bwd<16><<<nb, kBlock, 0, st>>>(last.a, u->params + u->head_w, u->params + u->head_b, f, g, df_out, dg_out, last.da, u->hpart, npix); break;
            case 32: k_head_bwd<32><<<nb, kBlock, 0, st>>>(last.a, u->params + u->head_w, u->params + u->head_b, f, g, df_out, dg_out, last.da, u->hpart, npix); break;
            default: k_head_bwd<64><<<nb, kBlock, 0, st>>>(last.a, u->params + u->head_w, u->params + u->head_b, f, g, df_out, dg_out, last.da, u->hpart, npix); break;
        }
        ++u->launches;
        k_sum_parts<<<width, 256, 0, st>>>(u->hpart, nb, width, u->grads + u->head_w);
    }
    // one layer: BN/ReLU adjoint, weight gradient, and (unless first) dgrad into out0/out1
    auto layer_bwd = [&](Layer& l, float* out0, float* out1, int split, int acc0, int acc1) -> cudaError_t {
        const long long px = (long long)n * l.H * l.W;
        const int C = l.cout, pix_per_cta = bn_pix_per_cta(u, px, C);
        const int nparts = (int)((px + pix_per_cta - 1) / pix_per_cta);
        u->launches += 3;
        k_bn_bwd_reduce<<<nparts, 256, 0, st>>>(l.y, l.da, l.bn, u->params + l.g_off, u->params + l.b_off, px, C,
                                                pix_per_cta, u->bnpart);
        k_bn_bwd_finalize<<<C, 256, 0, st>>>(u->bnpart, nparts, C, 1.f / (float)px, u->grads + l.g_off,
                                             u->grads + l.b_off, l.bsums);
        k_bn_bwd_dy<<<blocks(px * C / 4), kBlock, 0, st>>>(l.y, l.da, l.bn, u->params + l.g_off,
                                                           u->params + l.b_off, l.bsums, l.dy, px * C / 4, C);
        // weight gradient
        const WgradGeom w = l.gemm_w ? gemm_wgrad_geom(u, l, n) : wgrad_geom(l, n);
        u->launches += 2;
        if (l.gemm_w)
            k_wgrad_gemm<<<dim3(w.used, w.gy, w.gz), 256, kGemmWgradSmem, st>>>(l.dy, l.cout, l.in0, l.c0, l.in1, l.c1,
                                                                             n, l.H, l.W, w.tpc, u->wpart);
        else if (l.planes) wgrad_run<8, true>(l, w, n, f, g, u->wpart, st);
        else if (l.wg_cib == 64) wgrad_run<64, false>(l, w, n, f, g, u->wpart, st);
        else if (l.wg_cib == 32) wgrad_run<32, false>(l, w, n, f, g, u->wpart, st);
        else if (l.wg_cib == 16) wgrad_run<16, false>(l, w, n, f, g, u->wpart, st);
        else wgrad_run<8, false>(l, w, n, f, g, u->wpart, st);
        const int total = C * 9 * l.cin;
        k_wgrad_reduce<<<(total + 31) / 32, 256, 0, st>>>(u->wpart, w.used, C, l.cin, u->grads + l.w_off);
        cudaError_t r = cudaGetLastError();
        if (r != cudaSuccess || !out0) return r;
        return conv_dispatch(u, l, n, true, st, out0, out1, split, acc0, acc1, nullptr);
    };
    // decoder, last layer first
    for (int j = L - 2; j >= 0 && e == cudaSuccess; --j) {
        const int i = L - 2 - j;
        Layer& la = u->layers[2 * L + 2 * j];
        Layer& lb = u->layers[2 * L + 2 * j + 1];
        e = layer_bwd(lb, la.da, nullptr, lb.cin, 0, 0);
        if (e != cudaSuccess) break;
        Layer& skip = u->layers[2 * i + 1];
        e = layer_bwd(la, u->dup[i], skip.da, u->ch[i + 1], 0, 0);
        if (e != cudaSuccess) break;
        Layer& deep = (j == 0) ? u->layers[2 * L - 1] : u->layers[2 * L + 2 * (j - 1) + 1];
        ++u->launches;
        k_upsample_bwd<<<row_grid((deep.W / 2) * (deep.cout / 4), n * (deep.H / 2)), kBlock, 0, st>>>(
            u->dup[i], deep.da, n, deep.H, deep.W, deep.cout);
        e = cudaGetLastError();
    }
    // encoder, deepest first
    for (int i = L - 1; i >= 0 && e == cudaSuccess; --i) {
        Layer& la = u->layers[2 * i];
        Layer& lb = u->layers[2 * i + 1];
        e = layer_bwd(lb, la.da, nullptr, lb.cin, 0, 0);
        if (e != cudaSuccess) break;
        if (i == 0) {
            e = layer_bwd(la, nullptr, nullptr, 0, 0, 0);
            break;
        }
        e = layer_bwd(la, u->dpool[i], nullptr, la.cin, 0, 0);
        if (e != cudaSuccess) break;
        Layer& prev = u->layers[2 * i - 1];
        ++u->launches;
        k_maxpool_bwd<<<blocks((long long)n * (prev.H / 2) * (prev.W / 2) * (prev.cout / 4)), kBlock, 0, st>>>(
            prev.a, u->dpool[i], prev.da, n, prev.H, prev.W, prev.cout);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return ucuda(u, e, "U-Net backward");
    return tc_status(u, st, "U-Net backward");
}

int fmbym_unet_adam(fmbym_unet* u, void* stream, float lr, float beta1, float beta2, float eps, int step) {
    if (!u) return ufail(nullptr, FMBYM_ERR_INVALID_ARG, "handle is NULL");
    if (step < 1) return ufail(u, FMBYM_ERR_INVALID_ARG, "step counts from 1");
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    ++u->launches;
    k_adam<<<blocks(u->n_params), kBlock, 0, (cudaStream_t)stream>>>(u->params, u->grads, u->adam_m, u->adam_v,
                                                                    u->n_params, lr, beta1, beta2, eps, c1, c2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ucuda(u, e, "Adam");
    return FMBYM_OK;
}

}  // extern "C"
