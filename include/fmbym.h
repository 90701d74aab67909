/*
 * fmbym.h -- C ABI of the GB300 decoupled Fourier pose search (Fast-MbyM, arXiv 2203.00459).
 *
 * The library implements ScanMatch of Alg. 1 for batches of scan pairs on one GPU:
 *   stage 1 (rotation, Eq. 4-7): Hann window -> 2D FFT -> band-pass -> |.| -> Cart2Pol ->
 *            circular correlation along angle -> soft-argmax over the angle candidates;
 *   stage 2 (translation, Eq. 8): Rotate(source, theta) -> ZeroPad -> 2D FFT correlation ->
 *            soft-argmax over the translation candidates;
 * and the adjoint of the whole search (the differentiability of Sec. III-C that the masking
 * network of Sec. III-D trains through, Eq. 13).
 *
 * Conventions shared by every call
 *   - Scans are float32, row-major [N][N], y = row, x = column.  Scores are stored in lag order:
 *     index 0 is the most negative lag (-N/2 for translations, -n_theta/2 for angles).
 *   - The pose of a pair is float32 [3] = (theta [rad], t_x, t_y [units of delta_xy]).  The
 *     source f is rotated by +theta about (N/2, N/2) (theta > 0 turns +x toward +y), after which
 *     g(x) ~ f'(x - t); Alg. 1's BuildSO2/MatMul step is the identity in this convention.
 *   - Device pointers are CUDA global memory on the handle's device; "host" pointers are CPU
 *     memory (pinned memory makes the copies asynchronous).  The caller owns every buffer it
 *     passes; the library owns only its workspace, which it allocates in fmbym_create.
 *   - Calls are asynchronous on the given stream (a cudaStream_t passed as void*; NULL is the
 *     legacy default stream) unless stated otherwise.  A handle must be used from one host
 *     thread and one stream at a time.
 *   - Every call returns a status code; fmbym_last_error() describes the last failure.
 *     FMBYM_ERR_CUDA is sticky: a CUDA error in the context is reported, not cleared.
 */
#ifndef FMBYM_H
#define FMBYM_H

#ifdef __cplusplus
extern "C" {
#endif

enum fmbym_status {
    FMBYM_OK = 0,
    FMBYM_ERR_INVALID_ARG = 1,      /* NULL or out-of-range argument                         */
    FMBYM_ERR_UNSUPPORTED_SIZE = 2, /* N not in {127,128,255,256,511,512}, n_theta not in 8..1024,
                                       or pad_mode 1 with an odd N                          */
    FMBYM_ERR_WORKSPACE = 3,        /* more pairs than the handle was created for            */
    FMBYM_ERR_CUDA = 4,             /* a CUDA runtime call or launch failed                  */
    FMBYM_ERR_TIMEOUT = 5           /* a bounded device-side wait ran out                    */
};

/* Parameters of one scan size: the arguments of ScanMatch in Alg. 1 plus the readings of
 * the places the paper leaves open.
 *   n           scan side N (n_xy of Alg. 1); supported: 128, 256, 512 and the paper's odd sides
 *               127, 255, 511 (Sec. IV-B cell sizes; Alg. 1's n_xy = 255), whose stage-1 DFTs run as
 *               Bluestein convolutions and whose stage 2 runs in the even frame N + 1 (pad_mode 0
 *               only)
 *   n_theta     number of angle candidates over a half turn (delta_theta = pi / n_theta,
 *               Alg. 1 first Linspace); 8..1024: 128, 256 and 400 take the FFT correlation,
 *               any other count (Alg. 1's default 733 among them) direct circular sums
 *   n_r         radii of the polar grid, rho_j = j * (N/2) / n_r, 1 <= n_r <= N/2 (Cart2Pol)
 *   temp_theta  T_theta > 0, temp_xy  T_xy > 0 (SoftArgMax temperatures of Alg. 1)
 *   delta_xy    translation bin size > 0 (the pose's t is lag * delta_xy)
 *   window      1: periodic Hann window before the stage-1 FFT (Alg. 1 HanningFilter); 0: none
 *   pad_mode    0: ZeroPad to 2N, linear correlation (Alg. 1 ZeroPad); 1: N-periodic
 *   score_norm  0: softmax(zscore(c) / T); 1: softmax(c / T) (the literal form)
 *   band_lo, band_hi  radial band-pass on the DFT grid, keep band_lo <= rho <= band_hi bins
 *               (Alg. 1 BandPassFilter) */
typedef struct fmbym_size_cfg {
    int n;
    int n_theta;
    int n_r;
    float temp_theta;
    float temp_xy;
    float delta_xy;
    int window;
    int pad_mode;
    int score_norm;
    float band_lo;
    float band_hi;
    int angle_score;   /* 0: Eq. 7, the angle correlation at radial lag 0, summed over radius (reading
                          A2); 1: the mean over radial lags of the circular 2D polar correlation that
                          Alg. 1 prints, i.e. the angle correlation of the radial sums over n_r */
    int full_circle;   /* 0: heading in [-pi/2, pi/2) (|F| of a real scan is centrosymmetric, reading
                          A9); 1: the full circle, stage 2 run at theta and theta + pi and the one
                          with the higher translation peak kept (the extension of Sec. V for
                          arbitrary headings; three stage-2 passes) */
    int rotate_target; /* 0: stage 2 rotates the source, f' = Rotate(f, theta), and t is the
                          translation's soft-argmax (reading A8); 1: Alg. 1's own stage 2, g turned
                          back by theta, f correlated with it, and t = R(theta) t' from that
                          soft-argmax t' (BuildSO2 / MatMul); half circle only (full_circle 0) */
} fmbym_size_cfg;

/* Handle flags.
 *   FMBYM_FLAG_GRAPH     capture each distinct call layout (forward or backward; pair count, sizes
 *                        and offsets; buffer pointers) into a CUDA graph on first use and replay it
 *                        with one launch afterwards (up to 16 layouts are kept, least recently used
 *                        released).  The first call of a layout must not happen while the caller's
 *                        stream is being captured.  Ignored while tracing is on.
 *   FMBYM_FLAG_AUTOTUNE  at creation, pick each size's launch schedules (fmbym_tune_knob) by
 *                        timing a training call (fmbym_pose_train) of max_pairs synthetic pairs
 *                        under every candidate, one schedule after another; the defaults are
 *                        used otherwise.  Every schedule computes the same results up to float
 *                        rounding order. */
enum fmbym_flags { FMBYM_FLAG_GRAPH = 1, FMBYM_FLAG_AUTOTUNE = 2 };

/* Launch schedules of a size (values for fmbym_get_tuning / fmbym_set_tuning):
 *   FMBYM_TUNE_COL_TILE     columns per CTA of the stage-2 column passes: for the zero-padded
 *                           lengths P = 3N/2 one of {C/2, C, 2C} with C = 192 / (P/16) (default C);
 *                           otherwise C = 256 / (P/16) only
 *   FMBYM_TUNE_ANGLE_RADII  radii per CTA of the angle correlation and its adjoint: 16 (default) or 8
 *   FMBYM_TUNE_ROT_PIXELS   pixels per thread of the Rotate adjoint: 4 (default), 1, 2 or 8
 *   FMBYM_TUNE_COL_PLAN     radix order of the stage-2 column FFTs: 0 (default) = 16, R, 3 with
 *                           R = P / 48; 1 = 16, 3, R (the middle and last radices swapped).  Both are
 *                           valid only for the zero-padded lengths P = 3N/2 (192, 384, 768);
 *                           otherwise 0 only */
enum fmbym_tune_knob { FMBYM_TUNE_COL_TILE = 0, FMBYM_TUNE_ANGLE_RADII = 1, FMBYM_TUNE_ROT_PIXELS = 2,
                       FMBYM_TUNE_COL_PLAN = 3, FMBYM_TUNE_COUNT = 4 };

/* Handle configuration: n_sizes size configurations (host array, copied by fmbym_create),
 * the largest number of pairs one call may carry, and flags (fmbym_flags).  Pairs of different
 * sizes in one call run as concurrent groups, one per size, on internal streams forked from and
 * joined back to the caller's stream.  A packed call (offsets NULL) of one size and 16 pairs or
 * more runs as two halves, one on the caller's stream and one on an internal stream forked from
 * and joined back to it, each in its own half of the handle's workspace; the results are those
 * of one call, pair by pair.  Calls on one handle must not overlap (one stream at a time). */
typedef struct fmbym_config {
    int n_sizes;
    const fmbym_size_cfg* sizes;
    int max_pairs;
    int flags;
} fmbym_config;

typedef struct fmbym_handle fmbym_handle;

/* Creates a handle on the current CUDA device: validates the sizes, builds the per-size plans
 * (twiddle, window and polar-sample tables) and allocates the whole workspace for max_pairs
 * pairs.  Synchronous.  On failure *out is NULL and the status says why. */
int fmbym_create(fmbym_handle** out, const fmbym_config* cfg);

/* Releases the handle and its device memory.  Synchronises the device.  NULL is a no-op. */
void fmbym_destroy(fmbym_handle* h);

/* Text of the last failure on this handle ("" if none); valid until the next call.  With a
 * NULL handle, the last failure of fmbym_create on this thread. */
const char* fmbym_last_error(const fmbym_handle* h);

/* Bytes of device workspace the handle holds. */
unsigned long long fmbym_workspace_bytes(const fmbym_handle* h);

/* Forward search (Alg. 1) for n_pairs scan pairs in one call.
 *   size_idx  host int[n_pairs]: index into cfg->sizes of each pair, or NULL for all 0
 *   offsets   host long long[n_pairs]: element offset of pair p's scan in f and g (and in
 *             c_xy), or NULL for packed order (offset of p = sum of N^2 over pairs < p); the
 *             offset of a pair of an even side must be a multiple of 4 (16-byte rows), that of an
 *             odd side (127, 255, 511) may be any
 *   f, g      device float32: source and target scans
 *   pose      device float32 [n_pairs][3] out: (theta, t_x, t_y)
 *   c_theta   device float32 out or NULL: the n_theta angle scores of each pair, packed in pair
 *             order (pair p starts at sum of n_theta over pairs < p), lag order
 *   c_xy      device float32 out or NULL: the N x N translation scores of each pair at the pair's
 *             offset, rows = t_y lags, columns = t_x lags, lag order
 * Pairs of different sizes may be mixed in any order.  Returns FMBYM_ERR_WORKSPACE if n_pairs
 * exceeds max_pairs. */
int fmbym_pose(fmbym_handle* h, void* stream, int n_pairs, const int* size_idx,
               const long long* offsets, const float* f, const float* g, float* pose,
               float* c_theta, float* c_xy);

/* Adjoint of fmbym_pose: given dL/dpose (device float32 [n_pairs][3]) writes dL/df and dL/dg
 * (device float32, laid out like f and g, overwritten).  Recomputes every forward intermediate
 * from f and g; keeps nothing between calls.  Differentiation follows Sec. III-C: soft-argmax,
 * FFTs, bilinear Rotate and Cart2Pol, |z| (derivative z/|z|, 0 at z = 0), Hann window. */
int fmbym_pose_backward(fmbym_handle* h, void* stream, int n_pairs, const int* size_idx,
                        const long long* offsets, const float* f, const float* g,
                        const float* dpose, float* df, float* dg);

/* Pose loss of Eq. 13 and its gradient, for training through the search (Sec. III-D).
 *   pose, gt  device float32 [n_pairs][3]: estimated and ground-truth (theta, t_x, t_y)
 *   kind      1: L1, |pose - gt| summed over the three components (Eq. 13);
 *             2: L2, (pose - gt)^2 summed over the three components
 *   loss      device float32 [1] out, or NULL: the mean over pairs (the expectation of Eq. 13)
 *   dpose     device float32 [n_pairs][3] out, or NULL: dloss/dpose (the L1 derivative is 0 at 0)
 * Deterministic.  Returns FMBYM_ERR_INVALID_ARG for another kind. */
int fmbym_pose_loss(fmbym_handle* h, void* stream, int n_pairs, const float* pose, const float* gt,
                    int kind, float* loss, float* dpose);

/* Exhaustive rotate-then-correlate search, the brute-force method the decoupled search replaces
 * (the "raw" rows of Tab. IIIa; Sec. I and III).  For every candidate heading angles[k] the source
 * is rotated and correlated with the target by the stage-2 steps of Alg. 1 (Rotate, ZeroPad and
 * correlation, soft-argmax); the heading is the candidate with the highest correlation peak (the
 * first on ties) and the translation that candidate's soft-argmax.
 *   size      index into cfg->sizes; every pair of the call has this size
 *   offsets   host long long[n_pairs] or NULL (packed), as fmbym_pose
 *   f, g      device float32 scans, 16-byte aligned
 *   n_angles  number of candidates (>= 1); angles host float[n_angles], radians
 *   pose      device float32 [n_pairs][3] out: (theta, t_x, t_y)
 *   peaks     device float32 [n_pairs][n_angles] out, or NULL: every candidate's correlation peak
 * Runs n_angles stage-2 passes over the batch, launched directly.  Returns FMBYM_ERR_WORKSPACE
 * if n_pairs exceeds max_pairs. */
int fmbym_pose_exhaustive(fmbym_handle* h, void* stream, int n_pairs, int size, const long long* offsets,
                          const float* f, const float* g, int n_angles, const float* angles, float* pose,
                          float* peaks);

/* The launch schedules of size `size` (host int[FMBYM_TUNE_COUNT] out, indexed by
 * fmbym_tune_knob). */
int fmbym_get_tuning(const fmbym_handle* h, int size, int* values);

/* Sets the launch schedules of size `size` (host int[FMBYM_TUNE_COUNT]); every value must be one
 * of its knob's candidates, else FMBYM_ERR_INVALID_ARG and nothing changes.  Releases the
 * handle's captured graphs (they hold the previous schedules); synchronises the device. */
int fmbym_set_tuning(fmbym_handle* h, int size, const int* values);

/* One training step of the search (Sec. III-D, Eq. 12-13): the forward of fmbym_pose, the loss of
 * fmbym_pose_loss against gt, and the adjoint of fmbym_pose_backward for that loss, in one call.
 * The adjoint reads the forward's intermediates from the handle's workspace, where this call's
 * forward left them, instead of recomputing them; the results equal those of the three separate
 * calls.
 *   f, g       device float32 scans (as fmbym_pose); gt device float32 [n_pairs][3]
 *   loss_kind  1 (L1, Eq. 13) or 2 (L2), as fmbym_pose_loss's kind
 *   pose       device float32 [n_pairs][3] out; loss device float32 [1] out
 *   dpose      device float32 [n_pairs][3] out: dloss/dpose
 *   df, dg     device float32 out, laid out like f and g (overwritten)
 * f, g, df and dg must be 16-byte aligned; every buffer is required.  Errors as fmbym_pose. */
int fmbym_pose_train(fmbym_handle* h, void* stream, int n_pairs, const int* size_idx,
                     const long long* offsets, const float* f, const float* g, const float* gt,
                     int loss_kind, float* pose, float* loss, float* dpose, float* df, float* dg);

/* fmbym_pose with HOST buffers: copies f and g (host float32, total elements as laid out by
 * offsets) into the handle's device staging area, runs the search on the stream, copies the
 * pose (host float32 [n_pairs][3]) back and synchronises the stream.  total_elems is the
 * length of f and of g in floats; it must not exceed what max_pairs scans of the largest
 * configured size hold. */
int fmbym_pose_host(fmbym_handle* h, void* stream, int n_pairs, const int* size_idx,
                    const long long* offsets, long long total_elems, const float* f_host,
                    const float* g_host, float* pose_host);

/* fmbym_pose_train with HOST buffers, for callers whose scans and gradients live in CPU memory:
 * copies f, g (host float32, total_elems each, laid out by offsets as in fmbym_pose) and gt (host
 * float32 [n_pairs][3]) into the handle's device staging area, runs the training call of
 * fmbym_pose_train there, copies the pose (host float32 [n_pairs][3]), the loss (host float32 [1])
 * and df, dg (host float32, total_elems each) back, and synchronises the stream.  Elements of df
 * and dg outside every pair's scan are unspecified.  total_elems must not exceed what max_pairs
 * scans of the largest configured size hold (FMBYM_ERR_WORKSPACE).  Pinned host memory makes the
 * copies asynchronous with respect to the host; pageable memory works but copies slower.  A packed
 * call (offsets NULL) of 16 pairs or more runs as a pipeline of 4 chunks of pairs (1/8, 3/8, 3/8
 * and 1/8 of them), the copies in and out on the handle's own streams overlapping the chunks'
 * training calls (with a single size, alternate chunks run on a second internal stream in the
 * second half of the handle's workspace, so consecutive chunks overlap); the results are
 * those of the one-piece call (each chunk's loss is normalised by the call's pair count, and the
 * loss is taken over every pair at the end).  Errors as fmbym_pose_train. */
int fmbym_pose_train_host(fmbym_handle* h, void* stream, int n_pairs, const int* size_idx,
                          const long long* offsets, long long total_elems, const float* f_host,
                          const float* g_host, const float* gt_host, int loss_kind, float* pose_host,
                          float* loss_host, float* df_host, float* dg_host);

/* Measures the FP32 multiply-add rate of the current device, the ALU ceiling of the search's FFT
 * arithmetic: a kernel of independent fmaf chains (16 per thread, 4 CTAs of 256 threads per SM)
 * is launched once to warm up and then timed `reps` times with CUDA events on the stream; the
 * best rate is written to *fma_per_s (multiply-adds per second; FLOP/s is twice that).  iters is
 * the chain length per thread (>= 1; 50000 runs about 3 ms on a GB300).  Synchronous.  Allocates
 * nothing.  Returns FMBYM_ERR_INVALID_ARG for iters < 1, reps < 1 or a NULL output. */
int fmbym_fp32_fma_rate(void* stream, int iters, int reps, double* fma_per_s);

/* Launch tracing (the CUDA-event timing of Sec. IV-C, per kernel).  With on = 1 the handle records a
 * CUDA event on the launching stream before each kernel launch and after the last launch of each
 * call, so that every kernel's device time is the interval to the next event; on = 0 stops
 * recording.  Either way the recorded intervals are cleared.  Synchronises the device. */
int fmbym_set_tracing(fmbym_handle* h, int on);

/* Sums the recorded intervals per kernel kind: total_ms[k] and count[k] for k < cap (host
 * arrays); *n_kinds (optional) receives the number of kinds.  Waits for the last recorded event. */
int fmbym_trace_summary(fmbym_handle* h, int cap, double* total_ms, long long* count, int* n_kinds);

/* Name of kernel kind k ("" if out of range); static storage. */
const char* fmbym_trace_kind_name(int kind);

/* Number of kernels the handle has launched since it was created. */
long long fmbym_launch_count(const fmbym_handle* h);

/* fmbym_pose without a handle and without any device allocation.  (The paper has no counterpart:
 * this is a deployment convenience.)  Some callers cannot call cudaMalloc: a plug-in inside a host
 * framework that owns every device allocation, or a real-time process whose device memory is
 * fixed at start-up.  This call uses the same kernels as fmbym_pose, but all of its scratch (the
 * size tables, the pair table, counters and every intermediate) lives in one static device array
 * of fmbym_noalloc_capacity() bytes (16 MiB) inside the library, which every device that loads the
 * library reserves until the process exits.
 *   cfg       host pointer to one size configuration, validated as in fmbym_create except that
 *             n_theta must be 128, 256 or 400 (the counts with an FFT plan along angle; other counts
 *             return FMBYM_ERR_UNSUPPORTED_SIZE)
 *   n_pairs   pairs packed back to back: pair p at element offset p * N * N of f, g and c_xy
 *   f, g, pose, c_theta, c_xy  as in fmbym_pose (device, caller-owned; c_theta and c_xy may be NULL)
 * Limit: the whole footprint must fit the array (with the benchmark grids: one 512x512 pair, six
 * 256x256 pairs or 29 128x128 pairs); larger requests return FMBYM_ERR_WORKSPACE and the message
 * gives the bytes needed.  The first call on a device does a one-time set-up (it looks up the array's
 * device address and sets kernel attributes), so make that first call before any stream capture.
 * Every call shares the one array, which keeps the last call's contents.  Each call therefore
 * rebuilds, with one small kernel on the stream, everything it reads before writing it: the size
 * tables, the pair table and the zeroed completion counters; it copies nothing from host memory.
 * Calls that overlap on the GPU (other streams, other host threads) race on the array.  Errors are
 * reported by fmbym_noalloc_last_error(). */
int fmbym_pose_noalloc(void* stream, const fmbym_size_cfg* cfg, int n_pairs, const float* f,
                       const float* g, float* pose, float* c_theta, float* c_xy);

/* Bytes of the static scratch array used by fmbym_pose_noalloc. */
unsigned long long fmbym_noalloc_capacity(void);

/* Text of the last failure of fmbym_pose_noalloc on this host thread ("" if none). */
const char* fmbym_noalloc_last_error(void);

/* ---------------------------------------------------------------------------------------------
 * Radar front end.  The search takes Cartesian scans of side N and cell size delta_xy (Alg. 1),
 * recorded by a rotating FMCW radar (Sec. IV-A, Navtech CTS350-X: 400 azimuths, 3768 range bins
 * of 0.0438 m).  The paper does not state the polar-to-Cartesian conversion; this one is bilinear:
 * azimuth a looks along phi_a = 2 pi a / n_azimuths, from +x (column) toward +y (row); range bin
 * k is centred at (k + 1/2) range_res; pixel (y, x) sits at ((x - n/2) delta_xy, (y - n/2)
 * delta_xy), the sensor at the rotation centre of fmbym_pose; its value interpolates the scan
 * at (phi / (2 pi / n_azimuths), rho / range_res - 1/2), periodic in azimuth, held at range index
 * 0 inside the first bin centre and 0 beyond the last bin centre; the sensor pixel takes azimuth 0.
 *   stream      cudaStream_t or NULL; the call is asynchronous on it
 *   n_scans     number of scans (>= 0; 0 does nothing)
 *   polar       device float32 [n_scans][n_azimuths][n_range], row-major, caller-owned
 *   n_azimuths  >= 1;  n_range >= 1;  range_res > 0 (metres per range bin)
 *   n           side of the Cartesian images (1..16384);  delta_xy > 0 (metres per pixel)
 *   cart        device float32 [n_scans][n][n] out, caller-owned, overwritten
 * Returns FMBYM_ERR_INVALID_ARG for an out-of-range size or a NULL buffer with n_scans > 0, and
 * FMBYM_ERR_CUDA when the launch fails.  Needs no handle and allocates nothing. */
int fmbym_polar_to_cartesian(void* stream, int n_scans, const float* polar, int n_azimuths, int n_range,
                             float range_res, int n, float delta_xy, float* cart);

/* ---------------------------------------------------------------------------------------------
 * Masking network h_alpha (Sec. III-D, Eq. 10-12; layout of Tab. II).  A U-Net over the two-channel
 * image [f, g]: per level two 3x3 convolutions (no bias) each followed by BatchNorm and ReLU,
 * 2x2 max-pool down, bilinear x2 up (align_corners = False) concatenated before the skip
 * ([up, skip]), and a 1x1 convolution to 2 channels with bias and a sigmoid giving the masks
 * m_f, m_g; the outputs are f o m_f and g o m_g (Eq. 11).  Convolutions run on bf16 tensor cores
 * with float32 accumulation; activations after BN + ReLU, pooling and upsampling are bf16;
 * parameters are float32 masters.  BatchNorm uses batch statistics in training (population
 * variance; running mean/var updated with momentum 0.1 and the unbiased variance; eps 1e-5) and the
 * running statistics in evaluation.
 *
 * Flat parameter layout (float32): for every convolution in the order enc0a, enc0b, enc1a, ...,
 * enc{L-1}b, dec{L-2}a, dec{L-2}b, ..., dec0a, dec0b: weight [c_out][c_in][3][3], BN gamma [c_out],
 * BN beta [c_out]; then the head weight [2][c_1] and bias [2].  Running statistics: per convolution
 * in the same order, mean [c_out] then var [c_out].  Gradients use the parameter layout.
 * --------------------------------------------------------------------------------------------- */
typedef struct fmbym_unet fmbym_unet;

/* levels L in [2, 8]; channels c_1..c_L each 8, 16, 32, 64, 128 or 256, non-decreasing, c_1 <= 64
 * (Tab. II is L = 6 with 8, 16, 32, 64, 128, 256); height and width multiples of 8 * 2^(L-1), the
 * width also of 32; max_batch = the largest number of scan pairs per call.  Levels whose images
 * are narrower than 32 pixels, and layers whose weights do not fit in shared memory, run on the
 * flat-GEMM convolution kernels. */
typedef struct fmbym_unet_config {
    int levels;
    int channels[8];
    int height;
    int width;
    int max_batch;
} fmbym_unet_config;

/* Allocates parameters (zero), Adam moments (zero), running statistics (mean 0, var 1), and every
 * activation and gradient buffer for max_batch pairs.  Synchronous. */
int fmbym_unet_create(fmbym_unet** out, const fmbym_unet_config* cfg);
void fmbym_unet_destroy(fmbym_unet* u);
const char* fmbym_unet_last_error(const fmbym_unet* u);

/* Element counts of the parameter and running-statistics arrays, and their device addresses
 * (owned by the handle; the caller may read and write them between calls). */
long long fmbym_unet_param_count(const fmbym_unet* u);
long long fmbym_unet_running_count(const fmbym_unet* u);
float* fmbym_unet_params(fmbym_unet* u);
float* fmbym_unet_grads(fmbym_unet* u);
float* fmbym_unet_running(fmbym_unet* u);

/* Copies parameters and/or running statistics (device float32 in the flat layouts, or NULL to keep
 * the current ones) into the handle; loading parameters also resets the Adam moments.  Store copies
 * the handle's parameters, running statistics and gradients out (each device pointer or NULL). */
int fmbym_unet_load(fmbym_unet* u, void* stream, const float* params, const float* running);
int fmbym_unet_store(fmbym_unet* u, void* stream, float* params, float* running, float* grads);

/* The optimiser state for checkpoint / resume: copies the Adam first and second moments (device
 * float32 [param_count] each, in the parameter layout) out of (store) or into (load) the handle;
 * a NULL pointer skips that moment.  Load after fmbym_unet_load, which resets them. */
int fmbym_unet_store_adam(fmbym_unet* u, void* stream, float* m, float* v);
int fmbym_unet_load_adam(fmbym_unet* u, void* stream, const float* m, const float* v);

/* Inspection: copies one tensor of convolution layer `layer` (0-based, in the parameter order) for
 * the first n pairs of the last call, widened to float32 NHWC, into dst (device): which = 0 the
 * convolution output y (pre-BN), 1 the bf16 activation a (post-ReLU), 2 dL/da, 3 the bf16 dL/dy.
 * Synchronous. */
int fmbym_unet_layer_tensor(fmbym_unet* u, void* stream, int layer, int which, int n, float* dst);

/* Forward (Eq. 10-11) for n pairs: f, g device float32 [n][height][width]; training = 1 uses and
 * updates batch statistics (and keeps the activations for fmbym_unet_backward), 0 uses the running
 * statistics.  f_out, g_out (device float32 like f, or NULL) receive f o m_f and g o m_g; masks
 * (device float32 [n][2][height][width], or NULL) the masks. */
int fmbym_unet_forward(fmbym_unet* u, void* stream, int n, const float* f, const float* g, int training,
                       float* f_out, float* g_out, float* masks);

/* Backward of the last training forward (same n, f and g): given dL/d(f o m_f) and dL/d(g o m_g)
 * (device float32 like f), overwrites the gradient array with dL/dparameters.  Deterministic. */
int fmbym_unet_backward(fmbym_unet* u, void* stream, int n, const float* f, const float* g,
                        const float* df_out, const float* dg_out);

/* One Adam step (the optimiser of Sec. IV-B) on the parameters with the current gradients;
 * step counts from 1 (bias correction). */
int fmbym_unet_adam(fmbym_unet* u, void* stream, float lr, float beta1, float beta2, float eps, int step);

/* Number of kernels the network handle has launched. */
long long fmbym_unet_launch_count(const fmbym_unet* u);

/* Tensor-core path of the flat-GEMM convolutions (the layers that do not fit the tile kernels,
 * e.g. the 16^2 and 8^2 levels of Tab. II's network at 256^2): 0 = mma.sync (the default),
 * 1 = tcgen05 with the accumulator in tensor memory, for layers whose output channels are a
 * multiple of 64 (the others stay on mma.sync).  Results agree to float32 summation order.
 * FMBYM_ERR_INVALID_ARG for another value. */
int fmbym_unet_set_conv_path(fmbym_unet* u, int path);

/* Number of tcgen05 convolution CTAs whose bounded mbarrier wait gave up since creation (their
 * outputs are not written); 0 in a healthy run.  Synchronous.
 * A call of fmbym_unet_forward or fmbym_unet_backward that runs tcgen05 convolutions waits for its
 * stream at the end and returns FMBYM_ERR_TIMEOUT when one of its CTAs gave up: the producer's wait
 * for a shared-memory slot ran out, the CTA issued no further MMA, waited for the MMAs it had issued
 * to finish (a drain of seconds, far beyond any MMA), released its tensor memory and wrote nothing.
 * The handle stays usable. */
long long fmbym_unet_tc_timeouts(fmbym_unet* u);

/* Polls after which a tcgen05 producer's wait for a shared-memory slot gives up (0 restores the
 * default of 2^22, far beyond a healthy wait).  The drain of issued MMAs is not shortened.  A small
 * limit makes waits run out on purpose, so that the FMBYM_ERR_TIMEOUT path can be exercised. */
int fmbym_unet_set_tc_wait_limit(fmbym_unet* u, unsigned polls);

/* Library version as major*10000 + minor*100 + patch. */
int fmbym_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FMBYM_H */
