// Radar front end: a polar (azimuth x range) scan resampled onto the N x N Cartesian grid that the
// pose search takes.  The paper runs Alg. 1 on Cartesian scans of side N and cell size delta_xy,
// taken by a rotating FMCW radar (Sec. IV-A, Navtech CTS350-X); it does not state the conversion.
// The reading implemented here: azimuth a looks along phi_a = 2 pi a / n_az, from +x (column)
// toward +y (row); range bin k is centred at (k + 1/2) range_res; pixel (y, x) sits at
// ((x - N/2) delta_xy, (y - N/2) delta_xy) with the sensor at the rotation centre; its value is
// the bilinear interpolation of the scan at (phi / (2 pi / n_az), rho / range_res - 1/2), periodic
// in azimuth, held at range index 0 inside the first bin centre, 0 beyond the last bin centre;
// the sensor pixel (no bearing) takes azimuth 0.
//
// One thread per output pixel, grid-stride over every pixel of every scan.  Neighbouring pixels
// read neighbouring (azimuth, range) cells, so the gathers of a warp fall on a few rows of the scan.
#include <cmath>
#include <cuda_runtime.h>

#include "../../include/fmbym.h"

namespace {

constexpr int kFrontThreads = 256;

__global__ void __launch_bounds__(kFrontThreads) k_polar_to_cart(const float* __restrict__ polar, long long n_scans,
                                                                 int n_az, int n_range, float range_res, int n,
                                                                 float delta, float* __restrict__ cart) {
    const long long npix = (long long)n * n, total = n_scans * npix;
    const float two_pi = 6.28318530717958647692f;
    const float az_per_rad = (float)n_az / two_pi, inv_res = 1.f / range_res;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const long long q = i / npix;
        const int pix = (int)(i - q * npix), y = pix / n, x = pix - y * n;
        const float X = (float)(x - n / 2) * delta, Y = (float)(y - n / 2) * delta;
        float phi = atan2f(Y, X);
        if (phi < 0.f) phi += two_pi;
        const float fa = phi * az_per_rad;
        const float fk = fmaxf(sqrtf(X * X + Y * Y) * inv_res - 0.5f, 0.f);
        float v = 0.f;
        if (fk <= (float)(n_range - 1)) {
            int a0 = (int)floorf(fa);
            const float ta = fa - (float)a0;
            if (a0 >= n_az) a0 -= n_az;   // phi rounded up to 2 pi
            const int a1 = a0 + 1 == n_az ? 0 : a0 + 1;
            const int k0 = min((int)floorf(fk), n_range - 1), k1 = min(k0 + 1, n_range - 1);
            const float tk = fk - (float)k0;
            const float* P = polar + q * (long long)n_az * n_range;
            const float* r0 = P + (long long)a0 * n_range;
            const float* r1 = P + (long long)a1 * n_range;
            const float v0 = fmaf(tk, __ldg(r0 + k1) - __ldg(r0 + k0), __ldg(r0 + k0));
            const float v1 = fmaf(tk, __ldg(r1 + k1) - __ldg(r1 + k0), __ldg(r1 + k0));
            v = fmaf(ta, v1 - v0, v0);
        }
        cart[i] = v;
    }
}

}  // namespace

extern "C" int fmbym_polar_to_cartesian(void* stream, int n_scans, const float* polar, int n_azimuths, int n_range,
                                        float range_res, int n, float delta_xy, float* cart) {
    // n <= 16384 keeps a scan's pixel index in 32 bits
    if (n_scans < 0 || n_azimuths < 1 || n_range < 1 || n < 1 || n > 16384 || !(range_res > 0.f) || !(delta_xy > 0.f))
        return FMBYM_ERR_INVALID_ARG;
    if (n_scans == 0) return FMBYM_OK;
    if (!polar || !cart) return FMBYM_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FMBYM_ERR_CUDA;
    const long long total = (long long)n_scans * n * n;
    const long long need = (total + kFrontThreads - 1) / kFrontThreads;
    const int blocks = (int)(need < (long long)sms * 8 ? need : (long long)sms * 8);   // 8 CTAs of 256 per SM
    k_polar_to_cart<<<blocks, kFrontThreads, 0, (cudaStream_t)stream>>>(polar, n_scans, n_azimuths, n_range, range_res,
                                                                         n, delta_xy, cart);
    return cudaGetLastError() == cudaSuccess ? FMBYM_OK : FMBYM_ERR_CUDA;
}
