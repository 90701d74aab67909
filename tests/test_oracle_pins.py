"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test checks one oracle step against something other than the oracle itself: a library
routine the step reduces to (numpy's Hann, scipy's bilinear map_coordinates, scipy's 2D
correlation), a closed form worked out by hand, an exact invariance the paper proves (Eq. 6),
or brute force on tiny inputs.  A dropped term, a wrong sign or index, or a transposed operand in
any step fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.ndimage as ndi
import scipy.signal as sig

import oracle as O
from paper_2203_00459_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(1234)


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(1e-300, np.max(np.abs(b))))


def rot90_about_centre(x):
    """Exact +90 deg turn about pixel (N/2, N/2) on the N-periodic grid: out[Y, X] = x[(N-X)%N, Y]."""
    n = x.shape[0]
    Y, X = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    return x[np.mod(n - X, n), Y]


# ---------------------------------------------------------------------------------------------
# paper-printed values
# ---------------------------------------------------------------------------------------------

def test_alg1_defaults_fix_the_angle_span():
    """Alg. 1 prints delta_theta = pi / n_theta: the candidate angles tile a half turn (A9)."""
    gd = json.load(open(os.path.join(GOLDEN, "alg1_defaults.json")))
    nt = gd["n_theta"]
    k = O.lags(nt)
    assert k.size == nt and k[0] == -(nt // 2) and k[-1] == nt - 1 - nt // 2
    span = (k[-1] - k[0] + 1) * (math.pi / nt)
    assert abs(span / math.pi - gd["delta_theta_times_n_theta_over_pi"]) < 1e-15
    for d, n in gd["resolutions"]:
        assert abs(d * n - gd["delta_xy_m"] * gd["n_xy"]) < 0.5  # ~102 m field of view each


# ---------------------------------------------------------------------------------------------
# stage 1 pieces
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("n", [8, 128, 512, 127, 255])   # 127, 255: the paper's odd sizes
def test_hann_is_periodic_hann(n):
    assert rel(O.hann(n), np.hanning(n + 1)[:n]) < 1e-15


def test_band_mask_hand_values():
    m = O.band_mask(16, 2.0, 8.0)
    assert m.shape == (16, 9)
    assert m[0, 0] == 0 and m[0, 1] == 0 and m[1, 1] == 0      # rho = 0, 1, sqrt 2
    assert m[0, 2] == 1 and m[15, 2] == 1 and m[14, 0] == 1      # rho = 2, sqrt 5, 2 (v = -2)
    assert m[8, 0] == 1 and m[0, 8] == 1                          # rho = 8 (inclusive)
    assert m[8, 8] == 0 and m[7, 4] == 0 and m[8, 1] == 0         # rho = 11.3, 8.06, 8.06
    assert m[6, 5] == 1 and m[10, 5] == 1                         # rho = 7.81 (v = 6 and -6)


@pytest.mark.parametrize("n", [16, 15])
def test_spectrum_of_delta_is_a_phase_ramp(n):
    y0, x0 = 3, 5
    x = np.zeros((n, n))
    x[y0, x0] = 1.0
    F = O.spectrum(x, O.make_cfg(n, 8, 4, window=0))
    v = np.arange(n)[:, None]
    u = np.arange(n // 2 + 1)[None, :]
    assert rel(F, np.exp(-2j * np.pi * (v * y0 + u * x0) / n)) < 1e-13


@pytest.mark.parametrize("n,window", [(12, 1), (15, 1), (8, 0)])
def test_spectrum_matches_the_direct_dft_sum(n, window):
    """Eq. 4 written out: F[v, u] = sum_y sum_x w[y] w[x] f[y, x] exp(-2 pi i (v y + u x) / N) for
    u <= N/2, by plain loops on a tiny scan."""
    x = RNG.random((n, n))
    w = O.hann(n) if window else np.ones(n)
    ref = np.zeros((n, n // 2 + 1), complex)
    for v in range(n):
        for u in range(n // 2 + 1):
            acc = 0j
            for yy in range(n):
                for xx in range(n):
                    acc += w[yy] * w[xx] * x[yy, xx] * complex(math.cos(-2 * math.pi * (v * yy + u * xx) / n),
                                                               math.sin(-2 * math.pi * (v * yy + u * xx) / n))
            ref[v, u] = acc
    assert rel(O.spectrum(x, O.make_cfg(n, 8, 4, window=window)), ref) < 1e-12


def test_spectrum_of_plane_wave():
    n, u0, v0 = 32, 3, 5
    Y, X = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    x = np.cos(2 * np.pi * (u0 * X + v0 * Y) / n)
    a = O.magnitude(O.spectrum(x, O.make_cfg(n, 8, 4, window=0)),
                    O.make_cfg(n, 8, 4, window=0, band_lo=0, band_hi=1e9))
    expect = np.zeros_like(a)
    expect[v0, u0] = n * n / 2
    assert rel(a, expect) < 1e-12


def test_windowed_spectrum_of_constant():
    """Periodic Hann: sum w = N/2 and its DFT at u = 1 is -N/4, so F[0,0] = N^2/4,
    F[0,1] = F[1,0] = -N^2/8, F[1,1] = N^2/16 and F vanishes beyond |u|, |v| > 1."""
    n = 16
    F = O.spectrum(np.ones((n, n)), O.make_cfg(n, 8, 4, window=1))
    expect = np.zeros_like(F)
    expect[0, 0] = n * n / 4
    expect[0, 1] = expect[1, 0] = expect[n - 1, 0] = -n * n / 8
    expect[1, 1] = expect[n - 1, 1] = n * n / 16
    assert rel(F, expect) < 1e-13


def test_magnitude_is_translation_invariant():
    """Eq. 6: |F| does not depend on the translation (circular shift, no window)."""
    n = 64
    x = RNG.random((n, n))
    cfg = O.make_cfg(n, 32, 16, window=0)
    a1 = O.magnitude(O.spectrum(x, cfg), cfg)
    a2 = O.magnitude(O.spectrum(np.roll(x, (7, -11), axis=(0, 1)), cfg), cfg)
    assert rel(a2, a1) < 1e-12


@pytest.mark.parametrize("n,nt,nr", [(32, 16, 8), (64, 50, 32), (128, 128, 64), (33, 20, 8), (127, 733, 16)])
def test_cart2pol_matches_scipy_bilinear_on_full_periodic_spectrum(n, nt, nr):
    x = RNG.random((n, n))
    cfg = O.make_cfg(n, nt, nr, window=1, band_lo=0, band_hi=1e9)
    a = O.magnitude(O.spectrum(x, cfg), cfg)
    w = np.hanning(n + 1)[:n]
    full = np.abs(np.fft.fft2(x * w[:, None] * w[None, :]))
    alpha = np.arange(nt) * np.pi / nt
    rho = np.arange(nr) * (n / 2) / nr
    u = rho[None, :] * np.cos(alpha)[:, None]
    v = rho[None, :] * np.sin(alpha)[:, None]
    ref = ndi.map_coordinates(full, [v.ravel(), u.ravel()], order=1, mode="grid-wrap").reshape(nt, nr)
    assert rel(O.cart2pol(a, cfg), ref) < 1e-12


def test_cart2pol_reproduces_a_bilinear_spectrum():
    """a(v, u) = 3 + u v / 4 is bilinear and centrosymmetric, so Cart2Pol returns it exactly:
    3 + rho^2 cos(alpha) sin(alpha) / 4."""
    n, nt, nr = 64, 40, 16
    v = np.arange(n)
    vs = np.where(v <= n // 2, v, v - n)[:, None]
    u = np.arange(n // 2 + 1)[None, :]
    a = 3.0 + 0.25 * vs * u
    cfg = O.make_cfg(n, nt, nr)
    alpha = np.arange(nt) * np.pi / nt
    rho = np.arange(nr) * (n / 2) / nr
    expect = 3.0 + 0.25 * (rho ** 2)[None, :] * (np.cos(alpha) * np.sin(alpha))[:, None]
    assert rel(O.cart2pol(a, cfg), expect) < 1e-13


def test_quarter_turn_shifts_polar_spectrum_by_half_the_angle_bins():
    """A 90 deg turn permutes the grid exactly, so the polar magnitudes move by n_theta/2 rows
    and the rotation score peaks at lag -n_theta/2 (same bin as +n_theta/2 on a half turn)."""
    n, nt, nr = 64, 48, 24
    x = RNG.random((n, n))
    cfg = O.make_cfg(n, nt, nr)
    p1 = O.cart2pol(O.magnitude(O.spectrum(x, cfg), cfg), cfg)
    p2 = O.cart2pol(O.magnitude(O.spectrum(rot90_about_centre(x), cfg), cfg), cfg)
    assert rel(p2, np.roll(p1, nt // 2, axis=0)) < 1e-12
    c = O.angle_scores(p1, p2)
    assert int(np.argmax(c)) == 0


@pytest.mark.parametrize("nt,nr", [(30, 7), (733, 5)])   # 733: Alg. 1's n_theta, odd and prime
def test_angle_scores_match_fft_correlation(nt, nr):
    af = RNG.random((nt, nr))
    ag = RNG.random((nt, nr))
    c = O.angle_scores(af, ag)
    viafft = np.real(np.fft.ifft(np.conj(np.fft.fft(af, axis=0)) * np.fft.fft(ag, axis=0), axis=0)).sum(1)
    assert rel(c, viafft[np.mod(O.lags(nt), nt)]) < 1e-13


@pytest.mark.parametrize("nt", [40, 41])
def test_angle_scores_peak_at_the_roll(nt):
    af = RNG.random((nt, 9))
    for k0 in (-(nt // 2), -3, 0, 5, nt - 1 - nt // 2):
        c = O.angle_scores(af, np.roll(af, k0, axis=0))
        i = int(np.argmax(c))
        assert O.lags(nt)[i] == k0
        assert abs(c[i] - np.sum(af * af)) < 1e-12 * c[i]


def test_soft_argmax_two_scores_closed_form():
    """Two candidates with scores a < b z-score to (-1, 1), so p = (1, e^{2/T}) / (1 + e^{2/T})."""
    for T in (0.5, 1.0, 2.0):
        p = O.soft_argmax(np.array([3.0, 7.5]), T, 0)
        e = math.exp(2.0 / T)
        assert rel(p, np.array([1.0, e]) / (1.0 + e)) < 1e-15
    p = O.soft_argmax(np.array([0.0, math.log(3.0)]), 1.0, 1)     # raw scores: (1, 3)/4
    assert rel(p, np.array([0.25, 0.75])) < 1e-15


def test_soft_argmax_scale_invariance_and_hard_limit():
    """softmax(zscore(c) / T) ignores affine rescaling of c, and as T -> 0 it tends to the one-hot
    argmax: the mass off the top score is at most (n - 1) exp(-(z_1 - z_2) / T)."""
    c = np.random.default_rng(4).random(50)
    p = O.soft_argmax(c, 1.0, 0)
    assert rel(O.soft_argmax(7.0 * c + 3.0, 1.0, 0), p) < 1e-12
    T = 1e-4
    hard = O.soft_argmax(c, T, 0)
    assert int(np.argmax(hard)) == int(np.argmax(c))
    z = np.sort((c - c.mean()) / c.std())[::-1]
    assert 1.0 - hard.max() <= 49 * np.exp(-(z[0] - z[1]) / T) + 1e-15


# ---------------------------------------------------------------------------------------------
# stage 2 pieces
# ---------------------------------------------------------------------------------------------

def test_rotate_zero_is_identity():
    x = RNG.random((32, 32))
    assert rel(O.rotate(x, 0.0), x) < 1e-15


@pytest.mark.parametrize("n", [32, 31])
def test_rotate_quarter_turn_is_the_index_permutation(n):
    x = RNG.random((n, n))
    r = O.rotate(x, np.pi / 2)
    expect = rot90_about_centre(x)
    expect[:, 0] = 0.0      # X = 0 samples row N, outside the scan
    assert np.max(np.abs(r - expect)) < 1e-12


@pytest.mark.parametrize("theta", [0.3, -0.07, 2.5])
def test_rotate_matches_scipy_bilinear_with_zero_fill(theta):
    n = 48
    x = RNG.random((n, n))
    c = n / 2
    Y, X = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float), indexing="ij")
    px = c + math.cos(theta) * (X - c) + math.sin(theta) * (Y - c)
    py = c - math.sin(theta) * (X - c) + math.cos(theta) * (Y - c)
    ref = ndi.map_coordinates(x, [py.ravel(), px.ravel()], order=1, mode="grid-constant", cval=0.0)
    assert rel(O.rotate(x, theta), ref.reshape(n, n)) < 1e-12


@pytest.mark.parametrize("n", [8, 16, 24, 9, 15])
def test_xcorr2d_matches_scipy_correlate(n):
    fr = RNG.random((n, n))
    g = RNG.random((n, n))
    full = sig.correlate2d(g, fr, mode="full")          # full[s + N - 1] = sum_x g(x + s) fr(x)
    s = O.lags(n) + n - 1
    assert rel(O.xcorr2d(fr, g, 0), full[np.ix_(s, s)]) < 1e-12


def test_xcorr2d_transform_routes_equal_the_direct_sum():
    """Both routes of the correlation theorem (direct DFT sums, numpy FFT) give the definition's
    value at single lags, the +-N/2 edges among them."""
    n = 40
    fr = RNG.random((n, n))
    g = RNG.random((n, n))
    for pad in (0, 1):
        for route in ("direct", "fft"):
            c = O.xcorr2d(fr, g, pad, route)
            for sy, sx in [(-20, -20), (-20, 19), (0, 0), (7, -3), (19, 19), (-1, 12)]:
                d = O.xcorr2d_direct(fr, g, sy, sx, pad)
                assert abs(c[sy + n // 2, sx + n // 2] - d) < 1e-11 * abs(d), (pad, route, sy, sx)


@pytest.mark.parametrize("n", [16, 17])
def test_xcorr2d_brute_is_the_definition(n):
    """The brute-force surface against scipy's correlate2d (zero outside the scan) and against the
    sum with np.roll (N-periodic), over every lag."""
    fr = RNG.random((n, n))
    g = RNG.random((n, n))
    full = sig.correlate2d(g, fr, mode="full")
    s = O.lags(n) + n - 1
    assert rel(O.xcorr2d_brute(fr, g, 0), full[np.ix_(s, s)]) < 1e-13
    ref = np.array([[np.sum(fr * np.roll(g, (-sy, -sx), axis=(0, 1))) for sx in O.lags(n)] for sy in O.lags(n)])
    assert rel(O.xcorr2d_brute(fr, g, 1), ref) < 1e-13
    lag_list = [(int(O.lags(n)[0]), int(O.lags(n)[-1])), (0, 0), (3, -2)]
    vals = O.xcorr2d_brute(fr, g, 0, lag_list)
    for (sy, sx), v in zip(lag_list, vals):
        assert v == full[sy + n - 1, sx + n - 1] or abs(v - full[sy + n - 1, sx + n - 1]) < 1e-12 * abs(v)


def test_dft_matrix_is_the_unitary_root_table():
    """W[k, j] = exp(-2 pi i k j / n): symmetric, unit modulus, W W^H = n I, row 1 the first root."""
    for n in (12, 127, 768):
        W = O.dft_matrix(n)
        assert np.max(np.abs(W - W.T)) == 0.0
        assert np.max(np.abs(np.abs(W) - 1.0)) < 1e-15
        assert np.max(np.abs(W @ np.conj(W).T - n * np.eye(n))) < 1e-10 * n
        assert abs(W[1, 1] - complex(math.cos(2 * math.pi / n), -math.sin(2 * math.pi / n))) < 1e-16
        rows = [0, 5, n - 1]
        assert np.array_equal(O.dft_matrix(n, rows), W[rows])
        assert np.array_equal(O.dft_matrix(n, rows, +1), np.conj(W[rows]))


@pytest.mark.parametrize("n,nt,nr", [(128, 128, 64), (127, 733, 16), (64, 50, 32)])
def test_direct_sum_route_agrees_with_the_fft_route(n, nt, nr):
    """Every DFT of the search by its direct sum against numpy's FFT on the same sums: spectra,
    the padded correlation and both adjoints, and the whole forward and backward search."""
    f, g = RNG.random((n, n)), RNG.random((n, n))
    c = O.make_cfg(n, nt, nr)
    cf = dict(c, route="fft")
    assert rel(O.spectrum(f, c), O.spectrum(f, cf)) < 1e-13
    dF = RNG.standard_normal((n, n // 2 + 1)) + 1j * RNG.standard_normal((n, n // 2 + 1))
    assert rel(O.spectrum_backward(dF, c), O.spectrum_backward(dF, cf)) < 1e-13
    dc = RNG.standard_normal((n, n))
    for pad in (0, 1):
        assert rel(O.xcorr2d(f, g, pad), O.xcorr2d(f, g, pad, "fft")) < 1e-13
        a = O.xcorr2d_backward(f, g, dc, pad)
        b = O.xcorr2d_backward(f, g, dc, pad, "fft")
        assert rel(a[0], b[0]) < 1e-13 and rel(a[1], b[1]) < 1e-13
    r, rf = O.pose(f, g, c), O.pose(f, g, cf)
    for k in ("theta", "tx", "ty"):
        assert abs(r[k] - rf[k]) < 1e-12
    assert rel(r["c_xy"], rf["c_xy"]) < 1e-13 and rel(r["c_theta"], rf["c_theta"]) < 1e-13
    dp = np.array([0.7, -0.2, 0.4])
    a, b = O.pose_backward(f, g, c, dp), O.pose_backward(f, g, cf, dp)
    assert rel(a[0], b[0]) < 1e-11 and rel(a[1], b[1]) < 1e-11


def test_brute_force_scores_of_a_benchmark_pair_at_128():
    """The padded correlation of a 128^2 benchmark pair, every one of its 128^2 lags by the sum of
    the definition, against the direct-DFT route that pose() takes (and the circular variant)."""
    from paper_2203_00459_gb300 import synth
    f, g, _ = synth.make_batch("single128", pairs=1)
    fr = O.rotate(f[0], 0.05)
    for pad in (0, 1):
        assert rel(O.xcorr2d_brute(fr, g[0], pad), O.xcorr2d(fr, g[0], pad)) < 1e-13


@pytest.mark.parametrize("n", [64, 63])
def test_circular_integer_shift_peaks_at_the_shift(n):
    f = RNG.random((n, n))
    for ty, tx in [(3, -5), (-4, 4), (0, 0), (-(n // 2), n - 1 - n // 2)]:
        c = O.xcorr2d(f, np.roll(f, (ty, tx), axis=(0, 1)), 1)
        iy, ix = np.unravel_index(np.argmax(c), c.shape)
        assert (iy - n // 2, ix - n // 2) == (ty, tx)
        assert abs(c[iy, ix] - np.sum(f * f)) < 1e-12 * c[iy, ix]


def test_zero_padded_shift_of_points_peaks_exactly():
    n = 32
    f = np.zeros((n, n))
    pts = [(5, 7, 2.0), (20, 11, 3.0), (12, 25, 1.5)]
    for y, x, a in pts:
        f[y, x] = a
    ty, tx = -4, 6
    g = np.zeros_like(f)
    for y, x, a in pts:
        g[y + ty, x + tx] = a
    c = O.xcorr2d(f, g, 0)
    iy, ix = np.unravel_index(np.argmax(c), c.shape)
    assert (iy - n // 2, ix - n // 2) == (ty, tx)
    assert abs(c[iy, ix] - sum(a * a for _, _, a in pts)) < 1e-12


# ---------------------------------------------------------------------------------------------
# the whole search
# ---------------------------------------------------------------------------------------------

def test_identical_scans_give_zero_bins():
    f, _, _ = synth.make_batch("single128", pairs=1)
    cfg = O.make_cfg(128, 128, 64)
    r = O.pose(f[0], f[0], cfg)
    assert int(np.argmax(r["c_theta"])) == 64
    assert np.unravel_index(np.argmax(r["c_xy"]), r["c_xy"].shape) == (64, 64)
    # the angle score of a scan with itself is symmetric in the lag (bar the unpaired -n/2 lag)
    ct = r["c_theta"]
    assert rel(ct[1:], ct[1:][::-1]) < 1e-12
    # so is the translation score of an unrotated scan with itself
    cxy = O.xcorr2d(f[0], f[0], 0)
    assert rel(cxy[1:, 1:], cxy[1:, 1:][::-1, ::-1]) < 1e-12


def test_grid_aligned_workload_recovers_its_bins():
    """single128 pairs rotate by k * 360/128 deg = 2k bins of pi/128 and shift by integers: the
    angle score peaks at lag 2k, and at the true angle the translation score peaks at t."""
    f, g, gt = synth.make_batch("single128", pairs=6)
    cfg = O.make_cfg(128, 128, 64)
    for i in range(6):
        r = O.pose(f[i], g[i], cfg)
        k = int(np.argmax(r["c_theta"])) - 64
        assert k == int(round(gt[i, 0] / (np.pi / 128)))
        c = O.xcorr2d(O.rotate(f[i], gt[i, 0]), g[i], 0)
        iy, ix = np.unravel_index(np.argmax(c), c.shape)
        assert (ix - 64, iy - 64) == (int(gt[i, 1]), int(gt[i, 2]))


def test_pose_is_invariant_to_positive_scan_scaling():
    f, g, _ = synth.make_batch("single128", pairs=1)
    cfg = O.make_cfg(128, 128, 64)
    f64, g64 = f[0].astype(np.float64), g[0].astype(np.float64)
    a = O.pose(f64, g64, cfg)
    b = O.pose(3.0 * f64, 0.25 * g64, cfg)
    for k in ("theta", "tx", "ty"):
        assert abs(a[k] - b[k]) < 1e-10


# ---------------------------------------------------------------------------------------------
# adjoints: dot-product identities per linear stage, central differences end to end
# ---------------------------------------------------------------------------------------------

def test_adjoint_dot_products():
    n, nt, nr = 32, 24, 12
    cfg = O.make_cfg(n, nt, nr)
    x = RNG.random((n, n))
    y = RNG.random((n, n))
    # rotate at fixed theta
    dx, _ = O.rotate_backward(np.zeros((n, n)), 0.37, y)
    assert abs(np.sum(O.rotate(x, 0.37) * y) - np.sum(x * dx)) < 1e-11
    # cart2pol
    a = RNG.random((n, n // 2 + 1))
    dp = RNG.random((nt, nr))
    assert abs(np.sum(O.cart2pol(a, cfg) * dp) - np.sum(a * O.cart2pol_backward(dp, cfg))) < 1e-11
    # angle correlation, linear in each operand
    af, ag, dc = RNG.random((nt, nr)), RNG.random((nt, nr)), RNG.random(nt)
    daf, dag = O.angle_scores_backward(af, ag, dc)
    lhs = np.dot(O.angle_scores(af, ag), dc)
    assert abs(lhs - np.sum(af * daf)) < 1e-10 * lhs and abs(lhs - np.sum(ag * dag)) < 1e-10 * lhs
    # padded 2D correlation, linear in each operand
    for pad in (0, 1):
        dcx = RNG.random((n, n))
        dfr, dg = O.xcorr2d_backward(x, y, dcx, pad)
        lhs = np.sum(O.xcorr2d(x, y, pad) * dcx)
        assert abs(lhs - np.sum(x * dfr)) < 1e-10 * lhs and abs(lhs - np.sum(y * dg)) < 1e-10 * lhs
    # windowed half-plane DFT (real inner product on (Re, Im))
    dF = RNG.random((n, n // 2 + 1)) + 1j * RNG.random((n, n // 2 + 1))
    F = O.spectrum(x, cfg)
    lhs = np.sum(F.real * dF.real + F.imag * dF.imag)
    assert abs(lhs - np.sum(x * O.spectrum_backward(dF, cfg))) < 1e-10 * abs(lhs)


@pytest.mark.parametrize("score_norm,n", [(0, 32), (1, 32), (0, 33)])   # 33: an odd side (no Nyquist column)
def test_pose_gradient_matches_central_differences(score_norm, n):
    spec = dict(n=n, n_points=10, n_walls=2, n_theta=32, n_r=16, pairs=1, seed_id=9,
                theta_deg=8.0, t_px=3.0)
    f, g, _ = synth.make_batch("custom", spec=spec)
    f = f[0].astype(np.float64)
    g = g[0].astype(np.float64)
    if score_norm == 1:          # raw scores: keep the softmax soft by scaling the scans down
        f, g = f * 0.02, g * 0.02
        cfg = O.make_cfg(n, 32, 16, temp_theta=2.0, temp_xy=2.0, score_norm=1)
    else:
        cfg = O.make_cfg(n, 32, 16, temp_theta=0.5, temp_xy=0.5)
    dp = np.array([0.7, -0.3, 0.45])

    def loss(a, b):
        r = O.pose(a, b, cfg)
        return dp[0] * r["theta"] + dp[1] * r["tx"] + dp[2] * r["ty"]

    df, dg, _ = O.pose_backward(f, g, cfg, dp)
    rng = np.random.default_rng(7)
    h = 1e-4
    for which, grad in (("f", df), ("g", dg)):
        for _ in range(5):
            y, x = rng.integers(0, n, 2)
            a, b = f.copy(), g.copy()
            (a if which == "f" else b)[y, x] += h
            lp = loss(a, b)
            (a if which == "f" else b)[y, x] -= 2 * h
            lm = loss(a, b)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grad[y, x]) <= 1e-6 * np.max(np.abs(grad)) + 1e-6 * abs(fd)


def test_generator_is_deterministic_and_pairs_differ():
    f1, g1, p1 = synth.make_batch("batch256", pairs=2)
    f2, g2, p2 = synth.make_batch("batch256", pairs=2)
    assert np.array_equal(f1, f2) and np.array_equal(g1, g2) and np.array_equal(p1, p2)
    assert not np.array_equal(f1[0], f1[1])
    f3, _, p3 = synth.make_batch("batch256", pairs=1, start=1)
    assert np.array_equal(f3[0], f1[1]) and np.array_equal(p3[0], p1[1])


def test_exhaustive_search_recovers_a_grid_rotation_and_circular_shift():
    # g is f turned by a quarter turn (an exact index permutation) and circularly shifted by an
    # integer t: among headings 0, 45, ..., 315 degrees the exhaustive rotate-then-correlate
    # search must pick 90 degrees, and its translation is t (a sharp soft-argmax, circular lags)
    rng = np.random.default_rng(11)
    n = 32
    f = rng.random((n, n))
    fr = O.rotate(f, np.pi / 2)
    g = np.roll(fr, (-5, 3), axis=(0, 1))
    cfg = O.make_cfg(n, 32, 16, temp_xy=0.01, pad_mode=1)
    angles = np.arange(-4, 4) * (np.pi / 4)
    r = O.pose_exhaustive(f, g, cfg, angles)
    assert r["k"] == 6 and r["theta"] == np.pi / 2
    assert abs(r["tx"] - 3) < 1e-6 and abs(r["ty"] + 5) < 1e-6
    # the winning peak is the energy sum of the rotated source (Cauchy-Schwarz bound attained)
    assert abs(r["peaks"][6] - np.sum(fr * fr)) <= 1e-9 * np.sum(fr * fr)
    assert np.all(r["peaks"][np.arange(8) != 6] < r["peaks"][6])


def test_exhaustive_search_of_identical_scans_is_the_identity():
    f, _, _ = synth.make_batch("single128", pairs=1, start=3)
    cfg = O.make_cfg(128, 128, 64)
    r = O.pose_exhaustive(f[0], f[0], cfg, np.radians(np.arange(-10, 11)))
    assert r["theta"] == 0.0
    # (the unpaired -N/2 lag row and column leave a bias far below 1e-4 px)
    assert abs(r["tx"]) < 1e-4 and abs(r["ty"]) < 1e-4


def test_marginal_angle_score_is_the_radial_mean_of_the_2d_circular_correlation():
    # Alg. 1 literally: 2D correlation of the wrap-padded (circular) polar arrays, then the mean
    # over the radial lag dimension -- computed here by brute force over both lags
    rng = np.random.default_rng(21)
    nt, nr = 12, 5
    af, ag = rng.random((nt, nr)), rng.random((nt, nr))
    c2 = np.zeros((nt, nr))
    for k in range(nt):
        for ll in range(nr):
            c2[k, ll] = np.sum(af * np.roll(np.roll(ag, -k, axis=0), -ll, axis=1))
    want = np.array([c2[k % nt].mean() for k in O.lags(nt)])
    got = O.angle_scores_marginal(af, ag)
    assert np.allclose(got, want, rtol=1e-12, atol=0)
    # it differs from Eq. 7's radial lag 0 in general
    assert not np.allclose(got, O.angle_scores(af, ag) / nr)


def test_marginal_angle_score_adjoint_dot_product():
    rng = np.random.default_rng(22)
    af, ag = rng.random((16, 6)), rng.random((16, 6))
    dc = rng.standard_normal(16)
    daf, dag = O.angle_scores_marginal_backward(af, ag, dc)
    u, v = rng.standard_normal(af.shape), rng.standard_normal(ag.shape)
    h = 1e-6
    lhs = (np.dot(dc, O.angle_scores_marginal(af + h * u, ag + h * v))
           - np.dot(dc, O.angle_scores_marginal(af - h * u, ag - h * v))) / (2 * h)
    assert abs(lhs - (np.sum(daf * u) + np.sum(dag * v))) <= 1e-7 * max(1.0, abs(lhs))


def test_pose_gradient_matches_central_differences_marginal_score():
    f, g, _ = synth.make_batch("single128", pairs=1, start=5)
    cfg = O.make_cfg(128, 128, 64, angle_score=1)
    dpose = np.array([0.6, -0.3, 0.8])
    df, dg, _ = O.pose_backward(f[0], g[0], cfg, dpose)
    rng = np.random.default_rng(9)
    h = 1e-4
    for _ in range(4):
        y, x = rng.integers(8, 120, 2)
        for img, grad, which in ((f[0].astype(np.float64), df, 0), (g[0].astype(np.float64), dg, 1)):
            e = np.zeros_like(img)
            e[y, x] = h
            a = (img + e, g[0]) if which == 0 else (f[0], img + e)
            b = (img - e, g[0]) if which == 0 else (f[0], img - e)
            ra, rb = O.pose(*a, cfg), O.pose(*b, cfg)
            fd = sum(dpose[i] * (ra[k] - rb[k]) / (2 * h) for i, k in enumerate(("theta", "tx", "ty")))
            assert abs(fd - grad[y, x]) <= 1e-6 * max(1.0, np.max(np.abs(grad))), (which, y, x, fd, grad[y, x])


@pytest.mark.parametrize("deg,flip", [(170.0, True), (-125.0, True), (12.0, False)])
def test_full_circle_heading(deg, flip):
    # a scene turned by more than a quarter turn: the half-circle search reports the heading less
    # half a turn; the full-circle search finds it, with the translation
    n = 128
    th, tx, ty = math.radians(deg), 3.0, -2.0
    f, g = synth.make_pair(n, 60, 8, th, tx, ty, seed=777, index=int(deg) + 500)
    # a sharp angle soft-argmax (T = 0.2 on z-scores) so that stage 1 resolves large headings
    half = O.pose(f, g, O.make_cfg(n, 128, 64, temp_theta=0.2))
    full = O.pose(f, g, O.make_cfg(n, 128, 64, temp_theta=0.2, full_circle=1))
    wrap = lambda a: (a + math.pi) % (2 * math.pi) - math.pi
    assert abs(wrap(full["theta"] - th)) < math.radians(1.5)
    assert -math.pi < full["theta"] <= math.pi       # the flipped heading is reported in (-pi, pi]
    assert abs(full["theta"] - th) < math.radians(1.5) or abs(th) > math.pi - math.radians(1.5)
    assert abs(full["tx"] - tx) < 0.5 and abs(full["ty"] - ty) < 0.5
    assert abs(wrap(half["theta"] - th + (math.pi if flip else 0.0))) < math.radians(1.5)
    if not flip:
        assert full["theta"] == half["theta"] and full["tx"] == half["tx"]


def test_pose_gradient_matches_central_differences_full_circle():
    n = 128
    f, g = synth.make_pair(n, 40, 6, math.radians(160.0), 2.0, 1.0, seed=778, index=1)
    cfg = O.make_cfg(n, 128, 64, temp_theta=0.2, full_circle=1)
    dpose = np.array([0.5, 0.7, -0.4])
    assert abs(O.pose(f, g, cfg)["theta"]) > math.pi / 2      # the flipped branch
    df, dg, _ = O.pose_backward(f, g, cfg, dpose)
    rng = np.random.default_rng(10)
    h = 1e-4
    for _ in range(3):
        y, x = rng.integers(20, 108, 2)
        for which in (0, 1):
            img = (f if which == 0 else g).astype(np.float64)
            e = np.zeros_like(img)
            e[y, x] = h
            a = (img + e, g) if which == 0 else (f, img + e)
            b = (img - e, g) if which == 0 else (f, img - e)
            ra, rb = O.pose(*a, cfg), O.pose(*b, cfg)
            fd = sum(dpose[i] * (ra[k] - rb[k]) / (2 * h) for i, k in enumerate(("theta", "tx", "ty")))
            grad = (df if which == 0 else dg)
            assert abs(fd - grad[y, x]) <= 1e-6 * max(1.0, np.max(np.abs(grad))), (which, y, x, fd, grad[y, x])


@pytest.mark.parametrize("deg,tx,ty", [(20.0, 6.0, -3.0), (-14.0, -4.0, 5.0)])
def test_rotate_target_g_recovers_the_pose(deg, tx, ty):
    # Alg. 1's own stage 2 (g turned back by theta, then t = R(theta) t'): on a scene with a known
    # pose the scores peak at t' = R(-theta) t -- more than a pixel away from t at these angles, so
    # a wrong sign in either rotation shows -- and the reported translation is t
    n = 128
    th = math.radians(deg)
    f, g = synth.make_pair(n, 60, 8, th, tx, ty, seed=781, index=int(deg) + 900)
    lit = O.pose(f, g, O.make_cfg(n, 128, 64, temp_theta=0.2, rotate_target=1))
    src = O.pose(f, g, O.make_cfg(n, 128, 64, temp_theta=0.2))
    assert lit["theta"] == src["theta"]                          # stage 1 is the same
    assert abs(lit["theta"] - th) < math.radians(1.0)
    ct, st = math.cos(th), math.sin(th)
    tp = (ct * tx + st * ty, -st * tx + ct * ty)
    assert math.hypot(tp[0] - tx, tp[1] - ty) > 1.0
    assert abs(lit["tpx"] - tp[0]) < 0.5 and abs(lit["tpy"] - tp[1]) < 0.5
    assert abs(lit["tx"] - tx) < 0.5 and abs(lit["ty"] - ty) < 0.5
    with pytest.raises(ValueError):
        O.make_cfg(n, 128, 64, rotate_target=1, full_circle=1)


def test_pose_gradient_matches_central_differences_rotate_target_g():
    n = 128
    f, g = synth.make_pair(n, 40, 6, math.radians(15.0), 3.0, -2.0, seed=782, index=2)
    cfg = O.make_cfg(n, 128, 64, temp_theta=0.5, rotate_target=1)
    dpose = np.array([0.4, -0.6, 0.9])
    df, dg, _ = O.pose_backward(f, g, cfg, dpose)
    rng = np.random.default_rng(11)
    h = 1e-4
    for _ in range(3):
        y, x = rng.integers(20, 108, 2)
        for which in (0, 1):
            img = (f if which == 0 else g).astype(np.float64)
            e = np.zeros_like(img)
            e[y, x] = h
            a = (img + e, g) if which == 0 else (f, img + e)
            b = (img - e, g) if which == 0 else (f, img - e)
            ra, rb = O.pose(*a, cfg), O.pose(*b, cfg)
            fd = sum(dpose[i] * (ra[k] - rb[k]) / (2 * h) for i, k in enumerate(("theta", "tx", "ty")))
            grad = (df if which == 0 else dg)
            assert abs(fd - grad[y, x]) <= 1e-6 * max(1.0, np.max(np.abs(grad))), (which, y, x, fd, grad[y, x])


@pytest.mark.parametrize("n", [127, 255])
def test_paper_odd_sizes_recover_a_known_pose(n):
    """Alg. 1 at the paper's own odd scan sizes and n_theta = 733 (Sec. IV-B, Alg. 1): a pair
    rendered with a continuous pose comes back within 0.05 deg and 0.05 px."""
    f, g = synth.make_pair(n, n * n // 300, n // 16, math.radians(10.0), 3.0, -2.0, seed=77, index=0)
    r = O.pose(f, g, O.make_cfg(n, 733, n // 2, temp_theta=0.2))
    assert abs(math.degrees(r["theta"]) - 10.0) < 0.05, r["theta"]
    assert abs(r["tx"] - 3.0) < 0.05 and abs(r["ty"] + 2.0) < 0.05, (r["tx"], r["ty"])
