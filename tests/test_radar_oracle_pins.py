"""Pins of the radar front-end oracle (polar scan -> Cartesian grid, reading A16) against closed
forms, an exact symmetry and scipy's bilinear interpolation."""
import numpy as np
import pytest

from oracle import radar_oracle as R

RNG = np.random.default_rng(20220302)
N, DXY, NAZ, NRANGE, RES = 64, 0.4, 400, 200, 0.0438 * 4   # a Navtech-like scan, coarser range


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(1e-300, np.max(np.abs(b))))


def test_constant_scan_fills_the_disc_of_the_last_bin_centre():
    c = R.polar_to_cartesian(np.full((NAZ, NRANGE), 3.0), N, DXY, RES)
    X, Y = R.cartesian_points(N, DXY)
    inside = np.hypot(X, Y) <= (NRANGE - 0.5) * RES
    assert np.all(c[inside] == 3.0) and np.all(c[~inside] == 0.0)
    small = R.polar_to_cartesian(np.full((NAZ, 20), 3.0), N, DXY, RES)   # 20 bins: 3.4 m
    X, Y = R.cartesian_points(N, DXY)
    assert np.all(small[np.hypot(X, Y) > 19.5 * RES] == 0.0) and small[N // 2, N // 2] == 3.0


def test_scan_linear_in_range_gives_the_radius():
    """Bilinear interpolation reproduces a linear function: value = rho / res - 1/2, held at 0."""
    p = np.tile(np.arange(NRANGE, dtype=np.float64), (NAZ, 1))
    c = R.polar_to_cartesian(p, N, DXY, RES)
    X, Y = R.cartesian_points(N, DXY)
    expect = np.maximum(np.hypot(X, Y) / RES - 0.5, 0.0)
    assert np.max(np.abs(c - expect)) < 1e-10


def test_scan_linear_in_azimuth_gives_the_bearing():
    """value = phi / (2 pi / n_az), phi from +x toward +y, away from the seam at phi -> 2 pi."""
    p = np.tile(np.arange(NAZ, dtype=np.float64)[:, None], (1, NRANGE))
    c = R.polar_to_cartesian(p, N, DXY, RES)
    X, Y = R.cartesian_points(N, DXY)
    phi = np.mod(np.arctan2(Y, X), 2 * np.pi)
    ok = phi < (NAZ - 1) * 2 * np.pi / NAZ
    assert np.max(np.abs(c[ok] - phi[ok] * NAZ / (2 * np.pi))) < 1e-9
    assert abs(c[N // 2, N - 1] - 0.0) < 1e-12                 # +x: azimuth 0
    assert abs(c[N - 1, N // 2] - NAZ / 4) < 1e-9               # +y: a quarter turn


def test_quarter_turn_of_the_scan_turns_the_image():
    """Rolling the azimuths by n_az/4 turns the Cartesian image by +90 deg about the sensor:
    C'[x, N - y] = C[y, x]."""
    p = RNG.random((NAZ, NRANGE))
    c = R.polar_to_cartesian(p, N, DXY, RES)
    c2 = R.polar_to_cartesian(np.roll(p, NAZ // 4, axis=0), N, DXY, RES)
    y, x = np.meshgrid(np.arange(1, N), np.arange(N), indexing="ij")
    off = ~((y == N // 2) & (x == N // 2))   # the sensor pixel: rho = 0 has no azimuth (A16 takes 0)
    assert rel(c2[x, N - y][off], c[y, x][off]) < 1e-12


@pytest.mark.parametrize("n_az", [NAZ, 16])   # 16: a 22.5 deg sector before the seam holds many pixels
def test_matches_scipy_bilinear_with_wrapped_azimuth(n_az):
    ndimage = pytest.importorskip("scipy.ndimage")
    p = RNG.random((n_az, NRANGE))
    c = R.polar_to_cartesian(p, N, DXY, RES)
    fa, fk = R.polar_indices(N, DXY, n_az, RES)
    wrapped = np.vstack([p, p[:1]])                               # row n_az = row 0
    ref = ndimage.map_coordinates(wrapped, [fa.ravel(), fk.ravel()], order=1, mode="nearest").reshape(N, N)
    inside = fk <= NRANGE - 1
    assert rel(c[inside], ref[inside]) < 1e-12
    assert np.count_nonzero(inside & (fa > n_az - 1)) > (10 if n_az == 16 else -1)


def test_seam_sector_interpolates_back_to_azimuth_zero():
    """P[a] = a with 16 azimuths: past the last azimuth the value falls linearly from 15 to the 0
    of azimuth 0, i.e. 15 (16 - fa) in the sector fa in [15, 16)."""
    p = np.tile(np.arange(16, dtype=np.float64)[:, None], (1, NRANGE))
    c = R.polar_to_cartesian(p, N, DXY, RES)
    fa, _ = R.polar_indices(N, DXY, 16, RES)
    seam = fa > 15
    assert seam.sum() > 10
    assert np.max(np.abs(c[seam] - 15.0 * (16.0 - fa[seam]))) < 1e-9


def test_polar_generator_is_seeded_and_navtech_shaped():
    from paper_2203_00459_gb300 import synth
    a = synth.make_polar_scans(2, seed=5)
    b = synth.make_polar_scans(2, seed=5)
    assert a.shape == (2, 400, 3768) and a.dtype == np.float32
    assert np.array_equal(a, b) and not np.array_equal(a[0], a[1])
    assert not np.array_equal(a, synth.make_polar_scans(2, seed=6))
    assert a.min() >= 0.0 and a.max() > 5.0   # |noise| floor plus returns of amplitude >= 5 x speckle
