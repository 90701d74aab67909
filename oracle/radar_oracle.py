"""FP64 CPU oracle of the radar front end: a polar (azimuth x range) scan resampled onto the
N x N Cartesian grid that the pose search takes -- test infrastructure only.

The paper feeds Cartesian scans of side N and cell size delta_xy to the search (Sec. IV, Alg. 1)
and takes them from a rotating FMCW radar (Sec. IV-A, Navtech CTS350-X, 4 Hz).  It does not state
the conversion, so this module fixes one reading (A16), written out as its definition:

* A16 the polar scan is [n_az][n_range] row-major; azimuth a looks along phi_a = 2 pi a / n_az,
      measured from +x (column) toward +y (row), the sense of a positive theta in A8; range bin k
      is centred at rho_k = (k + 1/2) range_res.  Cartesian pixel (y, x) sits at
      (X, Y) = ((x - N/2) delta_xy, (y - N/2) delta_xy), the sensor at the rotation centre of A8.
      Its value is the bilinear interpolation of the scan at fractional indices
      (phi / (2 pi / n_az), rho / range_res - 1/2), periodic in azimuth; inside the first bin
      centre the range index is held at 0, beyond the last bin centre the value is 0.  The sensor
      pixel (rho = 0) has no bearing and takes azimuth 0.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may call this.
"""
from __future__ import annotations

import numpy as np


def cartesian_points(n, delta_xy):
    """(X, Y) in metres of every pixel of the N x N grid, [N, N] each (A16)."""
    idx = (np.arange(n, dtype=np.float64) - n // 2) * delta_xy
    Y, X = np.meshgrid(idx, idx, indexing="ij")
    return X, Y


def polar_indices(n, delta_xy, n_az, range_res):
    """Fractional (azimuth, range) indices of every Cartesian pixel (A16), [N, N] each."""
    X, Y = cartesian_points(n, delta_xy)
    phi = np.mod(np.arctan2(Y, X), 2.0 * np.pi)
    rho = np.hypot(X, Y)
    fa = phi / (2.0 * np.pi / n_az)
    fk = np.maximum(rho / range_res - 0.5, 0.0)
    return fa, fk


def polar_to_cartesian(polar, n, delta_xy, range_res):
    """Bilinear resampling of one polar scan [n_az, n_range] onto the N x N grid (A16)."""
    p = np.asarray(polar, np.float64)
    n_az, n_range = p.shape
    fa, fk = polar_indices(n, delta_xy, n_az, range_res)
    a0 = np.floor(fa).astype(np.int64)
    ta = fa - a0
    a0 = np.mod(a0, n_az)
    a1 = np.mod(a0 + 1, n_az)
    inside = fk <= n_range - 1
    k0 = np.minimum(np.floor(fk).astype(np.int64), n_range - 1)
    tk = fk - k0
    k1 = np.minimum(k0 + 1, n_range - 1)
    v = ((1.0 - ta) * ((1.0 - tk) * p[a0, k0] + tk * p[a0, k1])
         + ta * ((1.0 - tk) * p[a1, k0] + tk * p[a1, k1]))
    return np.where(inside, v, 0.0)
