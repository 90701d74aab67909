"""Distance of an adjoint parity case from a bilinear cell edge (reading A14), on the CPU.

The Rotate adjoint's d theta term uses the gradient of the bilinear interpolant, which is constant
inside a cell and jumps across a cell edge.  The kernels place the samples in fp32 at an fp32
theta and the oracle in fp64, so a case whose theta lies within a few fp32 ulps of an edge compares
the two sides of a jump instead of the arithmetic.  ``dtheta_kink_margin`` evaluates the d theta
term with fp32 sample positions (each position one fused multiply-add rounded to fp32, as the
kernel forms it) at the fp32 thetas around the oracle's, and returns the largest relative change
against the oracle's fp64 value: near 1e-6 for a safe case, percent-level next to an edge.
"""
import math

import numpy as np

import oracle as O
from oracle import fmbym_oracle as core

f32 = np.float32


def _fma32(a, b, c):
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def _dtheta32(x, d, theta32):
    """The d theta term of the Rotate adjoint, sample positions in fp32 (about c = N/2, a
    half-integer for an odd side)."""
    n = x.shape[0]
    c = f32(n / 2)
    ct, st = f32(math.cos(float(theta32))), f32(math.sin(float(theta32)))
    Y, X = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    dX, dY = X.astype(f32) - c, Y.astype(f32) - c
    px = _fma32(ct, dX, _fma32(st, dY, c))
    py = _fma32(ct, dY, _fma32(-st, dX, c))
    x0, y0 = np.floor(px).astype(np.int64), np.floor(py).astype(np.int64)
    fx, fy = (px - np.floor(px)).astype(np.float64), (py - np.floor(py)).astype(np.float64)

    def at(yy, xx):
        ok = (yy >= 0) & (yy < n) & (xx >= 0) & (xx < n)
        return np.where(ok, x[np.clip(yy, 0, n - 1), np.clip(xx, 0, n - 1)], 0.0)

    v00, v01, v10, v11 = at(y0, x0), at(y0, x0 + 1), at(y0 + 1, x0), at(y0 + 1, x0 + 1)
    dvx = (1 - fy) * (v01 - v00) + fy * (v11 - v10)
    dvy = (1 - fx) * (v10 - v00) + fx * (v11 - v01)
    return float((d * (dvx * (py.astype(np.float64) - n / 2) - dvy * (px.astype(np.float64) - n / 2))).sum())


def dtheta_kink_margin(f, g, cfg, dpose, monkeypatch, ulps=6):
    """Largest relative change of the fp32 d theta term over the fp32 thetas within ``ulps`` of
    the oracle's, against the oracle's fp64 term, for one pair and one dL/dpose."""
    cap = {}
    orig = core.rotate_backward

    def spy(x, t, d):
        cap.update(x=np.asarray(x, np.float64), t=t, d=d)
        return orig(x, t, d)

    monkeypatch.setattr(core, "rotate_backward", spy)
    O.pose_backward(f, g, cfg, np.asarray(dpose, np.float64))
    monkeypatch.setattr(core, "rotate_backward", orig)
    _, ref = orig(cap["x"], cap["t"], cap["d"])
    t32 = f32(cap["t"])
    u = np.spacing(t32)
    scale = max(abs(ref), 1e-30)
    return max(abs(_dtheta32(cap["x"], cap["d"], f32(t32 + k * u)) - ref) / scale for k in range(-ulps, ulps + 1))
