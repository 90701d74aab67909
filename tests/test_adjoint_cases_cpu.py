"""The GPU adjoint parity cases sit away from bilinear cell edges (reading A14): at every fp32
theta within 6 ulps of the oracle's, the kernel's fp32 d theta term stays within 1e-3 of the
oracle's.  A case that fails here would compare the two sides of a jump on the GPU, whatever the
kernels do; the n_r = 100 case this check found is kept as the negative control."""
import math

import numpy as np
import pytest

import oracle as O
from kink_util import dtheta_kink_margin
from paper_2203_00459_gb300 import synth

DP = np.array([[0.8, -0.35, 0.6], [-0.5, 1.0, 0.25]])


def _turned(n, degs, seed):
    pairs = [synth.make_pair(n, n * n // 300, n // 16, math.radians(d), 3.0, -2.0, seed=seed, index=i)
             for i, d in enumerate(degs)]
    return [a for a, _ in pairs], [b for _, b in pairs]


@pytest.mark.parametrize("angle_score", [0, 1])
def test_n_theta_733_adjoint_cases(monkeypatch, angle_score):
    f, g = _turned(256, (12.0, -7.0), 913)
    cfg = O.make_cfg(256, 733, 92, temp_theta=0.5, angle_score=angle_score)
    for i in range(2):
        assert dtheta_kink_margin(f[i], g[i], cfg, DP[i], monkeypatch) < 1e-3, (angle_score, i)


def test_the_case_that_sat_on_an_edge_is_seen(monkeypatch):
    f, g = _turned(256, (12.0, -7.0), 913)
    cfg = O.make_cfg(256, 733, 100, temp_theta=0.5)
    assert dtheta_kink_margin(f[0], g[0], cfg, DP[0], monkeypatch) > 1e-3


@pytest.mark.parametrize("name,pairs", [("single128", 5), ("batch256", 2)])
def test_fft_route_adjoint_cases(monkeypatch, name, pairs):
    spec = synth.WORKLOADS[name]
    f, g, _ = synth.make_batch(name, pairs=pairs, start=3)
    cfg = O.make_cfg(spec["n"], spec["n_theta"], spec["n_r"])
    dps = np.array([[0.8, -0.35, 0.6], [-0.5, 1.0, 0.25], [0.3, 0.2, -0.9], [1.0, 0.0, 0.0], [0.0, 1.0, 1.0]])
    for i in range(pairs):
        assert dtheta_kink_margin(f[i], g[i], cfg, dps[i], monkeypatch) < 1e-3, (name, i)


def _pairs(n, pts, walls, degs, tx, ty, seed):
    ps = [synth.make_pair(n, pts, walls, math.radians(d), tx, ty, seed=seed, index=i) for i, d in enumerate(degs)]
    return [a for a, _ in ps], [b for _, b in ps]


def _batch(name, pairs, start):
    f, g, _ = synth.make_batch(name, pairs=pairs, start=start)
    return list(f), list(g)


CASES = {
    "raw scores, ragged radii": (lambda: _batch("batch256", 2, 0),
                                 dict(n=256, n_theta=256, n_r=100, temp_theta=2.0e8, temp_xy=1.0e4, window=0,
                                      score_norm=1, band_lo=3.5, band_hi=100.0)),
    "circular padding": (lambda: _batch("single128", 2, 11), dict(n=128, n_theta=128, n_r=64, pad_mode=1, temp_xy=0.5)),
    "radial mean": (lambda: _batch("batch256", 2, 61), dict(n=256, n_theta=400, n_r=128, temp_theta=2.0, angle_score=1)),
    "full circle": (lambda: _pairs(128, 40, 6, (160.0, -20.0), 2.0, 1.0, 780),
                    dict(n=128, n_theta=128, n_r=64, temp_theta=0.2, full_circle=1)),
    "Alg. 1 stage 2": (lambda: _pairs(128, 40, 6, (15.0, -9.0), 3.0, -2.0, 784),
                       dict(n=128, n_theta=128, n_r=64, temp_theta=0.5, rotate_target=1)),
}


@pytest.mark.parametrize("case", list(CASES))
def test_option_adjoint_cases(monkeypatch, case):
    make, kw = CASES[case]
    f, g = make()
    cfg = O.make_cfg(**kw)
    for i in range(2):
        assert dtheta_kink_margin(f[i], g[i], cfg, DP[i], monkeypatch) < 1e-3, (case, i)


def test_schedule_variant_case(monkeypatch):
    f, g = _batch("batch256", 2, 31)
    cfg = O.make_cfg(256, 400, 128)
    assert dtheta_kink_margin(f[0], g[0], cfg, np.array([0.7, -0.4, 0.5]), monkeypatch) < 1e-3


ODD_DP = np.array([[0.9, -0.4, 0.25], [-0.3, 0.6, 0.5], [0.2, 0.1, -0.8]])


@pytest.mark.parametrize("name,pairs,start,kw", [
    ("batch127", 3, 3, {}), ("batch255", 2, 3, {}), ("batch511", 1, 5, {}),
    ("batch127", 2, 31, dict(rotate_target=1, temp_theta=0.5)),
    ("batch127", 2, 33, dict(score_norm=1, temp_theta=2.0e8, temp_xy=1.0e4, window=0))])
def test_odd_side_adjoint_cases(monkeypatch, name, pairs, start, kw):
    """The odd-side adjoint parity cases (the paper's 127, 255, 511; rotation about the half-integer
    centre N/2) and the variants at 127."""
    spec = synth.WORKLOADS[name]
    f, g, _ = synth.make_batch(name, pairs=pairs, start=start)
    cfg = O.make_cfg(spec["n"], spec["n_theta"], spec["n_r"], **kw)
    for i in range(pairs):
        assert dtheta_kink_margin(f[i], g[i], cfg, ODD_DP[i], monkeypatch) < 1e-3, (name, start, i)


def test_the_odd_side_case_next_to_an_edge_is_seen(monkeypatch):
    spec = synth.WORKLOADS["batch511"]
    f, g, _ = synth.make_batch("batch511", pairs=1, start=3)
    cfg = O.make_cfg(spec["n"], spec["n_theta"], spec["n_r"])
    assert dtheta_kink_margin(f[0], g[0], cfg, ODD_DP[0], monkeypatch) > 1e-3


def test_radix_order_case_at_512(monkeypatch):
    """The 512^2 pair of the radix-order parity test (start 3; start 9 sits on an edge)."""
    spec = synth.WORKLOADS["batch512"]
    cfg = O.make_cfg(512, spec["n_theta"], spec["n_r"])
    dp = np.array([0.7, -0.4, 0.5])
    f, g, _ = synth.make_batch("batch512", pairs=1, start=3)
    assert dtheta_kink_margin(f[0], g[0], cfg, dp, monkeypatch) < 1e-3
    f, g, _ = synth.make_batch("batch512", pairs=1, start=9)
    assert dtheta_kink_margin(f[0], g[0], cfg, dp, monkeypatch) > 1e-3
