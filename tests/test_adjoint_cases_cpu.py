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
