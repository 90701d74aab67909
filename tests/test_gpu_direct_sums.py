"""The CUDA search against the oracle's brute-force sums of the definitions, through the C ABI:
the translation scores against c[s] = sum_x f'(x) g(x + s) summed lag by lag (Eq. 3 and 8), and
the angle scores against the circular double sum of Eq. 7.  At 128^2 (the single-pair
configuration) every lag of every pair is checked; at 512^2 the full 32-pair batch runs in the
launch configuration the benchmark times (graph replay, autotuned schedules) and sampled lags are
checked, the four corners and edge midpoints of the lag square (+-N/2) among them."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2203_00459_gb300 import synth  # noqa: E402
from gpu_util import TOL_SURF, TOL_T, TOL_THETA, argmax_ok, oracle_cfg, surf_err  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2203_00459_gb300 import build
    build.build()
    from paper_2203_00459_gb300 import _lib, search
    return search, _lib


def forward(search, cfg, f, g, flags=0):
    s = search.PoseSearch([cfg], max_pairs=f.shape[0], flags=flags)
    ft, gt = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    out = s.pose(ft, gt, want_c_theta=True, want_c_xy=True)
    out = {k: v.cpu().numpy() for k, v in out.items()}
    s.close()
    return out


@pytest.mark.parametrize("pad_mode", [0, 1])
def test_every_lag_at_128_against_the_brute_force_sums(lib, pad_mode):
    search, _ = lib
    f, g, _ = synth.make_batch("single128", pairs=5)
    cfg = search.size_cfg(128, 128, 64, pad_mode=pad_mode)
    oc = oracle_cfg(cfg)
    o = forward(search, cfg, f, g)
    for i in range(f.shape[0]):
        r = O.pose(f[i], g[i], oc, keep=True)
        assert abs(o["pose"][i, 0] - r["theta"]) <= TOL_THETA
        assert abs(o["pose"][i, 1] - r["tx"]) <= TOL_T and abs(o["pose"][i, 2] - r["ty"]) <= TOL_T
        ct = o["c_theta"][128 * i:128 * (i + 1)]
        ct_ref = O.angle_scores(r["pf"], r["pg"])           # the circular double sum of Eq. 7
        assert surf_err(ct, ct_ref) <= TOL_SURF and argmax_ok(ct, ct_ref), i
        th = float(np.float32(o["pose"][i, 0]))              # stage 2 at the GPU's own heading
        ref = O.xcorr2d_brute(O.rotate(f[i], th), g[i], pad_mode)
        assert surf_err(o["c_xy"][i], ref) <= TOL_SURF, (i, surf_err(o["c_xy"][i], ref))
        assert argmax_ok(o["c_xy"][i], ref), i


def test_sampled_lags_of_the_full_512_batch_against_the_brute_force_sum(lib):
    search, _lib = lib
    spec = synth.WORKLOADS["batch512"]
    f, g, _ = synth.make_batch("batch512")
    n = spec["n"]
    cfg = search.size_cfg(n, spec["n_theta"], spec["n_r"])
    o = forward(search, cfg, f, g, flags=_lib.FLAG_GRAPH | _lib.FLAG_AUTOTUNE)
    lo, hi = -n // 2, n // 2 - 1
    rng = np.random.default_rng(512)
    for i in (0, 9, 31):
        cxy = o["c_xy"][i]
        top = np.unravel_index(int(np.argmax(cxy)), cxy.shape)
        lag_list = [(lo, lo), (lo, hi), (hi, lo), (hi, hi), (lo, 0), (0, lo), (hi, 0), (0, hi), (0, 0),
                    (int(top[0]) + lo, int(top[1]) + lo)]
        lag_list += [tuple(int(v) for v in rng.integers(lo, hi + 1, 2)) for _ in range(6)]
        th = float(np.float32(o["pose"][i, 0]))
        ref = O.xcorr2d_brute(O.rotate(f[i], th), g[i], 0, lag_list)
        scale = float(np.max(np.abs(ref)))
        for (sy, sx), v in zip(lag_list, ref):
            got = float(cxy[sy - lo, sx - lo])
            assert abs(got - v) <= TOL_SURF * scale, (i, sy, sx, got, v, scale)
