"""Degenerate inputs of the search against the FP64 oracle, through the C ABI: empty scans (every
score surface flat, so both soft-argmaxes return the mean of their candidates and the z-score's
zero deviation must not divide), a pair with one empty scan, and identical scans (both
correlations peak at lag 0)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2203_00459_gb300 import synth  # noqa: E402
from gpu_util import TOL_T, TOL_THETA, check_pair, oracle_cfg  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = [("single128", 128, 128, 64), ("batch512", 512, 400, 256)]


@pytest.fixture(scope="module")
def search():
    from paper_2203_00459_gb300 import build
    build.build()
    from paper_2203_00459_gb300 import search as s
    return s


def run(search, cfg, f, g, dpose):
    s = search.PoseSearch([cfg], max_pairs=f.shape[0])
    ft, gt = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    out = s.pose(ft, gt, want_c_theta=True, want_c_xy=True)
    df, dg = s.pose_backward(ft, gt, torch.from_numpy(dpose.astype(np.float32)).cuda())
    torch.cuda.synchronize()
    res = (out["pose"].cpu().numpy(), out["c_theta"].cpu().numpy(), out["c_xy"].cpu().numpy(), df.cpu().numpy(),
           dg.cpu().numpy())
    s.close()
    return res


@pytest.mark.parametrize("name,n,nt,nr", CASES)
def test_empty_scans_give_the_mean_candidate_and_no_gradient(search, name, n, nt, nr):
    """Pair 0 has two empty scans: every surface is exactly zero on both sides, so the poses are
    the candidate means and the gradients vanish.  Pair 1 matches a scan against an empty one:
    stage 2 correlates separately transformed images and is exactly flat too, but stage 1 packs
    A_f + i A_g into one FFT along angle, whose rounding leaves conj(A^_f) A^_g at about 1e-7 of
    |A^_f|^2 where exact arithmetic gives 0; the z-score rescales that residue to unit spread, so
    the heading of such a pair is not defined by the scans (only finiteness is required)."""
    cfg = search.size_cfg(n, nt, nr)
    z = np.zeros((2, n, n), np.float32)
    scan = synth.make_batch(name, pairs=1, start=2)[0]
    f = np.concatenate([z[:1], scan])
    g = np.concatenate([z[:1], z[:1]])
    dpose = np.array([[0.7, -0.4, 0.5], [0.3, 0.9, -0.2]])
    pose, ct, cxy, df, dg = run(search, cfg, f, g, dpose)
    oc = oracle_cfg(cfg)
    r = O.pose(f[0].astype(np.float64), g[0].astype(np.float64), oc)
    assert np.all(r["c_theta"] == 0.0) and np.all(ct[:nt] == 0.0) and np.all(cxy[0] == 0.0)
    # flat surfaces: the means of the candidate grids, -delta/2 on each axis
    assert abs(r["theta"] + np.pi / nt / 2) < 1e-12 and abs(r["tx"] + 0.5) < 1e-12 and abs(r["ty"] + 0.5) < 1e-12
    assert abs(pose[0, 0] - r["theta"]) <= TOL_THETA and abs(pose[0, 1] - r["tx"]) <= TOL_T
    assert abs(pose[0, 2] - r["ty"]) <= TOL_T
    odf, odg, _ = O.pose_backward(f[0].astype(np.float64), g[0].astype(np.float64), oc, dpose[0])
    assert np.all(odf == 0.0) and np.all(odg == 0.0) and np.all(df[0] == 0.0) and np.all(dg[0] == 0.0)
    # pair 1: stage 2 is exactly flat, its translation the lag means; everything finite
    assert np.all(cxy[1] == 0.0)
    assert abs(pose[1, 1] + 0.5) <= TOL_T and abs(pose[1, 2] + 0.5) <= TOL_T
    assert np.all(np.isfinite(pose[1])) and np.all(np.isfinite(df[1])) and np.all(np.isfinite(dg[1]))


@pytest.mark.parametrize("name,n,nt,nr", CASES)
def test_identical_scans_peak_at_lag_zero(search, name, n, nt, nr):
    cfg = search.size_cfg(n, nt, nr)
    f = synth.make_batch(name, pairs=1, start=5)[0]
    pose, ct, cxy, df, dg = run(search, cfg, f, f.copy(), np.array([[0.7, -0.4, 0.5]]))
    r = check_pair(f[0], f[0], cfg, pose[0], ct, cxy[0], tag=name)
    k0 = int(np.argmax(r["c_theta"]))
    assert k0 == nt // 2                                   # lag 0 sits at index n_theta / 2
    assert np.unravel_index(int(np.argmax(cxy[0])), cxy[0].shape) == (n // 2, n // 2)
    assert abs(pose[0, 1]) < 0.5 and abs(pose[0, 2]) < 0.5
    assert np.all(np.isfinite(df)) and np.all(np.isfinite(dg))
