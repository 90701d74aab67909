"""Angle counts without an FFT plan (Alg. 1's own n_theta = 733, odd, prime; and the range ends
8 and 1024): the direct circular sums of the angle stage and their adjoint against the FP64
oracle, through the C ABI."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2203_00459_gb300 import synth  # noqa: E402
from gpu_util import check_pair, oracle_cfg  # noqa: E402

pytestmark = pytest.mark.gpu

TOL_GRAD = 1e-3   # max |gpu - reference| / max |reference| per gradient image
DP = np.array([[0.8, -0.35, 0.6], [-0.5, 1.0, 0.25], [0.3, 0.2, -0.9]])


@pytest.fixture(scope="module")
def lib():
    from paper_2203_00459_gb300 import build
    build.build()
    from paper_2203_00459_gb300 import search
    return search


def grad_err(a, b):
    return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / max(1e-300, np.max(np.abs(b))))


def forward(search, cfg, f, g, flags=0):
    s = search.PoseSearch([cfg], max_pairs=f.shape[0], flags=flags)
    ft, gt = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    out = s.pose(ft, gt, want_c_theta=True, want_c_xy=True)
    torch.cuda.synchronize()
    res = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
    s.close()
    return res


def turned_pairs(n, degs, seed):
    pairs = [synth.make_pair(n, n * n // 300, n // 16, math.radians(d), 3.0, -2.0, seed=seed, index=i)
             for i, d in enumerate(degs)]
    return np.stack([a for a, _ in pairs]), np.stack([b for _, b in pairs])


@pytest.mark.parametrize("angle_score", [0, 1])
@pytest.mark.parametrize("nr", [128, 100])   # 100: a partial chunk of radii
def test_alg1_angle_count_733(lib, angle_score, nr):
    """n = 256, n_theta = 733 (Alg. 1), per-radius score (Eq. 7) and the radial mean: the angle
    scores, c_xy and the pose against the oracle's, and the heading against the truth."""
    degs = (17.0, -31.0, 2.5)
    f, g = turned_pairs(256, degs, 911)
    cfg = lib.size_cfg(256, 733, nr, temp_theta=0.2, angle_score=angle_score)
    o = forward(lib, cfg, f, g)
    for i, d in enumerate(degs):
        check_pair(f[i], g[i], cfg, o["pose"][i], o["c_theta"][733 * i:733 * (i + 1)], o["c_xy"][i], f"733:{i}")
        assert abs(o["pose"][i][0] - math.radians(d)) < math.radians(1.0), (d, o["pose"][i])


def test_alg1_literal_configuration(lib):
    """Alg. 1 as printed: n_theta = 733, T_theta = 2, raw scores, g turned back by theta."""
    from paper_2203_00459_gb300 import _lib
    f, g, _ = synth.make_batch("batch256", pairs=2, start=5)
    cfg = lib.size_cfg(256, 733, 128, temp_theta=2.0, score_norm=1, angle_score=1, rotate_target=1)
    o = forward(lib, cfg, f, g, flags=_lib.FLAG_GRAPH)
    for i in range(2):
        check_pair(f[i], g[i], cfg, o["pose"][i], o["c_theta"][733 * i:733 * (i + 1)], o["c_xy"][i], f"lit:{i}")


@pytest.mark.parametrize("nt", [8, 129, 1024])
def test_range_ends_and_odd_count(lib, nt):
    f, g, _ = synth.make_batch("single128", pairs=2, start=9)
    cfg = lib.size_cfg(128, nt, 64, temp_theta=0.5)
    o = forward(lib, cfg, f, g)
    for i in range(2):
        check_pair(f[i], g[i], cfg, o["pose"][i], o["c_theta"][nt * i:nt * (i + 1)], o["c_xy"][i], f"{nt}:{i}")


def test_counts_outside_the_range_are_rejected(lib):
    from paper_2203_00459_gb300 import _lib
    for nt in (7, 1025):
        with pytest.raises(_lib.FmbymError):
            lib.PoseSearch([lib.size_cfg(128, nt, 64)], max_pairs=1)


@pytest.mark.parametrize("angle_score", [0, 1])
def test_adjoint_733(lib, angle_score):
    """n_r = 92 leaves a partial chunk of radii.  The Rotate adjoint's d theta term takes the
    bilinear cell of each fp32 sample point, so it jumps where a sample crosses a cell edge; these
    pairs have no such edge within 6 fp32 ulps of the oracle's theta (at n_r = 100 pair 0 has one
    2 ulps away, where a one-ulp change of theta moves d theta by 4 %)."""
    f, g = turned_pairs(256, (12.0, -7.0), 913)
    cfg = lib.size_cfg(256, 733, 92, temp_theta=0.5, angle_score=angle_score)
    s = lib.PoseSearch([cfg], max_pairs=2)
    df, dg = s.pose_backward(torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda(),
                             torch.from_numpy(DP[:2].astype(np.float32)).cuda())
    torch.cuda.synchronize()
    df, dg = df.cpu().numpy(), dg.cpu().numpy()
    s.close()
    oc = oracle_cfg(cfg)
    for i in range(2):
        odf, odg, _ = O.pose_backward(f[i], g[i], oc, DP[i])
        ef, eg = grad_err(df[i], odf), grad_err(dg[i], odg)
        assert ef <= TOL_GRAD and eg <= TOL_GRAD, (angle_score, i, ef, eg)


def test_training_call_mixed_with_an_fft_angle_count(lib):
    """A call that mixes n_theta = 733 (direct sums) and n_theta = 400 (FFT): the training call
    gives the bits of the three separate calls, and its 733 adjoint matches the oracle's."""
    from paper_2203_00459_gb300 import _lib
    cfgs = [lib.size_cfg(256, 733, 128, temp_theta=0.5), lib.size_cfg(256, 400, 128)]
    order = [0, 1, 0]
    scans = [synth.make_batch("batch256", pairs=1, start=70 + k) for k in range(3)]
    F = torch.from_numpy(np.concatenate([f.ravel() for f, _, _ in scans])).cuda()
    G = torch.from_numpy(np.concatenate([g.ravel() for _, g, _ in scans])).cuda()
    gt = torch.from_numpy(np.concatenate([p for _, _, p in scans]).astype(np.float32)).cuda()
    offs = [k * 256 * 256 for k in range(3)]
    s = lib.PoseSearch(cfgs, max_pairs=3, flags=_lib.FLAG_GRAPH)
    for _ in range(2):   # the second graph call replays the captured layout
        pose, loss, dpose, df, dg = s.pose_train(F, G, gt, kind=2, size_idx=order, offsets=offs)
    pose2 = s.pose(F, G, size_idx=order, offsets=offs)["pose"]
    loss2, dpose2 = s.pose_loss(pose2, gt, kind=2)
    df2, dg2 = s.pose_backward(F, G, dpose2, size_idx=order, offsets=offs)
    torch.cuda.synchronize()
    for a, b in ((pose, pose2), (loss, loss2), (dpose, dpose2), (df, df2), (dg, dg2)):
        assert torch.equal(a, b)
    f, g, _ = scans[0]
    odf, odg, _ = O.pose_backward(f[0], g[0], oracle_cfg(cfgs[0]), dpose.cpu().numpy()[0].astype(np.float64))
    assert grad_err(df.cpu().numpy()[:256 * 256].reshape(256, 256), odf) <= TOL_GRAD
    assert grad_err(dg.cpu().numpy()[:256 * 256].reshape(256, 256), odg) <= TOL_GRAD
    s.close()
