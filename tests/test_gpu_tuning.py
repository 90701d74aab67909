"""Every compiled launch schedule (column tile and radix order of the stage-2 column passes, radii
per CTA of the angle kernels, pixels per thread of the Rotate adjoint) gives the oracle's results,
and the autotuner picks among them."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2203_00459_gb300 import synth  # noqa: E402
from gpu_util import check_pair, oracle_cfg  # noqa: E402

pytestmark = pytest.mark.gpu

TOL_GRAD = 1e-3
VARIANTS = [dict(col_tile=4), dict(col_tile=16), dict(angle_radii=8), dict(rot_pixels=1), dict(rot_pixels=2),
            dict(rot_pixels=8), dict(col_plan=1), dict(col_plan=1, col_tile=4), dict(col_plan=1, col_tile=16)]
DP = np.array([[0.7, -0.4, 0.5], [-0.3, 0.9, 0.2]])


@pytest.fixture(scope="module")
def lib():
    from paper_2203_00459_gb300 import build
    build.build()
    from paper_2203_00459_gb300 import _lib, search
    return _lib, search


@pytest.fixture(scope="module")
def data():
    return synth.make_batch("batch256", pairs=2, start=31)


def grad_err(a, b):
    return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("variant", VARIANTS, ids=[",".join(f"{k}={v}" for k, v in d.items()) for d in VARIANTS])
def test_schedule_variant_matches_oracle(lib, data, variant):
    _, search = lib
    f, g, _ = data
    cfg = search.size_cfg(256, 400, 128)
    s = search.PoseSearch([cfg], max_pairs=2)
    s.set_tuning(0, **variant)
    assert all(s.tuning(0)[k] == v for k, v in variant.items())
    ft, gt_ = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    out = s.pose(ft, gt_, want_c_theta=True, want_c_xy=True)
    df, dg = s.pose_backward(ft, gt_, torch.from_numpy(DP.astype(np.float32)).cuda())
    torch.cuda.synchronize()
    pose, ct, cxy = out["pose"].cpu().numpy(), out["c_theta"].cpu().numpy(), out["c_xy"].cpu().numpy()
    df, dg = df.cpu().numpy(), dg.cpu().numpy()
    s.close()
    for i in range(2):
        check_pair(f[i], g[i], cfg, pose[i], ct[i * 400:(i + 1) * 400], cxy[i], tag=str(variant))
    odf, odg, _ = O.pose_backward(f[0], g[0], oracle_cfg(cfg), DP[0])
    assert grad_err(df[0], odf) <= TOL_GRAD and grad_err(dg[0], odg) <= TOL_GRAD, variant


def test_autotuner_picks_candidates_and_keeps_results(lib, data):
    _lib, search = lib
    f, g, _ = data
    cfg = search.size_cfg(256, 400, 128)
    tuned = search.PoseSearch([cfg], max_pairs=4, flags=_lib.FLAG_AUTOTUNE)
    plain = search.PoseSearch([cfg], max_pairs=4)
    t = tuned.tuning(0)
    assert t["col_tile"] in (4, 8, 16) and t["angle_radii"] in (8, 16) and t["rot_pixels"] in (1, 2, 4, 8), t
    assert t["col_plan"] in (0, 1), t
    assert plain.tuning(0) == dict(col_tile=8, angle_radii=16, rot_pixels=4, col_plan=0)
    ft, gt_ = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    a = tuned.pose(ft, gt_)["pose"].cpu().numpy()
    b = plain.pose(ft, gt_)["pose"].cpu().numpy()
    assert np.max(np.abs(a - b)) <= 1e-4, (t, a, b)
    with pytest.raises(_lib.FmbymError):
        plain.set_tuning(0, col_tile=3)
    with pytest.raises(_lib.FmbymError):
        plain.set_tuning(0, rot_pixels=16)
    with pytest.raises(_lib.FmbymError):
        plain.set_tuning(0, col_plan=2)
    assert plain.tuning(0) == dict(col_tile=8, angle_radii=16, rot_pixels=4, col_plan=0)
    tuned.close()
    plain.close()


@pytest.mark.parametrize("col_plan", [0, 1])
def test_radix_orders_at_512_match_oracle(lib, col_plan):
    """Both radix orders of the 768-point column passes (16, 16, 3 and 16, 3, 16) at 512^2: forward
    pose and surfaces, and the adjoint, against the FP64 oracle on one pair."""
    _, search = lib
    spec = synth.WORKLOADS["batch512"]
    f, g, _ = synth.make_batch("batch512", pairs=1, start=3)   # clear of cell edges (reading A14)
    cfg = search.size_cfg(512, spec["n_theta"], spec["n_r"])
    s = search.PoseSearch([cfg], max_pairs=1)
    s.set_tuning(0, col_plan=col_plan)
    ft, gt_ = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    out = s.pose(ft, gt_, want_c_theta=True, want_c_xy=True)
    df, dg = s.pose_backward(ft, gt_, torch.from_numpy(DP[:1].astype(np.float32)).cuda())
    torch.cuda.synchronize()
    check_pair(f[0], g[0], cfg, out["pose"].cpu().numpy()[0], out["c_theta"].cpu().numpy(), out["c_xy"].cpu().numpy()[0],
               tag=f"col_plan={col_plan}")
    odf, odg, _ = O.pose_backward(f[0], g[0], oracle_cfg(cfg), DP[0])
    assert grad_err(df.cpu().numpy()[0], odf) <= TOL_GRAD and grad_err(dg.cpu().numpy()[0], odg) <= TOL_GRAD
    s.close()
