"""The paper's odd scan sides 127, 255 and 511 (Sec. IV-B cell sizes 0.8, 0.4, 0.2 m; Alg. 1's
n_xy = 255) on the GPU, through the C ABI, against the FP64 oracle: the stage-1 N-point DFTs run as
Bluestein convolutions, stage 2 in the even frame N + 1 (the same padded length P = 3(N + 1)/2).
Forward (pose, angle and translation score surfaces), the adjoint, and the training call."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2203_00459_gb300 import synth  # noqa: E402
from gpu_util import check_pair, oracle_cfg  # noqa: E402

pytestmark = pytest.mark.gpu

TOL_GRAD = 1e-3   # max |gpu - oracle| / max |oracle| per gradient image


@pytest.fixture(scope="module")
def lib():
    from paper_2203_00459_gb300 import build
    build.build()
    from paper_2203_00459_gb300 import _lib, search
    return search, _lib


def grad_err(a, b):
    return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / max(1e-300, np.max(np.abs(b))))


def cfg_of(search, name, **kw):
    spec = synth.WORKLOADS[name]
    return search.size_cfg(spec["n"], spec["n_theta"], spec["n_r"], **kw)


@pytest.mark.parametrize("name,pairs", [("batch127", 6), ("batch255", 4), ("batch511", 2)])
def test_forward_parity(lib, name, pairs):
    search, _ = lib
    f, g, _ = synth.make_batch(name, pairs=pairs)
    cfg = cfg_of(search, name)
    nt = cfg["n_theta"]
    s = search.PoseSearch([cfg], max_pairs=pairs)
    o = s.pose(torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda(), want_c_theta=True, want_c_xy=True)
    o = {k: v.cpu().numpy() for k, v in o.items()}
    s.close()
    for i in range(pairs):
        check_pair(f[i], g[i], cfg, o["pose"][i], o["c_theta"][nt * i:nt * (i + 1)], o["c_xy"][i], f"{name}:{i}")


@pytest.mark.parametrize("kw", [dict(score_norm=1, temp_theta=2.0e8, temp_xy=1.0e4, window=0, band_lo=3.5, band_hi=50.0),
                                dict(angle_score=1, temp_theta=2.0), dict(rotate_target=1, temp_theta=0.5),
                                dict(full_circle=1, temp_theta=0.5)])
def test_forward_variants_at_127(lib, kw):
    search, _ = lib
    f, g, _ = synth.make_batch("batch127", pairs=3, start=20)
    cfg = cfg_of(search, "batch127", **kw)
    s = search.PoseSearch([cfg], max_pairs=3)
    o = s.pose(torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda(), want_c_theta=True, want_c_xy=True)
    o = {k: v.cpu().numpy() for k, v in o.items()}
    s.close()
    for i in range(3):
        check_pair(f[i], g[i], cfg, o["pose"][i], o["c_theta"][128 * i:128 * (i + 1)], o["c_xy"][i], f"var{i}")


def test_alg1_literal_configuration_255(lib):
    """Alg. 1's own signature: n_xy = 255, n_theta = 733 (direct angle sums), T_theta = 2,
    delta_xy = 0.4, the radial-mean angle score and Alg. 1's own stage 2 (g turned back)."""
    search, _ = lib
    f, g, _ = synth.make_batch("batch255", pairs=3, start=7)
    cfg = search.size_cfg(255, 733, 127, temp_theta=2.0, delta_xy=0.4, angle_score=1, rotate_target=1)
    s = search.PoseSearch([cfg], max_pairs=3)
    o = s.pose(torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda(), want_c_theta=True, want_c_xy=True)
    o = {k: v.cpu().numpy() for k, v in o.items()}
    s.close()
    for i in range(3):
        check_pair(f[i], g[i], cfg, o["pose"][i], o["c_theta"][733 * i:733 * (i + 1)], o["c_xy"][i], f"alg1:{i}")


DP = np.array([[0.9, -0.4, 0.25], [-0.3, 0.6, 0.5], [0.2, 0.1, -0.8]])


# The cases sit away from the bilinear cell edges of the Rotate adjoint's d theta term (reading
# A14; checked on the CPU in test_adjoint_cases_cpu.py): pair 3 of batch511 lies next to one
# (its fp32 d theta term moves by 0.3 % within a few ulps of theta), pair 5 does not.
@pytest.mark.parametrize("name,pairs,start", [("batch127", 3, 3), ("batch255", 2, 3), ("batch511", 1, 5)])
def test_adjoint_parity(lib, name, pairs, start):
    search, _ = lib
    f, g, _ = synth.make_batch(name, pairs=pairs, start=start)
    cfg = cfg_of(search, name)
    s = search.PoseSearch([cfg], max_pairs=pairs)
    df, dg = s.pose_backward(torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda(),
                             torch.from_numpy(DP[:pairs].astype(np.float32)).cuda())
    df, dg = df.cpu().numpy(), dg.cpu().numpy()
    s.close()
    oc = oracle_cfg(cfg)
    for i in range(pairs):
        odf, odg, _ = O.pose_backward(f[i], g[i], oc, DP[i])
        assert grad_err(df[i], odf) <= TOL_GRAD and grad_err(dg[i], odg) <= TOL_GRAD, \
            (name, i, grad_err(df[i], odf), grad_err(dg[i], odg))


def test_adjoint_variants_at_127(lib):
    """Alg. 1's stage 2 (g turned back) and raw scores without a window, odd side."""
    search, _ = lib
    for start, kw in ((31, dict(rotate_target=1, temp_theta=0.5)),
                      (33, dict(score_norm=1, temp_theta=2.0e8, temp_xy=1.0e4, window=0))):
        f, g, _ = synth.make_batch("batch127", pairs=2, start=start)
        cfg = cfg_of(search, "batch127", **kw)
        s = search.PoseSearch([cfg], max_pairs=2)
        df, dg = s.pose_backward(torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda(),
                                 torch.from_numpy(DP[:2].astype(np.float32)).cuda())
        df, dg = df.cpu().numpy(), dg.cpu().numpy()
        s.close()
        for i in range(2):
            odf, odg, _ = O.pose_backward(f[i], g[i], oracle_cfg(cfg), DP[i])
            assert grad_err(df[i], odf) <= TOL_GRAD and grad_err(dg[i], odg) <= TOL_GRAD, (kw, i)


def test_training_call_equals_separate_calls_mixed_odd_and_even(lib):
    """One training call over pairs of 255 and 256 mixed (concurrent size groups) against the
    forward, loss and adjoint as separate calls: bitwise equal; and against the oracle adjoint."""
    search, _ = lib
    a = synth.make_batch("batch255", pairs=2, start=50)
    b = synth.make_batch("batch256", pairs=2, start=50)
    cfgs = [cfg_of(search, "batch255"), cfg_of(search, "batch256")]
    order = [0, 1, 1, 0]
    scans = [(a[0][0], a[1][0], a[2][0]), (b[0][0], b[1][0], b[2][0]), (b[0][1], b[1][1], b[2][1]),
             (a[0][1], a[1][1], a[2][1])]
    offs, cur = [], 0
    for f, _, _ in scans:
        offs.append(cur)
        cur += f.size + (-f.size) % 4   # offsets stay multiples of 4
    F = np.zeros(cur, np.float32)
    G = np.zeros(cur, np.float32)
    for (f, g, _), o in zip(scans, offs):
        F[o:o + f.size] = f.ravel()
        G[o:o + g.size] = g.ravel()
    gt = torch.from_numpy(np.stack([p for _, _, p in scans]).astype(np.float32)).cuda()
    s = search.PoseSearch(cfgs, max_pairs=4)
    Ft, Gt = torch.from_numpy(F).cuda(), torch.from_numpy(G).cuda()
    pose, loss, dpose, df, dg = s.pose_train(Ft, Gt, gt, kind=2, size_idx=order, offsets=offs)
    pose2 = s.pose(Ft, Gt, size_idx=order, offsets=offs)["pose"]
    loss2, dpose2 = s.pose_loss(pose2, gt, kind=2)
    df2, dg2 = s.pose_backward(Ft, Gt, dpose2, size_idx=order, offsets=offs)
    torch.cuda.synchronize()
    assert torch.equal(pose, pose2) and torch.equal(loss, loss2)
    for k, o in enumerate(offs):
        n = cfgs[order[k]]["n"]
        assert torch.equal(df[o:o + n * n], df2[o:o + n * n]) and torch.equal(dg[o:o + n * n], dg2[o:o + n * n])
    f0, g0, _ = scans[0]
    odf, _, _ = O.pose_backward(f0, g0, oracle_cfg(cfgs[0]), dpose.cpu().numpy()[0].astype(np.float64))
    assert grad_err(df[:255 * 255].cpu().numpy().reshape(255, 255), odf) <= TOL_GRAD
    s.close()


def test_odd_side_with_circular_padding_is_refused(lib):
    search, _lib = lib
    with pytest.raises(_lib.FmbymError) as e:
        search.PoseSearch([search.size_cfg(255, 400, 127, pad_mode=1)], max_pairs=1)
    assert e.value.status == _lib.ERR_UNSUPPORTED_SIZE


def test_autotuned_graph_handle_at_255_equals_a_plain_handle(lib):
    """The autotuner (timed training calls of every schedule) and the graph cache at an odd side:
    the tuned, graph-replayed handle's forward and training call against a plain handle's with the
    same schedules, bitwise."""
    search, _lib = lib
    f, g, gt = synth.make_batch("batch255", pairs=6, start=90)
    cfg = cfg_of(search, "batch255")
    tuned = search.PoseSearch([cfg], max_pairs=6, flags=_lib.FLAG_GRAPH | _lib.FLAG_AUTOTUNE)
    plain = search.PoseSearch([cfg], max_pairs=6)
    plain.set_tuning(0, **tuned.tuning(0))
    F, G = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    GT = torch.from_numpy(gt.astype(np.float32)).cuda()
    for _ in range(2):   # the second call replays the captured graphs
        a = tuned.pose(F, G, want_c_xy=True)
        b = plain.pose(F, G, want_c_xy=True)
        ta = tuned.pose_train(F, G, GT, kind=2)
        tb = plain.pose_train(F, G, GT, kind=2)
        torch.cuda.synchronize()
        assert torch.equal(a["pose"], b["pose"]) and torch.equal(a["c_xy"], b["c_xy"])
        assert all(torch.equal(x, y) for x, y in zip(ta, tb))
    tuned.close()
    plain.close()
