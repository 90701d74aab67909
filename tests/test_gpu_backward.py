"""Parity of the CUDA adjoint (fmbym_pose_backward) with the FP64 oracle's hand-derived adjoint and
with FP64 central finite differences of the oracle's forward search, through the C ABI."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2203_00459_gb300 import synth  # noqa: E402
from gpu_util import oracle_cfg  # noqa: E402

pytestmark = pytest.mark.gpu

TOL_GRAD = 1e-3   # max |gpu - reference| / max |reference| per gradient image


@pytest.fixture(scope="module")
def lib():
    from paper_2203_00459_gb300 import build
    build.build()
    from paper_2203_00459_gb300 import search
    return search


def grad_err(a, b):
    return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / max(1e-300, np.max(np.abs(b))))


def gpu_backward(search, cfg, f, g, dpose):
    s = search.PoseSearch([cfg], max_pairs=f.shape[0])
    ft, gt = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    dp = torch.from_numpy(dpose.astype(np.float32)).cuda()
    df, dg = s.pose_backward(ft, gt, dp)
    torch.cuda.synchronize()
    out = df.cpu().numpy(), dg.cpu().numpy()
    s.close()
    return out


def check_against_oracle(cfg, f, g, dpose, df, dg, tag):
    oc = oracle_cfg(cfg)
    for i in range(f.shape[0]):
        odf, odg, _ = O.pose_backward(f[i], g[i], oc, dpose[i])
        ef, eg = grad_err(df[i], odf), grad_err(dg[i], odg)
        assert ef <= TOL_GRAD and eg <= TOL_GRAD, (tag, i, ef, eg)


DP = np.array([[0.8, -0.35, 0.6], [-0.5, 1.0, 0.25], [0.3, 0.2, -0.9], [1.0, 0.0, 0.0], [0.0, 1.0, 1.0]])


@pytest.mark.parametrize("name,pairs", [("single128", 5), ("batch256", 2), ("batch512", 1)])
def test_adjoint_matches_oracle(lib, name, pairs):
    spec = synth.WORKLOADS[name]
    f, g, _ = synth.make_batch(name, pairs=pairs, start=3)
    cfg = lib.size_cfg(spec["n"], spec["n_theta"], spec["n_r"])
    dpose = DP[:pairs]
    df, dg = gpu_backward(lib, cfg, f, g, dpose)
    check_against_oracle(cfg, f, g, dpose, df, dg, name)


def test_adjoint_raw_scores_no_window_ragged_radii(lib):
    f, g, _ = synth.make_batch("batch256", pairs=2)
    cfg = lib.size_cfg(256, 256, 100, temp_theta=2.0e8, temp_xy=1.0e4, window=0, score_norm=1, band_lo=3.5,
                       band_hi=100.0)
    df, dg = gpu_backward(lib, cfg, f, g, DP[:2])
    check_against_oracle(cfg, f, g, DP[:2], df, dg, "raw")


def test_adjoint_circular_padding(lib):
    f, g, _ = synth.make_batch("single128", pairs=2, start=11)
    cfg = lib.size_cfg(128, 128, 64, pad_mode=1, temp_xy=0.5)
    df, dg = gpu_backward(lib, cfg, f, g, DP[:2])
    check_against_oracle(cfg, f, g, DP[:2], df, dg, "circular")


def test_adjoint_matches_central_differences_512(lib):
    """The 512^2 configuration's check: the GPU gradient of an L2 pose loss against FP64 central
    finite differences (h = 1e-4) of the oracle's forward search on 64 random pixels, pixel by
    pixel.  Where |FD| is at least 1e-3 of the image's largest gradient the GPU gradient must lie
    within 1e-3 of FD relative to that pixel's own value (measured on a GB300: at most 1.4e-4);
    below that floor the float32 sums' cancellation sets the error, and the bound is 1e-3 of the
    largest gradient.  The oracle's own adjoint is held to 1e-4 of FD per pixel above the floor
    (measured: at most 1e-6).  The FD loop evaluates the oracle with its FFT route, the same sums
    as its direct route (pinned against each other), to keep 128 evaluations at 512^2 short."""
    spec = synth.WORKLOADS["batch512"]
    f, g, gt = synth.make_batch("batch512", pairs=1, start=5)
    cfg = lib.size_cfg(512, spec["n_theta"], spec["n_r"])
    oc = oracle_cfg(cfg)
    ofd = dict(oc, route="fft")
    f64, g64 = f[0].astype(np.float64), g[0].astype(np.float64)
    r = O.pose(f64, g64, oc)
    pose = np.array([r["theta"], r["tx"], r["ty"]])

    def loss(a, b):
        rr = O.pose(a, b, ofd)
        return float(np.sum((np.array([rr["theta"], rr["tx"], rr["ty"]]) - gt[0]) ** 2))

    dpose = 2.0 * (pose - gt[0])
    df, dg = gpu_backward(lib, cfg, f, g, dpose[None, :])
    odf, odg, _ = O.pose_backward(f64, g64, oc, dpose)
    rng = np.random.default_rng(64)
    h = 1e-4
    scale = max(np.max(np.abs(df[0])), np.max(np.abs(dg[0])))
    floor = 1e-3 * scale
    above = 0
    for k in range(64):
        which = k % 2
        y, x = rng.integers(0, 512, 2)
        a, b = f64.copy(), g64.copy()
        (a if which == 0 else b)[y, x] += h
        lp = loss(a, b)
        (a if which == 0 else b)[y, x] -= 2 * h
        lm = loss(a, b)
        fd = (lp - lm) / (2 * h)
        an = (df if which == 0 else dg)[0, y, x]
        ora = (odf if which == 0 else odg)[y, x]
        assert abs(fd - an) <= TOL_GRAD * scale, (k, which, y, x, fd, an, scale)
        if abs(fd) >= floor:
            above += 1
            assert abs(fd - an) <= 1e-3 * abs(fd), (k, which, y, x, fd, an)
            assert abs(fd - ora) <= 1e-4 * abs(fd), (k, which, y, x, fd, ora)
    assert above >= 48, above   # the per-pixel bound must cover most of the sample


def test_autograd_function_and_determinism(lib):
    from paper_2203_00459_gb300.search import PoseSearch, scan_match
    f, g, gt = synth.make_batch("batch256", pairs=3)
    s = PoseSearch([lib.size_cfg(256, 400, 128)], max_pairs=3)
    ft = torch.from_numpy(f).cuda().requires_grad_(True)
    gtn = torch.from_numpy(g).cuda().requires_grad_(True)
    target = torch.from_numpy(gt.astype(np.float32)).cuda()
    pose = scan_match(ft, gtn, s)
    loss = ((pose - target) ** 2).sum()
    loss.backward()
    dpose = 2.0 * (pose.detach() - target)
    df, dg = s.pose_backward(ft.detach(), gtn.detach(), dpose)
    torch.cuda.synchronize()
    assert torch.equal(ft.grad, df) and torch.equal(gtn.grad, dg)
    df2, dg2 = s.pose_backward(ft.detach(), gtn.detach(), dpose)
    torch.cuda.synchronize()
    assert torch.equal(df, df2) and torch.equal(dg, dg2)
    s.close()


def test_adjoint_mixed_sizes_in_one_call(lib):
    from paper_2203_00459_gb300.search import PoseSearch
    cfgs = [lib.size_cfg(128, 128, 64), lib.size_cfg(256, 400, 128)]
    names = ["single128", "batch256"]
    order = [1, 0, 0]
    scans = [synth.make_batch(names[s], pairs=1, start=20 + k) for k, s in enumerate(order)]
    offs, cur = [], 0
    for f, _, _ in scans:
        offs.append(cur)
        cur += f.size
    F = np.concatenate([f.ravel() for f, _, _ in scans])
    G = np.concatenate([g.ravel() for _, g, _ in scans])
    s = PoseSearch(cfgs, max_pairs=3)
    dp = torch.from_numpy(DP[:3].astype(np.float32)).cuda()
    df, dg = s.pose_backward(torch.from_numpy(F).cuda(), torch.from_numpy(G).cuda(), dp, size_idx=order,
                             offsets=offs)
    torch.cuda.synchronize()
    df, dg = df.cpu().numpy(), dg.cpu().numpy()
    for k, si in enumerate(order):
        n = cfgs[si]["n"]
        f, g, _ = scans[k]
        odf, odg, _ = O.pose_backward(f[0], g[0], oracle_cfg(cfgs[si]), DP[k])
        assert grad_err(df[offs[k]:offs[k] + n * n].reshape(n, n), odf) <= TOL_GRAD
        assert grad_err(dg[offs[k]:offs[k] + n * n].reshape(n, n), odg) <= TOL_GRAD
    s.close()


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("kind", [1, 2])
def test_training_call_equals_separate_calls(lib, graph, kind):
    """fmbym_pose_train (forward, loss, adjoint reading the forward's intermediates) gives the same
    bits as fmbym_pose + fmbym_pose_loss + fmbym_pose_backward (which recomputes the forward), for a
    mixed-size call."""
    from paper_2203_00459_gb300 import _lib
    from paper_2203_00459_gb300.search import PoseSearch
    cfgs = [lib.size_cfg(128, 128, 64), lib.size_cfg(512, 400, 256)]
    names = ["single128", "batch512"]
    order = [1, 0, 1, 0]
    scans = [synth.make_batch(names[s], pairs=1, start=40 + k) for k, s in enumerate(order)]
    offs, cur = [], 0
    for f, _, _ in scans:
        offs.append(cur)
        cur += f.size
    F = torch.from_numpy(np.concatenate([f.ravel() for f, _, _ in scans])).cuda()
    G = torch.from_numpy(np.concatenate([g.ravel() for _, g, _ in scans])).cuda()
    gt = torch.from_numpy(np.concatenate([p for _, _, p in scans]).astype(np.float32)).cuda()
    s = PoseSearch(cfgs, max_pairs=4, flags=_lib.FLAG_GRAPH if graph else 0)
    for _ in range(2):   # the second graph call replays the captured layout
        pose, loss, dpose, df, dg = s.pose_train(F, G, gt, kind=kind, size_idx=order, offsets=offs)
    pose2 = s.pose(F, G, size_idx=order, offsets=offs)["pose"]
    loss2, dpose2 = s.pose_loss(pose2, gt, kind=kind)
    df2, dg2 = s.pose_backward(F, G, dpose2, size_idx=order, offsets=offs)
    torch.cuda.synchronize()
    for a, b in ((pose, pose2), (loss, loss2), (dpose, dpose2), (df, df2), (dg, dg2)):
        assert torch.equal(a, b)
    # and the adjoint matches the oracle's adjoint for the loss gradient the call produced
    if kind == 2:
        k = 0
        n = cfgs[order[k]]["n"]
        f, g, _ = scans[k]
        odf, odg, _ = O.pose_backward(f[0], g[0], oracle_cfg(cfgs[order[k]]), dpose.cpu().numpy()[k].astype(np.float64))
        assert grad_err(df.cpu().numpy()[offs[k]:offs[k] + n * n].reshape(n, n), odf) <= TOL_GRAD
        assert grad_err(dg.cpu().numpy()[offs[k]:offs[k] + n * n].reshape(n, n), odg) <= TOL_GRAD
    s.close()


def test_adjoint_radial_mean_angle_score(lib):
    f, g, _ = synth.make_batch("batch256", pairs=2, start=61)
    cfg = lib.size_cfg(256, 400, 128, temp_theta=2.0, angle_score=1)
    df, dg = gpu_backward(lib, cfg, f, g, DP[:2])
    check_against_oracle(cfg, f, g, DP[:2], df, dg, "marginal")


def test_adjoint_full_circle(lib):
    import math
    pairs = [synth.make_pair(128, 40, 6, math.radians(d), 2.0, 1.0, seed=780, index=i)
             for i, d in enumerate((160.0, -20.0))]
    f = np.stack([a for a, _ in pairs])
    g = np.stack([b for _, b in pairs])
    cfg = lib.size_cfg(128, 128, 64, temp_theta=0.2, full_circle=1)
    df, dg = gpu_backward(lib, cfg, f, g, DP[:2])
    check_against_oracle(cfg, f, g, DP[:2], df, dg, "full_circle")


def test_adjoint_rotate_target_g(lib):
    """The adjoint of Alg. 1's own stage 2 (g turned back by theta, t = R(theta) t') against the
    oracle's, and the training call bitwise equal to the three separate calls under it."""
    import math
    from paper_2203_00459_gb300 import _lib
    from paper_2203_00459_gb300.search import PoseSearch
    pairs = [synth.make_pair(128, 40, 6, math.radians(d), 3.0, -2.0, seed=784, index=i)
             for i, d in enumerate((15.0, -9.0))]
    f = np.stack([a for a, _ in pairs])
    g = np.stack([b for _, b in pairs])
    cfg = lib.size_cfg(128, 128, 64, temp_theta=0.5, rotate_target=1)
    df, dg = gpu_backward(lib, cfg, f, g, DP[:2])
    check_against_oracle(cfg, f, g, DP[:2], df, dg, "rotate_target")
    s = PoseSearch([cfg], max_pairs=2, flags=_lib.FLAG_GRAPH)
    F, G = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    gt = torch.tensor([[0.25, 3.0, -2.0], [-0.15, 3.0, -2.0]], dtype=torch.float32).cuda()
    pose, loss, dpose, dF, dG = s.pose_train(F, G, gt, kind=1)
    pose2 = s.pose(F, G)["pose"]
    loss2, dpose2 = s.pose_loss(pose2, gt, kind=1)
    dF2, dG2 = s.pose_backward(F, G, dpose2)
    torch.cuda.synchronize()
    for a, b in ((pose, pose2), (dpose, dpose2), (dF, dF2), (dG, dG2)):
        assert torch.equal(a, b)
    with pytest.raises(_lib.FmbymError):
        PoseSearch([lib.size_cfg(128, 128, 64, rotate_target=1, full_circle=1)], max_pairs=1)
    s.close()


def test_host_buffer_training_call_equals_the_device_call(lib):
    """fmbym_pose_train_host (host f, g, gt in; host pose, loss, df, dg out) against
    fmbym_pose_train on device buffers of the same handle: bitwise equal, twice in a row."""
    from paper_2203_00459_gb300.search import PoseSearch
    f, g, gt = synth.make_batch("batch256", pairs=4, start=40)
    s = PoseSearch([lib.size_cfg(256, 400, 128)], max_pairs=4)
    F, G = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    GT = torch.from_numpy(gt.astype(np.float32)).cuda()
    pose, loss, _, df, dg = s.pose_train(F, G, GT, kind=2)
    torch.cuda.synchronize()
    fh, gh = torch.from_numpy(f).pin_memory(), torch.from_numpy(g).pin_memory()
    gth = torch.from_numpy(gt.astype(np.float32)).pin_memory()
    for _ in range(2):
        ph, lh, dfh, dgh = s.pose_train_host(fh, gh, gth, kind=2)
        assert torch.equal(ph, pose.cpu()) and torch.equal(lh, loss.cpu())
        assert torch.equal(dfh, df.cpu()) and torch.equal(dgh, dg.cpu())
    s.close()


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("sizes", [(0,) * 24, (0, 1) * 8])
def test_pipelined_host_buffer_training_call(lib, sizes, graph):
    """Packed calls of 16 pairs or more run the host-buffer training call as a pipeline of chunks
    (copies in and out on their own streams, overlapping the chunks' training calls; with one size,
    alternate chunks on a second stream in the workspace's second slot); pose, loss, df and dg must
    be bitwise those of fmbym_pose_train on device buffers, also with mixed sizes, launched directly
    or from captured graphs."""
    from paper_2203_00459_gb300 import _lib
    from paper_2203_00459_gb300.search import PoseSearch
    cfgs = [lib.size_cfg(128, 128, 64), lib.size_cfg(256, 400, 128)]
    names = ["single128", "batch256"]
    scans = [synth.make_batch(names[s], pairs=1, start=70 + k) for k, s in enumerate(sizes)]
    F = np.concatenate([f.ravel() for f, _, _ in scans])
    G = np.concatenate([g.ravel() for _, g, _ in scans])
    GT = np.concatenate([p for _, _, p in scans]).astype(np.float32)
    s = PoseSearch(cfgs, max_pairs=len(sizes), flags=_lib.FLAG_GRAPH if graph else 0)
    si = list(sizes)
    pose, loss, _, df, dg = s.pose_train(torch.from_numpy(F).cuda(), torch.from_numpy(G).cuda(),
                                         torch.from_numpy(GT).cuda(), kind=2, size_idx=si)
    torch.cuda.synchronize()
    fh, gh, gth = torch.from_numpy(F).pin_memory(), torch.from_numpy(G).pin_memory(), torch.from_numpy(GT).pin_memory()
    for _ in range(3):
        ph, lh, dfh, dgh = s.pose_train_host(fh, gh, gth, kind=2, size_idx=si)
        assert torch.equal(ph, pose.cpu()) and torch.equal(lh, loss.cpu())
        assert torch.equal(dfh, df.cpu()) and torch.equal(dgh, dg.cpu())
    s.close()
