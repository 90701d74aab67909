"""Parity of the CUDA forward search with the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2203_00459_gb300 import synth  # noqa: E402
from gpu_util import check_pair, surf_err, TOL_THETA  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2203_00459_gb300 import build
    build.build()
    from paper_2203_00459_gb300 import search
    return search


def run(search, cfg, f, g, **kw):
    s = search.PoseSearch([cfg], max_pairs=max(1, f.shape[0]))
    ft, gt = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    out = s.pose(ft, gt, want_c_theta=True, want_c_xy=True, **kw)
    torch.cuda.synchronize()
    res = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
    s.close()
    return res


def test_single_pair_128(lib):
    f, g, _ = synth.make_batch("single128", pairs=1)
    cfg = lib.size_cfg(128, 128, 64)
    o = run(lib, cfg, f, g)
    check_pair(f[0], g[0], cfg, o["pose"][0], o["c_theta"], o["c_xy"][0], "single128")


def test_batch_128_grid_aligned_bins(lib):
    f, g, gt = synth.make_batch("single128", pairs=7)
    cfg = lib.size_cfg(128, 128, 64)
    o = run(lib, cfg, f, g)
    for i in range(7):
        check_pair(f[i], g[i], cfg, o["pose"][i], o["c_theta"][128 * i:128 * (i + 1)], o["c_xy"][i], f"p{i}")
        assert int(np.argmax(o["c_theta"][128 * i:128 * (i + 1)])) - 64 == int(round(gt[i, 0] / (np.pi / 128)))


@pytest.mark.parametrize("name,pairs", [("batch256", 5), ("batch512", 3)])
def test_small_batches_256_512(lib, name, pairs):
    spec = synth.WORKLOADS[name]
    f, g, _ = synth.make_batch(name, pairs=pairs)
    cfg = lib.size_cfg(spec["n"], spec["n_theta"], spec["n_r"])
    o = run(lib, cfg, f, g)
    nt = spec["n_theta"]
    for i in range(pairs):
        check_pair(f[i], g[i], cfg, o["pose"][i], o["c_theta"][nt * i:nt * (i + 1)], o["c_xy"][i], f"{name}:{i}")


def test_ragged_radii_raw_scores_no_window(lib):
    """n_r = 100 leaves a partial chunk of radii; raw scores and no window exercise the switches."""
    f, g, _ = synth.make_batch("batch256", pairs=2)
    cfg = lib.size_cfg(256, 256, 100, temp_theta=2.0e8, temp_xy=1.0e4, window=0, score_norm=1, band_lo=3.5,
                       band_hi=100.0)
    o = run(lib, cfg, f, g)
    for i in range(2):
        check_pair(f[i], g[i], cfg, o["pose"][i], o["c_theta"][256 * i:256 * (i + 1)], o["c_xy"][i], f"raw{i}")


def test_circular_integer_shift_is_exact(lib):
    rng = np.random.default_rng(5)
    n = 128
    f = rng.random((3, n, n)).astype(np.float32)
    shifts = [(3, -5), (-4, 4), (0, 0)]
    g = np.stack([np.roll(f[i], s, axis=(0, 1)) for i, s in enumerate(shifts)])
    cfg = lib.size_cfg(n, 128, 64, pad_mode=1, temp_xy=0.05)
    o = run(lib, cfg, f, g)
    for i, (ty, tx) in enumerate(shifts):
        check_pair(f[i], g[i], cfg, o["pose"][i], None, o["c_xy"][i], f"circ{i}")


def test_mixed_sizes_in_one_call_with_offsets(lib):
    """Pairs of three sizes interleaved in one call, packed with explicit offsets and a gap."""
    from paper_2203_00459_gb300.search import PoseSearch
    names = ["single128", "batch256", "batch512"]
    cfgs = [lib.size_cfg(128, 128, 64), lib.size_cfg(256, 400, 128), lib.size_cfg(512, 400, 256)]
    order = [1, 0, 2, 0, 1]
    scans = []
    for k, s in enumerate(order):
        f, g, _ = synth.make_batch(names[s], pairs=1, start=k)
        scans.append((f[0], g[0]))
    offs, cur = [], 0
    for (f, _) in scans:
        offs.append(cur)
        cur += f.size + 64
    F = np.zeros(cur, np.float32)
    G = np.zeros(cur, np.float32)
    for o_, (f, g) in zip(offs, scans):
        F[o_:o_ + f.size] = f.ravel()
        G[o_:o_ + g.size] = g.ravel()
    s = PoseSearch(cfgs, max_pairs=8)
    Ft, Gt = torch.from_numpy(F).cuda(), torch.from_numpy(G).cuda()
    out = s.pose(Ft, Gt, size_idx=order, offsets=offs, want_c_theta=True, want_c_xy=True)
    torch.cuda.synchronize()
    pose = out["pose"].cpu().numpy()
    ct = out["c_theta"].cpu().numpy()
    cxy = out["c_xy"].cpu().numpy()
    ct_off = 0
    for k, sidx in enumerate(order):
        n, nt = cfgs[sidx]["n"], cfgs[sidx]["n_theta"]
        f, g = scans[k]
        check_pair(f, g, cfgs[sidx], pose[k], ct[ct_off:ct_off + nt], cxy[offs[k]:offs[k] + n * n].reshape(n, n),
                   f"mixed{k}")
        ct_off += nt
    # host-buffer entry point gives the same poses
    ph = s.pose_host(torch.from_numpy(F).pin_memory(), torch.from_numpy(G).pin_memory(), size_idx=order,
                     offsets=offs).numpy()
    assert np.max(np.abs(ph - pose)) == 0.0
    s.close()


@pytest.mark.parametrize("name,sample", [("batch256", [0, 77, 255]), ("batch512", [0, 13, 31])])
def test_full_size_batches_sampled(lib, name, sample):
    """The full benchmark batches in one call (the launch configuration the benchmark times);
    sampled pairs are checked against the oracle, every pair for finite, in-range poses."""
    spec = synth.WORKLOADS[name]
    f, g, _ = synth.make_batch(name)
    cfg = lib.size_cfg(spec["n"], spec["n_theta"], spec["n_r"])
    o = run(lib, cfg, f, g)
    nt, n = spec["n_theta"], spec["n"]
    assert np.all(np.isfinite(o["pose"]))
    assert np.all(np.abs(o["pose"][:, 0]) <= np.pi / 2 + TOL_THETA)
    assert np.all(np.abs(o["pose"][:, 1:]) <= n / 2)
    for i in sample:
        check_pair(f[i], g[i], cfg, o["pose"][i], o["c_theta"][nt * i:nt * (i + 1)], o["c_xy"][i], f"{name}:{i}")


def test_repeat_calls_are_deterministic(lib):
    from paper_2203_00459_gb300.search import PoseSearch
    f, g, _ = synth.make_batch("batch256", pairs=4)
    s = PoseSearch([lib.size_cfg(256, 400, 128)], max_pairs=4)
    ft, gt = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    a = s.pose(ft, gt, want_c_xy=True)
    b = s.pose(ft, gt, want_c_xy=True)
    torch.cuda.synchronize()
    assert torch.equal(a["pose"], b["pose"]) and torch.equal(a["c_xy"], b["c_xy"])
    s.close()


def test_empty_batch_and_errors(lib):
    from paper_2203_00459_gb300 import _lib
    from paper_2203_00459_gb300.search import PoseSearch
    s = PoseSearch([lib.size_cfg(128, 128, 64)], max_pairs=2)
    e = torch.empty((0, 128, 128), device="cuda")
    assert s.pose(e, e)["pose"].shape == (0, 3)
    big = torch.zeros((3, 128, 128), device="cuda")
    with pytest.raises(_lib.FmbymError) as ei:
        s.pose(big, big)
    assert ei.value.status == _lib.ERR_WORKSPACE
    flat = torch.zeros(2 * 128 * 128 + 8, device="cuda")
    with pytest.raises(_lib.FmbymError) as ei:
        s.pose(flat, flat, size_idx=[0, 0], offsets=[0, 128 * 128 + 2])
    assert ei.value.status == _lib.ERR_INVALID_ARG
    s.close()


@pytest.mark.parametrize("name,n,nt,nr,score_norm,temp", [("batch256", 256, 400, 128, 0, 2.0),
                                                          ("single128", 128, 128, 50, 1, 1.0e7)])
def test_radial_mean_angle_score(lib, name, n, nt, nr, score_norm, temp):
    """The angle score Alg. 1 prints (mean over radial lags of the 2D polar correlation) with the
    T_theta = 2 of Alg. 1 (z-scores), and with raw scores and a ragged chunk of radii."""
    f, g, _ = synth.make_batch(name, pairs=2, start=60)
    cfg = lib.size_cfg(n, nt, nr, temp_theta=temp, score_norm=score_norm, angle_score=1,
                       temp_xy=1.0 if score_norm == 0 else 1.0e4)
    o = run(lib, cfg, f, g)
    for i in range(2):
        check_pair(f[i], g[i], cfg, o["pose"][i], o["c_theta"][nt * i:nt * (i + 1)], o["c_xy"][i], f"marg{i}")


@pytest.mark.parametrize("n,nt,nr", [(128, 128, 64), (256, 400, 128)])
def test_full_circle_heading(lib, n, nt, nr):
    """Headings beyond a quarter turn: stage 2 at theta and theta + pi, the higher peak kept."""
    import math
    degs = [170.0, -125.0, 12.0]
    pairs = [synth.make_pair(n, n * n // 300, n // 16, math.radians(d), 3.0, -2.0, seed=779, index=i)
             for i, d in enumerate(degs)]
    f = np.stack([a for a, _ in pairs])
    g = np.stack([b for _, b in pairs])
    cfg = lib.size_cfg(n, nt, nr, temp_theta=0.2, full_circle=1)
    o = run(lib, cfg, f, g)
    for i in range(len(degs)):
        check_pair(f[i], g[i], cfg, o["pose"][i], o["c_theta"][nt * i:nt * (i + 1)], o["c_xy"][i], f"fc{i}")
        err = (o["pose"][i][0] - math.radians(degs[i]) + math.pi) % (2 * math.pi) - math.pi
        assert abs(err) < math.radians(1.5), (degs[i], o["pose"][i])


@pytest.mark.parametrize("n,nt,nr", [(128, 128, 64), (256, 400, 128)])
def test_rotate_target_g(lib, n, nt, nr):
    """Alg. 1's own stage 2 (rotate_target 1): g turned back by theta, f correlated with it, and
    t = R(theta) t'; the scores and the pose against the oracle's, and the pose against the truth."""
    import math
    poses = [(20.0, 6.0, -3.0), (-14.0, -4.0, 5.0), (3.0, 2.0, 1.0)]
    pairs = [synth.make_pair(n, n * n // 300, n // 16, math.radians(d), tx, ty, seed=783, index=i)
             for i, (d, tx, ty) in enumerate(poses)]
    f = np.stack([a for a, _ in pairs])
    g = np.stack([b for _, b in pairs])
    cfg = lib.size_cfg(n, nt, nr, temp_theta=0.2, rotate_target=1)
    o = run(lib, cfg, f, g)
    for i, (d, tx, ty) in enumerate(poses):
        check_pair(f[i], g[i], cfg, o["pose"][i], o["c_theta"][nt * i:nt * (i + 1)], o["c_xy"][i], f"rg{i}")
        assert abs(o["pose"][i][0] - math.radians(d)) < math.radians(1.0)
        assert abs(o["pose"][i][1] - tx) < 0.5 and abs(o["pose"][i][2] - ty) < 0.5, (poses[i], o["pose"][i])
