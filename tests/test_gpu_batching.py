"""Batching of uneven pairs: concurrent size groups and CUDA-graph replay give the same bits as
direct per-size calls, through the C ABI."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2203_00459_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mod():
    from paper_2203_00459_gb300 import build
    build.build()
    from paper_2203_00459_gb300 import search, _lib
    return search, _lib


CFGS = None


def mixed_batch(search, counts, seed_start=0):
    """Interleaved pairs of the three benchmark sizes, packed back to back (counts per size)."""
    names = ["single128", "batch256", "batch512"]
    cfgs = [search.size_cfg(128, 128, 64), search.size_cfg(256, 400, 128), search.size_cfg(512, 400, 256)]
    order = []
    for s, c in enumerate(counts):
        order += [s] * c
    rng = np.random.default_rng(3)
    rng.shuffle(order)
    F, G, offs, cur = [], [], [], 0
    for k, s in enumerate(order):
        f, g, _ = synth.make_batch(names[s], pairs=1, start=seed_start + k)
        F.append(f.ravel())
        G.append(g.ravel())
        offs.append(cur)
        cur += f.size
    return cfgs, order, offs, np.concatenate(F), np.concatenate(G)


def test_concurrent_groups_match_per_size_calls(mod):
    search, _lib = mod
    cfgs, order, offs, F, G = mixed_batch(search, [5, 4, 3])
    Ft, Gt = torch.from_numpy(F).cuda(), torch.from_numpy(G).cuda()
    s = search.PoseSearch(cfgs, max_pairs=len(order))
    out = s.pose(Ft, Gt, size_idx=order, offsets=offs, want_c_xy=True)
    dp = torch.linspace(-1, 1, 3 * len(order), device="cuda").reshape(-1, 3)
    df, dg = s.pose_backward(Ft, Gt, dp, size_idx=order, offsets=offs)
    torch.cuda.synchronize()
    for si, cfg in enumerate(cfgs):
        idx = [k for k, x in enumerate(order) if x == si]
        n = cfg["n"]
        one = search.PoseSearch([cfg], max_pairs=len(idx))
        f = torch.stack([Ft[offs[k]:offs[k] + n * n].reshape(n, n) for k in idx])
        g = torch.stack([Gt[offs[k]:offs[k] + n * n].reshape(n, n) for k in idx])
        o1 = one.pose(f, g, want_c_xy=True)
        d1f, d1g = one.pose_backward(f, g, dp[idx].contiguous())
        torch.cuda.synchronize()
        assert torch.equal(o1["pose"], out["pose"][idx])
        for j, k in enumerate(idx):
            assert torch.equal(o1["c_xy"][j].ravel(), out["c_xy"][offs[k]:offs[k] + n * n])
            assert torch.equal(d1f[j].ravel(), df[offs[k]:offs[k] + n * n])
            assert torch.equal(d1g[j].ravel(), dg[offs[k]:offs[k] + n * n])
        one.close()
    s.close()


def test_graph_replay_is_bitwise_identical(mod):
    search, _lib = mod
    cfgs, order, offs, F, G = mixed_batch(search, [3, 2, 1], seed_start=50)
    Ft, Gt = torch.from_numpy(F).cuda(), torch.from_numpy(G).cuda()
    direct = search.PoseSearch(cfgs, max_pairs=len(order))
    graph = search.PoseSearch(cfgs, max_pairs=len(order), flags=_lib.FLAG_GRAPH)
    dp = torch.linspace(-1, 1, 3 * len(order), device="cuda").reshape(-1, 3)
    ref = direct.pose(Ft, Gt, size_idx=order, offsets=offs)["pose"]
    rdf, rdg = direct.pose_backward(Ft, Gt, dp, size_idx=order, offsets=offs)
    pose = torch.empty_like(ref)
    for rep in range(3):                      # capture, then replays
        pose.zero_()
        graph.pose(Ft, Gt, size_idx=order, offsets=offs, out=pose)
        df, dg = graph.pose_backward(Ft, Gt, dp, size_idx=order, offsets=offs)
        torch.cuda.synchronize()
        assert torch.equal(pose, ref)
        assert torch.equal(df, rdf) and torch.equal(dg, rdg)
    # new inputs in the same buffers replay the same graph with the new data
    Ft.copy_(Gt)
    graph.pose(Ft, Gt, size_idx=order, offsets=offs, out=pose)
    ref2 = direct.pose(Ft, Gt, size_idx=order, offsets=offs)["pose"]
    torch.cuda.synchronize()
    assert torch.equal(pose, ref2)
    # a different layout (another pair order) captures another graph
    order2 = order[::-1]
    offs2 = offs[::-1]
    p2 = graph.pose(Ft, Gt, size_idx=order2, offsets=offs2)["pose"]
    r2 = direct.pose(Ft, Gt, size_idx=order2, offsets=offs2)["pose"]
    torch.cuda.synchronize()
    assert torch.equal(p2, r2)
    direct.close()
    graph.close()


def test_graph_cache_evicts_and_stays_correct(mod):
    search, _lib = mod
    cfg = search.size_cfg(128, 128, 64)
    f, g, _ = synth.make_batch("single128", pairs=20)
    ft, gt = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    graph = search.PoseSearch([cfg], max_pairs=20, flags=_lib.FLAG_GRAPH)
    direct = search.PoseSearch([cfg], max_pairs=20)
    for b in list(range(1, 20)) + [3, 7, 1]:    # 19 layouts > 16 cached graphs, then revisits
        p = graph.pose(ft[:b], gt[:b])["pose"]
        r = direct.pose(ft[:b], gt[:b])["pose"]
        torch.cuda.synchronize()
        assert torch.equal(p, r), b
    graph.close()
    direct.close()
