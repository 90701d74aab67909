"""A packed call of one size and 16 or more pairs runs as two halves on two streams, each in its own
half of the workspace.  Its results must be, bit for bit, those of the same pairs in one piece (the
same call with explicit offsets keeps one grid over all pairs): pose, both score surfaces, the
adjoint, and the training call's loss and gradients, for an odd pair count (halves of 8 and 9),
launched directly and from captured graphs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2203_00459_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2203_00459_gb300 import build
    build.build()
    from paper_2203_00459_gb300 import _lib, search
    return _lib, search


@pytest.mark.parametrize("graph", [False, True])
def test_two_halves_equal_one_piece(lib, graph):
    _lib, search = lib
    B, n = 17, 128
    f, g, gt = synth.make_batch("batch127", pairs=B, spec=dict(synth.WORKLOADS["batch127"], n=n, pairs=B))
    cfg = search.size_cfg(n, 128, 64)
    s = search.PoseSearch([cfg], max_pairs=B, flags=_lib.FLAG_GRAPH if graph else 0)
    F, G = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    GT = torch.from_numpy(gt.astype(np.float32)).cuda()
    DP = torch.from_numpy(np.random.default_rng(3).normal(size=(B, 3)).astype(np.float32)).cuda()
    offs = np.arange(B, dtype=np.int64) * n * n
    for _ in range(2):
        a = s.pose(F, G, want_c_theta=True, want_c_xy=True)
        b = s.pose(F, G, offsets=offs, want_c_theta=True, want_c_xy=True)
        da = s.pose_backward(F, G, DP)
        db = s.pose_backward(F, G, DP, offsets=offs)
        ta = s.pose_train(F, G, GT, kind=1)
        tb = s.pose_train(F, G, GT, kind=1, offsets=offs)
        torch.cuda.synchronize()
        for k in ("pose", "c_theta", "c_xy"):
            assert torch.equal(a[k], b[k]), k
        assert torch.equal(da[0], db[0]) and torch.equal(da[1], db[1])
        for x, y, name in zip(ta, tb, ("pose", "loss", "dpose", "df", "dg")):
            assert torch.equal(x, y), name
    s.close()
