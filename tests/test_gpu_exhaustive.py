"""Parity of the CUDA exhaustive rotate-then-correlate search (the comparison method of Tab. IIIa)
with the FP64 oracle's, through the C ABI: the same winning candidate, its correlation peaks, and
its translation."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2203_00459_gb300 import synth  # noqa: E402
from gpu_util import TOL_T, argmax_ok, oracle_cfg  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def search():
    from paper_2203_00459_gb300 import build
    build.build()
    from paper_2203_00459_gb300 import search as s
    return s


@pytest.mark.parametrize("name,n,nt,nr,pairs", [("single128", 128, 128, 64, 3), ("batch256", 256, 400, 128, 2),
                                                 ("batch127", 127, 128, 63, 2)])   # 127: an odd side
def test_exhaustive_matches_oracle(search, name, n, nt, nr, pairs):
    cfg = search.size_cfg(n, nt, nr)
    f, g, gt = synth.make_batch(name, pairs=pairs, start=7)
    angles = np.radians(np.arange(-12, 13, 1.0)).astype(np.float32)
    s = search.PoseSearch([cfg], max_pairs=pairs)
    out = s.pose_exhaustive(torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda(), angles, want_peaks=True)
    torch.cuda.synchronize()
    pose, peaks = out["pose"].cpu().numpy(), out["peaks"].cpu().numpy()
    s.close()
    oc = oracle_cfg(cfg)
    for i in range(pairs):
        r = O.pose_exhaustive(f[i].astype(np.float64), g[i].astype(np.float64), oc, angles.astype(np.float64))
        assert np.max(np.abs(peaks[i] - r["peaks"])) <= 1e-4 * np.max(np.abs(r["peaks"])), (name, i)
        assert argmax_ok(peaks[i], r["peaks"]), (name, i)
        if int(np.argmax(peaks[i])) == r["k"]:
            assert pose[i, 0] == np.float32(angles[r["k"]])
            assert abs(pose[i, 1] - r["tx"]) <= TOL_T and abs(pose[i, 2] - r["ty"]) <= TOL_T, (name, i)
        # a 1-degree grid finds the heading to within a step
        assert abs(pose[i, 0] - gt[i, 0]) <= np.radians(1.0) + 1e-6


def test_exhaustive_rejects_bad_arguments(search):
    from paper_2203_00459_gb300 import _lib
    s = search.PoseSearch([search.size_cfg(128, 128, 64)], max_pairs=1)
    f = torch.zeros((1, 128, 128), device="cuda")
    with pytest.raises(_lib.FmbymError):
        s.pose_exhaustive(f, f, np.zeros(0, np.float32))
    with pytest.raises(ValueError):    # the binding refuses a size index the handle lacks
        s.pose_exhaustive(f, f, np.zeros(3, np.float32), size=1)
    import ctypes
    ang = np.zeros(3, np.float32)
    pose = torch.empty((1, 3), device="cuda")
    st = _lib.lib().fmbym_pose_exhaustive(s.handle, None, 1, 1, None, ctypes.c_void_p(f.data_ptr()),
                                          ctypes.c_void_p(f.data_ptr()), 3, ang.ctypes.data_as(ctypes.c_void_p),
                                          ctypes.c_void_p(pose.data_ptr()), None)
    assert st == _lib.ERR_INVALID_ARG   # and so does the library
    f2 = torch.zeros((2, 128, 128), device="cuda")
    with pytest.raises(_lib.FmbymError):
        s.pose_exhaustive(f2, f2, np.zeros(3, np.float32))
    s.close()
    # the comparator rotates the source; Alg. 1's g-rotating stage 2 is refused there
    s = search.PoseSearch([search.size_cfg(128, 128, 64, rotate_target=1)], max_pairs=1)
    with pytest.raises(_lib.FmbymError):
        s.pose_exhaustive(f, f, np.zeros(3, np.float32))
    s.close()
