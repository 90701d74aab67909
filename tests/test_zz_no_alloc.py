"""The allocation-free entry point fmbym_pose_noalloc against fmbym_pose.

Callers that may not allocate device memory (a plug-in whose host framework owns every device
allocation, a real-time process with a device-memory budget fixed at start-up) use
fmbym_pose_noalloc, whose scratch is a static array inside the library.  Its results must match
the handle-based fmbym_pose on the same inputs, call after call, since the array keeps the last
call's contents.  This file is collected last so that a run that stops at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2203_00459_gb300 import synth  # noqa: E402
from gpu_util import TOL_SURF, TOL_T, TOL_THETA, surf_err  # noqa: E402

pytestmark = pytest.mark.gpu


def _entry():
    from paper_2203_00459_gb300 import build, _lib
    build.build()
    L = _lib.lib()
    fn = L.fmbym_pose_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.POINTER(_lib.SizeCfg), ctypes.c_int] + [ctypes.c_void_p] * 5
    L.fmbym_noalloc_last_error.restype = ctypes.c_char_p
    L.fmbym_noalloc_capacity.restype = ctypes.c_ulonglong
    return L, fn, _lib


def _noalloc(fn, _lib, cfg, f, g):
    b, n = f.shape[0], f.shape[1]
    pose = torch.full((b, 3), float("nan"), device="cuda")
    ct = torch.full((b * cfg["n_theta"],), float("nan"), device="cuda")
    cxy = torch.full_like(f, float("nan"))
    c = _lib.SizeCfg(**cfg)
    st = fn(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), ctypes.byref(c), b, f.data_ptr(),
            g.data_ptr(), pose.data_ptr(), ct.data_ptr(), cxy.data_ptr())
    torch.cuda.synchronize()
    return st, pose.cpu().numpy(), ct.cpu().numpy(), cxy.cpu().numpy()


def _reference(cfg, f, g):
    from paper_2203_00459_gb300.search import PoseSearch
    s = PoseSearch([cfg], max_pairs=f.shape[0])
    out = s.pose(f, g, want_c_theta=True, want_c_xy=True)
    torch.cuda.synchronize()
    r = (out["pose"].cpu().numpy(), out["c_theta"].cpu().numpy(), out["c_xy"].cpu().numpy())
    s.close()
    return r


def _compare(a, b, nt):
    pa, ca, xa = a
    pb, cb, xb = b
    assert np.max(np.abs(pa[:, 0] - pb[:, 0])) <= TOL_THETA
    assert np.max(np.abs(pa[:, 1:] - pb[:, 1:])) <= TOL_T
    for i in range(pa.shape[0]):
        assert surf_err(ca[i * nt:(i + 1) * nt], cb[i * nt:(i + 1) * nt].astype(np.float64)) <= TOL_SURF
        assert surf_err(xa[i], xb[i].astype(np.float64)) <= TOL_SURF


def test_noalloc_matches_fmbym_pose_on_consecutive_calls():
    L, fn, _lib = _entry()
    from paper_2203_00459_gb300.search import size_cfg
    runs = [("batch256", size_cfg(256, 400, 128), 3),
            ("single128", size_cfg(128, 128, 64, temp_xy=0.5), 5),
            ("batch256", size_cfg(256, 400, 128), 2)]
    for name, cfg, b in runs:
        f, g, _ = synth.make_batch(name, pairs=b, start=7)
        ft, gt = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
        st, pose, ct, cxy = _noalloc(fn, _lib, cfg, ft, gt)
        assert st == 0, L.fmbym_noalloc_last_error()
        _compare((pose, ct, cxy), _reference(cfg, ft, gt), cfg["n_theta"])


def test_noalloc_rejects_requests_beyond_its_array():
    L, fn, _lib = _entry()
    from paper_2203_00459_gb300.search import size_cfg
    assert L.fmbym_noalloc_capacity() == 16 << 20
    f = torch.zeros((2, 512, 512), device="cuda")
    st, *_ = _noalloc(fn, _lib, size_cfg(512, 400, 256), f, f)
    assert st == _lib.ERR_WORKSPACE
    assert b"bytes" in L.fmbym_noalloc_last_error()
