"""CPU-side checks of the CUDA library: it builds for sm_103a, loads, exports every entry point
that include/fmbym.h declares, and rejects bad configurations before touching the GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2203_00459_gb300 import build, _lib
    build.build()
    return _lib.lib()


def declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(fmbym_\w+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(L):
    names = declared_symbols()
    assert "fmbym_pose" in names and "fmbym_create" in names
    for n in names:
        assert hasattr(L, n), n


def test_version(L):
    assert L.fmbym_version() >= 10000


def _create(L, **over):
    from paper_2203_00459_gb300 import _lib
    from paper_2203_00459_gb300.search import size_cfg
    c = size_cfg(128, 128, 64)
    c.update(over)
    arr = (_lib.SizeCfg * 1)(_lib.SizeCfg(**c))
    cfg = _lib.Config(1, arr, 4, 0)
    h = ctypes.c_void_p()
    st = L.fmbym_create(ctypes.byref(h), ctypes.byref(cfg))
    return st, h, L.fmbym_last_error(None).decode()


@pytest.mark.parametrize("over,status", [
    (dict(n=100), 2), (dict(n=1024), 2), (dict(n_theta=7), 2), (dict(n_theta=1025), 2), (dict(n_r=0), 1), (dict(n_r=65), 1),
    (dict(temp_theta=0.0), 1), (dict(delta_xy=-1.0), 1), (dict(pad_mode=2), 1), (dict(score_norm=3), 1),
    (dict(window=7), 1), (dict(band_lo=5.0, band_hi=4.0), 1)])
def test_create_rejects_bad_sizes_before_any_cuda_call(L, over, status):
    st, h, msg = _create(L, **over)
    assert st == status and not h.value and msg


def test_null_arguments(L):
    assert L.fmbym_create(None, None) == 1
    h = ctypes.c_void_p()
    assert L.fmbym_create(ctypes.byref(h), None) == 1
    assert L.fmbym_pose(None, None, 1, None, None, None, None, None, None, None) == 1
    assert L.fmbym_pose_backward(None, None, 1, None, None, None, None, None, None, None) == 1
    L.fmbym_destroy(None)


def test_polar_to_cartesian_validates_before_any_cuda_call(L):
    f = L.fmbym_polar_to_cartesian
    good = dict(n_scans=1, n_az=400, n_range=3768, res=0.0438, n=256, dxy=0.4)
    def call(**kw):
        a = dict(good, **kw)
        return f(None, a["n_scans"], ctypes.c_void_p(16), a["n_az"], a["n_range"], a["res"], a["n"], a["dxy"],
                 ctypes.c_void_p(16))
    for bad in (dict(n_scans=-1), dict(n_az=0), dict(n_range=0), dict(res=0.0), dict(res=float("nan")), dict(n=0),
                dict(n=16385), dict(dxy=-0.4)):
        assert call(**bad) == 1, bad
    assert f(None, 1, None, 400, 3768, 0.0438, 256, 0.4, None) == 1          # NULL buffers
    assert f(None, 0, None, 400, 3768, 0.0438, 256, 0.4, None) == 0          # nothing to do


@pytest.mark.parametrize("n_theta,status", [(733, 2), (129, 2), (7, 2)])
def test_noalloc_keeps_the_fft_angle_counts(L, n_theta, status):
    """The allocation-free entry point takes only the angle counts with an FFT plan; the direct
    sums of other counts need the handle's workspace.  Rejected before any CUDA call."""
    from paper_2203_00459_gb300 import _lib
    from paper_2203_00459_gb300.search import size_cfg
    c = _lib.SizeCfg(**size_cfg(256, n_theta, 128))
    st = L.fmbym_pose_noalloc(None, ctypes.byref(c), 1, ctypes.c_void_p(16), ctypes.c_void_p(16),
                              ctypes.c_void_p(16), None, None)
    assert st == status and L.fmbym_noalloc_last_error().decode()


@pytest.mark.parametrize("n,n_theta,n_r,most", [(512, 400, 256, 1), (256, 400, 128, 6), (128, 128, 64, 29)])
def test_noalloc_limit_of_the_static_array(L, n, n_theta, n_r, most):
    """The pair counts the header states for the 16 MiB array with the benchmark grids: one more
    pair is FMBYM_ERR_WORKSPACE, decided on the host before any CUDA call (without a GPU the
    request that fits stops later, at the first CUDA call)."""
    from paper_2203_00459_gb300 import _lib
    from paper_2203_00459_gb300.search import size_cfg
    c = _lib.SizeCfg(**size_cfg(n, n_theta, n_r))
    p = ctypes.c_void_p(16)
    assert L.fmbym_pose_noalloc(None, ctypes.byref(c), most + 1, p, p, p, None, None) == _lib.ERR_WORKSPACE
    assert L.fmbym_pose_noalloc(None, ctypes.byref(c), most, p, p, p, None, None) != _lib.ERR_WORKSPACE


def test_polar_wrapper_rejects_host_tensors():
    torch = pytest.importorskip("torch")
    from paper_2203_00459_gb300.search import polar_to_cartesian
    with pytest.raises(ValueError):
        polar_to_cartesian(torch.zeros((1, 400, 100)), 64, 0.4, 0.0438)
    with pytest.raises(ValueError):
        polar_to_cartesian(torch.zeros((1, 400, 100), dtype=torch.float64), 64, 0.4, 0.0438)
