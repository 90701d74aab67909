"""The Python binding rejects buffers the kernels cannot use before it makes any library call:
host tensors, other dtypes, strided views, another device, wrong shapes, pairs reaching past the
end of the scans.  A host pointer reaching a kernel would be an illegal access on the GPU; a float64
or strided buffer would be read as garbage.  Runs without a GPU: the library is replaced by a stub
that fails the test on any call."""
import ctypes

import pytest
import torch

from paper_2203_00459_gb300 import _lib, search
from paper_2203_00459_gb300.search import PoseSearch, check_device_tensor, check_host_tensor, size_cfg


class _NoLibrary:
    def __getattr__(self, name):
        raise AssertionError(f"library call {name} made before the arguments were checked")


@pytest.fixture()
def handle(monkeypatch):
    monkeypatch.setattr(_lib, "lib", lambda: _NoLibrary())
    s = PoseSearch.__new__(PoseSearch)
    s.sizes = [size_cfg(128, 128, 64), size_cfg(256, 400, 128)]
    s.max_pairs = 4
    s.flags = 0
    s.device = torch.device("cuda", 0)
    s._h = ctypes.c_void_p(1)
    yield s
    s._h = None


class _FakeCuda(torch.Tensor):
    """A CPU tensor that reports itself as living on a CUDA device, to reach the checks that
    follow the device-type check without a GPU."""
    fake_device = torch.device("cuda", 0)

    @property
    def is_cuda(self):
        return True

    @property
    def device(self):
        return self.fake_device


def fake(t, device=0):
    x = torch.Tensor._make_subclass(_FakeCuda, t)
    x.fake_device = torch.device("cuda", device)
    return x


def test_host_tensors_are_rejected_by_every_device_call(handle):
    f = torch.zeros(2, 128, 128)
    p = torch.zeros(2, 3)
    with pytest.raises(ValueError, match="CUDA"):
        handle.pose(f, f)
    with pytest.raises(ValueError, match="CUDA"):
        handle.pose_backward(f, f, p)
    with pytest.raises(ValueError, match="CUDA"):
        handle.pose_train(f, f, p)
    with pytest.raises(ValueError, match="CUDA"):
        handle.pose_loss(p, p)
    with pytest.raises(ValueError, match="CUDA"):
        handle.pose_exhaustive(f, f, [0.0])
    with pytest.raises(TypeError):
        handle.pose(f.numpy(), f.numpy())


def test_a_host_dpose_or_gt_is_rejected_after_valid_scans(handle):
    f = fake(torch.zeros(2, 128, 128))
    with pytest.raises(ValueError, match="dpose must be a CUDA"):
        handle.pose_backward(f, f, torch.zeros(2, 3))
    with pytest.raises(ValueError, match="gt must be a CUDA"):
        handle.pose_train(f, f, torch.zeros(2, 3))
    with pytest.raises(ValueError, match="out must be a CUDA"):
        handle.pose(f, f, out=torch.zeros(2, 3))


@pytest.mark.parametrize("bad,msg", [
    (lambda: fake(torch.zeros(2, 128, 128, dtype=torch.float64)), "float32"),
    (lambda: fake(torch.zeros(2, 128, 256)[:, :, ::2]), "contiguous"),
    (lambda: fake(torch.zeros(2, 128, 128), device=1), "handle on"),
    (lambda: fake(torch.zeros(2, 64, 64)), "scan size"),
])
def test_wrong_scan_buffers_are_rejected(handle, bad, msg):
    good = fake(torch.zeros(2, 128, 128))
    with pytest.raises(ValueError, match=msg):
        handle.pose(bad(), bad())
    if msg != "scan size":
        with pytest.raises(ValueError, match=msg):
            handle.pose(good, bad())


def test_shapes_and_extents_are_checked(handle):
    f = fake(torch.zeros(2, 128, 128))
    with pytest.raises(ValueError, match="shape"):
        handle.pose(f, fake(torch.zeros(3, 128, 128)))
    with pytest.raises(ValueError, match="shape"):
        handle.pose_backward(f, f, fake(torch.zeros(3, 3)))
    with pytest.raises(ValueError, match="shape"):
        handle.pose_train(f, f, fake(torch.zeros(2, 3)), out=(fake(torch.zeros(2, 3)),) * 5)
    flat = fake(torch.zeros(128 * 128 + 256 * 256 - 4))
    with pytest.raises(ValueError, match="beyond"):   # packed 128^2 + 256^2 needs 4 more elements
        handle.pose(flat, flat, size_idx=[0, 1])
    with pytest.raises(ValueError, match="beyond"):
        handle.pose(flat, flat, size_idx=[0], offsets=[128 * 128 * 4])
    with pytest.raises(ValueError, match="size_idx"):
        handle.pose(flat, flat, size_idx=[-1])
    with pytest.raises(ValueError, match="size_idx"):
        handle.pose(flat, flat, size_idx=[2])
    with pytest.raises(ValueError, match="one entry per pair"):
        handle.pose(flat, flat, size_idx=[0, 0], offsets=[0])
    with pytest.raises(ValueError, match="beyond"):
        handle.pose_exhaustive(f, f, [0.0], offsets=[128 * 128 * 2])


def test_host_buffers_of_the_host_entry_point(handle):
    with pytest.raises(ValueError, match="float32"):
        handle.pose_host(torch.zeros(1, 128, 128, dtype=torch.float64), torch.zeros(1, 128, 128))
    with pytest.raises(ValueError, match="contiguous"):
        handle.pose_host(torch.zeros(1, 128, 256)[:, :, ::2], torch.zeros(1, 128, 128))
    with pytest.raises(ValueError, match="CPU"):
        handle.pose_host(fake(torch.zeros(1, 128, 128)), torch.zeros(1, 128, 128))
    with pytest.raises(ValueError, match="elements"):
        handle.pose_host(torch.zeros(1, 128, 128), torch.zeros(2, 128, 128))


def test_checks_accept_good_buffers():
    t = fake(torch.zeros(4, 3))
    assert check_device_tensor(t, "t", torch.device("cuda", 0), shape=(4, 3)) is t
    h = torch.zeros(5)
    assert check_host_tensor(h, "h", numel=5) is h
    assert search.check_device_tensor is check_device_tensor


def test_offsets_without_size_idx_place_pairs_of_size_0(handle):
    """Offsets given without size_idx are honoured (pairs of the handle's first size), not dropped."""
    f = torch.zeros((3, 128, 128))
    n_pairs, si, off, nts, ns = handle._layout(f, None, [0, 128 * 128 * 2])
    assert n_pairs == 2 and list(si) == [0, 0] and list(off) == [0, 128 * 128 * 2] and ns == [128, 128]
    n_pairs, si, off, _, _ = handle._layout(f, None, None)
    assert n_pairs == 3 and si is None and off is None
