"""Parity of the CUDA radar front end (fmbym_polar_to_cartesian) with the FP64 oracle (reading
A16), through the C ABI, on Navtech-sized synthetic scans."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import radar_oracle as R  # noqa: E402
from paper_2203_00459_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

# fp32 bearing (atan2f, a few ulps of 2 pi) and radius (sqrtf) put the fractional indices within
# about 1e-4 bins of the oracle's at these sizes (<= 3768 range bins, 400 azimuths); a bilinear
# value then moves by at most 1e-4 x (the largest neighbour difference <= 2 max|scan|) per index.
TOL = 1e-3   # max |gpu - oracle| / max |scan|


@pytest.fixture(scope="module")
def search():
    from paper_2203_00459_gb300 import build
    build.build()
    from paper_2203_00459_gb300 import search as s
    return s


def run(search, polar, n, dxy, res):
    out = search.polar_to_cartesian(torch.from_numpy(polar).cuda(), n, dxy, res)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def check(polar, cart, n, dxy, res, tag):
    n_range = polar.shape[2]
    _, fk = R.polar_indices(n, dxy, polar.shape[1], res)
    # where the oracle's range index sits on the outer edge, fp32 may fall on either side of it
    edge = np.abs(fk - (n_range - 1)) < 1e-3
    assert edge.sum() <= 8, (tag, int(edge.sum()))
    for i in range(polar.shape[0]):
        ref = R.polar_to_cartesian(polar[i], n, dxy, res)
        err = np.abs(cart[i] - ref)[~edge].max() / np.abs(polar[i]).max()
        assert err <= TOL, (tag, i, err)


@pytest.mark.parametrize("n,dxy", [(256, 0.4), (512, 0.2), (255, 0.4)])
def test_navtech_scan(search, n, dxy):
    polar = synth.make_polar_scans(3, seed=5)
    check(polar, run(search, polar, n, dxy, 0.0438), n, dxy, 0.0438, f"navtech {n}")


def test_outer_edge_inside_the_image_and_odd_azimuths(search):
    """300 bins of 0.175 m (52 m) end inside a 256 x 0.4 m image; 399 azimuths (not a multiple of 4)."""
    polar = synth.make_polar_scans(2, n_az=399, n_range=300, seed=6)
    cart = run(search, polar, 256, 0.4, 0.175)
    check(polar, cart, 256, 0.4, 0.175, "edge")
    X, Y = R.cartesian_points(256, 0.4)
    assert np.all(cart[:, np.hypot(X, Y) > 299.6 * 0.175] == 0.0)


def test_empty_and_invalid_calls(search):
    from paper_2203_00459_gb300 import _lib
    z = torch.zeros((0, 400, 100), device="cuda")
    assert search.polar_to_cartesian(z, 64, 0.4, 0.0438).shape == (0, 64, 64)
    with pytest.raises(_lib.FmbymError):
        search.polar_to_cartesian(torch.zeros((1, 400, 100), device="cuda"), 64, -0.4, 0.0438)
