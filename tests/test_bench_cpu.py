"""Host-side pieces of bench.py: the algorithmic-bytes model behind the roofline and the traffic
record, checked by hand counts (no GPU)."""
import math

import bench


def test_step_model_at_512():
    """N = 512, P = 768, n_theta = 400, n_r = 256, 16 chunks: 65.3 MB of compulsory kernel traffic
    per pair in the training step; k_b_cols reads the D rows and both column spectra and writes two
    adjoint spectra: (1 + 2 + 2) N (P/2) complex floats."""
    m = bench.kernel_model(512, 768, 400, 256, 16)
    assert abs(sum(v[0] for v in m.values()) / 1e6 - 65.28) < 0.01
    n, wp, c = 512, 384, 8
    assert m["b_cols"][0] == n * wp * c + 2 * 768 * wp * c + 2 * n * wp * c
    assert m["b_cols"][0] * 32 == 301989888                     # one 32-pair launch
    assert m["b_cols"][1] == 3 * wp * 5.0 * 768 * math.log2(768)  # three column FFT passes


def test_traffic_record_is_per_launch_of_the_recorded_tile():
    bytes_, h, pairs, tile, plan = bench.TRAFFIC["b_cols"]
    assert pairs == 32 and tile in (2, 4, 8) and plan in (0, 1) and len(h) == 16
    # ncu traffic below the algorithmic bytes of the same launch: nothing is re-read
    assert 0.8 < bytes_ / (bench.kernel_model(512, 768, 400, 256, 16)["b_cols"][0] * pairs) < 1.0
