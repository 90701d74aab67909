"""The KITTI-style drift of Sec. IV-C against closed forms on planar trajectories."""
import math

import numpy as np
import pytest

from paper_2203_00459_gb300 import odometry as od

T = 1000   # frames of 1 m


def straight(theta=0.0, scale=1.0):
    return np.tile([theta, scale * 1.0, 0.0], (T, 1))


def test_perfect_estimate_has_no_drift():
    rng = np.random.default_rng(3)
    gt = np.column_stack([rng.normal(0, 0.01, T), 1.0 + rng.random(T), rng.normal(0, 0.1, T)])
    d = od.drift(gt, gt)
    assert d["translation_pct"] < 1e-9 and d["rotation_deg_per_km"] < 1e-6 and d["segments"] > 0


def test_scale_error_on_a_straight_path():
    """Every step 1 m, estimated (1 + s) m: a segment of L frames is off by s L, so s of L."""
    s = 0.02
    d = od.drift(straight(), straight(scale=1.0 + s))
    assert abs(d["translation_pct"] - 100 * s) < 1e-9 and d["rotation_deg_per_km"] < 1e-9
    assert d["by_length"][800.0][2] == T - 800 + 1   # segments from frames 0 .. T - 800


def test_heading_bias_on_a_straight_path():
    """A bias of b rad per 1 m frame turns the estimate by b L over L frames: b rad/m."""
    b = 1e-4
    d = od.drift(straight(), straight(theta=b))
    assert abs(d["rotation_deg_per_km"] - math.degrees(b) * 1e3) < 1e-6


def test_scaled_circle_measures_the_chord():
    """On a circle of radius R (1 m steps, constant turn) the relative rotations are exact and the
    steps are (1 + s) long, so the estimate is the circle scaled by (1 + s) and a segment's
    residual translation is s times its chord 2 R sin(L / 2R); L = 100 m only."""
    R, s = 150.0, 0.05
    dth = 1.0 / R                        # arc of 1 m
    chord1 = 2 * R * math.sin(dth / 2)   # straight step between frames
    gt = np.tile([dth, chord1 * math.cos(dth / 2), chord1 * math.sin(dth / 2)], (400, 1))
    est = gt * np.array([1.0, 1.0 + s, 1.0 + s])
    d = od.drift(gt, est, lengths=(100.0,))
    D = od.travelled(od.chain(gt))
    j = int(np.searchsorted(D, 100.0))
    arc = j * dth                         # angle swept by the first frame reaching 100 m
    expect = s * 2 * R * math.sin(arc / 2) / 100.0
    assert abs(d["translation_pct"] - 100 * expect) < 1e-9 and d["rotation_deg_per_km"] < 1e-9


def test_short_trajectories_have_no_segments():
    d = od.drift(straight()[:50], straight()[:50])
    assert d["segments"] == 0 and math.isnan(d["translation_pct"])


def test_chain_of_an_l_shaped_path():
    """100 steps of 1 m along x, a +90 deg turn in place (+x toward +y), 100 steps along the new
    heading: the last frame sits at (100, 100) facing +y after 200 m, and a segment error seen
    from the turned leg is expressed in that leg's frame."""
    rel = np.array([[0.0, 1.0, 0.0]] * 100 + [[math.pi / 2, 0.0, 0.0]] + [[0.0, 1.0, 0.0]] * 100)
    T = od.chain(rel)
    assert np.allclose(T[-1][:2, 2], [100.0, 100.0], atol=1e-9)
    assert abs(math.atan2(T[-1][1, 0], T[-1][0, 0]) - math.pi / 2) < 1e-12
    assert abs(od.travelled(T)[-1] - 200.0) < 1e-9
    # an estimate 1 m short on the first step only: the one 100 m segment that contains step 0
    # (from frame 0) is off by exactly 1 m, the others by nothing; segments start at frames
    # 0 .. 101 (the turn frame adds no distance)
    est = rel.copy()
    est[0, 1] = 0.0
    d = od.drift(rel, est, lengths=(100.0,))
    assert d["by_length"][100.0][2] == 102
    assert abs(d["translation_pct"] - 100.0 * (1.0 / 100.0) / 102) < 1e-12


def test_drive_ground_truth_converts_to_the_commanded_motion():
    """make_drive's step k moves the vehicle speed pixels forward and then turns it by
    yaw sin(2 pi k / period); motion_from_pose of the scan-to-scan pose gives back exactly that,
    in metres."""
    from paper_2203_00459_gb300 import synth
    _, poses = synth.make_drive(64, 12, speed_px=3.0, yaw_deg=2.0, period=10, seed=2)
    m = od.motion_from_pose(poses, 0.4)
    k = np.arange(12)
    w = np.radians(2.0) * np.sin(2 * np.pi * k / 10)
    assert np.max(np.abs(m - np.column_stack([w, np.full(12, 3.0 * 0.4), np.zeros(12)]))) < 1e-12


def test_oracle_odometry_on_a_synthetic_drive():
    """Scan-to-scan poses of the FP64 oracle (the plain search, Alg. 1) chained over a 180 m
    synthetic drive score a few percent of drift; the same poses with the heading's sign flipped
    in the conversion score several times worse, so the check sees the convention."""
    import oracle as O
    from paper_2203_00459_gb300 import synth
    frames, poses = synth.make_drive(128, 45, speed_px=4.0, yaw_deg=1.0, period=30, seed=1)
    cfg = O.make_cfg(128, 256, 64, temp_theta=0.2)
    est = np.array([[r["theta"], r["tx"], r["ty"]] for r in (O.pose(frames[k], frames[k + 1], cfg) for k in range(45))])
    gt = od.motion_from_pose(poses, 1.0)
    d = od.drift(gt, od.motion_from_pose(est, 1.0), lengths=(100.0,))
    assert d["segments"] > 15 and d["translation_pct"] < 4.0 and d["rotation_deg_per_km"] < 40.0, d
    flipped = est * np.array([-1.0, 1.0, 1.0])
    bad = od.drift(gt, od.motion_from_pose(flipped, 1.0), lengths=(100.0,))
    assert bad["translation_pct"] > 3 * d["translation_pct"], (d, bad)
