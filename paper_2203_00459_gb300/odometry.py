"""Odometry drift in the KITTI style, as the paper scores its odometry (Sec. IV-C): over every
segment of 100, 200, ..., 800 m of a trajectory, the residual translation and rotation between the
estimated and the true motion across the segment, divided by the segment length, averaged over all
segments.  Host-side evaluation (numpy); it runs on trajectories, not on scans.

Poses are planar: a relative pose (theta, x, y) is frame k+1 expressed in frame k (radians,
metres), and frames are chained as T_{k+1} = T_k M(theta, x, y) from T_0 = I.  A segment starts at
frame i (every ``step`` frames) and ends at the first frame j whose travelled distance from i, along
the true trajectory, is at least L; segments that run past the end are skipped.
"""
from __future__ import annotations

import numpy as np

LENGTHS = (100.0, 200.0, 300.0, 400.0, 500.0, 600.0, 700.0, 800.0)


def se2(theta, x, y):
    c, s = np.cos(theta), np.sin(theta)
    return np.array([[c, -s, x], [s, c, y], [0.0, 0.0, 1.0]])


def chain(rel):
    """Absolute poses [T + 1, 3, 3] of the relative poses rel [T, 3], starting from the identity."""
    rel = np.asarray(rel, np.float64)
    out = np.empty((rel.shape[0] + 1, 3, 3))
    out[0] = np.eye(3)
    for k, (th, x, y) in enumerate(rel):
        out[k + 1] = out[k] @ se2(th, x, y)
    return out


def travelled(abs_poses):
    """Cumulative path length [T + 1] along the frame origins."""
    steps = np.hypot(*np.diff(abs_poses[:, :2, 2], axis=0).T)
    return np.concatenate([[0.0], np.cumsum(steps)])


def drift(gt_rel, est_rel, lengths=LENGTHS, step=1):
    """Segment errors of est_rel against gt_rel (both [T, 3]).  Returns dict with
    ``translation_pct`` (mean residual translation / L, in %), ``rotation_deg_per_km`` (mean
    residual rotation / L), ``segments`` (how many were averaged) and ``by_length``
    {L: (translation_pct, rotation_deg_per_km, count)}."""
    G, E = chain(gt_rel), chain(est_rel)
    d = travelled(G)
    per = {L: [] for L in lengths}
    for i in range(0, len(d), step):
        for L in lengths:
            j = int(np.searchsorted(d, d[i] + L, side="left"))
            if j >= len(d):
                continue
            dg = np.linalg.inv(G[i]) @ G[j]
            de = np.linalg.inv(E[i]) @ E[j]
            r = np.linalg.inv(de) @ dg
            per[L].append((np.hypot(r[0, 2], r[1, 2]) / L, abs(np.arctan2(r[1, 0], r[0, 0])) / L))
    allv = [v for L in lengths for v in per[L]]
    if not allv:
        return {"translation_pct": float("nan"), "rotation_deg_per_km": float("nan"), "segments": 0, "by_length": {}}
    t, r = np.mean(np.asarray(allv), axis=0)
    by = {L: (100.0 * float(np.mean([v[0] for v in per[L]])), float(np.degrees(np.mean([v[1] for v in per[L]]))) * 1e3,
              len(per[L])) for L in lengths if per[L]}
    return {"translation_pct": 100.0 * float(t), "rotation_deg_per_km": float(np.degrees(r)) * 1e3,
            "segments": len(allv), "by_length": by}


def motion_from_pose(pose, delta_xy):
    """Vehicle motion (frame k+1 in frame k: theta, x, y in radians and metres) from the search's
    pose between scans k and k+1 (theta, t_x, t_y in pixels; scan k+1 holds scan k's returns at
    c + R(theta)(p - c) + t): the scene turning by theta is the vehicle turning by -theta, and the
    vehicle's displacement is -delta_xy R(-theta) t."""
    p = np.asarray(pose, np.float64).reshape(-1, 3)
    th = -p[:, 0]
    c, s = np.cos(th), np.sin(th)
    tx, ty = p[:, 1], p[:, 2]
    return np.column_stack([th, -delta_xy * (c * tx - s * ty), -delta_xy * (s * tx + c * ty)])
