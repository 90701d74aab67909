"""Seeded synthetic radar-like scan pairs (stand-in for the Oxford Radar RobotCar scans, Sec. IV-A).

This module only makes inputs.  It holds none of the search's arithmetic: a scene of point
scatterers and line "walls" is rendered analytically, once in the source frame and once in the
target frame (Eq. 1: x' = R x + t about the image centre), so the ground-truth pose is exact to
sub-pixel precision and neither the oracle nor the CUDA library is needed to make a target.

Scene recipe (per scan pair):
* K point scatterers at uniform continuous positions, amplitude U(5, 20);
* W walls: centre uniform, length U(0.1 N, 0.5 N), orientation U[0, pi), sampled every 0.5 px,
  amplitude U(2, 8);
* every scatterer and wall sample carries an Exp(1) speckle factor (shared by both frames);
* each element is drawn as a normalised Gaussian footprint of sigma = 0.8 px on the N-periodic
  grid (the 3x3 blur of the recipe, evaluated analytically at the element's exact position);
* each scan then gets its own additive |N(0, 0.3)| noise.

The target carries the source scene moved by the pose (theta, t_x, t_y): an element at p in the
source is at c + R(theta) (p - c) + t in the target, wrapped onto the N-periodic grid, with
c = (N/2, N/2) and theta > 0 turning +x toward +y.  Random numbers come from numpy's Philox
counter-based generator keyed by (seed, pair index); all distributions are built from uniform
doubles so that the stream does not depend on numpy's sampling routines.
"""
from __future__ import annotations

import math

import numpy as np

SIGMA_PX = 0.8
FOOT = 3  # footprint half-width in pixels


def _rng(seed, index):
    return np.random.Generator(np.random.Philox(key=(int(seed) << 32) + int(index)))


def _exp1(rng, size):
    return -np.log1p(-rng.random(size))


def _abs_normal(rng, size, sd):
    u1 = rng.random(size)
    u2 = rng.random(size)
    return np.abs(sd * np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2))


def scene(rng, n, n_points, n_walls):
    """Element positions (x, y) and amplitudes of one random scene in the source frame."""
    px = rng.random(n_points) * n
    py = rng.random(n_points) * n
    amp = 5.0 + 15.0 * rng.random(n_points)
    xs, ys, amps = [px], [py], [amp]
    for _ in range(n_walls):
        cx, cy = rng.random() * n, rng.random() * n
        length = (0.1 + 0.4 * rng.random()) * n
        ang = rng.random() * np.pi
        a = 2.0 + 6.0 * rng.random()
        m = max(2, int(length / 0.5) + 1)
        s = np.linspace(-0.5 * length, 0.5 * length, m)
        xs.append(cx + s * math.cos(ang))
        ys.append(cy + s * math.sin(ang))
        amps.append(np.full(m, a))
    x = np.concatenate(xs)
    y = np.concatenate(ys)
    a = np.concatenate(amps) * _exp1(rng, x.size)
    return x, y, a


def render(n, x, y, a):
    """Sum of normalised Gaussian footprints on the N-periodic grid (float64 [N, N])."""
    ix = np.floor(x).astype(np.int64)
    iy = np.floor(y).astype(np.int64)
    acc = np.zeros(n * n, dtype=np.float64)
    offs = np.arange(-FOOT, FOOT + 2)
    norm = 1.0 / (2.0 * np.pi * SIGMA_PX * SIGMA_PX)
    for oy in offs:
        gy = iy + oy
        wy = np.exp(-((gy - y) ** 2) / (2 * SIGMA_PX ** 2))
        for ox in offs:
            gx = ix + ox
            w = wy * np.exp(-((gx - x) ** 2) / (2 * SIGMA_PX ** 2)) * norm * a
            idx = np.mod(gy, n) * n + np.mod(gx, n)
            acc += np.bincount(idx, weights=w, minlength=n * n)
    return acc.reshape(n, n)


def move(n, x, y, theta, tx, ty):
    """Element positions in the target frame: c + R(theta)(p - c) + t (Eq. 1 about the centre)."""
    c = n / 2.0
    ct, st = math.cos(theta), math.sin(theta)
    dx, dy = x - c, y - c
    return c + ct * dx - st * dy + tx, c + st * dx + ct * dy + ty


def make_pair(n, n_points, n_walls, theta, tx, ty, seed, index, noise_sd=0.3):
    """One (source, target) pair with pose (theta [rad], tx, ty [px]); float32 [N, N] each."""
    rng = _rng(seed, index)
    x, y, a = scene(rng, n, n_points, n_walls)
    f = render(n, x, y, a) + _abs_normal(rng, (n, n), noise_sd)
    x2, y2 = move(n, x, y, theta, tx, ty)
    g = render(n, x2, y2, a) + _abs_normal(rng, (n, n), noise_sd)
    return f.astype(np.float32), g.astype(np.float32)


# Workloads: the scene sizes and pose ranges of the benchmark configurations.
WORKLOADS = {
    # 128^2, integer circular shifts, rotations on the 128-bin angle grid spacing 2 x 180/128 deg
    "single128": dict(n=128, n_points=40, n_walls=6, n_theta=128, n_r=64, pairs=1, seed_id=1),
    # 256^2, continuous theta ~ U(-5, 5) deg, t ~ U(-8, 8) px
    "batch256": dict(n=256, n_points=150, n_walls=20, n_theta=400, n_r=128, pairs=256, seed_id=2,
                     theta_deg=5.0, t_px=8.0),
    # 512^2, theta ~ U(-8, 8) deg, t ~ U(-16, 16) px
    "batch512": dict(n=512, n_points=400, n_walls=40, n_theta=400, n_r=256, pairs=32, seed_id=3,
                     theta_deg=8.0, t_px=16.0),
    # the paper's odd sides (Sec. IV-B: 0.8, 0.4, 0.2 m cells): the same scenes and pose ranges as the
    # power-of-two workloads above, continuous poses, n_r <= N/2
    "batch127": dict(n=127, n_points=40, n_walls=6, n_theta=128, n_r=63, pairs=16, seed_id=4,
                     theta_deg=5.0, t_px=4.0),
    "batch255": dict(n=255, n_points=150, n_walls=20, n_theta=400, n_r=127, pairs=64, seed_id=5,
                     theta_deg=5.0, t_px=8.0),
    "batch511": dict(n=511, n_points=400, n_walls=40, n_theta=400, n_r=255, pairs=32, seed_id=6,
                     theta_deg=8.0, t_px=16.0),
}

SEED_BASE = 20220301


def draw_pose(rng, spec):
    """Ground-truth pose for one pair of a workload (see WORKLOADS)."""
    if spec["n"] == 128 and "theta_deg" not in spec:
        k = int(np.floor(rng.random() * 5)) - 2
        t = np.floor(rng.random(2) * 9).astype(int) - 4
        return k * (2.0 * np.pi / 128.0), float(t[0]), float(t[1])
    th = math.radians(spec["theta_deg"]) * (2.0 * rng.random() - 1.0)
    t = spec["t_px"] * (2.0 * rng.random(2) - 1.0)
    return th, float(t[0]), float(t[1])


def make_batch(name, pairs=None, start=0, spec=None):
    """Pairs [start, start+pairs) of a named workload: (f [B,N,N], g [B,N,N], pose [B,3]) float32."""
    spec = dict(WORKLOADS[name] if spec is None else spec)
    b = spec["pairs"] if pairs is None else pairs
    n = spec["n"]
    seed = SEED_BASE + spec["seed_id"]
    f = np.empty((b, n, n), np.float32)
    g = np.empty((b, n, n), np.float32)
    pose = np.empty((b, 3), np.float64)
    for i in range(b):
        idx = start + i
        prng = _rng(seed + 1000, idx)
        th, tx, ty = draw_pose(prng, spec)
        f[i], g[i] = make_pair(n, spec["n_points"], spec["n_walls"], th, tx, ty, seed, idx)
        pose[i] = (th, tx, ty)
    return f, g, pose


# ---------------------------------------------------------------------------------------------
# trajectories with moving scatterers (the learned-mask workload, 256^2)
# ---------------------------------------------------------------------------------------------

def make_trajectory(n_frames, seed, index, n=256, n_static=150, n_walls=20, moving_frac=0.1,
                    theta_deg=5.0, t_px=8.0, speed_px=6.0, moving_amp=(20.0, 60.0), noise_sd=0.3,
                    pixel_speckle=False):
    """Frames of one trajectory and the ego step between consecutive frames.

    A static scene (scatterers and walls, as in make_pair) plus moving_frac * n_static moving
    scatterers with amplitude U(moving_amp) and their own constant velocity (uniform in a disk of
    radius speed_px per frame).  Frame k+1 sees every element of frame k moved by the ego step
    (theta_k, t_k) ~ (U(+-theta_deg), U(+-t_px)^2) about the image centre (Eq. 1), and the moving
    scatterers additionally displaced by their velocity.  Each frame gets fresh |N(0, noise_sd)|
    noise and, with pixel_speckle, a fresh per-pixel Exp(1) multiplicative speckle (the image-level
    speckle of the recipe, independent in every frame).  Returns (frames float32 [n_frames, N, N],
    steps float64 [n_frames - 1, 3])."""
    rng = _rng(seed, index)
    xs, ys, amp = scene(rng, n, n_static, n_walls)
    m = max(1, int(round(moving_frac * n_static)))
    mx = rng.random(m) * n
    my = rng.random(m) * n
    ma = (moving_amp[0] + (moving_amp[1] - moving_amp[0]) * rng.random(m)) * _exp1(rng, m)
    sp = speed_px * np.sqrt(rng.random(m))
    ang = 2.0 * np.pi * rng.random(m)
    vx, vy = sp * np.cos(ang), sp * np.sin(ang)
    frames = np.empty((n_frames, n, n), np.float32)
    steps = np.empty((n_frames - 1, 3), np.float64)
    for k in range(n_frames):
        img = render(n, np.concatenate([xs, mx]), np.concatenate([ys, my]), np.concatenate([amp, ma]))
        if pixel_speckle:
            img = img * _exp1(rng, (n, n))
        frames[k] = (img + _abs_normal(rng, (n, n), noise_sd)).astype(np.float32)
        if k == n_frames - 1:
            break
        th = math.radians(theta_deg) * (2.0 * rng.random() - 1.0)
        t = t_px * (2.0 * rng.random(2) - 1.0)
        steps[k] = (th, t[0], t[1])
        xs, ys = move(n, xs, ys, th, t[0], t[1])
        mx, my = move(n, mx + vx, my + vy, th, t[0], t[1])
        # velocities turn with the sensor frame
        c, s = math.cos(th), math.sin(th)
        vx, vy = c * vx - s * vy, s * vx + c * vy
    return frames, steps


def trajectory_pairs(n_traj, n_frames, seed, **kw):
    """Consecutive-frame pairs of n_traj trajectories: (f, g, pose) with pose the ego step."""
    F, G, P = [], [], []
    for j in range(n_traj):
        fr, st = make_trajectory(n_frames, seed, j, **kw)
        F.append(fr[:-1])
        G.append(fr[1:])
        P.append(st)
    return np.concatenate(F), np.concatenate(G), np.concatenate(P)


def _trajectory_job(args):
    n_frames, seed, index, kw = args
    fr, st = make_trajectory(n_frames, seed, index, **kw)
    return fr[:-1], fr[1:], st


def trajectory_pairs_parallel(n_traj, n_frames, seed, processes=None, **kw):
    """trajectory_pairs over a spawn process pool (same pairs, same order)."""
    import multiprocessing as mp
    import os
    procs = processes or min(n_traj, os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(procs) as pool:
        parts = pool.map(_trajectory_job, [(n_frames, seed, j, kw) for j in range(n_traj)])
    return (np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts]),
            np.concatenate([p[2] for p in parts]))


def make_polar_scans(b, n_az=400, n_range=3768, n_targets=300, seed=0):
    """Seeded polar (azimuth x range) radar scans [b, n_az, n_range] float32, shaped like the
    Navtech CTS350-X scans of the Oxford Radar RobotCar data (Sec. IV-A: 400 azimuths, 3768 range
    bins): an |N(0, 0.3)| noise floor plus n_targets returns at uniform (azimuth, range), amplitude
    U(5, 20) x Exp(1) speckle, each a Gaussian footprint of sigma 1 azimuth bin (wrapped) by
    2 range bins."""
    out = np.empty((b, n_az, n_range), np.float32)
    da, dk = np.arange(-3, 4), np.arange(-6, 7)
    shape = np.exp(-0.5 * da[:, None] ** 2) * np.exp(-0.5 * (dk[None, :] / 2.0) ** 2)
    for i in range(b):
        rng = _rng(seed, 1000 + i)
        s = _abs_normal(rng, (n_az, n_range), 0.3)
        a = np.floor(rng.random(n_targets) * n_az).astype(np.int64)
        k = np.floor(rng.random(n_targets) * n_range).astype(np.int64)
        amp = (5.0 + 15.0 * rng.random(n_targets)) * _exp1(rng, n_targets)
        for t in range(n_targets):
            rows = np.mod(a[t] + da, n_az)
            cols = k[t] + dk
            ok = (cols >= 0) & (cols < n_range)
            s[np.ix_(rows, cols[ok])] += amp[t] * shape[:, ok]
        out[i] = s
    return out


def make_drive(n, n_frames, speed_px=1.0, yaw_deg=0.5, period=80, n_points=None, n_walls=None, seed=0,
               noise_sd=0.3, reach=0.45):
    """A vehicle driving through one static, non-periodic world: frames [n_frames + 1, N, N]
    float32 and the search pose between consecutive frames [n_frames, 3] = (theta, t_x, t_y) in the
    convention of make_pair (frame k+1 holds frame k's returns at c + R(theta)(p - c) + t).

    Step k moves the vehicle speed_px pixels along its heading and then turns it by
    yaw_deg sin(2 pi k / period) degrees.  The world holds the point scatterers and walls of
    make_pair's recipe at the same density per N x N area, spread over the path's bounding box
    grown by N.  Frame k renders the returns within reach * N of the vehicle (a radar sees a disc
    around itself) at p_k = c + R_k^T (p - T_k), with fresh |N(0, noise_sd)| noise."""
    rng = _rng(seed, 7)
    n_points = n * n // 300 if n_points is None else n_points
    n_walls = n // 16 if n_walls is None else n_walls
    # the path first: vehicle poses (phi_k, T_k), world origin at the start
    phis, Ts = [0.0], [np.zeros(2)]
    for k in range(n_frames):
        T1 = Ts[-1] + speed_px * np.array([math.cos(phis[-1]), math.sin(phis[-1])])
        phis.append(phis[-1] + math.radians(yaw_deg) * math.sin(2.0 * math.pi * k / period))
        Ts.append(T1)
    P = np.array(Ts)
    lo, hi = P.min(axis=0) - n, P.max(axis=0) + n
    area = float(np.prod(hi - lo)) / (n * n)
    x, y, a = scene(rng, 1, int(round(n_points * area)), 0)   # points in the unit square
    x, y = lo[0] + x * (hi[0] - lo[0]), lo[1] + y * (hi[1] - lo[1])
    xs, ys, amps = [x], [y], [a]
    for _ in range(int(round(n_walls * area))):
        cx, cy = lo[0] + rng.random() * (hi[0] - lo[0]), lo[1] + rng.random() * (hi[1] - lo[1])
        length = (0.1 + 0.4 * rng.random()) * n
        ang = rng.random() * np.pi
        m = max(2, int(length / 0.5) + 1)
        sv = np.linspace(-0.5 * length, 0.5 * length, m)
        xs.append(cx + sv * math.cos(ang))
        ys.append(cy + sv * math.sin(ang))
        amps.append(np.full(m, 2.0 + 6.0 * rng.random()) * _exp1(rng, m))
    x, y, a = np.concatenate(xs), np.concatenate(ys), np.concatenate(amps)
    c = n / 2.0
    frames = np.empty((n_frames + 1, n, n), np.float32)
    poses = np.empty((n_frames, 3))
    for k in range(n_frames + 1):
        cp, sp = math.cos(phis[k]), math.sin(phis[k])
        dx, dy = x - Ts[k][0], y - Ts[k][1]
        u, v = cp * dx + sp * dy, -sp * dx + cp * dy
        seen = u * u + v * v < (reach * n) ** 2
        frames[k] = render(n, c + u[seen], c + v[seen], a[seen]) + _abs_normal(rng, (n, n), noise_sd)
        if k < n_frames:
            c1, s1 = math.cos(phis[k + 1]), math.sin(phis[k + 1])
            d = Ts[k] - Ts[k + 1]
            poses[k] = (phis[k] - phis[k + 1], c1 * d[0] + s1 * d[1], -s1 * d[0] + c1 * d[1])
    return frames, poses
