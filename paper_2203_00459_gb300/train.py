"""End-to-end training of the masking network through the decoupled search (Sec. III-D, Eq. 10-13).

One step: masks and masked scans from the U-Net (Eq. 10-11), then one training call of the search
on the masked scans (the pose of Eq. 12 / Alg. 1, the L1 pose loss of Eq. 13 and the adjoint of
the search down to the masked scans), the adjoint of the network, and an Adam step -- every stage
a call into the CUDA library.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import masknet, synth
from .search import PoseSearch, size_cfg


def init_params(channels=(8, 16, 32, 64), seed=1):
    """Seeded initial parameters in the flat layout: He-uniform 3x3 weights (bound sqrt(6 / fan_in)),
    BN gamma 1 and beta 0, head weight uniform(+-1/sqrt(c_1)) and bias 0 (numpy Philox)."""
    rng = np.random.Generator(np.random.Philox(key=int(seed)))
    named = {}
    for name, ci, co in masknet.conv_names(channels):
        bound = math.sqrt(6.0 / (ci * 9))
        named[name + ".w"] = torch.from_numpy((2 * rng.random((co, ci, 3, 3)) - 1) * bound)
        named[name + ".gamma"] = torch.ones(co, dtype=torch.float64)
        named[name + ".beta"] = torch.zeros(co, dtype=torch.float64)
    b = 1.0 / math.sqrt(channels[0])
    named["head.w"] = torch.from_numpy((2 * rng.random((2, channels[0], 1, 1)) - 1) * b)
    named["head.b"] = torch.zeros(2, dtype=torch.float64)
    return masknet.flatten(named, channels)


class MaskedSearch:
    """The masking network in front of the decoupled search, trained through it."""

    def __init__(self, n=256, n_theta=400, n_r=128, channels=(8, 16, 32, 64), batch=64, seed=1, loss_kind=1,
                 delta_xy=1.0):
        # delta_xy: the cell size in the units the translation is wanted in (Alg. 1's delta_xy); the
        # pose's translation, and the ground truth given to train_step, are in those units
        self.cfg = size_cfg(n, n_theta, n_r, delta_xy=delta_xy)
        self.search = PoseSearch([self.cfg], max_pairs=batch)
        self.net = masknet.MaskNet(channels, n, n, max_batch=batch)
        self.net.load(init_params(channels, seed).cuda())
        self.loss_kind = loss_kind
        self.steps = 0

    def train_step(self, f, g, gt, lr=1e-3):
        """One Adam step on a batch (device tensors f, g [B, N, N], gt [B, 3]); returns the loss."""
        fo, go, _ = self.net.forward(f, g, training=True)
        _, loss, _, dfo, dgo = self.search.pose_train(fo, go, gt, kind=self.loss_kind)
        self.net.backward(f, g, dfo, dgo)
        self.steps += 1
        self.net.adam(lr, self.steps)
        return loss

    def save(self, path):
        """Checkpoint: float32 master parameters, BN running statistics, both Adam moments and the
        step count (the state a resumed run needs to continue bit for bit), as an .npz file."""
        p, r, _ = self.net.store()
        m, v = self.net.adam_state()
        torch.cuda.synchronize()
        np.savez(path, params=p.cpu().numpy(), running=r.cpu().numpy(), adam_m=m.cpu().numpy(),
                 adam_v=v.cpu().numpy(), steps=np.int64(self.steps), loss_kind=np.int64(self.loss_kind))

    def load(self, path):
        """Resumes from a checkpoint written by save()."""
        z = np.load(path)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        self.net.load(dev(z["params"]), dev(z["running"]))
        self.net.load_adam(dev(z["adam_m"]), dev(z["adam_v"]))
        self.steps = int(z["steps"])
        self.loss_kind = int(z["loss_kind"])
        torch.cuda.synchronize()

    def poses(self, f, g, masked=True):
        """Poses with the trained masks (evaluation statistics), or of the raw scans, computed in
        chunks of the handle's batch size."""
        out = []
        b = self.search.max_pairs
        for k in range(0, f.shape[0], b):
            fk, gk = f[k:k + b].contiguous(), g[k:k + b].contiguous()
            if masked:
                fk, gk, _ = self.net.forward(fk, gk, training=False)
            out.append(self.search.pose(fk, gk)["pose"])
        return torch.cat(out)

    def close(self):
        self.search.close()
        self.net.close()


def pose_errors(pose, gt):
    """Mean absolute error of (theta [rad], t_x, t_y [px]) over a batch (numpy)."""
    return np.mean(np.abs(np.asarray(pose, np.float64) - np.asarray(gt, np.float64)), axis=0)


def trajectory_data(n_traj, n_frames, seed, n=256, parallel=False):
    """Training or evaluation pairs of the learned-mask workload: consecutive frames of trajectories
    with 10 % moving scatterers and fresh per-frame speckle."""
    if parallel:
        return synth.trajectory_pairs_parallel(n_traj, n_frames, seed, n=n, pixel_speckle=True)
    return synth.trajectory_pairs(n_traj, n_frames, seed, n=n, pixel_speckle=True)
