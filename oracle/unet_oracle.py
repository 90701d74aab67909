"""FP64 CPU oracle of the masking network h_alpha (Sec. III-D, Eq. 10-12, Tab. II) -- test
infrastructure only (tests/, __graft_entry__.smoke(), bench.py's CPU legs).

Plain PyTorch CPU operations in float64 are the steps (conv2d, batch_norm statistics, max_pool2d,
bilinear interpolate, sigmoid); autograd gives the gradient.  The CUDA path computes with bf16
tensor-core operands and float32 accumulation, so the oracle rounds to bf16 at exactly the same
points -- the two scans entering the first convolution, every convolution weight, and every
post-activation tensor (after BN + ReLU, after max-pool, after the bilinear upsampling) -- and
keeps everything else in float64.  Rounding is to nearest even, the bf16 conversion both sides
use.  Gradients pass straight through the roundings.

Architecture readings (the paper leaves them open):
* levels with channels c_1..c_L (4 levels 8/16/32/64 for the 256^2 configuration; Tab. II's
  five encoder levels plus the 256-channel bottleneck are (8, 16, 32, 64, 128, 256));
* every convolution is 3x3, stride 1, zero padding 1, no bias, followed by BatchNorm (batch
  statistics in training, population variance; running statistics with momentum 0.1 updated with
  the unbiased variance; eps 1e-5) and ReLU;
* down: 2x2 max-pool, stride 2; up: bilinear x2 of the deeper feature (align_corners=False)
  concatenated before the skip, [up, skip];
* head: one 1x1 convolution 8 -> 2 with bias, then the sigmoid; masks m_f, m_g multiply the scans
  (Eq. 11).
"""
from __future__ import annotations

import math

import numpy as np
import torch
import torch.nn.functional as F

EPS = 1e-5
MOMENTUM = 0.1


def bf16(x):
    """Round a float64 tensor to bf16 and back (round to nearest even); gradient passes through."""
    return x + (x.detach().to(torch.bfloat16).to(x.dtype) - x.detach())


def conv_layers(channels=(8, 16, 32, 64), in_ch=2):
    """(name, c_in, c_out) of every 3x3 convolution in forward order: per level two convolutions
    down the encoder, then per level (deepest first) two convolutions up the decoder, the first of
    which takes [bilinear x2 of the deeper feature, skip]."""
    layers, c_prev = [], in_ch
    for i, c in enumerate(channels):
        layers += [(f"enc{i}a", c_prev, c), (f"enc{i}b", c, c)]
        c_prev = c
    deeper = channels[-1]
    for i in range(len(channels) - 2, -1, -1):
        layers += [(f"dec{i}a", deeper + channels[i], channels[i]), (f"dec{i}b", channels[i], channels[i])]
        deeper = channels[i]
    return layers


def init_params(channels=(8, 16, 32, 64), seed=1, in_ch=2, out_ch=2):
    """Seeded initial parameters (float64, PyTorch layouts): He-uniform conv weights, BN gamma 1,
    beta 0, head weight uniform(+-1/sqrt(c_1)) and bias 0.  Uses numpy's Philox generator."""
    rng = np.random.Generator(np.random.Philox(key=int(seed)))
    p = {}
    for name, ci, co in conv_layers(channels, in_ch):
        bound = math.sqrt(6.0 / (ci * 9))
        p[name + ".w"] = torch.from_numpy((2 * rng.random((co, ci, 3, 3)) - 1) * bound)
        p[name + ".gamma"] = torch.ones(co, dtype=torch.float64)
        p[name + ".beta"] = torch.zeros(co, dtype=torch.float64)
    b = 1.0 / math.sqrt(channels[0])
    p["head.w"] = torch.from_numpy((2 * rng.random((out_ch, channels[0], 1, 1)) - 1) * b)
    p["head.b"] = torch.zeros(out_ch, dtype=torch.float64)
    return p


def init_state(channels=(8, 16, 32, 64), in_ch=2):
    """BatchNorm running statistics (mean 0, variance 1)."""
    s = {}
    for name, _, co in conv_layers(channels, in_ch):
        s[name + ".mean"] = torch.zeros(co, dtype=torch.float64)
        s[name + ".var"] = torch.ones(co, dtype=torch.float64)
    return s


def conv_bn_relu(x, p, state, name, training):
    """3x3 convolution (bf16 weights), BatchNorm, ReLU; output rounded to bf16."""
    y = F.conv2d(x, bf16(p[name + ".w"]), padding=1)
    if training:
        mean = y.mean(dim=(0, 2, 3))
        var = y.var(dim=(0, 2, 3), unbiased=False)
        n = y.shape[0] * y.shape[2] * y.shape[3]
        with torch.no_grad():
            state[name + ".mean"].mul_(1 - MOMENTUM).add_(MOMENTUM * mean.detach())
            state[name + ".var"].mul_(1 - MOMENTUM).add_(MOMENTUM * var.detach() * n / max(1, n - 1))
    else:
        mean, var = state[name + ".mean"], state[name + ".var"]
    xhat = (y - mean[None, :, None, None]) / torch.sqrt(var[None, :, None, None] + EPS)
    return bf16(torch.relu(xhat * p[name + ".gamma"][None, :, None, None] + p[name + ".beta"][None, :, None, None]))


def down2(x):
    """Encoder step down: 2 x 2 max-pool, stride 2 (Tab. II)."""
    return F.max_pool2d(x, 2)


def up2(x):
    """Decoder step up: bilinear x2 with align_corners=False, rounded to bf16 like every
    post-activation tensor (Tab. II)."""
    return bf16(F.interpolate(x, scale_factor=2, mode="bilinear", align_corners=False))


def forward(p, state, f, g, channels=(8, 16, 32, 64), training=True):
    """Masks [B, 2, H, W] (float64) of Eq. 10 for scans f, g [B, H, W]."""
    x = bf16(torch.stack([f, g], dim=1))
    skips = []
    L = len(channels)
    for i in range(L):
        if i > 0:
            x = down2(x)
        x = conv_bn_relu(x, p, state, f"enc{i}a", training)
        x = conv_bn_relu(x, p, state, f"enc{i}b", training)
        skips.append(x)
    for i in range(L - 2, -1, -1):
        up = up2(x)
        x = torch.cat([up, skips[i]], dim=1)
        x = conv_bn_relu(x, p, state, f"dec{i}a", training)
        x = conv_bn_relu(x, p, state, f"dec{i}b", training)
    z = F.conv2d(x, bf16(p["head.w"]), p["head.b"])
    return torch.sigmoid(z)


def masked(p, state, f, g, channels=(8, 16, 32, 64), training=True):
    """(f o m_f, g o m_g) of Eq. 11 and the masks."""
    m = forward(p, state, f, g, channels, training)
    return f * m[:, 0], g * m[:, 1], m


def grads(p, state, f, g, dft, dgt, channels=(8, 16, 32, 64)):
    """Parameter gradients (float64) of <f o m_f, dft> + <g o m_g, dgt> in training mode."""
    q = {k: v.clone().requires_grad_(True) for k, v in p.items()}
    ft, gt, _ = masked(q, {k: v.clone() for k, v in state.items()}, f, g, channels, True)
    (ft * dft).sum().add((gt * dgt).sum()).backward()
    return {k: v.grad for k, v in q.items()}


def adam(p, grad, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba, the optimiser of Sec. IV-B) on the float64 master parameters."""
    out = {}
    for k in p:
        m[k] = b1 * m[k] + (1 - b1) * grad[k]
        v[k] = b2 * v[k] + (1 - b2) * grad[k] ** 2
        mh = m[k] / (1 - b1 ** step)
        vh = v[k] / (1 - b2 ** step)
        out[k] = p[k] - lr * mh / (torch.sqrt(vh) + eps)
    return out
