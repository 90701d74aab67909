"""Python face of the masking network h_alpha (Sec. III-D) in the CUDA library: a handle over the
U-Net with flat float32 parameters, and the layout helpers that map named tensors to that layout.
Marshalling only; every layer runs in the library's kernels."""
from __future__ import annotations

import ctypes

import torch

from . import _lib


def conv_names(channels):
    """(name, c_in, c_out) of the 3x3 convolutions in the order of the flat parameter layout."""
    out, prev = [], 2
    for i, c in enumerate(channels):
        out += [(f"enc{i}a", prev, c), (f"enc{i}b", c, c)]
        prev = c
    deeper = channels[-1]
    for i in range(len(channels) - 2, -1, -1):
        out += [(f"dec{i}a", deeper + channels[i], channels[i]), (f"dec{i}b", channels[i], channels[i])]
        deeper = channels[i]
    return out


def flatten(named, channels):
    """Named tensors {'enc0a.w', 'enc0a.gamma', ..., 'head.w', 'head.b'} -> flat float32 vector."""
    parts = []
    for name, _, _ in conv_names(channels):
        parts += [named[name + ".w"].reshape(-1), named[name + ".gamma"].reshape(-1), named[name + ".beta"].reshape(-1)]
    parts += [named["head.w"].reshape(-1), named["head.b"].reshape(-1)]
    return torch.cat([p.to(torch.float32) for p in parts])


def unflatten(flat, channels):
    """Inverse of flatten (views into flat)."""
    out, k = {}, 0
    for name, ci, co in conv_names(channels):
        out[name + ".w"] = flat[k:k + co * ci * 9].reshape(co, ci, 3, 3)
        k += co * ci * 9
        out[name + ".gamma"] = flat[k:k + co]
        k += co
        out[name + ".beta"] = flat[k:k + co]
        k += co
    out["head.w"] = flat[k:k + 2 * channels[0]].reshape(2, channels[0], 1, 1)
    k += 2 * channels[0]
    out["head.b"] = flat[k:k + 2]
    return out


def flatten_running(named, channels):
    parts = []
    for name, _, _ in conv_names(channels):
        parts += [named[name + ".mean"].reshape(-1), named[name + ".var"].reshape(-1)]
    return torch.cat([p.to(torch.float32) for p in parts])


def unflatten_running(flat, channels):
    out, k = {}, 0
    for name, _, co in conv_names(channels):
        out[name + ".mean"] = flat[k:k + co]
        out[name + ".var"] = flat[k + co:k + 2 * co]
        k += 2 * co
    return out


def _p(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _st(stream=None):
    return ctypes.c_void_p((torch.cuda.current_stream() if stream is None else stream).cuda_stream)


class MaskNet:
    """The U-Net h_alpha for scans of height x width, up to max_batch pairs per call."""

    def __init__(self, channels=(8, 16, 32, 64), height=256, width=256, max_batch=64):
        self.channels = tuple(int(c) for c in channels)
        L = _lib.lib()
        ch = (ctypes.c_int * 8)(*(list(self.channels) + [0] * (8 - len(self.channels))))
        cfg = _lib.UnetConfig(len(self.channels), ch, int(height), int(width), int(max_batch))
        h = ctypes.c_void_p()
        _lib.check_unet(L.fmbym_unet_create(ctypes.byref(h), ctypes.byref(cfg)), None)
        self._h = h
        self.height, self.width, self.max_batch = int(height), int(width), int(max_batch)
        self.n_params = int(L.fmbym_unet_param_count(h))
        self.n_running = int(L.fmbym_unet_running_count(h))

    def close(self):
        if getattr(self, "_h", None) is not None:
            _lib.lib().fmbym_unet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, params=None, running=None):
        st = _lib.lib().fmbym_unet_load(self._h, _st(), _p(params), _p(running))
        _lib.check_unet(st, self._h)

    def store(self):
        """(params, running, grads) as new device tensors."""
        p = torch.empty(self.n_params, device="cuda")
        r = torch.empty(self.n_running, device="cuda")
        g = torch.empty(self.n_params, device="cuda")
        _lib.check_unet(_lib.lib().fmbym_unet_store(self._h, _st(), _p(p), _p(r), _p(g)), self._h)
        return p, r, g

    def adam_state(self):
        """(first, second) Adam moments as new device tensors."""
        m = torch.empty(self.n_params, device="cuda")
        v = torch.empty(self.n_params, device="cuda")
        _lib.check_unet(_lib.lib().fmbym_unet_store_adam(self._h, _st(), _p(m), _p(v)), self._h)
        return m, v

    def load_adam(self, m=None, v=None):
        _lib.check_unet(_lib.lib().fmbym_unet_load_adam(self._h, _st(), _p(m), _p(v)), self._h)

    def forward(self, f, g, training=True, want_masks=False, f_out=None, g_out=None):
        n = f.shape[0]
        fo = torch.empty_like(f) if f_out is None else f_out
        go = torch.empty_like(g) if g_out is None else g_out
        m = torch.empty((n, 2) + tuple(f.shape[1:]), device=f.device) if want_masks else None
        st = _lib.lib().fmbym_unet_forward(self._h, _st(), n, _p(f), _p(g), int(bool(training)), _p(fo), _p(go), _p(m))
        _lib.check_unet(st, self._h)
        return fo, go, m

    def backward(self, f, g, dfo, dgo):
        st = _lib.lib().fmbym_unet_backward(self._h, _st(), f.shape[0], _p(f), _p(g), _p(dfo.contiguous()),
                                             _p(dgo.contiguous()))
        _lib.check_unet(st, self._h)

    def adam(self, lr, step, beta1=0.9, beta2=0.999, eps=1e-8):
        _lib.check_unet(_lib.lib().fmbym_unet_adam(self._h, _st(), lr, beta1, beta2, eps, int(step)), self._h)

    def layer_tensor(self, layer, which, n, shape):
        """Tensor `which` (0 y, 1 a, 2 dL/da, 3 dL/dy) of convolution `layer`, NHWC float32."""
        out = torch.empty(shape, device="cuda")
        st = _lib.lib().fmbym_unet_layer_tensor(self._h, _st(), int(layer), int(which), int(n), _p(out))
        _lib.check_unet(st, self._h)
        return out

    def launch_count(self):
        return int(_lib.lib().fmbym_unet_launch_count(self._h))

    def set_conv_path(self, path):
        """0: the flat-GEMM convolutions on mma.sync; 1: on tcgen05 (output channels a multiple of 64)."""
        _lib.check_unet(_lib.lib().fmbym_unet_set_conv_path(self._h, int(path)), self._h)

    def tc_timeouts(self):
        return int(_lib.lib().fmbym_unet_tc_timeouts(self._h))

    def set_tc_wait_limit(self, polls):
        """Polls before a tcgen05 producer's slot wait gives up (0: the default)."""
        _lib.check_unet(_lib.lib().fmbym_unet_set_tc_wait_limit(self._h, int(polls)), self._h)
