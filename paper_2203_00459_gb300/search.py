"""Python face of the C ABI: a handle object over torch CUDA tensors and an autograd Function.

Only marshalling happens here: every step of the search runs in the CUDA library.  torch supplies
device memory and the current stream.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib


def size_cfg(n, n_theta, n_r, temp_theta=1.0, temp_xy=1.0, delta_xy=1.0, window=1, pad_mode=0,
             score_norm=0, band_lo=2.0, band_hi=None, angle_score=0, full_circle=0, rotate_target=0):
    """Parameters of one scan size (fmbym_size_cfg); band_hi defaults to N/2."""
    return dict(n=int(n), n_theta=int(n_theta), n_r=int(n_r), temp_theta=float(temp_theta),
                temp_xy=float(temp_xy), delta_xy=float(delta_xy), window=int(window), pad_mode=int(pad_mode),
                score_norm=int(score_norm), band_lo=float(band_lo),
                band_hi=float(n / 2 if band_hi is None else band_hi), angle_score=int(angle_score),
                full_circle=int(full_circle), rotate_target=int(rotate_target))


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def check_device_tensor(t, name, device, shape=None, min_numel=None):
    """Rejects, before any library call, a buffer the kernels cannot read or write as float32
    device memory: not a tensor, not on CUDA, not float32, not contiguous, on another device than
    the handle's, of the wrong shape, or holding fewer than min_numel elements.  A CPU tensor's
    address handed to a kernel would be an illegal access, a float64 or strided one silent garbage."""
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor, got {type(t).__name__}")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (got device {t.device})")
    if t.dtype != torch.float32:
        raise ValueError(f"{name} must be float32 (got {t.dtype})")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if device is not None and t.device != device:
        raise ValueError(f"{name} is on {t.device}, the handle on {device}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)} (got {tuple(t.shape)})")
    if min_numel is not None and t.numel() < min_numel:
        raise ValueError(f"{name} holds {t.numel()} elements; the pairs need {min_numel}")
    return t


def check_host_tensor(t, name, numel=None):
    """Rejects a host buffer of fmbym_pose_host that is not a contiguous CPU float32 tensor."""
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor, got {type(t).__name__}")
    if t.is_cuda or t.device.type != "cpu":
        raise ValueError(f"{name} must be a CPU tensor (got device {t.device})")
    if t.dtype != torch.float32:
        raise ValueError(f"{name} must be float32 (got {t.dtype})")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} holds {t.numel()} elements, expected {numel}")
    return t


class PoseSearch:
    """A library handle: plans and workspace for the given sizes and up to max_pairs pairs per call."""

    def __init__(self, sizes, max_pairs, device=None, flags=0):
        self.sizes = [dict(s) for s in sizes]
        self.max_pairs = int(max_pairs)
        self.flags = int(flags)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        L = _lib.lib()
        arr = (_lib.SizeCfg * len(self.sizes))(*[_lib.SizeCfg(**s) for s in self.sizes])
        self._arr = arr
        cfg = _lib.Config(len(self.sizes), arr, self.max_pairs, self.flags)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _lib.check(L.fmbym_create(ctypes.byref(h), ctypes.byref(cfg)), None)
        self._h = h

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("handle is closed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            _lib.lib().fmbym_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tuning(self, size=0):
        """The launch schedules of a size: dict(col_tile, angle_radii, rot_pixels, col_plan)."""
        v = (ctypes.c_int * len(_lib.TUNE_KNOBS))()
        _lib.check(_lib.lib().fmbym_get_tuning(self.handle, int(size), v), self.handle)
        return dict(zip(_lib.TUNE_KNOBS, list(v)))

    def set_tuning(self, size=0, **values):
        """Sets launch schedules of a size (unnamed knobs keep their values)."""
        cur = self.tuning(size)
        cur.update(values)
        v = (ctypes.c_int * len(_lib.TUNE_KNOBS))(*[int(cur[k]) for k in _lib.TUNE_KNOBS])
        _lib.check(_lib.lib().fmbym_set_tuning(self.handle, int(size), v), self.handle)

    def workspace_bytes(self):
        return int(_lib.lib().fmbym_workspace_bytes(self.handle))

    # -- layout helpers ------------------------------------------------------------------------
    def _scans(self, f, g, size_idx, offsets):
        """Validates the scan buffers f and g against the handle and the pair layout (before any
        library call) and returns _layout's tuple."""
        check_device_tensor(f, "f", self.device)
        check_device_tensor(g, "g", self.device, shape=f.shape)
        lay = self._layout(f, size_idx, offsets)
        n_pairs, si, off, _, ns = lay
        if off is not None and off.size != n_pairs:
            raise ValueError("offsets must have one entry per pair")
        if off is None:
            end = sum(n * n for n in ns)
        else:
            end = max((int(o) + n * n for o, n in zip(off, ns)), default=0)
        if end > f.numel():
            raise ValueError(f"the pairs reach element {end}, beyond the {f.numel()} elements of f and g")
        return lay

    def _layout(self, f, size_idx, offsets):
        """Returns (n_pairs, size_idx array or None, offsets array or None, n_theta list, N list).
        Offsets without size_idx place pairs of size 0."""
        if size_idx is None and offsets is not None:
            size_idx = np.zeros(len(offsets), np.int32)
        if size_idx is None:
            if f.dim() != 3:
                raise ValueError("f must be [B, N, N] when size_idx is not given")
            n_pairs = f.shape[0]
            if f.shape[1] != self.sizes[0]["n"] or f.shape[2] != self.sizes[0]["n"]:
                raise ValueError("scan size does not match size 0 of the handle")
            return n_pairs, None, None, [self.sizes[0]["n_theta"]] * n_pairs, [self.sizes[0]["n"]] * n_pairs
        si = np.ascontiguousarray(np.asarray(size_idx, dtype=np.int32))
        n_pairs = si.size
        if n_pairs and (si.min() < 0 or si.max() >= len(self.sizes)):
            raise ValueError("size_idx out of range")
        off = None if offsets is None else np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        return n_pairs, si, off, [self.sizes[i]["n_theta"] for i in si], [self.sizes[i]["n"] for i in si]

    # -- calls ---------------------------------------------------------------------------------
    def pose(self, f, g, size_idx=None, offsets=None, want_c_theta=False, want_c_xy=False, stream=None,
             out=None):
        """Forward search; returns dict(pose [B,3], c_theta (flat) or None, c_xy (like f) or None)."""
        n_pairs, si, off, nts, _ = self._scans(f, g, size_idx, offsets)
        if out is not None:
            check_device_tensor(out, "out", self.device, shape=(n_pairs, 3))
        pose = out if out is not None else torch.empty((n_pairs, 3), device=f.device, dtype=torch.float32)
        ct = torch.empty(sum(nts), device=f.device, dtype=torch.float32) if want_c_theta else None
        cxy = torch.empty_like(f) if want_c_xy else None
        st = _lib.lib().fmbym_pose(self.handle, _stream(stream), n_pairs,
                                   None if si is None else si.ctypes.data_as(ctypes.c_void_p),
                                   None if off is None else off.ctypes.data_as(ctypes.c_void_p),
                                   _ptr(f), _ptr(g), _ptr(pose), _ptr(ct), _ptr(cxy))
        _lib.check(st, self.handle)
        return dict(pose=pose, c_theta=ct, c_xy=cxy)

    def pose_backward(self, f, g, dpose, size_idx=None, offsets=None, stream=None):
        """Adjoint: (df, dg) given dL/dpose [B, 3]."""
        n_pairs, si, off, _, _ = self._scans(f, g, size_idx, offsets)
        check_device_tensor(dpose, "dpose", self.device, shape=(n_pairs, 3))
        df = torch.empty_like(f)
        dg = torch.empty_like(g)
        st = _lib.lib().fmbym_pose_backward(self.handle, _stream(stream), n_pairs,
                                            None if si is None else si.ctypes.data_as(ctypes.c_void_p),
                                            None if off is None else off.ctypes.data_as(ctypes.c_void_p),
                                            _ptr(f), _ptr(g), _ptr(dpose), _ptr(df), _ptr(dg))
        _lib.check(st, self.handle)
        return df, dg

    def pose_train(self, f, g, gt, kind=1, size_idx=None, offsets=None, stream=None, out=None):
        """One training step of the search: forward, the Eq. 13 loss against gt [B, 3] (kind 1 = L1,
        2 = L2) and the adjoint of that loss, the adjoint reading the forward's intermediates instead
        of recomputing them.  out: optional preallocated (pose, loss, dpose, df, dg).  Returns
        (pose, loss, dpose, df, dg)."""
        n_pairs, si, off, _, _ = self._scans(f, g, size_idx, offsets)
        check_device_tensor(gt, "gt", self.device, shape=(n_pairs, 3))
        if out is not None:
            if len(out) != 5:
                raise ValueError("out must be (pose, loss, dpose, df, dg)")
            for t, nm, shp in zip(out, ("pose", "loss", "dpose", "df", "dg"),
                                  ((n_pairs, 3), (1,), (n_pairs, 3), tuple(f.shape), tuple(g.shape))):
                check_device_tensor(t, "out." + nm, self.device, shape=shp)
        if out is None:
            out = (torch.empty((n_pairs, 3), device=f.device, dtype=torch.float32),
                   torch.empty(1, device=f.device, dtype=torch.float32),
                   torch.empty((n_pairs, 3), device=f.device, dtype=torch.float32),
                   torch.empty_like(f), torch.empty_like(g))
        pose, loss, dpose, df, dg = out
        st = _lib.lib().fmbym_pose_train(self.handle, _stream(stream), n_pairs,
                                         None if si is None else si.ctypes.data_as(ctypes.c_void_p),
                                         None if off is None else off.ctypes.data_as(ctypes.c_void_p),
                                         _ptr(f), _ptr(g), _ptr(gt), int(kind), _ptr(pose), _ptr(loss),
                                         _ptr(dpose), _ptr(df), _ptr(dg))
        _lib.check(st, self.handle)
        return pose, loss, dpose, df, dg

    def pose_exhaustive(self, f, g, angles, size=0, offsets=None, want_peaks=False, stream=None, out=None):
        """Exhaustive rotate-then-correlate search over the candidate headings `angles` (radians):
        returns dict(pose [B, 3], peaks [B, len(angles)] or None).  Every pair has size `size`."""
        check_device_tensor(f, "f", self.device)
        check_device_tensor(g, "g", self.device, shape=f.shape)
        if not 0 <= int(size) < len(self.sizes):
            raise ValueError("size index out of range")
        nn = self.sizes[int(size)]["n"] ** 2
        if offsets is None:
            n_pairs = f.shape[0]
            off = None
        else:
            off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
            n_pairs = off.size
        end = n_pairs * nn if off is None else max((int(o) + nn for o in off), default=0)
        if end > f.numel():
            raise ValueError(f"the pairs reach element {end}, beyond the {f.numel()} elements of f and g")
        if out is not None:
            check_device_tensor(out, "out", self.device, shape=(n_pairs, 3))
        ang = np.ascontiguousarray(np.asarray(angles, dtype=np.float32))
        pose = out if out is not None else torch.empty((n_pairs, 3), device=f.device, dtype=torch.float32)
        peaks = torch.empty((n_pairs, ang.size), device=f.device, dtype=torch.float32) if want_peaks else None
        st = _lib.lib().fmbym_pose_exhaustive(self.handle, _stream(stream), n_pairs, int(size),
                                              None if off is None else off.ctypes.data_as(ctypes.c_void_p),
                                              _ptr(f), _ptr(g), int(ang.size), ang.ctypes.data_as(ctypes.c_void_p),
                                              _ptr(pose), _ptr(peaks))
        _lib.check(st, self.handle)
        return dict(pose=pose, peaks=peaks)

    def pose_loss(self, pose, gt, kind=1, loss=None, dpose=None, stream=None):
        """Eq. 13 loss (kind 1 = L1, 2 = L2; mean over pairs) and dloss/dpose, on the device."""
        check_device_tensor(pose, "pose", self.device)
        n_pairs = pose.shape[0]
        check_device_tensor(pose, "pose", self.device, shape=(n_pairs, 3))
        check_device_tensor(gt, "gt", self.device, shape=(n_pairs, 3))
        if loss is not None:
            check_device_tensor(loss, "loss", self.device, shape=(1,))
        if dpose is not None:
            check_device_tensor(dpose, "dpose", self.device, shape=(n_pairs, 3))
        loss = torch.empty(1, device=pose.device) if loss is None else loss
        dpose = torch.empty_like(pose) if dpose is None else dpose
        st = _lib.lib().fmbym_pose_loss(self.handle, _stream(stream), n_pairs, _ptr(pose),
                                        _ptr(gt), int(kind), _ptr(loss), _ptr(dpose))
        _lib.check(st, self.handle)
        return loss, dpose

    def pose_host(self, f_host, g_host, size_idx=None, offsets=None, stream=None):
        """Forward search from host (CPU, ideally pinned) tensors; returns the pose as a CPU tensor.
        Copies in, computes and copies out inside the call, which synchronises the stream."""
        check_host_tensor(f_host, "f_host")
        check_host_tensor(g_host, "g_host", numel=f_host.numel())
        if size_idx is None:
            n_pairs = f_host.shape[0]
            si = off = None
        else:
            si = np.ascontiguousarray(np.asarray(size_idx, dtype=np.int32))
            n_pairs = si.size
            off = None if offsets is None else np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        pose = torch.empty((n_pairs, 3), dtype=torch.float32, pin_memory=f_host.is_pinned())
        st = _lib.lib().fmbym_pose_host(self.handle, _stream(stream), n_pairs,
                                        None if si is None else si.ctypes.data_as(ctypes.c_void_p),
                                        None if off is None else off.ctypes.data_as(ctypes.c_void_p),
                                        ctypes.c_longlong(f_host.numel()), _ptr(f_host), _ptr(g_host), _ptr(pose))
        _lib.check(st, self.handle)
        return pose


    def pose_train_host(self, f_host, g_host, gt_host, kind=1, size_idx=None, offsets=None, stream=None, out=None):
        """fmbym_pose_train from host (CPU float32, ideally pinned) tensors: copies f, g, gt in, runs
        the training call, copies pose, loss, df and dg out, and synchronises the stream.  out:
        optional preallocated host (pose [B, 3], loss [1], df like f, dg like g).  Returns
        (pose, loss, df, dg) as CPU tensors."""
        check_host_tensor(f_host, "f_host")
        check_host_tensor(g_host, "g_host", numel=f_host.numel())
        if size_idx is None:
            n_pairs = f_host.shape[0]
            si = off = None
        else:
            si = np.ascontiguousarray(np.asarray(size_idx, dtype=np.int32))
            n_pairs = si.size
            off = None if offsets is None else np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        check_host_tensor(gt_host, "gt_host", numel=3 * n_pairs)
        pin = f_host.is_pinned()
        if out is None:
            out = (torch.empty((n_pairs, 3), dtype=torch.float32, pin_memory=pin),
                   torch.empty(1, dtype=torch.float32, pin_memory=pin),
                   torch.empty_like(f_host, pin_memory=pin), torch.empty_like(g_host, pin_memory=pin))
        for t, nm, k in zip(out, ("pose", "loss", "df", "dg"), (3 * n_pairs, 1, f_host.numel(), g_host.numel())):
            check_host_tensor(t, "out." + nm, numel=k)
        pose, loss, df, dg = out
        st = _lib.lib().fmbym_pose_train_host(self.handle, _stream(stream), n_pairs,
                                              None if si is None else si.ctypes.data_as(ctypes.c_void_p),
                                              None if off is None else off.ctypes.data_as(ctypes.c_void_p),
                                              ctypes.c_longlong(f_host.numel()), _ptr(f_host), _ptr(g_host),
                                              _ptr(gt_host), int(kind), _ptr(pose), _ptr(loss), _ptr(df), _ptr(dg))
        _lib.check(st, self.handle)
        return pose, loss, df, dg


def fp32_fma_rate(iters=50000, reps=3, stream=None):
    """The device's measured FP32 multiply-add rate (fmbym_fp32_fma_rate), in multiply-adds/s."""
    v = ctypes.c_double()
    st = _lib.lib().fmbym_fp32_fma_rate(_stream(stream), int(iters), int(reps), ctypes.byref(v))
    if st != 0:
        raise _lib.FmbymError(st, "fmbym_fp32_fma_rate")
    return v.value


class PoseFunction(torch.autograd.Function):
    """pose = ScanMatch(f, g) with the library's hand-written adjoint as backward."""

    @staticmethod
    def forward(ctx, f, g, search, size_idx=None, offsets=None):
        ctx.search, ctx.size_idx, ctx.offsets = search, size_idx, offsets
        ctx.save_for_backward(f, g)
        return search.pose(f.contiguous(), g.contiguous(), size_idx, offsets)["pose"]

    @staticmethod
    def backward(ctx, dpose):
        f, g = ctx.saved_tensors
        df, dg = ctx.search.pose_backward(f.contiguous(), g.contiguous(), dpose.contiguous(), ctx.size_idx,
                                          ctx.offsets)
        return df, dg, None, None, None


def scan_match(f, g, search, size_idx=None, offsets=None):
    """Differentiable batched ScanMatch (Alg. 1): pose [B, 3] = (theta, t_x, t_y)."""
    return PoseFunction.apply(f, g, search, size_idx, offsets)


def polar_to_cartesian(polar, n, delta_xy, range_res, out=None, stream=None):
    """Radar front end (fmbym_polar_to_cartesian): polar scans [B, n_az, n_range] (CUDA float32,
    contiguous) -> Cartesian scans [B, n, n] for the search."""
    if polar.dim() == 2:
        polar = polar.unsqueeze(0)
    if not (polar.is_cuda and polar.dtype == torch.float32 and polar.is_contiguous()):
        raise ValueError("polar must be a contiguous CUDA float32 tensor [B, n_az, n_range]")
    b, n_az, n_range = polar.shape
    if out is None:
        out = torch.empty((b, n, n), dtype=torch.float32, device=polar.device)
    st = _lib.lib().fmbym_polar_to_cartesian(_stream(stream), b, _ptr(polar), n_az, n_range, float(range_res), int(n),
                                            float(delta_xy), _ptr(out))
    if st != 0:
        raise _lib.FmbymError(st, "fmbym_polar_to_cartesian")
    return out
