"""Helpers shared by the GPU parity tests: run the library and the FP64 oracle on the same seeded
inputs and compare them with the tolerances of the parity bar."""
import numpy as np

import oracle as O

TOL_THETA = 1e-4   # rad
TOL_T = 1e-3       # px (delta_xy units)
TOL_SURF = 1e-4    # max |gpu - oracle| / max |oracle| per score surface


def surf_err(a, b):
    return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / max(1e-300, np.max(np.abs(b))))


def argmax_ok(gpu, ref):
    """Identical argmax unless the oracle's top two are within 1e-5 of the max (a tie), in
    which case either of them passes."""
    ref = np.asarray(ref).ravel()
    gi = int(np.argmax(np.asarray(gpu).ravel()))
    order = np.argsort(ref)[::-1]
    if ref[order[0]] - ref[order[1]] > 1e-5 * abs(ref[order[0]]):
        return gi == int(order[0])
    return gi in (int(order[0]), int(order[1]))


def oracle_cfg(c):
    return O.make_cfg(c["n"], c["n_theta"], c["n_r"], c["temp_theta"], c["temp_xy"], c["delta_xy"],
                      c["window"], c["pad_mode"], c["score_norm"], c["band_lo"], c["band_hi"],
                      c.get("angle_score", 0), c.get("full_circle", 0), c.get("rotate_target", 0))


def check_pair(f, g, cfg, pose, c_theta=None, c_xy=None, tag=""):
    """Compares one pair's GPU outputs with the oracle.  The translation surface is compared with
    the oracle's stage 2 evaluated at the GPU's own theta, so that it measures the stage-2 kernels
    rather than the propagation of stage-1 rounding; the end-to-end pose is compared directly."""
    oc = oracle_cfg(cfg)
    r = O.pose(f, g, oc)
    assert abs(pose[0] - r["theta"]) <= TOL_THETA, (tag, "theta", pose[0], r["theta"])
    assert abs(pose[1] - r["tx"]) <= TOL_T, (tag, "tx", pose[1], r["tx"])
    assert abs(pose[2] - r["ty"]) <= TOL_T, (tag, "ty", pose[2], r["ty"])
    if c_theta is not None:
        assert surf_err(c_theta, r["c_theta"]) <= TOL_SURF, (tag, "c_theta", surf_err(c_theta, r["c_theta"]))
        assert argmax_ok(c_theta, r["c_theta"]), (tag, "argmax c_theta")
    if c_xy is not None:
        th = float(np.float32(pose[0]))
        if oc.get("rotate_target", 0) == 1:   # Alg. 1's own stage 2 correlates f with g turned back
            ref = O.xcorr2d(f, O.rotate(g, -th), oc["pad_mode"])
        else:
            ref = O.xcorr2d(O.rotate(f, th), g, oc["pad_mode"])
        assert surf_err(c_xy, ref) <= TOL_SURF, (tag, "c_xy", surf_err(c_xy, ref))
        assert argmax_ok(c_xy, ref), (tag, "argmax c_xy")
    return r
