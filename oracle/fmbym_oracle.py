"""Plain FP64 CPU oracle of the decoupled Fourier pose search (Fast-MbyM, Sec. III-C, Alg. 1).

TEST INFRASTRUCTURE ONLY. Nothing on the product path imports this module: only the
tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs
of ``bench.py`` may call it.  It shares no code with the CUDA library.

Every function follows one step of Alg. 1 in the paper's order, in float64.  Every 2D DFT is the
direct sum of its definition (Eq. 4), F[v, u] = sum_y sum_x x[y, x] exp(-2 pi i (v y + u x) / N),
evaluated separably as a product with explicit DFT matrices whose exponents are reduced modulo N
in integers (a matrix product is the only library primitive).  The translation scores are the
correlation theorem over those direct DFTs, as Alg. 1 computes them; xcorr2d_brute is the sum of
the definition itself, sum_x f'(x) g(x + s), lag by lag, and the angle scores are the
brute-force circular double sum.  numpy's FFT survives only behind cfg["route"] = "fft", a faster
route of the same sums kept as a cross-check and for the central-difference loops.  Readings of
the places where the paper is silent or ambiguous:

* A1  correlations conjugate the first operand: c = iFFT(conj(FFT a) * FFT b)  (Eq. 3, 7, 8
      define correlation; Alg. 1 prints the product without the conjugate).
* A2  the rotation score is Eq. 7 at radial lag 0: c_theta[k] = sum_r sum_a a_f[a,r] a_g[a+k,r].
* A3  a periodic Hann window w[n] = 0.5 - 0.5 cos(2 pi n / N), applied in stage 1 only.
* A4  band-pass = hard radial annulus band_lo <= rho <= band_hi on the DFT grid (rho in bins).
* A5  soft-argmax scores are z-scored (population std) before softmax(z / T); score_norm=1
      gives the literal softmax(c / T).
* A6  candidates are integer lags times the bin size: k in [-(n//2), n - n//2).
* A7  zero padding to P = 2N (linear correlation), lags s in [-N/2, N/2) per axis;
      pad_mode=1 is the N-periodic (circular) correlation.
* A8  the source f is rotated by +theta about c = (N/2, N/2) (bilinear, zero outside); the
      translation is then the stage-2 soft-argmax directly, so BuildSO2 / MatMul of Alg. 1
      reduce to the identity.  theta > 0 turns +x (column) toward +y (row).
* A9  polar angles span [0, pi) (|F| of a real image is centrosymmetric).
* A14 |z| has derivative z/|z| (0 at z = 0); bilinear weights use the floor cell.

Layouts: images are [N, N] row-major, y = row, x = column.  Score surfaces are stored in lag
order (index 0 is the most negative lag).  The pose is (theta [rad], t_x, t_y [delta_xy units]).
"""
from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------------------------------------
# configuration (Alg. 1 signature; defaults are the readings listed above)
# ----------------------------------------------------------------------------------------------

def make_cfg(n, n_theta, n_r, temp_theta=1.0, temp_xy=1.0, delta_xy=1.0, window=1, pad_mode=0,
             score_norm=0, band_lo=2.0, band_hi=None, angle_score=0, full_circle=0, rotate_target=0,
             route="direct"):
    """Alg. 1 parameters (n_theta, T_theta, n_xy = n, delta_xy, T_xy) plus the A3-A7 switches;
    angle_score 0 is Eq. 7 (reading A2), 1 the mean over radial lags that Alg. 1 prints;
    full_circle 1 resolves the heading over the full circle (see pose()); rotate_target 0 rotates
    the source f by theta (reading A8), 1 is Alg. 1's own stage 2: g turned back by theta, then the
    translation found between f and it turned by theta (see pose()); route "direct" evaluates the
    DFTs as their direct sums, "fft" through numpy's FFT (the same sums, faster)."""
    if int(rotate_target) == 1 and int(full_circle) == 1:
        raise ValueError("rotate_target 1 is defined for the half-circle search only")
    if route not in ("direct", "fft"):
        raise ValueError("route must be 'direct' or 'fft'")
    return dict(n=int(n), n_theta=int(n_theta), n_r=int(n_r), temp_theta=float(temp_theta),
                temp_xy=float(temp_xy), delta_xy=float(delta_xy), window=int(window),
                pad_mode=int(pad_mode), score_norm=int(score_norm), band_lo=float(band_lo),
                band_hi=float(n / 2 if band_hi is None else band_hi), angle_score=int(angle_score),
                full_circle=int(full_circle), rotate_target=int(rotate_target), route=route)


def lags(n):
    """Candidate integer lags of a length-n circular score vector (A6): -(n//2) ... n-1-n//2."""
    return np.arange(n) - n // 2


# ----------------------------------------------------------------------------------------------
# stage 1: rotation (Alg. 1 stage 1, Eq. 4-7)
# ----------------------------------------------------------------------------------------------

def hann(n):
    """Periodic Hann window (Alg. 1 HanningFilter; reading A3)."""
    i = np.arange(n, dtype=np.float64)
    return 0.5 - 0.5 * np.cos(2.0 * np.pi * i / n)


def band_mask(n, band_lo, band_hi):
    """Radial band-pass on the half spectrum [N, N/2+1] (Alg. 1 BandPassFilter; reading A4)."""
    v = np.arange(n)
    vs = np.where(v <= n // 2, v, v - n).astype(np.float64)
    u = np.arange(n // 2 + 1, dtype=np.float64)
    rho = np.sqrt(vs[:, None] ** 2 + u[None, :] ** 2)
    return ((rho >= band_lo) & (rho <= band_hi)).astype(np.float64)


def dft_matrix(n, rows=None, sign=-1):
    """The kernel of the length-n DFT sum: W[k, j] = exp(sign 2 pi i k j / n) for frequency (or lag)
    k in `rows` (default 0..n-1) and sample j < n.  The product k j is reduced modulo n in integers
    first, so every entry is a root of unity rounded once."""
    k = np.arange(n) if rows is None else np.asarray(rows, dtype=np.int64)
    kj = np.mod(np.outer(k, np.arange(n, dtype=np.int64)), n)
    return np.exp(sign * 2j * np.pi * kj.astype(np.float64) / n)


def spectrum(x, cfg):
    """Windowed 2D DFT of a real scan, half plane u in [0, N/2] (Alg. 1 FFT2d; Eq. 4).

    F[v, u] = sum_y sum_x w[y] w[x] x[y, x] exp(-2 pi i (v y + u x) / N), the direct sum done as
    the separable matrix product W_N X W_half^T."""
    n = cfg["n"]
    x = np.asarray(x, dtype=np.float64)
    if cfg["window"]:
        w = hann(n)
        x = x * w[:, None] * w[None, :]
    if cfg.get("route", "direct") == "fft":
        return np.fft.rfft2(x)
    return dft_matrix(n) @ x @ dft_matrix(n, np.arange(n // 2 + 1)).T


def magnitude(F, cfg):
    """Band-passed magnitude spectrum a = |h_band o F| on the half plane (Alg. 1 Abs; Eq. 6)."""
    return np.abs(F) * band_mask(cfg["n"], cfg["band_lo"], cfg["band_hi"])


def polar_points(n, n_theta, n_r):
    """Sample points of Cart2Pol: alpha_a = a pi / n_theta, rho_r = r (N/2) / n_r (A9, A4).

    Returns (u, v) arrays [n_theta, n_r]: u = rho cos(alpha) along x, v = rho sin(alpha) along y."""
    alpha = np.arange(n_theta, dtype=np.float64) * np.pi / n_theta
    rho = np.arange(n_r, dtype=np.float64) * (n / 2.0) / n_r
    return rho[None, :] * np.cos(alpha)[:, None], rho[None, :] * np.sin(alpha)[:, None]


def half_index(n, vi, ui):
    """Map integer frequencies (vi, ui) of the N-periodic full spectrum onto the half plane.

    |F| of a real image satisfies |F(-v,-u)| = |F(v,u)| (Hermitian), so a column ui > N/2 is
    read at (-vi, -ui).  Returns index arrays into the [N, N/2+1] half spectrum."""
    vi = np.mod(vi, n)
    ui = np.mod(ui, n)
    mirror = ui > n // 2
    vv = np.where(mirror, np.mod(-vi, n), vi)
    uu = np.where(mirror, n - ui, ui)
    return vv, uu


def cart2pol(a, cfg):
    """Bilinear resampling of the magnitude spectrum onto the (angle x radius) grid (Alg. 1
    Cart2Pol; bilinear as in the spatial transformer, Sec. III-C).  Returns [n_theta, n_r]."""
    n = cfg["n"]
    u, v = polar_points(n, cfg["n_theta"], cfg["n_r"])
    x0 = np.floor(u)
    y0 = np.floor(v)
    fx = u - x0
    fy = v - y0
    x0 = x0.astype(np.int64)
    y0 = y0.astype(np.int64)
    out = np.zeros_like(u)
    for dy, wy in ((0, 1.0 - fy), (1, fy)):
        for dx, wx in ((0, 1.0 - fx), (1, fx)):
            vv, uu = half_index(n, y0 + dy, x0 + dx)
            out += wy * wx * a[vv, uu]
    return out


def angle_scores(af, ag):
    """Circular cross-correlation along angle summed over radius (Eq. 7 with reading A2):
    c[k] = sum_a sum_r af[a, r] ag[(a + k) mod n_theta, r] for k in lags(n_theta)."""
    n = af.shape[0]
    c = np.empty(n, dtype=np.float64)
    for i, k in enumerate(lags(n)):
        c[i] = np.sum(af * np.roll(ag, -k, axis=0))
    return c


def angle_scores_marginal(af, ag):
    """The rotation score Alg. 1 prints: the 2D correlation of the (angle x radius) polar arrays,
    circular in both (WrapPad), averaged over the radial lags.  Summing a circular correlation over
    all radial lags pairs every radius with every other once, so it is the circular correlation
    along angle of the radial sums, divided by n_r:
    c[k] = (1/n_r) sum_a m_f[a] m_g[(a + k) mod n_theta], m = sum over radius."""
    n_r = af.shape[1]
    return angle_scores(af.sum(axis=1, keepdims=True), ag.sum(axis=1, keepdims=True)) / n_r


def angle_scores_any(af, ag, cfg):
    return angle_scores_marginal(af, ag) if cfg.get("angle_score", 0) == 1 else angle_scores(af, ag)


def normalise_scores(c, score_norm):
    """A5: z = (c - mean) / std (population) for score_norm=0, the raw scores for 1."""
    c = np.asarray(c, dtype=np.float64)
    if score_norm == 1:
        return c.copy()
    mu = c.mean()
    sd = np.sqrt(np.mean((c - mu) ** 2))
    if sd == 0.0:
        return np.zeros_like(c)
    return (c - mu) / sd


def soft_argmax(c, temp, score_norm):
    """Temperature softmax over the scores (Alg. 1 SoftArgMax; Sec. III-C).

    Returns the probabilities p (same shape as c); the expectation is taken by the caller
    over the candidate coordinates."""
    z = normalise_scores(c, score_norm).ravel() / temp
    z = z - z.max()
    e = np.exp(z)
    return (e / e.sum()).reshape(np.shape(c))


# ----------------------------------------------------------------------------------------------
# stage 2: translation (Alg. 1 stage 2, Eq. 8)
# ----------------------------------------------------------------------------------------------

def rotate(x, theta):
    """Rotate a scan by +theta about c = (N/2, N/2) with bilinear sampling and zero fill
    (Alg. 1 Rotate; reading A8).  out[Y, X] = bilinear(x, c + R(-theta) ([X, Y] - c))."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    c = n / 2.0
    Y, X = np.meshgrid(np.arange(n, dtype=np.float64), np.arange(n, dtype=np.float64), indexing="ij")
    ct, st = np.cos(theta), np.sin(theta)
    dx, dy = X - c, Y - c
    px = c + ct * dx + st * dy
    py = c - st * dx + ct * dy
    x0 = np.floor(px)
    y0 = np.floor(py)
    fx = px - x0
    fy = py - y0
    x0 = x0.astype(np.int64)
    y0 = y0.astype(np.int64)
    out = np.zeros_like(px)
    for oy, wy in ((0, 1.0 - fy), (1, fy)):
        for ox, wx in ((0, 1.0 - fx), (1, fx)):
            yy, xx = y0 + oy, x0 + ox
            inside = (yy >= 0) & (yy < n) & (xx >= 0) & (xx < n)
            out += np.where(inside, wy * wx * x[np.clip(yy, 0, n - 1), np.clip(xx, 0, n - 1)], 0.0)
    return out


def xcorr2d(fr, g, pad_mode, route="direct"):
    """Translation scores c[s] = sum_x fr(x) g(x + s), s in lags(N)^2 (Eq. 3 and 8), through the
    correlation theorem as in Alg. 1: ZeroPad to P = 2N, then iDFT2d(conj(DFT2d(fr)) o DFT2d(g))
    at the kept lags (A1, A7).  pad_mode=1: N-periodic correlation (P = N).

    route "direct": each DFT is its direct sum.  The padded entries are zero, so the forward sums
    run over the N x N scan, Fp = W_P[:, :N] fr W_P[:, :N]^T, and the inverse sum
    c[s] = P^-2 sum_k sum_l conj(Fp) Gp exp(+2 pi i (k s_y + l s_x) / P) is evaluated only at the
    kept lags s mod P."""
    n = fr.shape[0]
    p = n if pad_mode == 1 else 2 * n
    fr = np.asarray(fr, np.float64)
    g = np.asarray(g, np.float64)
    s = np.mod(lags(n), p)
    if route == "fft":
        Fp = np.fft.fft2(fr, s=(p, p))
        Gp = np.fft.fft2(g, s=(p, p))
        full = np.real(np.fft.ifft2(np.conj(Fp) * Gp))
        return full[np.ix_(s, s)]
    Wp = dft_matrix(p)[:, :n]
    Fp = Wp @ fr @ Wp.T
    Gp = Wp @ g @ Wp.T
    Wi = dft_matrix(p, s, sign=+1)
    return np.real(Wi @ (np.conj(Fp) * Gp) @ Wi.T) / (p * p)


def xcorr2d_brute(fr, g, pad_mode, lag_list=None):
    """The translation scores by brute force, c[s] = sum_x fr(x) g(x + s) summed for each lag on
    its own (Eq. 3, 8; no transform).  Returns the full surface over lags(N)^2 in lag order, or,
    given lag_list [(s_y, s_x), ...], the scores at those lags."""
    n = fr.shape[0]
    if lag_list is not None:
        return np.array([xcorr2d_direct(fr, g, int(sy), int(sx), pad_mode) for sy, sx in lag_list])
    L = lags(n)
    c = np.empty((n, n))
    for i, sy in enumerate(L):
        for j, sx in enumerate(L):
            c[i, j] = xcorr2d_direct(fr, g, int(sy), int(sx), pad_mode)
    return c


def xcorr2d_direct(fr, g, sy, sx, pad_mode):
    """One translation score by its definition, sum_x fr(x) g(x + s) (Eq. 3), no FFT.
    Zero outside the scan for pad_mode=0, N-periodic for pad_mode=1."""
    n = fr.shape[0]
    fr = np.asarray(fr, np.float64)
    g = np.asarray(g, np.float64)
    if pad_mode == 1:
        return float(np.sum(fr * np.roll(g, (-sy, -sx), axis=(0, 1))))
    y0, y1 = max(0, -sy), min(n, n - sy)
    x0, x1 = max(0, -sx), min(n, n - sx)
    if y0 >= y1 or x0 >= x1:
        return 0.0
    return float(np.sum(fr[y0:y1, x0:x1] * g[y0 + sy:y1 + sy, x0 + sx:x1 + sx]))


# ----------------------------------------------------------------------------------------------
# the whole search (Alg. 1)
# ----------------------------------------------------------------------------------------------

def pose(f, g, cfg, keep=False):
    """ScanMatch(f, g) of Alg. 1 under the readings above.

    Returns dict(theta, tx, ty, c_theta [n_theta], c_xy [N, N]) and, with keep=True, every
    intermediate the backward pass needs."""
    n, nt = cfg["n"], cfg["n_theta"]
    f = np.asarray(f, np.float64)
    g = np.asarray(g, np.float64)
    # stage 1 (Alg. 1 stage 1)
    Ff, Fg = spectrum(f, cfg), spectrum(g, cfg)
    af, ag = magnitude(Ff, cfg), magnitude(Fg, cfg)
    pf, pg = cart2pol(af, cfg), cart2pol(ag, cfg)
    c_theta = angle_scores_any(pf, pg, cfg)
    p_theta = soft_argmax(c_theta, cfg["temp_theta"], cfg["score_norm"])
    d_theta = np.pi / nt
    theta = float(np.sum(p_theta * lags(nt) * d_theta))
    # stage 2 (Alg. 1 stage 2)
    if cfg.get("rotate_target", 0) == 1:
        # Alg. 1 as printed: Rotate g, correlate f with it, then BuildSO2 / MatMul on the translation.
        # With g(x) = f'(x - t) and f' = rotate(f, theta) (reading A8), g turned back by theta is f
        # shifted by t' = R(-theta) t, so the scores peak at t' and t = R(theta) t'
        gr = rotate(g, -theta)
        c_xy = xcorr2d(f, gr, cfg["pad_mode"], cfg.get("route", "direct"))
        p_xy = soft_argmax(c_xy, cfg["temp_xy"], cfg["score_norm"])
        s = lags(n) * cfg["delta_xy"]
        tpx = float(np.sum(p_xy * s[None, :]))
        tpy = float(np.sum(p_xy * s[:, None]))
        ct, st = np.cos(theta), np.sin(theta)
        out = dict(theta=theta, tx=float(ct * tpx - st * tpy), ty=float(st * tpx + ct * tpy), c_theta=c_theta,
                   c_xy=c_xy, tpx=tpx, tpy=tpy)
        if keep:
            out.update(Ff=Ff, Fg=Fg, af=af, ag=ag, pf=pf, pg=pg, p_theta=p_theta, gr=gr, p_xy=p_xy)
        return out
    fr = rotate(f, theta)
    c_xy = xcorr2d(fr, g, cfg["pad_mode"], cfg.get("route", "direct"))
    if cfg.get("full_circle", 0) == 1:
        # |F| cannot tell theta from theta + pi (Sec. V suggests the decoupled search for arbitrary
        # headings): correlate at both and keep the one whose translation peak is higher
        theta_b = theta + np.pi if theta < 0 else theta - np.pi
        fr_b = rotate(f, theta_b)
        c_b = xcorr2d(fr_b, g, cfg["pad_mode"], cfg.get("route", "direct"))
        if c_b.max() > c_xy.max():
            theta, fr, c_xy = theta_b, fr_b, c_b
    p_xy = soft_argmax(c_xy, cfg["temp_xy"], cfg["score_norm"])
    s = lags(n) * cfg["delta_xy"]
    tx = float(np.sum(p_xy * s[None, :]))
    ty = float(np.sum(p_xy * s[:, None]))
    out = dict(theta=theta, tx=tx, ty=ty, c_theta=c_theta, c_xy=c_xy)
    if keep:
        out.update(Ff=Ff, Fg=Fg, af=af, ag=ag, pf=pf, pg=pg, p_theta=p_theta, fr=fr, p_xy=p_xy)
    return out


def pose_exhaustive(f, g, cfg, angles):
    """The exhaustive rotate-then-correlate search that the decoupled search replaces (the
    brute-force "raw" method of Tab. IIIa, Sec. I and III): every candidate heading theta_k is
    tried by rotating the source (as stage 2 does) and correlating it with the target over the
    same lags; the heading is the candidate with the highest correlation peak, the translation
    that candidate's soft-argmax.  Returns dict(k, theta, tx, ty, peaks [len(angles)])."""
    n = cfg["n"]
    f = np.asarray(f, np.float64)
    g = np.asarray(g, np.float64)
    s = lags(n) * cfg["delta_xy"]
    peaks = np.empty(len(angles))
    best = None
    for k, th in enumerate(angles):
        c_xy = xcorr2d(rotate(f, float(th)), g, cfg["pad_mode"], cfg.get("route", "direct"))
        peaks[k] = c_xy.max()
        if best is None or peaks[k] > peaks[best[0]]:
            best = (k, c_xy)
    k, c_xy = best
    p_xy = soft_argmax(c_xy, cfg["temp_xy"], cfg["score_norm"])
    return dict(k=k, theta=float(angles[k]), tx=float(np.sum(p_xy * s[None, :])),
                ty=float(np.sum(p_xy * s[:, None])), peaks=peaks)


def pose_batch(fs, gs, cfg):
    """Alg. 1 applied to each pair of a batch; returns (pose [B,3], c_theta [B,n_theta], c_xy [B,N,N])."""
    res = [pose(f, g, cfg) for f, g in zip(fs, gs)]
    P = np.array([[r["theta"], r["tx"], r["ty"]] for r in res])
    return P, np.stack([r["c_theta"] for r in res]), np.stack([r["c_xy"] for r in res])


# ----------------------------------------------------------------------------------------------
# adjoint of the whole search (differentiability, Sec. III-C and III-D): hand-derived, FP64
# ----------------------------------------------------------------------------------------------

def soft_argmax_backward(c, p, q, temp, score_norm):
    """Adjoint of E_p[coord] with p = softmax(normalise(c) / T), given q = dL/dp.

    softmax: dy = p (q - <p, q>); temperature: dz = dy / T; z-score (population std):
    dc = (dz - mean(dz) - z mean(dz z)) / std."""
    shape = np.shape(c)
    p = np.asarray(p, np.float64).ravel()
    q = np.asarray(q, np.float64).ravel()
    dz = p * (q - np.dot(p, q)) / temp
    if score_norm == 1:
        return dz.reshape(shape)
    c = np.asarray(c, np.float64).ravel()
    mu = c.mean()
    sd = np.sqrt(np.mean((c - mu) ** 2))
    if sd == 0.0:
        return np.zeros(shape)
    z = (c - mu) / sd
    return ((dz - dz.mean() - z * np.mean(dz * z)) / sd).reshape(shape)


def xcorr2d_backward(fr, g, dc, pad_mode, route="direct"):
    """Adjoint of c[s] = sum_x fr(x) g(x + s) (Eq. 3, lags s in lags(N)^2).

    d fr(x) = sum_s dc[s] g(x + s)  (correlation of dc with g)
    d g(y)  = sum_s dc[s] fr(y - s) (convolution of dc with fr)
    both evaluated through the same padded transforms as the forward pass: with D the lag surface
    embedded at s mod P, d fr = iDFT(conj(DFT D) DFT g) and d g = iDFT(DFT D DFT fr), read on the
    scan x < N.  route "direct" takes every DFT as its direct sum (the forward sums over the
    non-zero support, the inverse sums at the scan's N positions only)."""
    n = fr.shape[0]
    p = n if pad_mode == 1 else 2 * n
    fr = np.asarray(fr, np.float64)
    g = np.asarray(g, np.float64)
    s = np.mod(lags(n), p)
    if route == "fft":
        D = np.zeros((p, p))
        D[np.ix_(s, s)] = dc
        Dh = np.fft.fft2(D)
        Gh = np.fft.fft2(g, s=(p, p))
        Fh = np.fft.fft2(fr, s=(p, p))
        dfr = np.real(np.fft.ifft2(np.conj(Dh) * Gh))[:n, :n]
        dg = np.real(np.fft.ifft2(Dh * Fh))[:n, :n]
        return dfr, dg
    W = dft_matrix(p)
    Wn = W[:, :n]
    Ws = W[:, s]                     # D is non-zero only at the lag positions s mod P
    Dh = Ws @ np.asarray(dc, np.float64) @ Ws.T
    Gh = Wn @ g @ Wn.T
    Fh = Wn @ fr @ Wn.T
    Wi = dft_matrix(p, np.arange(n), sign=+1)
    dfr = np.real(Wi @ (np.conj(Dh) * Gh) @ Wi.T) / (p * p)
    dg = np.real(Wi @ (Dh * Fh) @ Wi.T) / (p * p)
    return dfr, dg


def rotate_backward(x, theta, dout):
    """Adjoint of rotate(): d x (transpose of the bilinear gather) and d theta.

    With p(X) = c + R(-theta)(X - c):  d px / d theta = py - c,  d py / d theta = -(px - c)."""
    x = np.asarray(x, np.float64)
    n = x.shape[0]
    c = n / 2.0
    Y, X = np.meshgrid(np.arange(n, dtype=np.float64), np.arange(n, dtype=np.float64), indexing="ij")
    ct, st = np.cos(theta), np.sin(theta)
    dx, dy = X - c, Y - c
    px = c + ct * dx + st * dy
    py = c - st * dx + ct * dy
    x0 = np.floor(px)
    y0 = np.floor(py)
    fx = px - x0
    fy = py - y0
    x0 = x0.astype(np.int64)
    y0 = y0.astype(np.int64)

    def tap(oy, ox):
        yy, xx = y0 + oy, x0 + ox
        inside = (yy >= 0) & (yy < n) & (xx >= 0) & (xx < n)
        return yy, xx, inside, np.where(inside, x[np.clip(yy, 0, n - 1), np.clip(xx, 0, n - 1)], 0.0)

    t00, t01, t10, t11 = tap(0, 0), tap(0, 1), tap(1, 0), tap(1, 1)
    dxin = np.zeros_like(x)
    for (yy, xx, inside, _), w in ((t00, (1 - fy) * (1 - fx)), (t01, (1 - fy) * fx),
                                   (t10, fy * (1 - fx)), (t11, fy * fx)):
        np.add.at(dxin, (yy[inside], xx[inside]), (w * dout)[inside])
    v00, v01, v10, v11 = t00[3], t01[3], t10[3], t11[3]
    dv_dpx = (1 - fy) * (v01 - v00) + fy * (v11 - v10)
    dv_dpy = (1 - fx) * (v10 - v00) + fx * (v11 - v01)
    dtheta = float(np.sum(dout * (dv_dpx * (py - c) - dv_dpy * (px - c))))
    return dxin, dtheta


def angle_scores_backward(af, ag, dc):
    """Adjoint of angle_scores(): d af[a] = sum_k dc[k] ag[a + k], d ag[b] = sum_k dc[k] af[b - k]."""
    daf = np.zeros_like(af)
    dag = np.zeros_like(ag)
    for i, k in enumerate(lags(af.shape[0])):
        daf += dc[i] * np.roll(ag, -k, axis=0)
        dag += dc[i] * np.roll(af, k, axis=0)
    return daf, dag


def angle_scores_marginal_backward(af, ag, dc):
    """Adjoint of angle_scores_marginal(): the radial sums' adjoint, spread back over radius."""
    n_r = af.shape[1]
    dmf, dmg = angle_scores_backward(af.sum(axis=1, keepdims=True), ag.sum(axis=1, keepdims=True), dc)
    return np.repeat(dmf / n_r, n_r, axis=1), np.repeat(dmg / n_r, n_r, axis=1)


def cart2pol_backward(dp, cfg):
    """Transpose of the bilinear polar gather onto the [N, N/2+1] half spectrum."""
    n = cfg["n"]
    u, v = polar_points(n, cfg["n_theta"], cfg["n_r"])
    x0 = np.floor(u)
    y0 = np.floor(v)
    fx = u - x0
    fy = v - y0
    x0 = x0.astype(np.int64)
    y0 = y0.astype(np.int64)
    da = np.zeros((n, n // 2 + 1))
    for dy, wy in ((0, 1.0 - fy), (1, fy)):
        for dx, wx in ((0, 1.0 - fx), (1, fx)):
            vv, uu = half_index(n, y0 + dy, x0 + dx)
            np.add.at(da, (vv, uu), wy * wx * dp)
    return da


def magnitude_backward(F, da, cfg):
    """Adjoint of a = band |F| w.r.t. (Re F, Im F), returned as dRe + i dIm; z/|z| is 0 at z = 0."""
    m = np.abs(F)
    unit = np.where(m > 0, F / np.where(m > 0, m, 1.0), 0.0)
    return da * band_mask(cfg["n"], cfg["band_lo"], cfg["band_hi"]) * unit


def spectrum_backward(dF, cfg):
    """Adjoint of the windowed half-plane DFT: d x[y,x] = w[y] w[x] Re sum_{v, u<=N/2} dF[v,u]
    exp(+2 pi i (v y + u x) / N), as the direct sum conj(W_N) dF conj(W_half)."""
    n = cfg["n"]
    if cfg.get("route", "direct") == "fft":
        D = np.zeros((n, n), dtype=np.complex128)
        D[:, : n // 2 + 1] = dF
        dx = np.real(np.fft.ifft2(D)) * (n * n)
    else:
        dx = np.real(np.conj(dft_matrix(n)) @ dF @ np.conj(dft_matrix(n, np.arange(n // 2 + 1))))
    if cfg["window"]:
        w = hann(n)
        dx = dx * w[:, None] * w[None, :]
    return dx


def pose_backward(f, g, cfg, dpose):
    """Gradient of L with respect to f and g given dL/d(theta, tx, ty) (Eq. 13 drives this in
    training).  Recomputes the forward intermediates; the stage-2 translation depends on theta
    through Rotate, so d theta collects the direct term and the term through the rotated source."""
    n, nt = cfg["n"], cfg["n_theta"]
    r = pose(f, g, cfg, keep=True)
    dth_out, dtx, dty = (float(v) for v in dpose)
    s = lags(n) * cfg["delta_xy"]
    if cfg.get("rotate_target", 0) == 1:
        # t = R(theta) t': dt' = R(theta)^T dt, and d theta gains dt . (dR/dtheta) t'; the
        # scores' adjoint reaches f directly and g through Rotate(., -theta)
        th = r["theta"]
        ct, st = np.cos(th), np.sin(th)
        dtpx, dtpy = ct * dtx + st * dty, -st * dtx + ct * dty
        dth_t = dtx * (-st * r["tpx"] - ct * r["tpy"]) + dty * (ct * r["tpx"] - st * r["tpy"])
        q_xy = dtpx * s[None, :] + dtpy * s[:, None]
        dc_xy = soft_argmax_backward(r["c_xy"], r["p_xy"], q_xy, cfg["temp_xy"], cfg["score_norm"])
        df, dgr = xcorr2d_backward(np.asarray(f, np.float64), r["gr"], dc_xy, cfg["pad_mode"],
                                   cfg.get("route", "direct"))
        dg, dth_rot_arg = rotate_backward(g, -th, dgr)
        dth_rot = dth_t - dth_rot_arg
    else:
        q_xy = dtx * s[None, :] + dty * s[:, None]
        dc_xy = soft_argmax_backward(r["c_xy"], r["p_xy"], q_xy, cfg["temp_xy"], cfg["score_norm"])
        dfr, dg = xcorr2d_backward(r["fr"], g, dc_xy, cfg["pad_mode"], cfg.get("route", "direct"))
        df, dth_rot = rotate_backward(f, r["theta"], dfr)
    dth = dth_out + dth_rot
    q_t = dth * lags(nt) * (np.pi / nt)
    dc_t = soft_argmax_backward(r["c_theta"], r["p_theta"], q_t, cfg["temp_theta"], cfg["score_norm"])
    if cfg.get("angle_score", 0) == 1:
        dpf, dpg = angle_scores_marginal_backward(r["pf"], r["pg"], dc_t)
    else:
        dpf, dpg = angle_scores_backward(r["pf"], r["pg"], dc_t)
    df = df + spectrum_backward(magnitude_backward(r["Ff"], cart2pol_backward(dpf, cfg), cfg), cfg)
    dg = dg + spectrum_backward(magnitude_backward(r["Fg"], cart2pol_backward(dpg, cfg), cfg), cfg)
    return df, dg, dict(dtheta_total=dth, dtheta_rot=dth_rot, dc_xy=dc_xy, dc_theta=dc_t)
