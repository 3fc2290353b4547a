"""FP64 numpy statement of the FDK initialisation (Sec. 4.1).  Test infrastructure
only: used by tests/, the smoke check and the bench's CPU baseline, never by the
product path.

Sec. 4.1 initialises the Gaussians from a preliminary FDK reconstruction
(Feldkamp, Davis & Kress 1984): voxels with density above tau are candidates, M
of them are drawn at random as kernel positions, each kernel's scale is the
nearest-neighbour distance (3DGS convention: the mean distance to the three
nearest other positions), there is no rotation, and the central density is the
FDK value scaled by k.  The paper gives no FDK formulas; this module writes the
circular-orbit, flat-detector FDK out in its textbook form (Kak & Slaney,
Sec. 3.6.3):

  * pre-weighting  R'(xi, eta) = R(xi, eta) * L_SD / sqrt(L_SD^2 + xi^2 + eta^2)
    (cone beam; parallel beam leaves R unchanged);
  * ramp filtering along each detector row with the band-limited ramp
    (Ram-Lak) sampled at the row spacing tau: h(0) = 1/(4 tau^2), h(n tau) = 0
    for even n != 0, h(n tau) = -1/(n^2 pi^2 tau^2) for odd n, times 1/2 for the
    full-circle redundancy and times tau for the discrete convolution;
  * weighted back-projection f(p) = dbeta * sum_v w_v(p) F_v(xi(p), eta(p)).

With detector coordinates scaled to the isocentre (distance D_v = t_v[2] from
the source) the row spacing is tau = pitch_u D/L_SD and the FDK distance weight
is (D/u2)^2.  Written in the detector's own coordinates this becomes

  F(xi_n) = (1 / pitch_u) sum_k R'(xi_k) c_{n-k},  c_0 = 1/8,
            c_n = -1 / (2 n^2 pi^2) for odd n, 0 for even n != 0,
  w_v(p)  = D_v L_SD / u2^2 (cone),  1 (parallel),

and F is read at the voxel's projection (xi, eta) = L_SD (u0, u1) / u2 (cone) or
(u0, u1) (parallel), u = W p + t, by bilinear interpolation between pixel
centres, samples outside the detector counting as zero.  dbeta is the angular
step (2 pi / V for V evenly spaced views on a full circle).

The sampling step draws without replacement by a counter-based generator so that
any implementation can reproduce the draw: candidate voxel j (flat [z][y][x]
index) gets the key SplitMix64(seed + (j + 1) * 0x9E3779B97F4A7C15) (Steele,
Lea & Flood 2014: one Weyl-sequence step followed by the variant-13 finaliser),
and the M candidates with the smallest keys are chosen, listed in increasing
voxel index.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


# ----------------------------------------------------------------------------- filtering


def ramp_taps(n_max: int) -> np.ndarray:
    """c_n for n = -n_max .. n_max: the Ram-Lak ramp in units of 1/tau^2, times 1/2
    (full-circle redundancy): 1/8 at 0, -1/(2 n^2 pi^2) at odd n, 0 at even n."""
    n = np.arange(-n_max, n_max + 1)
    c = np.zeros(n.size)
    c[n == 0] = 0.125
    odd = (n % 2) != 0
    c[odd] = -1.0 / (2.0 * np.pi ** 2 * n[odd].astype(np.float64) ** 2)
    return c


def detector_coords(cam):
    """Pixel-centre coordinates (xi [W], eta [H]) in detector length units."""
    xi = (np.arange(cam.W) + 0.5 - 0.5 * cam.W) * cam.pitch_u + cam.off_u
    eta = (np.arange(cam.H) + 0.5 - 0.5 * cam.H) * cam.pitch_v + cam.off_v
    return xi, eta


def fdk_filter(proj, cam, rows=None) -> np.ndarray:
    """Weighted, ramp-filtered projections F [V, H, W] (float64) from log projections
    [V, H, W]: pre-weighting (cone beam), then each detector row convolved with the
    taps c_n over the whole row (no wrap-around), divided by pitch_u.  rows: an
    optional boolean mask [V, H] of the rows to compute (the others are NaN)."""
    proj = np.asarray(proj, dtype=np.float64)
    V, H, W = proj.shape
    if cam.beam == 1:
        xi, eta = detector_coords(cam)
        XI, ETA = np.meshgrid(xi, eta)
        proj = proj * (cam.L_SD / np.sqrt(cam.L_SD ** 2 + XI ** 2 + ETA ** 2))
    c = ramp_taps(W - 1)
    out = np.full_like(proj, np.nan)
    for v in range(V):
        for r in range(H):
            if rows is not None and not rows[v, r]:
                continue
            # full convolution has length 2W-1 + W-1; the outputs at the pixel
            # centres are the middle W samples
            out[v, r] = np.convolve(proj[v, r], c)[W - 1:2 * W - 1]
    return out / cam.pitch_u


# ----------------------------------------------------------------------------- back-projection


def _bilinear(img, x, y):
    """img [H, W] at continuous pixel indices (x column, y row); corners outside
    the image contribute zero."""
    H, W = img.shape
    x0 = np.floor(x).astype(np.int64)
    y0 = np.floor(y).astype(np.int64)
    fx = x - x0
    fy = y - y0
    out = np.zeros(x.shape)
    for dy, wy in ((0, 1.0 - fy), (1, fy)):
        for dx, wx in ((0, 1.0 - fx), (1, fx)):
            xi = x0 + dx
            yi = y0 + dy
            ok = (xi >= 0) & (xi < W) & (yi >= 0) & (yi < H)
            val = np.zeros(x.shape)
            val[ok] = img[yi[ok], xi[ok]]
            out += wx * wy * val
    return out


def voxel_centres(gdesc) -> np.ndarray:
    """Centres [Z*Y*X, 3] of one grid in [z][y][x] order."""
    g = np.asarray(gdesc, dtype=np.float64)
    o, vs, d = g[0:3], g[3:6], g[6:9].astype(int)
    x = o[0] + (np.arange(d[0]) + 0.5) * vs[0]
    y = o[1] + (np.arange(d[1]) + 0.5) * vs[1]
    z = o[2] + (np.arange(d[2]) + 0.5) * vs[2]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def fdk_backproject(filt, views, cam, gdesc, dbeta, points=None) -> np.ndarray:
    """f(p) = dbeta sum_v w_v(p) F_v(xi(p), eta(p)) at every voxel centre of gdesc
    (flat [z][y][x]) or at the given points [N, 3].  Cone beam: views whose depth
    u2 <= near_plane leave the voxel out."""
    filt = np.asarray(filt, dtype=np.float64)
    views = np.asarray(views, dtype=np.float64)
    P = voxel_centres(gdesc) if points is None else np.asarray(points, dtype=np.float64)
    acc = np.zeros(P.shape[0])
    for v in range(views.shape[0]):
        Wm = views[v, :9].reshape(3, 3)
        t = views[v, 9:12]
        u = P @ Wm.T + t
        if cam.beam == 1:
            keep = u[:, 2] > cam.near_plane
            u2 = np.where(keep, u[:, 2], 1.0)
            xi = cam.L_SD * u[:, 0] / u2
            eta = cam.L_SD * u[:, 1] / u2
            w = np.where(keep, t[2] * cam.L_SD / (u2 * u2), 0.0)
        else:
            xi, eta, w = u[:, 0], u[:, 1], np.ones(P.shape[0])
        x = (xi - cam.off_u) / cam.pitch_u + 0.5 * cam.W - 0.5
        y = (eta - cam.off_v) / cam.pitch_v + 0.5 * cam.H - 0.5
        acc += w * _bilinear(filt[v], x, y)
    return dbeta * acc


def fdk(proj, views, cam, gdesc, dbeta) -> np.ndarray:
    return fdk_backproject(fdk_filter(proj, cam), views, cam, gdesc, dbeta)


# ----------------------------------------------------------------------------- sampling and scales


def splitmix64(x: np.ndarray) -> np.ndarray:
    """The SplitMix64 output function (variant-13 finaliser) of 64-bit states x."""
    z = np.asarray(x, dtype=np.uint64).copy()
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64_stream(seed: int, n: int) -> np.ndarray:
    """The first n outputs of a SplitMix64 generator started at state `seed`."""
    i = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return splitmix64(np.uint64(seed) + i * GOLDEN)


def sample_candidates(vol, tau: float, M: int, seed: int) -> np.ndarray:
    """Flat voxel indices of the M candidates (vol > tau) with the smallest keys
    SplitMix64(seed + (j + 1) * golden), in increasing index order; all candidates
    if there are at most M.  The threshold comparison is made in the volume's own
    precision (tau rounded to it), as the kernel makes it."""
    v = np.asarray(vol).ravel()
    cand = np.flatnonzero(v > v.dtype.type(tau))
    if cand.size <= M:
        return cand
    with np.errstate(over="ignore"):
        keys = splitmix64(np.uint64(seed) + (cand.astype(np.uint64) + np.uint64(1)) * GOLDEN)
    pick = np.argsort(keys, kind="stable")[:M]
    return np.sort(cand[pick])


def knn3_mean_distance(points, chunk: int = 2048, lone: float = np.nan, which=None) -> np.ndarray:
    """Mean Euclidean distance from each point to its three nearest other points, by
    brute force; with fewer than four points, to all the others; a single point
    gets `lone`.  which: optional indices of the points to compute (default all)."""
    P = np.asarray(points, dtype=np.float64)
    n = P.shape[0]
    q = np.arange(n) if which is None else np.asarray(which, dtype=np.int64)
    out = np.empty(q.size)
    kk = min(3, n - 1)
    if kk <= 0:
        out[:] = lone
        return out
    for a in range(0, q.size, chunk):
        b = min(q.size, a + chunk)
        d2 = ((P[q[a:b], None, :] - P[None, :, :]) ** 2).sum(-1)
        d2[np.arange(b - a), q[a:b]] = np.inf
        part = np.sort(d2, axis=1)[:, :kk] if n <= 4 else np.partition(d2, kk, axis=1)[:, :kk]
        out[a:b] = np.sqrt(part).mean(axis=1)
    return out


def init_gaussians(vol, gdesc, tau: float, M: int, seed: int, k: float):
    """Sec. 4.1: positions at the chosen voxel centres, isotropic scales = the mean
    3-NN distance (a lone position: the smallest voxel edge), identity rotations,
    rho = k * vol.  Returns (mean [n, 3], scale [n, 3], quat [n, 4] (w, x, y, z),
    rho [n]) in float64."""
    idx = sample_candidates(vol, tau, M, seed)
    mean = voxel_centres(gdesc)[idx]
    s = knn3_mean_distance(mean, lone=float(np.min(np.asarray(gdesc, dtype=np.float64)[3:6])))
    scale = np.repeat(s[:, None], 3, axis=1)
    quat = np.zeros((idx.size, 4))
    quat[:, 0] = 1.0
    rho = k * np.asarray(vol, dtype=np.float64).ravel()[idx]
    return mean, scale, quat, rho
