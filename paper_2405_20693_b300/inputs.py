"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module holds input generation only -- random Gaussian sets, scanner view
tables, ellipsoid phantoms with their analytic line integrals, and the
phantom-based initialisation -- and none of the splatting arithmetic of the
method.  All randomness is numpy PCG64 with an explicit seed.

Units: one world unit is 128 mm, so the reconstruction volume [-1, 1]^3 is a
256 mm cube.  The paper's cone-beam scanner (source-to-origin 1000 mm,
source-to-detector 1500 mm, 512^2 detector at 0.8 mm; Sec. 5.1 and App. B)
becomes L_SO = 7.8125, L_SD = 11.71875, pitch = 0.00625 in these units.
Densities live in [0, 1] (App. B normalises volumes to [0, 1]).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

MM_PER_UNIT = 128.0
CONE_L_SO = 1000.0 / MM_PER_UNIT
CONE_L_SD = 1500.0 / MM_PER_UNIT
CONE_PITCH = 0.8 / MM_PER_UNIT


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# --------------------------------------------------------------------------- Gaussians


@dataclass
class GaussianSet:
    """Radiative Gaussians (Eq. 3): SoA float32 arrays, scales already positive."""

    mean: np.ndarray   # [M, 3]
    scale: np.ndarray  # [M, 3]
    quat: np.ndarray   # [M, 4]  (w, x, y, z), not necessarily unit length
    rho: np.ndarray    # [M]

    @property
    def M(self) -> int:
        return int(self.mean.shape[0])

    def astype(self, dt) -> "GaussianSet":
        return GaussianSet(*(np.ascontiguousarray(a, dtype=dt) for a in (self.mean, self.scale, self.quat, self.rho)))

    def subset(self, idx) -> "GaussianSet":
        return GaussianSet(self.mean[idx], self.scale[idx], self.quat[idx], self.rho[idx])


def random_quats(g: np.random.Generator, M: int) -> np.ndarray:
    q = g.standard_normal((M, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def uniform_gaussians(M: int, seed: int, scale_lo=0.01, scale_hi=0.1, box=1.0, rho_lo=0.0, rho_hi=1.0) -> GaussianSet:
    """Means U[-box, box]^3, per-axis scales log-uniform in [scale_lo, scale_hi],
    uniform random unit quaternions, densities U[rho_lo, rho_hi]."""
    g = rng(seed)
    mean = g.uniform(-box, box, (M, 3))
    scale = np.exp(g.uniform(math.log(scale_lo), math.log(scale_hi), (M, 3)))
    quat = random_quats(g, M)
    rho = g.uniform(rho_lo, rho_hi, M)
    return GaussianSet(mean, scale, quat, rho).astype(np.float32)


# --------------------------------------------------------------------------- scanner geometry


@dataclass
class Camera:
    """Detector and beam description shared by every view of one scan."""

    beam: int          # 0 = parallel, 1 = cone
    H: int
    W: int
    L_SD: float = 0.0
    pitch_u: float = 1.0
    pitch_v: float = 1.0
    off_u: float = 0.0
    off_v: float = 0.0
    near_plane: float = 0.0

    def as_vector(self) -> np.ndarray:
        return np.array([self.beam, self.H, self.W, self.L_SD, self.pitch_u, self.pitch_v,
                         self.off_u, self.off_v, self.near_plane], dtype=np.float64)


def view_table(thetas_rad, L_SO: float, dtype=np.float32) -> np.ndarray:
    """Per-view world->scanner transform [V, 12] = W (row-major 3x3) then t (App. A):
    W = [[-sin, cos, 0], [0, 0, -1], [-cos, -sin, 0]], t = (0, 0, L_SO).
    Evaluated in float64 and rounded once to float32; every consumer uses the
    float32 table (the oracle widens it).  dtype=float64 keeps W orthonormal to
    double precision, for closed-form checks."""
    th = np.asarray(thetas_rad, dtype=np.float64)
    out = np.zeros((th.size, 12), dtype=np.float64)
    s, c = np.sin(th), np.cos(th)
    out[:, 0], out[:, 1], out[:, 2] = -s, c, 0.0
    out[:, 3], out[:, 4], out[:, 5] = 0.0, 0.0, -1.0
    out[:, 6], out[:, 7], out[:, 8] = -c, -s, 0.0
    out[:, 9], out[:, 10], out[:, 11] = 0.0, 0.0, L_SO
    return out.astype(dtype)


def parallel_camera(H: int, W: int, pitch: float) -> Camera:
    return Camera(beam=0, H=H, W=W, pitch_u=pitch, pitch_v=pitch)


def cone_camera(H=512, W=512, L_SO=CONE_L_SO, L_SD=CONE_L_SD, pitch=CONE_PITCH) -> Camera:
    # Gaussians closer than 1% of L_SO to the source plane are dropped.
    return Camera(beam=1, H=H, W=W, L_SD=L_SD, pitch_u=pitch, pitch_v=pitch, near_plane=0.01 * L_SO)


def even_angles(V: int, span_deg: float = 360.0) -> np.ndarray:
    return np.deg2rad(np.arange(V) * (span_deg / V))


def limited_angles(V: int, span_deg: float) -> np.ndarray:
    """Limited-angle scan (App. E): V projection angles evenly
    spaced over [0, span_deg], both ends included."""
    return np.deg2rad(np.linspace(0.0, span_deg, V))


def grid_desc(origin, voxel, dims) -> np.ndarray:
    """One voxel grid: origin (3), voxel size (3), dims (X, Y, Z); centre of voxel
    (i, j, k) is origin + (index + 1/2) * voxel."""
    return np.array(list(origin) + list(voxel) + list(dims), dtype=np.float64)


def cube_grid(n: int, lo=-1.0, hi=1.0) -> np.ndarray:
    v = (hi - lo) / n
    return grid_desc((lo, lo, lo), (v, v, v), (n, n, n))


def patch_grid(offset_vox, D: int, n_full=256, lo=-1.0, hi=1.0) -> np.ndarray:
    """A D^3 patch of the n_full^3 output grid starting at integer voxel offset."""
    v = (hi - lo) / n_full
    o = [lo + offset_vox[k] * v for k in range(3)]
    return grid_desc(o, (v, v, v), (D, D, D))


# --------------------------------------------------------------------------- ellipsoid phantom


@dataclass
class Phantom:
    """Additive sum of constant-density ellipsoids."""

    centre: np.ndarray   # [E, 3]
    axes: np.ndarray     # [E, 3] semi-axes
    rot: np.ndarray      # [E, 3, 3] columns = ellipsoid axes in world frame
    density: np.ndarray  # [E]

    def quadric(self):
        # x inside  <=>  (x-c)^T A (x-c) <= 1,  A = R diag(1/a^2) R^T
        return np.einsum("eij,ej,ekj->eik", self.rot, 1.0 / self.axes ** 2, self.rot)

    def volume(self, gdesc: np.ndarray, chunk: int = 1 << 21) -> np.ndarray:
        """Density at voxel centres, [Z, Y, X] float64."""
        o, v, d = gdesc[0:3], gdesc[3:6], gdesc[6:9].astype(int)
        xs = o[0] + (np.arange(d[0]) + 0.5) * v[0]
        ys = o[1] + (np.arange(d[1]) + 0.5) * v[1]
        zs = o[2] + (np.arange(d[2]) + 0.5) * v[2]
        A = self.quadric()
        out = np.zeros((d[2], d[1], d[0]))
        for e in range(self.centre.shape[0]):
            c, a = self.centre[e], self.axes[e].max()
            # restrict to the bounding box of the circumscribed sphere
            sl = []
            for ax, k in ((zs, 2), (ys, 1), (xs, 0)):
                i0 = int(np.searchsorted(ax, c[k] - a))
                i1 = int(np.searchsorted(ax, c[k] + a, side="right"))
                sl.append((i0, i1))
            (z0, z1), (y0, y1), (x0, x1) = sl
            if z0 >= z1 or y0 >= y1 or x0 >= x1:
                continue
            Z, Y, X = np.meshgrid(zs[z0:z1] - c[2], ys[y0:y1] - c[1], xs[x0:x1] - c[0], indexing="ij")
            P = np.stack([X, Y, Z], axis=-1)
            q = np.einsum("...i,ij,...j->...", P, A[e], P)
            out[z0:z1, y0:y1, x0:x1] += self.density[e] * (q <= 1.0)
        return out

    def line_integrals(self, s: np.ndarray, w: np.ndarray) -> np.ndarray:
        """Exact integral of the density along rays s + t w (|w| = 1), t over R:
        sum over ellipsoids of density x chord length (ray-quadric intersection)."""
        s = s.reshape(-1, 3)
        w = w.reshape(-1, 3)
        A = self.quadric()
        out = np.zeros(s.shape[0])
        for e in range(self.centre.shape[0]):
            d = s - self.centre[e]
            Aw = w @ A[e]
            a = np.einsum("ij,ij->i", Aw, w)
            b = np.einsum("ij,ij->i", Aw, d)
            c = np.einsum("ij,ij->i", d @ A[e], d) - 1.0
            disc = b * b - a * c
            chord = np.where(disc > 0, 2.0 * np.sqrt(np.maximum(disc, 0.0)) / a, 0.0)
            out += self.density[e] * chord
        return out


def random_phantom(seed: int, n: int = 40, r_max: float = 0.6, axis_lo=0.05, axis_hi=0.4) -> Phantom:
    """n ellipsoids: centres uniform in the ball |c| <= r_max, semi-axes U[axis_lo, axis_hi],
    uniform random orientation, density U[0, 1]."""
    g = rng(seed)
    dirs = g.standard_normal((n, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    radii = r_max * g.uniform(0, 1, n) ** (1.0 / 3.0)
    centre = dirs * radii[:, None]
    axes = g.uniform(axis_lo, axis_hi, (n, 3))
    q = random_quats(g, n)
    rot = np.stack([quat_rotation(qq) for qq in q])
    density = g.uniform(0.0, 1.0, n)
    return Phantom(centre, axes, rot, density)


def quat_rotation(q) -> np.ndarray:
    w, x, y, z = np.asarray(q, dtype=np.float64) / np.linalg.norm(q)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def normalised_phantom(seed: int, n_grid: int = 256, **kw) -> tuple[Phantom, np.ndarray]:
    """Phantom rescaled so that the largest voxel of its n_grid^3 volume over
    [-1, 1]^3 equals 1; returns (phantom, volume)."""
    ph = random_phantom(seed, **kw)
    vol = ph.volume(cube_grid(n_grid))
    m = vol.max()
    if m > 0:
        ph = Phantom(ph.centre, ph.axes, ph.rot, ph.density / m)
        vol = vol / m
    return ph, vol


def detector_rays(view: np.ndarray, cam: Camera):
    """World-space rays (s, w) of every pixel of one view, [H*W, 3] each.
    Cone: from the source through the pixel centre on the plane u2 = L_SD.
    Parallel: along the scanner's third axis through (xi, eta, 0)."""
    Wm = view[:9].astype(np.float64).reshape(3, 3)
    t = view[9:12].astype(np.float64)
    c = np.arange(cam.W)
    r = np.arange(cam.H)
    xi = (c + 0.5 - cam.W / 2) * cam.pitch_u + cam.off_u
    eta = (r + 0.5 - cam.H / 2) * cam.pitch_v + cam.off_v
    XI, ETA = np.meshgrid(xi, eta)
    n = XI.size
    if cam.beam == 1:
        us = np.zeros((n, 3))
        ud = np.stack([XI.ravel(), ETA.ravel(), np.full(n, cam.L_SD)], axis=1)
    else:
        us = np.stack([XI.ravel(), ETA.ravel(), np.zeros(n)], axis=1)
        ud = np.tile(np.array([0.0, 0.0, 1.0]), (n, 1))
    ud /= np.linalg.norm(ud, axis=1, keepdims=True)
    s = (us - t) @ Wm      # W^T (u - t)
    w = ud @ Wm            # W^T d
    return s, w


def phantom_projections(ph: Phantom, views: np.ndarray, cam: Camera, device=None) -> np.ndarray:
    """Noise-free log projections (Eq. 1) of the phantom, [V, H, W] float64.
    device=None evaluates with numpy; a torch device name evaluates the same
    ray-quadric chords with torch in float64 there (much faster for full scans)."""
    out = np.zeros((views.shape[0], cam.H, cam.W))
    if device is None:
        for v in range(views.shape[0]):
            s, w = detector_rays(views[v], cam)
            out[v] = ph.line_integrals(s, w).reshape(cam.H, cam.W)
        return out
    import torch

    A = torch.as_tensor(ph.quadric(), dtype=torch.float64, device=device)
    C = torch.as_tensor(ph.centre, dtype=torch.float64, device=device)
    dens = torch.as_tensor(ph.density, dtype=torch.float64, device=device)
    for v in range(views.shape[0]):
        s, w = detector_rays(views[v], cam)
        s = torch.as_tensor(s, device=device)
        w = torch.as_tensor(w, device=device)
        acc = torch.zeros(s.shape[0], dtype=torch.float64, device=device)
        for e in range(C.shape[0]):
            d = s - C[e]
            Aw = w @ A[e]
            a = (Aw * w).sum(1)
            b = (Aw * d).sum(1)
            c = ((d @ A[e]) * d).sum(1) - 1.0
            disc = b * b - a * c
            acc += dens[e] * torch.where(disc > 0, 2.0 * torch.sqrt(torch.clamp(disc, min=0.0)) / a, 0.0)
        out[v] = acc.reshape(cam.H, cam.W).cpu().numpy()
    return out


def poisson_noise(proj: np.ndarray, seed: int, n0: float = 1e5) -> np.ndarray:
    """Counts N ~ Poisson(N0 exp(-I)); returns -ln(max(N, 1) / N0) (Sec. 5.1, App. B noise,
    photon term only)."""
    g = rng(seed)
    counts = g.poisson(n0 * np.exp(-proj))
    return -np.log(np.maximum(counts, 1) / n0)


# --------------------------------------------------------------------------- initialisation


def init_from_volume(vol: np.ndarray, gdesc: np.ndarray, M: int, seed: int, tau=0.05, k=0.15,
                     scale_override=None, random_rot=False) -> GaussianSet:
    """Sec. 4.1 initialisation with a given volume standing in for FDK: sample M
    voxel centres with density > tau, scales = mean distance to the 3 nearest
    sampled neighbours (isotropic), identity rotation, rho = k * volume.
    scale_override=(lo, hi) draws per-axis log-uniform scales instead, and
    random_rot draws random rotations (the densified configuration)."""
    from scipy.spatial import cKDTree

    g = rng(seed)
    o, v, d = gdesc[0:3], gdesc[3:6], gdesc[6:9].astype(int)
    idx = np.flatnonzero(vol.ravel() > tau)
    pick = g.choice(idx, size=M, replace=idx.size < M)
    z, y, x = np.unravel_index(pick, vol.shape)
    mean = np.stack([o[0] + (x + 0.5) * v[0], o[1] + (y + 0.5) * v[1], o[2] + (z + 0.5) * v[2]], axis=1)
    if scale_override is None:
        dist, _ = cKDTree(mean).query(mean, k=4)
        s = np.maximum(dist[:, 1:].mean(axis=1), 1e-4)
        scale = np.repeat(s[:, None], 3, axis=1)
    else:
        lo, hi = scale_override
        scale = np.exp(g.uniform(math.log(lo), math.log(hi), (M, 3)))
    quat = random_quats(g, M) if random_rot else np.tile(np.array([1.0, 0, 0, 0]), (M, 1))
    rho = k * vol.ravel()[pick]
    return GaussianSet(mean, scale, quat, rho).astype(np.float32)


def random_init(M: int, seed: int, radius=0.9, half_height=0.9, rho=0.05) -> GaussianSet:
    """Random initialisation: means uniform in the cylinder r <= radius, |z| <=
    half_height, isotropic scales = mean distance to 3 nearest neighbours, identity
    rotation, constant density."""
    from scipy.spatial import cKDTree

    g = rng(seed)
    r = radius * np.sqrt(g.uniform(0, 1, M))
    phi = g.uniform(0, 2 * np.pi, M)
    z = g.uniform(-half_height, half_height, M)
    mean = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    dist, _ = cKDTree(mean).query(mean, k=4)
    s = np.maximum(dist[:, 1:].mean(axis=1), 1e-4)
    scale = np.repeat(s[:, None], 3, axis=1)
    quat = np.tile(np.array([1.0, 0, 0, 0]), (M, 1))
    return GaussianSet(mean, scale, quat, np.full(M, rho)).astype(np.float32)


# --------------------------------------------------------------------------- multi-scan workload


@dataclass
class ScanSpec:
    """One scan of the uneven multi-scan workload."""

    seed: int
    M: int
    V: int
    det: int      # detector edge in pixels (the detector always spans 409.6 mm)
    n_out: int    # output volume edge in voxels (TV patch spacing 2 / n_out)
    span: float = 360.0  # scanned arc in degrees; < 360 = limited-angle (ends included)


def batched_specs(n_scans: int = 16, seed: int = 5):
    """Gaussian counts log-uniform in [5k, 300k]; 25, 50 or 75 views; 256^2 or 512^2
    detectors; 128^3 or 256^3 output volumes."""
    g = rng(seed)
    out = []
    for j in range(n_scans):
        M = int(round(math.exp(g.uniform(math.log(5e3), math.log(3e5)))))
        V = int(g.choice([25, 50, 75]))
        det = int(g.choice([256, 512]))
        n_out = int(g.choice([128, 256]))
        out.append(ScanSpec(100 + j, M, V, det, n_out))
    return out


def make_scan(spec: ScanSpec, device=None):
    """Phantom (seed spec.seed), cone-beam geometry with the detector scaled to
    409.6 mm, measured projections, and the random initialisation (means in the
    inscribed cylinder, 3-NN isotropic scales, density 0.05).  Returns
    (gaussians, camera, views, measured projections, phantom volume)."""
    ph, vol = normalised_phantom(spec.seed, spec.n_out)
    cam = cone_camera(spec.det, spec.det, pitch=CONE_PITCH * 512 / spec.det)
    ang = even_angles(spec.V) if spec.span >= 360.0 else limited_angles(spec.V, spec.span)
    views = view_table(ang, CONE_L_SO)
    meas = phantom_projections(ph, views, cam, device=device).astype(np.float32)
    G = random_init(spec.M, spec.seed)
    return G, cam, views, meas, vol
