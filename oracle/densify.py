"""FP64 numpy statement of the adaptive density control (Sec. 4.2.3).  Test
infrastructure only.

Sec. 4.2.3 keeps 3DGS's adaptive control with two changes: empty Gaussians are
removed but large ones never are, and densification (clone or split of the
Gaussians with large loss gradients) halves the density of both the original and
the copy.  Sec. 5.1 runs it from iteration 500 to 15k with a gradient threshold of
5e-5.  The paper states nothing else; the readings here follow 3DGS where it is
silent:
  * statistic: per Gaussian, the mean over the (iteration, view) records in which
    it received a gradient of |dL/dp^| in normalised device coordinates (the pixel
    gradient times (W/2, H/2));
  * densify where that mean >= grad_threshold; clone where the largest scale is at
    most split_scale, else split into two children with scales / split_factor and
    means drawn from N(p, Sigma), the original removed; densities of the original
    and of every copy halved (rho / 2);
  * prune where rho < min_density (no size-based pruning);
  * surviving Gaussians keep their Adam moments, new ones start at zero;
  * at most max_gaussians after the step: candidates beyond that are left as they
    are, in index order;
  * layout of the result: survivors in index order, then the copies in the order
    of their originals (a clone's copy, or a split's two children).
The split offsets are drawn by a counter-based generator so that any implementation
reproduces them: draw j has u_j = ((SplitMix64(seed + (j + 1) * 0x9E3779B97F4A7C15)
>> 40) + 1/2) / 2^24, and child c (0, 1) of Gaussian i has the standard normal
offset z_k = sqrt(-2 ln u_j) cos(2 pi u_{j+1}) with j = ((2 i + c) 3 + k) 2 for
component k (Box & Muller 1958).
"""
from __future__ import annotations

import numpy as np

from .fdk import GOLDEN, splitmix64

GROUPS = ("quat", "mean", "scale", "rho")
WIDTH = {"quat": 4, "mean": 3, "scale": 3, "rho": 1}


def split_state(flat: np.ndarray, M: int) -> dict:
    """Views of a flat [quat 4M | mean 3M | scale 3M | rho M] array by group."""
    out, off = {}, 0
    for g in GROUPS:
        w = WIDTH[g]
        out[g] = flat[off:off + w * M].reshape(M, w) if w > 1 else flat[off:off + M]
        off += w * M
    return out


def join_state(parts: dict) -> np.ndarray:
    return np.concatenate([np.asarray(parts[g], np.float64).ravel() for g in GROUPS])


def uniforms(seed: int, j: np.ndarray) -> np.ndarray:
    """u_j in (0, 1): the top 24 bits of SplitMix64(seed + (j + 1) golden), plus 1/2, over 2^24."""
    with np.errstate(over="ignore"):
        x = splitmix64(np.uint64(seed) + (np.asarray(j, np.uint64) + np.uint64(1)) * GOLDEN)
    return ((x >> np.uint64(40)).astype(np.float64) + 0.5) / 16777216.0


def split_normals(seed: int, i: int, child: int) -> np.ndarray:
    """The standard normal offset (3) of child `child` of Gaussian i (Box-Muller)."""
    j = ((2 * i + child) * 3 + np.arange(3)) * 2
    u1, u2 = uniforms(seed, j), uniforms(seed, j + 1)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def rotation(q) -> np.ndarray:
    """Rotation matrix of the normalised quaternion (w, x, y, z)."""
    w, x, y, z = np.asarray(q, np.float64) / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def inv_softplus(y):
    y = np.asarray(y, np.float64)
    return y + np.log(-np.expm1(-y))


def classify(act: np.ndarray, M: int, grad_sum, count, grad_threshold, min_density, split_scale):
    """Per Gaussian: 0 prune, 1 keep, 2 clone, 3 split (before the capacity cap)."""
    a = split_state(np.asarray(act, np.float64), M)
    cnt = np.asarray(count, np.float64)
    avg = np.where(cnt > 0, np.asarray(grad_sum, np.float64) / np.maximum(cnt, 1.0), 0.0)
    prune = a["rho"] < min_density
    dens = ~prune & (avg >= grad_threshold)
    big = a["scale"].max(axis=1) > split_scale
    kind = np.ones(M, np.int64)
    kind[prune] = 0
    kind[dens & ~big] = 2
    kind[dens & big] = 3
    return kind


def densify(raw, act, m, v, M: int, grad_sum, count, grad_threshold=5e-5, min_density=1e-5, split_scale=0.02,
            split_factor=1.6, seed=0, max_gaussians=None):
    """One densify-and-prune step.  Returns (raw, act, m, v) flat float64 arrays of the
    new state and its Gaussian count."""
    kind = classify(act, M, grad_sum, count, grad_threshold, min_density, split_scale)
    cap = M * 4 if max_gaussians is None else int(max_gaussians)
    base = int((kind > 0).sum())                 # every non-pruned Gaussian kept as is
    cand = np.flatnonzero(kind >= 2)
    room = max(0, cap - base)
    accepted = np.zeros(M, bool)
    accepted[cand[:room]] = True                 # each accepted candidate adds one Gaussian
    kind = np.where((kind >= 2) & ~accepted, 1, kind)
    R, A, Mo, Vo = (split_state(np.asarray(x, np.float64), M) for x in (raw, act, m, v))
    out = {k: {g: [] for g in GROUPS} for k in ("raw", "act", "m", "v")}

    def emit(i, quat_a, mean_a, scale_a, rho_a, keep_moments):
        vals_a = {"quat": quat_a, "mean": mean_a, "scale": scale_a, "rho": rho_a}
        vals_r = {"quat": quat_a, "mean": mean_a, "scale": np.log(scale_a), "rho": inv_softplus(rho_a)}
        for g in GROUPS:
            out["act"][g].append(np.atleast_1d(vals_a[g]))
            out["raw"][g].append(np.atleast_1d(vals_r[g]))
            out["m"][g].append(np.atleast_1d(Mo[g][i]) if keep_moments else np.zeros(WIDTH[g]))
            out["v"][g].append(np.atleast_1d(Vo[g][i]) if keep_moments else np.zeros(WIDTH[g]))

    def emit_survivor(i, halve):
        for k, src in (("raw", R), ("act", A), ("m", Mo), ("v", Vo)):
            for g in GROUPS:
                out[k][g].append(np.atleast_1d(src[g][i]).astype(np.float64))
        if halve:
            out["act"]["rho"][-1] = np.atleast_1d(A["rho"][i] / 2)
            out["raw"]["rho"][-1] = np.atleast_1d(inv_softplus(A["rho"][i] / 2))

    for i in range(M):
        if kind[i] in (1, 2):
            emit_survivor(i, halve=kind[i] == 2)
    for i in range(M):
        if kind[i] == 2:
            emit(i, A["quat"][i], A["mean"][i], A["scale"][i], A["rho"][i] / 2, False)
        elif kind[i] == 3:
            Rm = rotation(A["quat"][i])
            for c in range(2):
                z = split_normals(seed, i, c)
                emit(i, A["quat"][i], A["mean"][i] + Rm @ (A["scale"][i] * z), A["scale"][i] / split_factor,
                     A["rho"][i] / 2, False)
    n = sum(1 for _ in out["act"]["rho"])
    res = tuple(np.concatenate([np.concatenate(out[k][g]) for g in GROUPS]) for k in ("raw", "act", "m", "v"))
    return res, n


def grad_stats(record_grads: np.ndarray, cam):
    """(sum of |dL/dp^| in normalised device coordinates, count of records with a
    gradient) per Gaussian from per-(view, Gaussian) record gradients [V, M, 6]
    (p^ in detector units: pixel gradient = detector gradient x pitch)."""
    rg = np.asarray(record_grads, np.float64)
    gx = rg[..., 1] * cam.pitch_u * cam.W / 2
    gy = rg[..., 2] * cam.pitch_v * cam.H / 2
    seen = np.any(rg != 0, axis=-1)
    return np.where(seen, np.hypot(gx, gy), 0.0).sum(axis=0), seen.sum(axis=0).astype(np.float64)
