"""FP64 numpy statement of the training losses and the optimizer step.  Test
infrastructure only.

Eq. 8: L_total = L1(I_r, I_m) + lambda_ssim * D-SSIM(I_r, I_m) + lambda_tv * TV(V_tv),
with lambda_ssim = 0.25, lambda_tv = 0.05 (Sec. 5.1).  The paper names the
losses without formulas; the readings used here:
  * L1   = mean |I_r - I_m| over all pixels of all views in the batch;
  * SSIM = Wang et al. 2004: 11x11 Gaussian window, sigma 1.5, zero-padded
    "same" filtering, C1 = (0.01 L)^2, C2 = (0.03 L)^2 with L = 1, mean of the
    SSIM map over all pixels; D-SSIM = 1 - SSIM;
  * TV   = anisotropic L1: for each of the three axes, the mean of |forward
    difference| over all valid differences, summed over the axes (the isotropic
    form sqrt(sum of squared forward differences + eps), averaged over voxels, is
    the option tv3d_iso);
  * Adam (Kingma & Ba) with the paper's per-group learning rates, decayed
    exponentially to 0.1x over the run (Sec. 5.1).
Each function that returns a gradient derives it by hand; the tests pin those
against complex-step derivatives of the forward functions.
"""
from __future__ import annotations

import numpy as np

LAMBDA_SSIM = 0.25
LAMBDA_TV = 0.05
C1 = 0.01 ** 2
C2 = 0.03 ** 2


def gaussian_window(size: int = 11, sigma: float = 1.5) -> np.ndarray:
    k = np.arange(size) - (size - 1) / 2.0
    g = np.exp(-(k * k) / (2 * sigma * sigma))
    g /= g.sum()
    return np.outer(g, g)


def filt(img: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Zero-padded 'same' correlation of a 2D image with a square window, by
    explicit shifted sums (works for complex input)."""
    H, W = img.shape
    k = w.shape[0]
    r = k // 2
    pad = np.zeros((H + 2 * r, W + 2 * r), dtype=img.dtype)
    pad[r:r + H, r:r + W] = img
    out = np.zeros_like(img)
    for i in range(k):
        for j in range(k):
            out = out + w[i, j] * pad[i:i + H, j:j + W]
    return out


def ssim_parts(x, y, w):
    mx, my = filt(x, w), filt(y, w)
    exx, eyy, exy = filt(x * x, w), filt(y * y, w), filt(x * y, w)
    sxx, syy, sxy = exx - mx * mx, eyy - my * my, exy - mx * my
    A1, A2 = 2 * mx * my + C1, 2 * sxy + C2
    B1, B2 = mx * mx + my * my + C1, sxx + syy + C2
    S = (A1 * A2) / (B1 * B2)
    return mx, my, A1, A2, B1, B2, S


def ssim(x: np.ndarray, y: np.ndarray) -> float:
    """Mean SSIM of one 2D image pair (Wang et al. 2004)."""
    w = gaussian_window()
    return ssim_parts(x, y, w)[-1].mean()


def ssim_grad(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """d mean-SSIM / d x.  With raw moments mu_x = w*x, E_xx = w*(x^2), E_xy = w*(xy):
      dS/dmu_x = 2 mu_y (A2 - A1) / (B1 B2) - 2 mu_x S (B2 - B1) / (B1 B2)
      dS/dE_xx = -S / B2
      dS/dE_xy = 2 A1 / (B1 B2)
    and the adjoint of the zero-padded filter is the same filter (symmetric window)."""
    w = gaussian_window()
    mx, my, A1, A2, B1, B2, S = ssim_parts(x, y, w)
    d_mu = (2 * my * (A2 - A1) - 2 * mx * S * (B2 - B1)) / (B1 * B2)
    d_exx = -S / B2
    d_exy = 2 * A1 / (B1 * B2)
    N = x.size
    return (filt(d_mu, w) + 2 * x * filt(d_exx, w) + y * filt(d_exy, w)) / N


def projection_loss(render: np.ndarray, meas: np.ndarray, lam_ssim: float = LAMBDA_SSIM):
    """L1 + lambda_ssim * (1 - SSIM) over a [V, H, W] batch; SSIM averaged over views.
    Returns (loss, d loss / d render)."""
    render = np.asarray(render, dtype=np.float64)
    meas = np.asarray(meas, dtype=np.float64)
    V = render.shape[0]
    diff = render - meas
    l1 = np.abs(diff).mean()
    g = np.sign(diff) / diff.size
    s = 0.0
    for v in range(V):
        s += ssim(render[v], meas[v])
        g[v] -= lam_ssim * ssim_grad(render[v], meas[v]) / V
    loss = l1 + lam_ssim * (1.0 - s / V)
    return loss, g


def tv3d(vol: np.ndarray, lam_tv: float = LAMBDA_TV):
    """lambda_tv * anisotropic TV of a [Z, Y, X] volume; returns (loss, gradient)."""
    vol = np.asarray(vol, dtype=np.float64)
    loss = 0.0
    g = np.zeros_like(vol)
    for ax in range(3):
        d = np.diff(vol, axis=ax)
        n = d.size
        loss += np.abs(d).mean()
        sg = np.sign(d) / n
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, -1)
        hi[ax] = slice(1, None)
        g[tuple(hi)] += sg
        g[tuple(lo)] -= sg
    return lam_tv * loss, lam_tv * g


def tv3d_iso(vol: np.ndarray, lam_tv: float = LAMBDA_TV, eps: float = 1e-6):
    """lambda_tv * isotropic TV of a [Z, Y, X] volume: the mean over all voxels of
    sqrt(sum_k d_k^2 + eps), d_k the forward difference along axis k (0 where the
    neighbour lies outside); returns (loss, gradient).  With n(x) that root,
    dn(x)/dV(x) = -sum_k d_k(x) / n(x) and dn(x)/dV(x + e_k) = d_k(x) / n(x)."""
    vol = np.asarray(vol)
    N = vol.size
    d = []
    for ax in range(3):
        dk = np.zeros_like(vol)
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, -1)
        hi[ax] = slice(1, None)
        dk[tuple(lo)] = vol[tuple(hi)] - vol[tuple(lo)]
        d.append(dk)
    n = np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2 + eps)
    loss = n.mean()
    g = np.zeros_like(vol)
    for ax in range(3):
        r = d[ax] / n
        g -= r
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, -1)
        hi[ax] = slice(1, None)
        g[tuple(hi)] += r[tuple(lo)]
    return lam_tv * loss, lam_tv * g / N


# ----------------------------------------------------------------------------- optimizer

LR0 = {"mean": 2e-4, "rho": 1e-2, "scale": 5e-3, "quat": 1e-3}
LR_FINAL_FACTOR = 0.1


def lr_at(group: str, it: int, total: int = 30000) -> float:
    """Exponential decay from the initial rate to 0.1x at the last iteration."""
    t = min(max(it / float(total), 0.0), 1.0)
    return LR0[group] * LR_FINAL_FACTOR ** t


def softplus(x):
    return np.log1p(np.exp(-np.abs(x))) + np.maximum(x, 0.0)


def inv_softplus(y):
    return y + np.log(-np.expm1(-y))


def adam_step(raw: dict, grads_act: dict, m: dict, v: dict, it: int, total: int = 30000,
              b1=0.9, b2=0.999, eps=1e-15):
    """One Adam step on the raw parameters (mean, log-scale, quat, softplus^-1 rho)
    given gradients with respect to the activated ones (mean, scale = exp(log-scale),
    quat, rho = softplus(raw)).  `it` is the 0-based iteration; returns the new
    activated parameters.  Arrays are updated in place."""
    chain = {
        "mean": lambda r: 1.0,
        "quat": lambda r: 1.0,
        "scale": lambda r: np.exp(r),
        "rho": lambda r: 1.0 / (1.0 + np.exp(-r)),
    }
    out = {}
    for k in ("mean", "scale", "quat", "rho"):
        g = grads_act[k] * chain[k](raw[k])
        m[k][...] = b1 * m[k] + (1 - b1) * g
        v[k][...] = b2 * v[k] + (1 - b2) * g * g
        mh = m[k] / (1 - b1 ** (it + 1))
        vh = v[k] / (1 - b2 ** (it + 1))
        raw[k][...] = raw[k] - lr_at(k, it, total) * mh / (np.sqrt(vh) + eps)
    out["mean"] = raw["mean"].copy()
    out["scale"] = np.exp(raw["scale"])
    out["quat"] = raw["quat"].copy()
    out["rho"] = softplus(raw["rho"])
    return out
