"""FP64 numpy statement of the reconstruction metrics of Sec. 5.1.  Test
infrastructure only.

The paper scores a reconstructed volume by PSNR over the whole 3D volume and by
SSIM averaged over 2D slices in the axial, coronal and sagittal directions.
Readings used here (the paper gives no formulas):
  * PSNR = 10 log10(L^2 / MSE) with data range L = 1 (volumes normalised to
    [0, 1]) and MSE the mean over all voxels;
  * slice SSIM = the 2D SSIM of losses.ssim (Wang et al. 2004: 11x11 Gaussian
    window, sigma 1.5, zero-padded "same" filtering, C1 = (0.01 L)^2,
    C2 = (0.03 L)^2, mean of the SSIM map over the slice's pixels);
  * for a [Z][Y][X] volume with z the rotation axis: axial slices are the z = const
    images (rows y, columns x), coronal the y = const images (rows z, columns x),
    sagittal the x = const images (rows z, columns y);
  * per orientation the mean over its slices; the 3D SSIM is the mean of the three
    orientation means.
"""
from __future__ import annotations

import numpy as np

from . import losses

ORIENTATIONS = ("axial", "coronal", "sagittal")


def slices(vol: np.ndarray, orientation: str):
    """The 2D slices of a [Z][Y][X] volume in one orientation, as a [n, rows, cols] view."""
    v = np.asarray(vol)
    if orientation == "axial":
        return v                       # [z][y][x]
    if orientation == "coronal":
        return v.transpose(1, 0, 2)    # [y][z][x]
    if orientation == "sagittal":
        return v.transpose(2, 0, 1)    # [x][z][y]
    raise ValueError(orientation)


def ssim_orientation(a: np.ndarray, b: np.ndarray, orientation: str) -> float:
    sa, sb = slices(np.asarray(a, np.float64), orientation), slices(np.asarray(b, np.float64), orientation)
    return float(np.mean([losses.ssim(sa[k], sb[k]) for k in range(sa.shape[0])]))


def ssim3d(a: np.ndarray, b: np.ndarray) -> dict:
    """{'axial', 'coronal', 'sagittal': mean slice SSIM, 'ssim': their mean}."""
    out = {o: ssim_orientation(a, b, o) for o in ORIENTATIONS}
    out["ssim"] = float(np.mean([out[o] for o in ORIENTATIONS]))
    return out


def psnr3d(a: np.ndarray, b: np.ndarray, data_range: float = 1.0):
    """(MSE, PSNR in dB) over the whole volume."""
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return mse, (10.0 * np.log10(data_range ** 2 / mse) if mse > 0 else np.inf)
