"""Central differences of the oracle's FP64 Eq. 8 loss in one parameter of one
Gaussian, taken on windows so that they stay affordable at full size (test
infrastructure shared by the CPU pin of the windowing and the GPU checks at scale).

A parameter of Gaussian k changes the image only inside its pixel box in each view
and the SSIM map only within 5 pixels of it, so each view is rendered on a window of
the box widened by 10 pixels (every Gaussian whose box meets the window, the whole
set at the window's pixels), and the loss change is summed there; the TV change is
summed over the patches Gaussian k reaches.  The gate of Gaussian k is held at the
unperturbed parameters (core.render_gated / voxelize_gated), as an adjoint's is.
Beside the difference it returns two bounds in the same units: the kinks of |.| in
L1 and TV that the two evaluations can straddle, and the gate band (pixels within
1e-4 Q of Gaussian k's gate, where an FP32 gate may decide the other way) weighted
by |dL/dI| there."""
import numpy as np

from oracle import core, losses
from paper_2405_20693_b300 import inputs as I

LAMBDA_SSIM = 0.25
LAMBDA_TV = 0.05


def crop_camera(cam, c0, c1, r0, r1):
    """The detector window of columns c0..c1 and rows r0..r1 as a camera of its own:
    the same pixel centres, (c + 1/2 - W/2) pitch + off."""
    w, h = c1 - c0 + 1, r1 - r0 + 1
    return I.Camera(beam=cam.beam, H=h, W=w, L_SD=cam.L_SD, pitch_u=cam.pitch_u, pitch_v=cam.pitch_v,
                    off_u=cam.off_u + (c0 + 0.5 * w - 0.5 * cam.W) * cam.pitch_u,
                    off_v=cam.off_v + (r0 + 0.5 * h - 0.5 * cam.H) * cam.pitch_v, near_plane=cam.near_plane)


def pixel_boxes(G, views, cam, Q=9.0):
    """Per view and Gaussian, the oracle's inclusive pixel box of its gate (q <= Q),
    widened by a pixel as the oracle's scatter form widens it: [V, M, 4] int32 =
    c0, c1, r0, r1 (c0 > c1 when it projects nowhere)."""
    V, M = views.shape[0], G.M
    out = np.zeros((V, M, 4), np.int32)
    for v in range(V):
        pr = core.project(G, views[v:v + 1], cam)[0]
        ok = pr[:, 0] == 1.0
        ex, ey = np.sqrt(Q * np.maximum(pr[:, 3], 0)), np.sqrt(Q * np.maximum(pr[:, 5], 0))
        a = (pr[:, 1] - ex - cam.off_u) / cam.pitch_u + 0.5 * cam.W - 0.5
        b = (pr[:, 1] + ex - cam.off_u) / cam.pitch_u + 0.5 * cam.W - 0.5
        c = (pr[:, 2] - ey - cam.off_v) / cam.pitch_v + 0.5 * cam.H - 0.5
        d = (pr[:, 2] + ey - cam.off_v) / cam.pitch_v + 0.5 * cam.H - 0.5
        c0 = np.clip(np.ceil(a) - 1, 0, cam.W - 1)
        c1 = np.clip(np.floor(b) + 1, -1, cam.W - 1)
        r0 = np.clip(np.ceil(c) - 1, 0, cam.H - 1)
        r1 = np.clip(np.floor(d) + 1, -1, cam.H - 1)
        c1 = np.where(ok & (np.ceil(a) - 1 <= cam.W - 1) & (np.floor(b) + 1 >= 0), c1, -1)
        r1 = np.where(ok & (np.ceil(c) - 1 <= cam.H - 1) & (np.floor(d) + 1 >= 0), r1, -1)
        out[v] = np.stack([c0, c1, r0, r1], axis=1).astype(np.int32)
    return out


def one(G, k, kind=None, comp=None, h=0.0):
    """Gaussian k alone (float64), optionally with one parameter moved by h."""
    a = [np.array(x[k:k + 1], np.float64) for x in (G.mean, G.scale, G.quat, G.rho)]
    if kind is not None:
        if kind == 3:
            a[3][0] += h
        else:
            a[kind][0, comp] += h
    return I.GaussianSet(*a)


class OracleLossFD:
    """Central differences of the oracle's Eq. 8 loss in one parameter of one
    Gaussian, summed over windows (see the module docstring).  patch_gds: the TV
    patches [P, 9] (each D^3); Q, Q3: the gates."""

    def __init__(self, G, views, cam, meas, patch_gds, Q=9.0, Q3=11.345):
        self.G, self.views, self.cam, self.meas = G, views, cam, meas
        self.V = views.shape[0]
        self.N = self.V * cam.H * cam.W
        self.patch_gds = np.atleast_2d(patch_gds)
        self.Q, self.Q3 = Q, Q3
        self.D = int(self.patch_gds[0, 6])
        self.boxes = pixel_boxes(G, views, cam, Q)
        self.patch_base, _ = core.voxelize(G, self.patch_gds, Q3)
        self.windows_checked = []  # (v, window, oracle image, band) of the base renders

    def view_terms(self, k, v, kind, comp, eps):
        cam = self.cam
        c0, c1, r0, r1 = self.boxes[v, k]
        if c0 > c1 or r0 > r1:
            return 0.0, 0.0, 0.0
        wc0, wc1 = max(0, c0 - 10), min(cam.W - 1, c1 + 10)
        wr0, wr1 = max(0, r0 - 10), min(cam.H - 1, r1 + 10)
        bx = self.boxes[v]
        cand = np.flatnonzero((bx[:, 0] <= wc1) & (bx[:, 1] >= wc0) & (bx[:, 2] <= wr1) & (bx[:, 3] >= wr0))
        ccam = crop_camera(cam, wc0, wc1, wr0, wr1)
        vw = self.views[v:v + 1]
        Q = self.Q
        base, _, band_img = core.render(self.G.subset(cand), vw, ccam, Q=Q, want_band=True)
        base = base[0]
        if len(self.windows_checked) < 40:
            self.windows_checked.append((v, (wc0, wc1, wr0, wr1), base, band_img[0]))
        g0 = one(self.G, k)
        own = core.render_gated(g0, g0, vw, ccam, Q)[0]
        plus = base - own + core.render_gated(one(self.G, k, kind, comp, eps), g0, vw, ccam, Q)[0]
        minus = base - own + core.render_gated(one(self.G, k, kind, comp, -eps), g0, vw, ccam, Q)[0]
        m = self.meas[v, wr0:wr1 + 1, wc0:wc1 + 1]
        # L1: mean over all N pixels of the batch
        d_l1 = (np.abs(plus - m) - np.abs(minus - m)).sum() / self.N
        lo, hi = np.minimum(plus, minus), np.maximum(plus, minus)
        tiny = 1e-5 * np.maximum(np.abs(m), 1.0)
        kink = ((lo - tiny <= m) & (m <= hi + tiny)) | (np.abs(base - m) <= tiny)
        kink_bound = (np.abs(plus - minus)[kink]).sum() / self.N / eps
        # SSIM: the map changes only within 5 pixels of the box; the window keeps 10
        w = losses.gaussian_window()
        sp = losses.ssim_parts(plus, m, w)[-1]
        sm = losses.ssim_parts(minus, m, w)[-1]
        rr = slice(max(0, r0 - 5) - wr0, min(cam.H - 1, r1 + 5) - wr0 + 1)
        cc = slice(max(0, c0 - 5) - wc0, min(cam.W - 1, c1 + 5) - wc0 + 1)
        d_ssim = (sp[rr, cc] - sm[rr, cc]).sum() / (cam.H * cam.W) / self.V
        # dL/dI on the box (exact there: the window keeps 10 pixels) for the gate band
        n_crop = base.size
        dldi = np.sign(base - m) / self.N - LAMBDA_SSIM * losses.ssim_grad(base, m) * n_crop / (
            cam.H * cam.W) / self.V
        dc = (plus - minus) / (2 * eps)
        gx = (np.arange(wc0, wc1 + 1) + 0.5 - 0.5 * cam.W) * cam.pitch_u + cam.off_u
        gy = (np.arange(wr0, wr1 + 1) + 0.5 - 0.5 * cam.H) * cam.pitch_v + cam.off_v
        pr = core.project(g0, vw, cam)[0, 0]
        a, b_, c = pr[3], pr[4], pr[5]
        det = a * c - b_ * b_
        X, Y = np.meshgrid(gx - pr[1], gy - pr[2])
        qk = (c * X * X - 2 * b_ * X * Y + a * Y * Y) / det
        inband = np.abs(qk - Q) <= 1e-4 * Q
        band = (np.abs(dldi) * np.abs(dc))[inband].sum()
        return d_l1 - LAMBDA_SSIM * d_ssim, kink_bound, band

    def tv_terms(self, k, kind, comp, eps):
        Q3, D = self.Q3, self.D
        g0 = one(self.G, k)
        own = core.voxelize_gated(g0, g0, self.patch_gds, Q3)
        if not own.any():
            return 0.0, 0.0
        plus = self.patch_base - own + core.voxelize_gated(one(self.G, k, kind, comp, eps), g0, self.patch_gds, Q3)
        minus = self.patch_base - own + core.voxelize_gated(one(self.G, k, kind, comp, -eps), g0, self.patch_gds, Q3)
        dtv, kink = 0.0, 0.0
        n3 = D ** 3
        for p in range(self.patch_gds.shape[0]):
            sl = slice(p * n3, (p + 1) * n3)
            if not own[sl].any():
                continue
            vp, vm = plus[sl].reshape(D, D, D), minus[sl].reshape(D, D, D)
            dtv += losses.tv3d(vp, LAMBDA_TV)[0] - losses.tv3d(vm, LAMBDA_TV)[0]
            for ax in range(3):
                dp, dm = np.diff(vp, axis=ax), np.diff(vm, axis=ax)
                straddle = (np.sign(dp) != np.sign(dm)) | (np.abs(dp) + np.abs(dm) <= 1e-12)
                kink += LAMBDA_TV * np.abs(dp - dm)[straddle].sum() / dp.size / eps
        return dtv, kink

    def grad(self, k, kind, comp, eps):
        """(FD of the loss, kink bound, gate-band bound), all per unit of the parameter."""
        tot, kink, band = 0.0, 0.0, 0.0
        for v in range(self.V):
            d, kb, bb = self.view_terms(k, v, kind, comp, eps)
            tot += d
            kink += kb
            band += bb
        dtv, ktv = self.tv_terms(k, kind, comp, eps)
        return (tot + dtv) / (2 * eps), kink + ktv, band


