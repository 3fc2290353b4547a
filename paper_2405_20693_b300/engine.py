"""Workspaces, autograd bridge and the training step built on the C ABI.

Everything numeric runs in libr2g.so; this module sizes and owns the device
workspaces (torch uint8 tensors), grows a workspace when the device reports
that the per-tile / per-brick lists did not fit, and chains the calls of one
training iteration (Eq. 8): rasterize -> L1 + D-SSIM -> voxelize a TV patch ->
TV -> both backward passes -> fused Adam.
"""
from __future__ import annotations

import numpy as np
import torch

from . import r2g

Q_PIXEL = 9.0        # 3-sigma pixel gate
Q_VOXEL = 11.345     # chi^2_3 0.99 quantile: the 0.99-probability culling of Sec. 4.2.2
LAMBDA_SSIM = 0.25   # Sec. 5.1
LAMBDA_TV = 0.05     # Sec. 5.1
SCAN_TILE = (32, 32)  # tile shape of the training step's rasterizer (fewest list entries at 512^2)


def _bytes(n: int, device) -> torch.Tensor:
    return torch.empty(int(n), dtype=torch.uint8, device=device)


class Rasterizer:
    """Owns the workspace of one (M, V, camera, tile) configuration."""

    def __init__(self, M: int, V: int, cam, Q=Q_PIXEL, tile=(16, 16), device="cuda", capacity=None, biased=False,
                 dilation=0.0, view_chunk=0):
        """view_chunk > 0: views processed that many at a time, the workspace sized for
        one chunk, and the backward rebuilding each chunk's lists (r2g_raster_opts)."""
        self.M, self.V = int(M), int(V)
        self.cam = r2g.camera(cam)
        self.opts = r2g.raster_opts(Q, tile, biased=biased, dilation=dilation, view_chunk=view_chunk)
        self.copts = r2g.raster_opts(Q, tile, count_pairs=True, biased=biased, dilation=dilation,
                                     view_chunk=view_chunk)
        self.device = device
        Vc = view_chunk if 0 < view_chunk < self.V else self.V
        self.capacity = int(capacity or max(1 << 16, 4 * self.M * Vc))
        self.ws = None
        self._alloc()

    def _alloc(self):
        n = r2g.r2g_raster_workspace_size(self.M, self.V, self.cam, self.opts, self.capacity)
        self.ws = _bytes(n, self.device)

    def forward(self, mean, scale, quat, rho, views, image=None, check=True, count=False):
        """Image [V, H, W].  check=True polls the device status (one sync) and re-runs
        with a larger workspace if the lists overflowed."""
        if image is None:
            image = torch.empty((self.V, self.cam.H, self.cam.W), dtype=torch.float32, device=self.device)
        while True:
            r2g.r2g_rasterize(mean, scale, quat, rho, views, self.cam, self.copts if count else self.opts, image,
                              self.ws)
            if not check:
                return image
            st, needed = r2g.r2g_poll(self.ws)
            if st == r2g.R2G_OK:
                return image
            if st != r2g.R2G_E_CAPACITY:
                raise r2g.R2GError(st, "rasterize: " + r2g.last_error())
            self.capacity = int(needed * 1.25) + 1024
            self._alloc()

    def backward(self, mean, scale, quat, rho, views, dimage, dmean, dscale, dquat, drho):
        r2g.r2g_rasterize_backward(mean, scale, quat, rho, views, self.cam, self.opts, dimage.contiguous(), dmean,
                                   dscale, dquat, drho, self.ws)

    def pair_count(self) -> int:
        return r2g.r2g_pair_count(self.ws)


class Voxelizer:
    """Owns the workspace of one (M, grids) configuration."""

    def __init__(self, M: int, gdescs, Q3=Q_VOXEL, device="cuda", capacity=None):
        self.M = int(M)
        self.gd = np.atleast_2d(np.asarray(gdescs, dtype=np.float64))
        self.grids = r2g.grids(self.gd)
        self.Q3 = float(Q3)
        self.device = device
        self.n_vox = int(sum(int(d[6] * d[7] * d[8]) for d in self.gd))
        self.capacity = int(capacity or max(1 << 16, 2 * self.M * len(self.gd)))
        self._alloc()

    def _alloc(self):
        n = r2g.r2g_voxel_workspace_size(self.M, self.grids, self.capacity)
        self.ws = _bytes(n, self.device)

    def set_grids(self, gdescs):
        """Same grid count and sizes, new origins (e.g. a new TV patch position)."""
        gd = np.atleast_2d(np.asarray(gdescs, dtype=np.float64))
        assert gd.shape == self.gd.shape and np.all(gd[:, 6:] == self.gd[:, 6:])
        self.gd = gd
        self.grids = r2g.grids(gd)

    def forward(self, mean, scale, quat, rho, vol=None, check=True, count=False):
        if vol is None:
            vol = torch.empty(self.n_vox, dtype=torch.float32, device=self.device)
        while True:
            r2g.r2g_voxelize(mean, scale, quat, rho, self.grids, self.Q3, vol, self.ws, counted=count)
            if not check:
                return vol
            st, needed = r2g.r2g_poll(self.ws)
            if st == r2g.R2G_OK:
                return vol
            if st != r2g.R2G_E_CAPACITY:
                raise r2g.R2GError(st, "voxelize: " + r2g.last_error())
            self.capacity = int(needed * 1.25) + 1024
            self._alloc()

    def backward(self, mean, scale, quat, rho, dvol, dmean, dscale, dquat, drho):
        r2g.r2g_voxelize_backward(mean, scale, quat, rho, self.grids, self.Q3, dvol.contiguous(), dmean, dscale,
                                  dquat, drho, self.ws)

    def pair_count(self) -> int:
        return r2g.r2g_pair_count(self.ws)


# ----------------------------------------------------------------------------- autograd bridge


class _RasterizeFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mean, scale, quat, rho, views, rast):
        ctx.rast = rast
        ctx.save_for_backward(mean, scale, quat, rho, views)
        return rast.forward(mean.detach(), scale.detach(), quat.detach(), rho.detach(), views)

    @staticmethod
    def backward(ctx, dimage):
        mean, scale, quat, rho, views = ctx.saved_tensors
        g = [torch.zeros_like(t) for t in (mean, scale, quat, rho)]
        ctx.rast.backward(mean, scale, quat, rho, views, dimage.float(), *g)
        return (*g, None, None)


class _VoxelizeFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mean, scale, quat, rho, vox):
        ctx.vox = vox
        ctx.save_for_backward(mean, scale, quat, rho)
        return vox.forward(mean.detach(), scale.detach(), quat.detach(), rho.detach())

    @staticmethod
    def backward(ctx, dvol):
        mean, scale, quat, rho = ctx.saved_tensors
        g = [torch.zeros_like(t) for t in (mean, scale, quat, rho)]
        ctx.vox.backward(mean, scale, quat, rho, dvol.float(), *g)
        return (*g, None)


class _ProjectionLossFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, render, meas, lam, ws):
        loss = torch.empty(1, dtype=torch.float32, device=render.device)
        drender = torch.empty_like(render)
        r2g.r2g_projection_loss(render.detach().contiguous(), meas, lam, loss, drender, ws)
        ctx.save_for_backward(drender)
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        (drender,) = ctx.saved_tensors
        return drender * g, None, None, None


class _TVFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vol, G, D, lam, ws):
        loss = torch.empty(1, dtype=torch.float32, device=vol.device)
        dvol = torch.empty_like(vol)
        r2g.r2g_tv3d(vol.detach().contiguous().view(G, D, D, D), lam, loss, dvol.view(G, D, D, D), ws)
        ctx.save_for_backward(dvol)
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        (dvol,) = ctx.saved_tensors
        return dvol * g, None, None, None, None


def projection_loss(render, meas, lam=LAMBDA_SSIM, ws=None):
    """Eq. 8's projection term L1 + lam (1 - SSIM) of a [V, H, W] render against the
    measured [V, H, W] projections, differentiable in the render (r2g_projection_loss)."""
    V, H, W = render.shape
    if ws is None:
        ws = _bytes(r2g.r2g_loss_workspace_size(V, H, W), render.device)
    return _ProjectionLossFn.apply(render, meas.contiguous(), float(lam), ws)


def tv3d(vol, G: int, D: int, lam=LAMBDA_TV, ws=None):
    """lam x the anisotropic 3D TV summed over G concatenated D^3 volumes (Eq. 8,
    r2g_tv3d), differentiable in the volumes."""
    if ws is None:
        ws = _bytes(r2g.r2g_tv_workspace_size(G, D), vol.device)
    return _TVFn.apply(vol, int(G), int(D), float(lam), ws)


def rasterize(mean, scale, quat, rho, views, rast: Rasterizer):
    """Differentiable X-ray projection (Eq. 5, Eq. 7): [V, H, W]."""
    return _RasterizeFn.apply(mean, scale, quat, rho, views, rast)


def voxelize(mean, scale, quat, rho, vox: Voxelizer):
    """Differentiable density query (Eq. 4): concatenated grid volumes."""
    return _VoxelizeFn.apply(mean, scale, quat, rho, vox)


# ----------------------------------------------------------------------------- FDK initialisation


INIT_TAU = 0.05   # Sec. 5.1: density threshold of the candidate voxels
INIT_K = 0.15     # Sec. 5.1: scale-down of the queried densities
INIT_M = 50_000   # Sec. 5.1: Gaussians at initialisation


def fdk_volume(views, meas, cam, gdesc, dbeta=None, device="cuda"):
    """FDK reconstruction (Sec. 4.1) of one grid from the measured log projections:
    views [V, 12] and meas [V, H, W] float32 device tensors; returns the volume
    [Z, Y, X] on the device.  dbeta defaults to 2 pi / V (a full circle)."""
    V = int(views.shape[0])
    c = r2g.camera(cam)
    filt = torch.empty_like(meas)
    r2g.r2g_fdk_filter(meas, c, filt)
    g = r2g.grids(gdesc)[0]
    vol = torch.empty((g.dims[2], g.dims[1], g.dims[0]), dtype=torch.float32, device=device)
    r2g.r2g_fdk_backproject(views, c, filt, g, 2 * np.pi / V if dbeta is None else dbeta, vol)
    return vol


def init_gaussians(vol, gdesc, M=INIT_M, tau=INIT_TAU, k=INIT_K, seed=0, device="cuda"):
    """Sec. 4.1's Gaussians from a device volume on grid gdesc: returns device
    tensors (mean [n, 3], scale [n, 3], quat [n, 4], rho [n]), n <= M."""
    g = r2g.grids(gdesc)[0]
    mean = torch.empty((M, 3), dtype=torch.float32, device=device)
    scale = torch.empty_like(mean)
    quat = torch.empty((M, 4), dtype=torch.float32, device=device)
    rho = torch.empty(M, dtype=torch.float32, device=device)
    n_out = torch.zeros(1, dtype=torch.int64, device=device)
    ws = _bytes(r2g.r2g_init_workspace_size(g, M), device)
    r2g.r2g_init_gaussians(vol, g, tau, M, seed, k, mean, scale, quat, rho, n_out, ws)
    n = int(n_out.item())
    return mean[:n], scale[:n], quat[:n], rho[:n]


def fdk_init(views, meas, cam, n_out: int, M=INIT_M, tau=INIT_TAU, k=INIT_K, seed=0, device="cuda"):
    """FDK volume on the n_out^3 output grid over [-1, 1]^3, then the initial
    Gaussians; returns (GaussianSet on the host, volume on the device)."""
    from .inputs import GaussianSet, cube_grid

    gd = cube_grid(n_out)
    vol = fdk_volume(views, meas, cam, gd, device=device)
    mean, scale, quat, rho = init_gaussians(vol, gd, M, tau, k, seed, device)
    G = GaussianSet(*(t.cpu().numpy() for t in (mean, scale, quat, rho)))
    return G, vol


# ----------------------------------------------------------------------------- volume metrics


METRIC_KEYS = ("mse", "psnr", "ssim", "ssim_axial", "ssim_coronal", "ssim_sagittal")


def volume_metrics(vol, ref, device="cuda") -> dict:
    """Sec. 5.1's scores of a [Z, Y, X] device volume against a reference (float32
    device tensors): MSE, PSNR (data range 1) and SSIM averaged over the axial,
    coronal and sagittal slices (and each orientation's mean)."""
    Z, Y, X = vol.shape
    out = torch.empty(6, dtype=torch.float64, device=device)
    ws = _bytes(r2g.r2g_metrics_workspace_size(X, Y, Z), device)
    r2g.r2g_volume_metrics(vol.contiguous(), ref.contiguous(), out, ws)
    return dict(zip(METRIC_KEYS, out.cpu().tolist()))


# ----------------------------------------------------------------------------- training state


def inv_softplus(y: np.ndarray) -> np.ndarray:
    return y + np.log(-np.expm1(-y))


class TrainState:
    """Gaussian parameters, gradients and Adam moments, resident on the device in the
    C ABI's flat layout [quat 4M | mean 3M | scale 3M | rho M]."""

    def __init__(self, G, device="cuda"):
        M = G.M
        self.M = M
        raw = np.concatenate([np.asarray(G.quat, np.float64).ravel(), np.asarray(G.mean, np.float64).ravel(),
                              np.log(np.asarray(G.scale, np.float64)).ravel(),
                              inv_softplus(np.maximum(np.asarray(G.rho, np.float64), 1e-6)).ravel()])
        self.raw = torch.tensor(raw, dtype=torch.float32, device=device)
        act = np.concatenate([np.asarray(G.quat, np.float64).ravel(), np.asarray(G.mean, np.float64).ravel(),
                              np.asarray(G.scale, np.float64).ravel(),
                              np.maximum(np.asarray(G.rho, np.float64), 1e-6).ravel()])
        self.act = torch.tensor(act, dtype=torch.float32, device=device)
        self.grad = torch.zeros_like(self.act)
        self.m = torch.zeros_like(self.act)
        self.v = torch.zeros_like(self.act)

    def adopt(self, raw, act, m, v, M: int):
        """Take over a state of M Gaussians (flat layout, arrays of at least 11 M floats)."""
        self.M = int(M)
        self.raw, self.act, self.m, self.v = raw, act, m, v
        self.grad = torch.zeros_like(act)

    def views_of(self, t):
        M = self.M
        return t[0:4 * M].view(M, 4), t[4 * M:7 * M].view(M, 3), t[7 * M:10 * M].view(M, 3), t[10 * M:11 * M]

    def params(self):
        """(mean, scale, quat, rho) views of the activated parameters."""
        q, m, s, r = self.views_of(self.act)
        return m, s, q, r

    def grads(self):
        q, m, s, r = self.views_of(self.grad)
        return m, s, q, r


class TrainStep:
    """One iteration of Eq. 8 on one projection view and one D^3 TV patch."""

    def __init__(self, state: TrainState, views: torch.Tensor, meas: torch.Tensor, cam, D=32, n_out=256,
                 tile=None, total_iters=30000, device="cuda"):
        self.s = state
        self.views = views            # [V, 12] device
        self.meas = meas              # [V, H, W] device
        self.cam = cam
        self.D = D
        self.n_out = n_out
        self.rast = Rasterizer(state.M, 1, cam, tile=tile or SCAN_TILE, device=device)
        from .inputs import patch_grid
        self._patch = patch_grid
        self.vox = Voxelizer(state.M, patch_grid((0, 0, 0), D, n_out), device=device)
        self.image = torch.empty((1, cam.H, cam.W), dtype=torch.float32, device=device)
        self.dimage = torch.empty_like(self.image)
        self.vol = torch.empty(D ** 3, dtype=torch.float32, device=device)
        self.dvol = torch.empty_like(self.vol)
        self.loss = torch.zeros(2, dtype=torch.float32, device=device)
        self.loss_ws = _bytes(r2g.r2g_loss_workspace_size(1, cam.H, cam.W), device)
        self.tv_ws = _bytes(r2g.r2g_tv_workspace_size(1, D), device)
        self.adam = r2g.adam_opts(total_iters=total_iters)

    def run(self, it: int, view: int, offset, check=False):
        """One full iteration; returns nothing (loss stays on the device in self.loss)."""
        mean, scale, quat, rho = self.s.params()
        dmean, dscale, dquat, drho = self.s.grads()
        v = self.views[view:view + 1]
        self.rast.forward(mean, scale, quat, rho, v, self.image, check=check)
        r2g.r2g_projection_loss(self.image, self.meas[view:view + 1], LAMBDA_SSIM, self.loss[0:1], self.dimage,
                                self.loss_ws)
        self.vox.set_grids(self._patch(offset, self.D, self.n_out))
        self.vox.forward(mean, scale, quat, rho, self.vol, check=check)
        r2g.r2g_tv3d(self.vol.view(1, self.D, self.D, self.D), LAMBDA_TV, self.loss[1:2],
                     self.dvol.view(1, self.D, self.D, self.D), self.tv_ws)
        self.rast.backward(mean, scale, quat, rho, v, self.dimage, dmean, dscale, dquat, drho)
        self.vox.backward(mean, scale, quat, rho, self.dvol, dmean, dscale, dquat, drho)
        r2g.r2g_adam_step(self.s.raw, self.s.act, self.s.grad, self.s.m, self.s.v, it, self.adam)


# ----------------------------------------------------------------------------- multi-scan batching


class Scan:
    """One reconstruction job resident on the device: parameters, Adam state,
    views, measured projections, step buffers and workspaces, and the C job
    descriptor for r2g_train_step."""

    def __init__(self, G, views_np, meas_np, cam, n_out=256, D=32, tile=None, total_iters=30000,
                 device="cuda", headroom=1.5, seed=0, biased=False, tv_eps=0.0, dilation=0.0, all_views=False,
                 n_patches=1, full_volume=False, view_chunk=0):
        """all_views: every step rasterizes all V views in one launch (the batch form of
        r2g_train_step) instead of one view picked per step; n_patches: TV patches per
        step (> 1: their origins come from `patch_origins`, a device [n_patches, 3]
        tensor the caller fills before each step); full_volume: every step also
        voxelizes the whole n_out^3 output volume into `full_vol` (forward only);
        view_chunk > 0: the all-views rasterizer works that many views at a time and
        rebuilds each chunk's lists in the backward (a workspace for one chunk)."""
        self.state = TrainState(G, device=device)
        self.all_views = bool(all_views)
        self.n_patches = max(1, int(n_patches))
        self.full_volume = bool(full_volume)
        self.biased = bool(biased)
        self.dilation = float(dilation)  # low-pass dilation of the footprint, pixels^2 (0: none, the paper's)
        self.tv_eps = float(tv_eps)   # > 0: isotropic TV with this eps; 0: anisotropic (default)
        self.version = 0              # bumped whenever the C job changes (densification)
        self.dens_grad = self.dens_count = None
        self.dens_schedule = None
        self.dens_seed = seed
        self.rng = np.random.Generator(np.random.PCG64(seed + 2))  # this scan's view / patch choices
        self.it = 0
        self.M = G.M
        self.cam = cam
        self.D = D
        self.n_out = n_out
        self.views = torch.as_tensor(np.ascontiguousarray(views_np, np.float32), device=device)
        self.meas = torch.as_tensor(np.ascontiguousarray(meas_np, np.float32), device=device)
        self.V = int(self.views.shape[0])
        self.Vs = self.V if self.all_views else 1   # views rasterized per step
        NP = self.n_patches
        self.image = torch.empty((self.Vs, cam.H, cam.W), dtype=torch.float32, device=device)
        self.dimage = torch.empty_like(self.image)
        self.vol = torch.empty(NP * D ** 3, dtype=torch.float32, device=device)
        self.dvol = torch.empty_like(self.vol)
        self.loss = torch.zeros(2, dtype=torch.float32, device=device)
        self.patch_origins = torch.zeros((NP, 3), dtype=torch.float32, device=device)
        self.view_chunk = int(view_chunk)
        self.rast = Rasterizer(self.M, self.Vs, cam, tile=tile or SCAN_TILE, device=device, biased=biased,
                               dilation=self.dilation, view_chunk=self.view_chunk)
        from .inputs import cube_grid, patch_grid

        self.vox = Voxelizer(self.M, [patch_grid((0, 0, 0), D, n_out)] * NP, device=device)
        self.full_vox = Voxelizer(self.M, cube_grid(n_out), device=device) if self.full_volume else None
        self.full_vol = (torch.empty((n_out, n_out, n_out), dtype=torch.float32, device=device)
                         if self.full_volume else None)
        self.loss_ws = _bytes(r2g.r2g_loss_workspace_size(self.Vs, cam.H, cam.W), device)
        self.tv_ws = _bytes(r2g.r2g_tv_workspace_size(NP, D), device)
        self.adam = r2g.adam_opts(total_iters=total_iters)
        self.device = device
        self.headroom = headroom
        self._size_workspaces(headroom)
        self.job = self._make_job()

    def enable_adaptive(self, max_gaussians: int, opts=None, start=500, stop=15000, every=100):
        """Adaptive density control (Sec. 4.2.3, schedule of Sec. 5.1): from then on each
        step accumulates the position-gradient statistics, and `densify()` runs after
        the steps whose iteration count is a multiple of `every` in [start, stop]."""
        self.max_gaussians = int(max_gaussians)
        self.dens_opts = opts or r2g.densify_opts()
        self.dens_schedule = (int(start), int(stop), int(every))
        self.dens_ws = _bytes(r2g.r2g_densify_workspace_size(), self.device)
        self.dens_grad = torch.zeros(self.max_gaussians, dtype=torch.float32, device=self.device)
        self.dens_count = torch.zeros_like(self.dens_grad)
        self.job = self._make_job()

    def densify_due(self) -> bool:
        if getattr(self, "dens_schedule", None) is None:
            return False
        a, b, e = self.dens_schedule
        return a <= self.it <= b and self.it % e == 0

    def densify(self):
        """One prune/clone/split step (r2g_densify) into a new state; the statistics
        restart, the workspaces are re-sized for the new count, and the C job is
        rebuilt (a captured round graph must be recaptured: `version` changes)."""
        s, cap = self.state, self.max_gaussians
        out = [torch.empty(11 * cap, dtype=torch.float32, device=self.device) for _ in range(4)]
        m_new = torch.zeros(1, dtype=torch.int64, device=self.device)
        opts = self.dens_opts
        opts.seed = (int(self.dens_seed) * 1_000_003 + self.it) & (2 ** 64 - 1)
        r2g.r2g_densify(s.M, s.raw, s.act, s.m, s.v, self.dens_grad, self.dens_count, opts, cap, *out, m_new,
                        self.dens_ws)
        M2 = int(m_new.item())
        s.adopt(*out, M2)
        self.M = M2
        self.dens_grad.zero_()
        self.dens_count.zero_()
        self.rast.M = M2
        self.vox.M = M2
        self._size_workspaces(self.headroom, probes=2)
        self.job = self._make_job()
        self.version += 1
        return M2

    def checkpoint(self) -> dict:
        """A snapshot of this scan's training state in host memory: the raw and activated
        parameters and both Adam moments (flat layout, 11 M floats each), the Gaussian
        count, the iteration counter (which drives the learning-rate schedule), the
        state of the scan's view / TV-patch generator and, under adaptive density
        control, the position-gradient statistics.  Waits for the scan's queued work.
        `restore` puts it back; `save_checkpoint` / `load_checkpoint` write and read it."""
        torch.cuda.synchronize(self.device)
        s = self.state
        n = 11 * s.M
        ck = {"M": int(s.M), "it": int(self.it), "rng": self.rng.bit_generator.state,
              "raw": s.raw[:n].cpu().numpy().copy(), "act": s.act[:n].cpu().numpy().copy(),
              "m": s.m[:n].cpu().numpy().copy(), "v": s.v[:n].cpu().numpy().copy()}
        if self.dens_grad is not None:
            ck["dens_grad"] = self.dens_grad.cpu().numpy().copy()
            ck["dens_count"] = self.dens_count.cpu().numpy().copy()
        return ck

    def restore(self, ck: dict):
        """Continue from a `checkpoint` of a scan with the same projections, views, camera
        and options (this scan's own, or one built alike).  The parameters and moments are
        copied to new device arrays (sized for the adaptive-control capacity when it is
        on), the workspaces are re-sized for the snapshot's Gaussian count and the C job is
        rebuilt, so a captured round graph is recaptured (`version` changes).  From a
        restored state the next iteration's forward pass and losses are those the original
        run computed, bit for bit; its update may differ in the last bits, because the
        backward sums the gradient moments with float atomics."""
        M = int(ck["M"])
        n = 11 * M
        cap = 11 * max(M, getattr(self, "max_gaussians", 0) if self.dens_grad is not None else 0)
        out = []
        for key in ("raw", "act", "m", "v"):
            a = np.asarray(ck[key], np.float32)
            if a.shape != (n,):
                raise ValueError(f"checkpoint array {key} has shape {a.shape}, expected ({n},)")
            t = torch.zeros(cap, dtype=torch.float32, device=self.device)
            t[:n].copy_(torch.from_numpy(a))
            out.append(t)
        self.state.adopt(*out, M)
        self.M = M
        self.rast.M = M
        self.vox.M = M
        if self.full_vox is not None:
            self.full_vox.M = M
        self.it = int(ck["it"])
        self.rng.bit_generator.state = ck["rng"]
        if self.dens_grad is not None:
            if "dens_grad" in ck:
                self.dens_grad.copy_(torch.from_numpy(np.asarray(ck["dens_grad"], np.float32)))
                self.dens_count.copy_(torch.from_numpy(np.asarray(ck["dens_count"], np.float32)))
            else:
                self.dens_grad.zero_()
                self.dens_count.zero_()
        self._size_workspaces(self.headroom, probes=2)
        self.job = self._make_job()
        self.version += 1

    def volume_params(self):
        """(mean, scale, quat, rho) for the voxelizer.  The rectified model's densities
        are the 3D densities; the X-3DGS variant (biased=True) learned mu rho per view,
        so each density is divided by its Gaussian's mean mu over the training views
        (Sec. 4.2.1) -- in the r2g_mean_mu kernel."""
        mean, scale, quat, rho = self.state.params()
        if not self.biased:
            return mean, scale, quat, rho
        rv = torch.empty_like(rho)
        r2g.r2g_mean_mu(mean, scale, quat, self.views, self.rast.cam, rho=rho, rho_vol=rv)
        return mean, scale, quat, rv

    def _size_workspaces(self, headroom, probes=6):
        """Size the list workspaces on a spread of views and patch positions with
        checked runs, then add headroom: the captured graph cannot regrow them."""
        from .inputs import patch_grid

        mean, scale, quat, rho = self.state.params()
        need_r, need_v = 0, 0
        if self.all_views:
            self.rast.forward(mean, scale, quat, rho, self.views, self.image, check=True)
            need_r = r2g.r2g_poll(self.rast.ws)[1]
        else:
            for v in np.linspace(0, self.V - 1, min(self.V, probes)).astype(int):
                self.rast.forward(mean, scale, quat, rho, self.views[v:v + 1], self.image, check=True)
                need_r = max(need_r, r2g.r2g_poll(self.rast.ws)[1])
        NP = self.n_patches
        for off in ((0, 0, 0), ((self.n_out - self.D) // 2,) * 3, (self.n_out - self.D,) * 3):
            # every patch of the step at the densest of the probed positions
            self.vox.set_grids([patch_grid(off, self.D, self.n_out)] * NP)
            self.vox.forward(mean, scale, quat, rho, self.vol, check=True)
            need_v = max(need_v, r2g.r2g_poll(self.vox.ws)[1])
        self.rast.capacity = int(need_r * headroom) + 4096
        self.rast._alloc()
        self.vox.capacity = int(need_v * headroom) + 4096
        self.vox._alloc()
        if self.full_vox is not None:
            self.full_vox.forward(mean, scale, quat, rho, self.full_vol.view(-1), check=True)
            self.full_vox.capacity = int(r2g.r2g_poll(self.full_vox.ws)[1] * headroom) + 4096
            self.full_vox._alloc()

    def _make_job(self):
        s = self.state
        J = r2g.Job()
        J.M = self.M
        J.raw, J.act, J.grad = s.raw.data_ptr(), s.act.data_ptr(), s.grad.data_ptr()
        J.adam_m, J.adam_v = s.m.data_ptr(), s.v.data_ptr()
        J.V = self.V
        J.views, J.meas = self.views.data_ptr(), self.meas.data_ptr()
        J.cam = self.rast.cam
        J.ropts = self.rast.opts
        J.Q3 = Q_VOXEL
        J.D = self.D
        J.voxel = 2.0 / self.n_out
        J.lambda_ssim, J.lambda_tv = LAMBDA_SSIM, LAMBDA_TV
        J.adam = self.adam
        J.image, J.dimage = self.image.data_ptr(), self.dimage.data_ptr()
        J.vol, J.dvol, J.loss = self.vol.data_ptr(), self.dvol.data_ptr(), self.loss.data_ptr()
        J.raster_ws, J.raster_ws_bytes = self.rast.ws.data_ptr(), self.rast.ws.numel()
        J.voxel_ws, J.voxel_ws_bytes = self.vox.ws.data_ptr(), self.vox.ws.numel()
        J.loss_ws, J.loss_ws_bytes = self.loss_ws.data_ptr(), self.loss_ws.numel()
        J.tv_ws, J.tv_ws_bytes = self.tv_ws.data_ptr(), self.tv_ws.numel()
        J.tv_eps = self.tv_eps
        J.views_per_step = self.V if self.all_views else 0
        J.n_patches = self.n_patches if self.n_patches > 1 else 0
        J.patch_origins = self.patch_origins.data_ptr() if self.n_patches > 1 else None
        if self.full_vox is not None:
            J.full_vol = self.full_vol.data_ptr()
            J.full_grid = self.full_vox.grids[0]
            J.full_ws, J.full_ws_bytes = self.full_vox.ws.data_ptr(), self.full_vox.ws.numel()
        if self.dens_grad is not None:
            J.dens_grad, J.dens_count = self.dens_grad.data_ptr(), self.dens_count.data_ptr()
        return J

    def autotune_tile(self, tiles=((8, 8), (16, 16), (32, 8), (32, 32)), steps=4):
        """Pick the rasterizer tile shape with the shortest fused training step for this
        scan: each candidate is timed over `steps` steps (CUDA events, after one warm-up
        step) on a copy of the state, which is restored afterwards, so the scan's
        trajectory does not change.  Returns {tile: ms per step} and keeps the fastest."""
        import ctypes

        s = self.state
        saved = [t.clone() for t in (s.raw, s.act, s.m, s.v)]
        stream = torch.cuda.current_stream()
        t = np.zeros((steps + 1, 8), np.int32)
        f = t.view(np.float32)
        g = np.random.Generator(np.random.PCG64(12345))
        for k in range(steps + 1):
            off = g.integers(0, self.n_out - self.D + 1, 3)
            t[k, 0], t[k, 1] = int(g.integers(0, self.V)), self.it
            f[k, 2:5] = -1.0 + off * (2.0 / self.n_out)
        table = torch.as_tensor(t, device=self.device)
        elem = ctypes.sizeof(r2g.RoundEntry)
        sep = int(self.rast.opts.separate_lists)
        times = {}
        for tile in tiles:
            self.rast = Rasterizer(self.M, self.Vs, self.cam, tile=tile, device=self.device, biased=self.biased,
                                   dilation=self.dilation, view_chunk=self.view_chunk)
            self.rast.opts.separate_lists = sep
            self._size_workspaces(self.headroom, probes=2)
            self.job = self._make_job()
            r2g.r2g_train_step(self.job, table.data_ptr(), stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k in range(1, steps + 1):
                r2g.r2g_train_step(self.job, table.data_ptr() + k * elem, stream)
            e1.record(stream)
            e1.synchronize()
            times[tuple(tile)] = e0.elapsed_time(e1) / steps
            for dst, src in zip((s.raw, s.act, s.m, s.v), saved):
                dst.copy_(src)
        best = min(times, key=times.get)
        self.rast = Rasterizer(self.M, self.Vs, self.cam, tile=best, device=self.device, biased=self.biased,
                               dilation=self.dilation, view_chunk=self.view_chunk)
        self.rast.opts.separate_lists = sep
        self._size_workspaces(self.headroom, probes=2)
        self.job = self._make_job()
        self.version += 1
        return times

    def next_entry(self):
        """(view, iteration, TV patch origin) of this scan's next iteration."""
        v = int(self.rng.integers(0, self.V))
        off = self.rng.integers(0, self.n_out - self.D + 1, 3)
        e = (v, self.it, tuple(float(x) for x in (-1.0 + off * (2.0 / self.n_out))))
        self.it += 1
        return e

    def footprint_bytes(self) -> int:
        """Device bytes this scan holds (parameters, Adam state, views, measurements,
        step buffers and workspaces)."""
        s = self.state
        n = sum(t.numel() * t.element_size() for t in (s.raw, s.act, s.grad, s.m, s.v, self.views, self.meas,
                                                         self.image, self.dimage, self.vol, self.dvol, self.loss))
        if self.full_vox is not None:
            n += self.full_vol.numel() * 4 + self.full_vox.ws.numel()
        return int(n + self.rast.ws.numel() + self.vox.ws.numel() + self.loss_ws.numel() + self.tv_ws.numel())

    def overflowed(self) -> bool:
        bad = r2g.r2g_poll(self.rast.ws)[0] != r2g.R2G_OK or r2g.r2g_poll(self.vox.ws)[0] != r2g.R2G_OK
        return bad or (self.full_vox is not None and r2g.r2g_poll(self.full_vox.ws)[0] != r2g.R2G_OK)


class HostFeed:
    """Training one scan from host memory (r2g_train_step_host_batch): its measured
    projections [V][H][W] and view table [V][12] stay in pinned host memory; each
    step's measurements, geometry rows, TV patch origins and round entry go into
    one of n_slots device staging slots on a copy stream while the steps before it
    run, and its losses come back to pinned host memory.  A one-view scan stages the
    step's view; an all-views scan (Scan(all_views=True)) stages all V views every
    step.  step() returns the losses of the step n_slots - 1 calls earlier (None
    for the first n_slots - 1 calls); finish() returns those still in flight."""

    def __init__(self, scan: "Scan", meas_host: torch.Tensor, views_host: torch.Tensor, n_slots=3, stream=None):
        if not (meas_host.is_pinned() and views_host.is_pinned()):
            raise ValueError("HostFeed needs pinned host tensors")
        H, W = scan.cam.H, scan.cam.W
        if tuple(meas_host.shape[1:]) != (H, W) or views_host.shape[1] != 12:
            raise ValueError("measurements must be [V][H][W] and views [V][12]")
        dev = scan.device
        self.scan, self.n = scan, int(n_slots)
        Vs, NP = scan.Vs, scan.n_patches
        self.meas_host, self.views_host = meas_host.contiguous(), views_host.contiguous()
        self.meas_stage = torch.empty((self.n, Vs, H, W), dtype=torch.float32, device=dev)
        self.views_stage = torch.empty((self.n, Vs, 12), dtype=torch.float32, device=dev)
        self.ent_stage = torch.zeros((self.n, 8), dtype=torch.int32, device=dev)
        self.ent_host = torch.zeros((self.n, 8), dtype=torch.int32).pin_memory()
        self.org_stage = torch.zeros((self.n, NP, 3), dtype=torch.float32, device=dev)
        self.loss_dev = torch.zeros((self.n, 2), dtype=torch.float32, device=dev)
        self.loss_host = torch.zeros((self.n, 2), dtype=torch.float32).pin_memory()
        self.loss_np = self.loss_host.numpy()
        self.stg = r2g.Staging(self.n, self.meas_stage.data_ptr(), self.views_stage.data_ptr(),
                               self.ent_stage.data_ptr(), self.ent_host.data_ptr(), self.loss_dev.data_ptr(),
                               self.org_stage.data_ptr())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._meas0, self._img = self.meas_host.data_ptr(), 4 * H * W
        self._views0, self._loss0 = self.views_host.data_ptr(), self.loss_host.data_ptr()
        self.bytes_in = 4 * Vs * H * W + 48 * Vs + 32 + (12 * NP if NP > 1 else 0)  # per step, host -> device
        self.k = 0   # steps queued
        self.r = 0   # first step whose losses have not been returned

    def _take(self):
        r = self.r
        r2g.r2g_train_step_host_wait(self.stg, r, self.stream)
        self.r = r + 1
        return float(self.loss_np[r % self.n, 0]), float(self.loss_np[r % self.n, 1])

    def step(self, view: int, entry_ptr: int, origins_ptr: int | None = None):
        """Queue one iteration on the measurement and geometry of `view` (all views for
        an all-views scan) with the round entry at host address entry_ptr and, for a
        scan with several TV patches, their origins at host address origins_ptr
        (pinned float32 [n_patches][3]; both read during the call)."""
        k, n = self.k, self.n
        v0 = 0 if self.scan.all_views else view
        r2g.r2g_train_step_host_batch(self.scan.job, self.stg, k, self._meas0 + v0 * self._img,
                                      self._views0 + 48 * v0, origins_ptr, entry_ptr, self._loss0 + 8 * (k % n),
                                      self.stream)
        self.k = k + 1
        # step k + 1 reuses the loss buffer of step k + 1 - n: return that step's first
        return self._take() if self.k - self.r >= n else None

    def finish(self):
        """Wait for every queued step; their losses, in step order."""
        return [self._take() for _ in range(self.k - self.r)]


class BatchTrainer:
    """Runs one training iteration of every resident scan per round.

    The per-round choices (view, TV patch origin, iteration; each scan draws them
    from its own seeded generator) live in a device round table [J][8]
    (r2g_round_entry) filled from pinned host memory by a copy that is part of the
    round.  With graph=True the whole round -- the table upload and every scan's
    r2g_train_step, one branch per scan on its own stream -- is captured once as a
    CUDA graph and replayed; with graph=False the same calls are issued eagerly on
    the same streams."""

    def __init__(self, scans, n_streams=None, graph=True, seed=0, device="cuda", separate_lists=None,
                 autotune=False):
        self.scans = list(scans)
        self.J = len(self.scans)
        # with several scans in flight the list builds run as separate launches: a
        # cooperative launch holds its SMs until its whole grid runs, which limits the
        # overlap between the scans' branches (measured: 1.55 vs 1.86 ms per 16-scan round)
        sep = self.J > 1 if separate_lists is None else bool(separate_lists)
        for sc in self.scans:
            if bool(sc.rast.opts.separate_lists) != sep:
                sc.rast.opts.separate_lists = int(sep)
                sc.job = sc._make_job()
                sc.version += 1
        # per-scan tile shape by measurement (each scan alone, state restored)
        self.tiles = [sc.autotune_tile() if autotune else None for sc in self.scans]
        self.device = device
        self.table_host = torch.zeros((self.J, 8), dtype=torch.int32).pin_memory()
        self.table_dev = torch.zeros((self.J, 8), dtype=torch.int32, device=device)
        n_streams = self.J if n_streams is None else n_streams  # one branch per scan by default
        self.streams = [torch.cuda.Stream(device=device) for _ in range(max(1, n_streams))]
        self.graph = None
        self.use_graph = graph
        self._versions = [sc.version for sc in self.scans]
        self.elem = ctypes_sizeof_entry()

    def _fill(self):
        t = self.table_host.numpy()
        f = t.view(np.float32)
        for j, sc in enumerate(self.scans):
            v, it, origin = sc.next_entry()
            t[j, 0] = v
            t[j, 1] = it
            f[j, 2:5] = origin

    @property
    def it(self):
        return [sc.it for sc in self.scans]

    def _issue(self):
        main = torch.cuda.current_stream()
        r2g.r2g_upload_round(self.table_dev, self.table_host, self.J, main)
        base = self.table_dev.data_ptr()
        for j, sc in enumerate(self.scans):
            s = self.streams[j % len(self.streams)]
            s.wait_stream(main)
            with torch.cuda.stream(s):
                r2g.r2g_train_step(sc.job, base + j * self.elem, s)
        for s in self.streams[:min(self.J, len(self.streams))]:  # only the branches that were forked
            main.wait_stream(s)

    def round(self):
        """One iteration of every scan.  The host table is rewritten only after the
        previous round has finished.  With graph=True the first round runs eagerly
        (which also loads every kernel) and is then captured; later rounds replay.
        Scans with adaptive control densify after the round when due, and the graph
        is recaptured at the next round."""
        torch.cuda.current_stream().synchronize()
        versions = [sc.version for sc in self.scans]
        if versions != self._versions:
            self.graph = None
            self._versions = versions
        self._fill()
        self._round()
        due = [sc for sc in self.scans if sc.densify_due()]
        if due:
            torch.cuda.current_stream().synchronize()
            for sc in due:
                sc.densify()

    def _round(self):
        if not self.use_graph:
            self._issue()
            return
        if self.graph is None:
            self._issue()
            torch.cuda.synchronize()
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph):
                self._issue()
            return
        self.graph.replay()

    def losses(self):
        return torch.stack([sc.loss for sc in self.scans]).cpu().numpy()


def _npz(path: str) -> str:
    return path if str(path).endswith(".npz") else str(path) + ".npz"


def save_checkpoint(ck: dict, path: str):
    """Write a `Scan.checkpoint` snapshot to one .npz file (arrays as stored, the
    count, iteration and generator state as JSON); ".npz" is appended to a path
    without it, as `load_checkpoint` expects."""
    import json

    path = _npz(path)
    arrays = {k: np.asarray(v) for k, v in ck.items() if isinstance(v, np.ndarray)}
    meta = {k: v for k, v in ck.items() if not isinstance(v, np.ndarray)}
    np.savez(path, __meta__=np.frombuffer(json.dumps(meta).encode(), dtype=np.uint8), **arrays)


def load_checkpoint(path: str) -> dict:
    """Read a snapshot written by `save_checkpoint`."""
    import json

    with np.load(_npz(path)) as z:
        ck = json.loads(bytes(z["__meta__"]).decode())
        for k in z.files:
            if k != "__meta__":
                ck[k] = z[k].copy()
    return ck


def ctypes_sizeof_entry() -> int:
    import ctypes

    return ctypes.sizeof(r2g.RoundEntry)
