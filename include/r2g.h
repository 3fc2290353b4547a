/* r2g.h -- C ABI of the B300 (sm_103a) R^2-Gaussian X-ray rasterizer and voxelizer.
 *
 * The method (arXiv 2405.20693): a scanned object is a sum of radiative 3D
 * Gaussians G_i(x) = rho_i exp(-1/2 (x-p_i)^T Sigma_i^{-1} (x-p_i)), Sigma_i =
 * R_i S_i S_i^T R_i^T (Eq. 3, Sec. 4.1), density sigma(x) = sum_i G_i(x) (Eq. 4).
 * A log-projection pixel is the line integral of sigma (Eq. 1), which splits into
 * per-Gaussian integrals (Eq. 5).  Each Gaussian is carried into ray space by the
 * scanner transform W, t and the local-affine Jacobian J of the cone-beam map
 * (Eq. 6, App. A) and integrated in closed form into a 2D Gaussian of amplitude
 * rho_hat = mu rho, mu = sqrt(2 pi |Sigma~| / |Sigma^|) (Eq. 7); the image is
 * the plain sum of those 2D Gaussians (no alpha compositing).  The voxelizer
 * evaluates Eq. 4 on voxel grids through 8^3 bricks (Sec. 4.2.2).
 *
 * Conventions shared by every entry point
 *  - Pointers named "device" are CUDA device memory owned by the caller.
 *    Structs passed by pointer (camera, options, grids) are host memory, read
 *    during the call only.  The library never allocates: scratch lives in a
 *    caller-owned device workspace whose size the *_workspace_size functions give.
 *  - Every call is asynchronous on `stream` (a cudaStream_t; NULL is the legacy
 *    default stream) and never synchronises the host, except the functions
 *    documented as synchronising (r2g_poll, r2g_*_lists, r2g_pair_count).
 *  - Gaussian parameters are float32 structure-of-arrays: mean[M][3],
 *    scale[M][3] (> 0, already activated), quat[M][4] as (w, x, y, z) -- it is
 *    normalised inside and gradients flow through the normalisation -- and
 *    rho[M] (any sign).  1 <= M < 2^31.
 *  - Gradients are ACCUMULATED (+=) into dmean, dscale, dquat, drho.
 *  - Errors: argument errors are found on the host and returned at once
 *    (R2G_E_INVAL, nothing launched); a failed launch returns R2G_E_CUDA.  Errors
 *    found on the device (a list longer than the workspace's key capacity) are
 *    written to a status word in the workspace and read by r2g_poll.
 *    r2g_last_error() gives a thread-local message for the last failure.
 */
#ifndef R2G_H
#define R2G_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* r2g_stream; /* identical to cudaStream_t */

typedef enum {
    R2G_OK = 0,
    R2G_E_INVAL = 1,    /* bad argument; nothing was launched */
    R2G_E_CAPACITY = 2, /* more tile/brick list entries than the workspace holds */
    R2G_E_CUDA = 3,     /* a CUDA call or launch failed */
    R2G_E_TIMEOUT = 4,  /* a bounded device-side wait gave up (see r2g_set_wait_limit) */
    R2G_E_NUMERIC = 5   /* a training step met a non-finite loss and skipped its update */
} r2g_status;

/* Detector and beam of one scan (App. A).  Pixel (r, c) has its centre at
 *   xi  = (c + 1/2 - W/2) * pitch_u + off_u,  eta = (r + 1/2 - H/2) * pitch_v + off_v
 * on the detector plane, in the same length unit as the Gaussians. */
typedef struct {
    int32_t beam;      /* 0 = parallel beam (the L_SO -> infinity limit, J = I); 1 = cone beam */
    int32_t H, W;      /* detector rows and columns, 1..32768 */
    float L_SD;        /* source-to-detector distance (cone) */
    float pitch_u, pitch_v;
    float off_u, off_v;
    float near_plane;  /* cone: a Gaussian whose scanner depth u2 <= near_plane is dropped */
} r2g_camera;

/* Rasterizer options. */
typedef struct {
    float Q;             /* pixel gate: a Gaussian adds to a pixel when q = d^T Sigma^^{-1} d <= Q (9 = 3 sigma) */
    int32_t tile_w;      /* tile shape: 16x16 (default), 8x8, 32x8 or 32x32 */
    int32_t tile_h;
    int32_t count_pairs; /* 1: also count the gated pairs (bookkeeping runs only; slower) */
    int32_t biased;      /* 1: the un-rectified amplitude rho_hat = rho of the 3DGS-style X-ray splatting that
                          * Sec. 4.2.1 corrects (mu = 1, view-dependent projected mass); 0 (default): Eq. 7 */
    int32_t separate_lists; /* 1: build the per-tile lists in separate launches; 0 (default): one cooperative
                             * launch when the grid can be resident (fewer launches; it holds its SMs until
                             * the whole grid runs, which limits overlap with other streams' kernels).  The
                             * lists are the same either way.  r2g_train_step applies it to both branches. */
    float dilation;      /* low-pass dilation in pixels^2, 0 (default) = none.  > 0: the footprint evaluated at
                          * the pixels (and its pixel box) is Sigma^ + diag(dilation pitch_u^2, dilation
                          * pitch_v^2), as 3DGS adds 0.3 px^2 for anti-aliasing; rho_hat keeps Eq. 7's mu of the
                          * undilated Sigma^, so the projected mass is no longer the Gaussian's (the paper uses
                          * none).  Negative or non-finite: R2G_E_INVAL. */
    int32_t view_chunk;  /* 0 (default): the workspace holds every view's records and lists, the forward
                          * stores them and the backward reuses them.  k > 0 (and < V): views are processed k
                          * at a time, the workspace holds one chunk of k views (its size is that of k views),
                          * and the backward rebuilds each chunk's records and lists instead of reading them
                          * stored -- the memory of a many-view launch for a second projection and list build
                          * of all but the last chunk.  The image and the gradients are those of the stored
                          * form (the forward bit for bit).  r2g_raster_lists then returns the last chunk's
                          * lists.  Negative: R2G_E_INVAL. */
} r2g_raster_opts;

/* One voxel grid: the centre of voxel (x, y, z) is origin + (index + 1/2) * voxel;
 * the volume is stored [Z][Y][X], x fastest. */
typedef struct {
    float origin[3];
    float voxel[3];
    int32_t dims[3];   /* X, Y, Z, each 1..4096 */
} r2g_grid;

/* ---------------------------------------------------------------- rasterizer
 *
 * Views: a DEVICE float table views[V][12] = W (3x3 row-major) then t (3), the
 * world->scanner transform u = W p + t of App. A for each projection angle.
 * Per (Gaussian, view) the library forms, in FP32, in this order (the stated
 * sequence the per-tile lists are defined by; no fused multiply-add):
 *   q <- q / |q|;  R(q);  M = R diag(s);  u = W p + t;
 *   cone:  f = L_SD / u2, j02 = -(f u0)/u2, j12 = -(f u1)/u2, p^ = (f u0, f u1),
 *          T = [[f W0 + j02 W2], [f W1 + j12 W2]]  (the first two rows of J W);
 *   parallel: T = [W0; W1], p^ = (u0, u1);
 *   N = T M;  Sigma^ = N N^T = [[alpha, beta], [beta, gamma]];
 *   |Sigma^| = sum of the squared 2x2 minors of N (Cauchy-Binet);
 *   drop if (cone) u2 <= near_plane or |Sigma^| <= 0;
 *   e_x = sqrt(Q alpha), e_y = sqrt(Q gamma);
 *   cx = (p^x - off_u)/pitch_u + (W/2 - 1/2),  rx = e_x / pitch_u  (rows alike);
 *   pixel columns ceil(cx - rx) .. floor(cx + rx) clamped to the detector
 *   (empty -> dropped); tiles = those columns / tile_w (rows / tile_h).
 * Every pixel of every listed tile then evaluates the gate q <= Q exactly, so the
 * image does not depend on the tile shape.  Per-tile lists hold Gaussian ids in
 * ascending order (stable radix sort), so the forward image is deterministic.
 * The amplitude uses mu = sqrt(2 pi / (omega^T Sigma^{-1} omega)), omega the unit
 * direction from the source to the mean (cone) or the beam direction (parallel),
 * which equals Eq. 7's determinant ratio. */

/* Bytes of workspace for M Gaussians x V views with room for key_capacity
 * (tile, Gaussian) list entries.  1 <= key_capacity <= 2^32 - 1.  Returns 0 for
 * invalid arguments. */
size_t r2g_raster_workspace_size(int64_t M, int32_t V, const r2g_camera* cam, const r2g_raster_opts* opts,
                                 int64_t key_capacity);

/* Eq. 5 + Eq. 7: image[V][H][W] (device, float32, overwritten) =
 * sum over Gaussians of rho_hat exp(-q/2) [q <= Q] at each pixel centre.
 * The workspace keeps the per-view records and tile lists for the matching
 * r2g_rasterize_backward call.  Sets R2G_E_CAPACITY in the workspace status (see
 * r2g_poll) when the lists need more than the workspace's key capacity; the image
 * is then incomplete. */
r2g_status r2g_rasterize(int64_t M, const float* mean, const float* scale, const float* quat, const float* rho,
                         int32_t V, const float* views, const r2g_camera* cam, const r2g_raster_opts* opts,
                         float* image, void* ws, size_t ws_bytes, r2g_stream stream);

/* Gradient of sum(dimage * image) with respect to the parameters, accumulated into
 * dmean[M][3], dscale[M][3], dquat[M][4], drho[M] (device).  Must follow the
 * r2g_rasterize call that filled `ws` with the same parameters, views and options,
 * with no other use of `ws` in between.  Gradient accumulation uses float atomics,
 * so the last bits may vary from run to run. */
r2g_status r2g_rasterize_backward(int64_t M, const float* mean, const float* scale, const float* quat,
                                  const float* rho, int32_t V, const float* views, const r2g_camera* cam,
                                  const r2g_raster_opts* opts, const float* dimage, float* dmean, float* dscale,
                                  float* dquat, float* drho, void* ws, size_t ws_bytes, r2g_stream stream);

/* The projection step alone (Eq. 6, Eq. 7; the stated FP32 sequence above), for
 * inspection and tests: proj[V][M][8] (device) = p^x, p^y (detector units),
 * alpha, beta, gamma (Sigma^), |Sigma^|, rho_hat, valid (1.0 / 0.0);
 * rect[V][M][4] (device int32) = pixel columns c_lo, c_hi and rows r_lo, r_hi
 * of the bound (zeros when dropped).  No workspace. */
r2g_status r2g_project(int64_t M, const float* mean, const float* scale, const float* quat, const float* rho,
                       int32_t V, const float* views, const r2g_camera* cam, const r2g_raster_opts* opts,
                       float* proj, int32_t* rect, r2g_stream stream);

/* Eq. 7's factor averaged over views, for the X-3DGS variant (Sec. 4.2.1).
 * mu_mean[M] (device, may be NULL) = the mean over the V views of
 * mu = sqrt(2 pi / (omega^T Sigma^-1 omega)) of each Gaussian, omega the unit ray
 * through its mean (views that drop it by the near plane are left out; 0 if every
 * view drops it).  rho_vol[M] (device, may be NULL; needs rho) = rho / mu_mean, 0
 * where mu_mean is 0: a model trained with `biased` = 1 learns per-view amplitudes
 * mu rho, and rho_vol is the density that variant hands to the voxelizer.  At
 * least one output must be given.  No workspace; M = 0 is a no-op. */
r2g_status r2g_mean_mu(int64_t M, const float* mean, const float* scale, const float* quat, const float* rho,
                       int32_t V, const float* views, const r2g_camera* cam, float* mu_mean, float* rho_vol,
                       r2g_stream stream);

/* The per-tile lists of the last r2g_rasterize on `ws`.  Synchronises `stream`.
 * ranges[n_tiles][2] (device uint32, [start, end) into ids) with n_tiles =
 * V * ceil(H/tile_h) * ceil(W/tile_w), tiles numbered (v, ty, tx) row-major;
 * ids[capacity] (device uint32) = Gaussian id of each entry.  *n_entries (host)
 * receives the entry count; R2G_E_CAPACITY if it exceeds `capacity` (nothing
 * copied). */
r2g_status r2g_raster_lists(int64_t M, int32_t V, const r2g_camera* cam, const r2g_raster_opts* opts,
                            const void* ws, size_t ws_bytes, uint32_t* ranges, uint32_t* ids, int64_t capacity,
                            int64_t* n_entries, r2g_stream stream);

/* Count of (pixel or voxel, Gaussian) pairs that passed the gate in the last
 * counting call on `ws`: r2g_rasterize with opts->count_pairs = 1, or
 * r2g_voxelize_counted.  Bookkeeping for throughput figures; timed runs do not
 * count.  Synchronises `stream`. */
r2g_status r2g_pair_count(const void* ws, size_t ws_bytes, int64_t* pairs, r2g_stream stream);

/* ---------------------------------------------------------------- voxelizer
 *
 * Bricks of 8^3 voxels per grid; a Gaussian is listed in every brick meeting the
 * voxel-centre box |x_k - p_k| <= sqrt(Q3 Sigma_kk), formed in FP32 as
 *   Sigma_kk = (M_k0^2 + M_k1^2) + M_k2^2 (M = R diag(s) as above),
 *   c_k = (p_k - origin_k)/voxel_k - 1/2, r_k = sqrt(Q3 Sigma_kk)/voxel_k,
 *   voxels ceil(c_k - r_k) .. floor(c_k + r_k) clamped, bricks = voxels / 8.
 * Each voxel then applies the gate q <= Q3 exactly.  Q3 = 11.345 is the 0.99
 * quantile of chi^2_3 (Sec. 4.2.2 culls at probability 0.99). */

size_t r2g_voxel_workspace_size(int64_t M, int32_t G, const r2g_grid* grids, int64_t key_capacity);

/* Eq. 4: vol (device float32, overwritten) = the G grids' volumes concatenated in
 * order, each [Z][Y][X]; V[x] = sum_i rho_i exp(-1/2 (x-p_i)^T Sigma_i^{-1} (x-p_i)) [q <= Q3].
 * 1 <= G <= 64.  The workspace keeps the brick lists for r2g_voxelize_backward. */
r2g_status r2g_voxelize(int64_t M, const float* mean, const float* scale, const float* quat, const float* rho,
                        int32_t G, const r2g_grid* grids, float Q3, float* vol, void* ws, size_t ws_bytes,
                        r2g_stream stream);

/* r2g_voxelize that also counts the gated (voxel, Gaussian) pairs (read them with
 * r2g_pair_count). */
r2g_status r2g_voxelize_counted(int64_t M, const float* mean, const float* scale, const float* quat,
                                const float* rho, int32_t G, const r2g_grid* grids, float Q3, float* vol, void* ws,
                                size_t ws_bytes, r2g_stream stream);

/* Gradient of sum(dvol * vol), accumulated (+=).  Must follow the matching
 * r2g_voxelize on `ws` (same parameters and grids). */
r2g_status r2g_voxelize_backward(int64_t M, const float* mean, const float* scale, const float* quat,
                                 const float* rho, int32_t G, const r2g_grid* grids, float Q3, const float* dvol,
                                 float* dmean, float* dscale, float* dquat, float* drho, void* ws,
                                 size_t ws_bytes, r2g_stream stream);

/* Per-brick lists of the last r2g_voxelize on `ws` (synchronises `stream`):
 * ranges[n_bricks][2], bricks numbered per grid in order, (bz, by, bx) row-major
 * within a grid; ids[capacity] Gaussian ids; *n_entries the count. */
r2g_status r2g_voxel_lists(int64_t M, int32_t G, const r2g_grid* grids, const void* ws, size_t ws_bytes,
                           uint32_t* ranges, uint32_t* ids, int64_t capacity, int64_t* n_entries,
                           r2g_stream stream);

/* ---------------------------------------------------------------- losses (Eq. 8)
 *
 * Projection loss L1 + lambda_ssim (1 - SSIM) over a batch render/meas[V][H][W]
 * (device): L1 = mean |render - meas| over all V*H*W pixels; SSIM (Wang 2004) with
 * an 11x11 Gaussian window (sigma 1.5), zero padding, C1 = 1e-4, C2 = 9e-4, mean of
 * the SSIM map per view, averaged over views.  Writes the loss to *loss (device
 * float) and d loss / d render to drender[V][H][W] (device, overwritten). */
size_t r2g_loss_workspace_size(int32_t V, int32_t H, int32_t W);
r2g_status r2g_projection_loss(int32_t V, int32_t H, int32_t W, const float* render, const float* meas,
                               float lambda_ssim, float* loss, float* drender, void* ws, size_t ws_bytes,
                               r2g_stream stream);

/* lambda_tv x anisotropic 3D total variation (Sec. 4.2.3): for each axis, the mean
 * of |forward difference| over all valid differences, summed over the 3 axes, of
 * each of G volumes vol[G][D][D][D] (device), summed over the G volumes.  Writes
 * *loss (device) and dvol (device, overwritten).  2 <= D <= 1024.  The loss is
 * reduced in a fixed order through a workspace of r2g_tv_workspace_size bytes. */
size_t r2g_tv_workspace_size(int32_t G, int32_t D);
r2g_status r2g_tv3d(int32_t G, int32_t D, const float* vol, float lambda_tv, float* loss, float* dvol, void* ws,
                    size_t ws_bytes, r2g_stream stream);

/* lambda_tv x isotropic 3D total variation, an alternative to the anisotropic form
 * of r2g_tv3d (Sec. 4.2.3 names 3D TV without fixing the norm): per volume, the
 * mean over its D^3 voxels of sqrt(sum over the 3 axes of the squared forward
 * difference + eps), a difference being 0 where the forward neighbour lies outside
 * the volume; summed over the G volumes.  eps > 0 keeps the gradient finite in
 * flat regions.  Same layouts, workspace (r2g_tv_workspace_size) and errors as
 * r2g_tv3d; eps <= 0 returns R2G_E_INVAL. */
r2g_status r2g_tv3d_iso(int32_t G, int32_t D, const float* vol, float lambda_tv, float eps, float* loss, float* dvol,
                        void* ws, size_t ws_bytes, r2g_stream stream);

/* The same TV loss and gradient as r2g_tv3d, for callers that cannot allocate
 * device memory where they call it (a host that fixes the device budget up front,
 * a real-time loop that must not stall on an allocation, a plugin that only
 * receives input and output buffers).  No workspace argument: the partial sums go
 * to a fixed 256 KiB array inside the library, so G * D^3 <= 16777216 voxels
 * (larger volumes return R2G_E_INVAL; use r2g_tv3d).  Nothing is allocated.
 * The first call on each device looks up that array's device address once
 * (cudaGetSymbolAddress) -- make it before any stream capture; the address is kept
 * for the process, so it is not valid after a cudaDeviceReset or from another
 * (non-primary) context on that device.  Calls share the
 * array: calls that overlap on the GPU race; calls ordered on one stream do not.
 * The paper has no counterpart to this entry point. */
r2g_status r2g_tv3d_noalloc(int32_t G, int32_t D, const float* vol, float lambda_tv, float* loss, float* dvol,
                            r2g_stream stream);

/* ---------------------------------------------------------------- optimizer
 *
 * One Adam step (Sec. 5.1) on the raw parameters, given gradients with respect to
 * the ACTIVATED parameters that the rasterizer/voxelizer consumed.  Raw ->
 * activated: mean as is, scale = exp(raw_scale), quat as is, rho = softplus(raw_rho).
 * The step reads the gradients, updates the raw parameters and both moments,
 * writes the new activated parameters, and zeroes the gradients for the next
 * iteration.  Learning rate per group: lr0 * final_factor^(it / total_iters);
 * `it` is the 0-based iteration.  raw, act, grad, m, v are device float32 arrays
 * of M*11 entries laid out group after group: quat [M][4], mean [M][3],
 * scale [M][3], rho [M] (quat first, so that it keeps the 16-byte alignment the
 * rasterizer needs). */
typedef struct {
    float lr0[4];        /* mean, scale, quat, rho: 2e-4, 5e-3, 1e-3, 1e-2 in the paper */
    float final_factor;  /* 0.1; must be > 0 (R2G_E_INVAL otherwise) */
    int32_t total_iters; /* 30000 */
    float beta1, beta2, eps;
} r2g_adam_opts;

r2g_status r2g_adam_step(int64_t M, float* raw, float* act, float* grad, float* m, float* v, int32_t it,
                         const r2g_adam_opts* opts, r2g_stream stream);

/* ---------------------------------------------------------------- status */

/* Waits for `stream`, then returns the device status of the last call on `ws`
 * (R2G_OK, R2G_E_CAPACITY, R2G_E_TIMEOUT, or -- on a training step's raster
 * workspace -- R2G_E_NUMERIC) and, if needed_keys is not NULL, the number of list
 * entries that call needed.  Clears nothing. */
r2g_status r2g_poll(const void* ws, size_t ws_bytes, r2g_stream stream, int64_t* needed_keys);

/* Bound of the library's device-side waits: the grid barriers of the cooperative
 * list builds (one launch for projection + lists when the whole grid can be
 * resident) give up after `polls` polls (about 20 ns apart) instead of waiting on;
 * the call's workspace status then reads R2G_E_TIMEOUT (r2g_poll), the blocks leave
 * the build, and the kernels that would read its lists (the splat and voxel kernels
 * of that call and of the backward on the same workspace) skip their work, so the
 * outputs of that call are not valid but every kernel ends.  0 restores the default
 * (2^22 polls, about 0.1 s, far beyond any healthy barrier).  Process-wide; applies
 * to launches issued after the call.  Always R2G_OK. */
r2g_status r2g_set_wait_limit(uint64_t polls);

/* ---------------------------------------------------------------- training step
 *
 * One iteration of Eq. 8 for one scan (rasterize one view, L1 + lambda_ssim
 * D-SSIM against its measurement, voxelize one D^3 TV patch, lambda_tv TV, both
 * backward passes, Adam), launched on `stream` with no host synchronisation.  The
 * batch form (r2g_job.views_per_step, n_patches, full_vol) rasterizes every view of
 * the scan in one launch, takes several TV patches and voxelizes the full volume.
 * Every per-iteration choice comes from a DEVICE round entry, read when the
 * kernels run, so a sequence of r2g_train_step calls over many scans can be
 * captured once in a CUDA graph and replayed each round after rewriting the
 * entries.  Workspaces are sized for M Gaussians x 1 view (raster), 1 grid of D^3
 * (voxel), 1 x H x W (loss) and 1 x D (TV); list overflow is reported in the
 * raster/voxel workspace status (r2g_poll).  The TV branch runs on a side stream
 * forked from `stream` and joined back before the gradients are summed; every
 * `stream` gets its own side stream, created by its first call (so make that
 * first call outside stream capture) and kept for the life of the process. */
typedef struct {
    int32_t view;      /* index of the view (and measured projection) this iteration */
    int32_t it;        /* 0-based iteration for the learning-rate schedule and bias correction */
    float origin[3];   /* origin of the TV patch grid */
    int32_t pad[3];
} r2g_round_entry;

typedef struct {
    int64_t M;
    float *raw, *act, *grad, *adam_m, *adam_v;  /* device [11 M]: quat | mean | scale | rho (see r2g_adam_step) */
    int32_t V;                                  /* views in the scan */
    const float* views;                         /* device [V][12] */
    const float* meas;                          /* device [V][H][W] measured log projections */
    r2g_camera cam;
    r2g_raster_opts ropts;
    float Q3;                                   /* voxel gate */
    int32_t D;                                  /* TV patch edge in voxels */
    float voxel;                                /* TV patch voxel size (the output volume's spacing) */
    float lambda_ssim, lambda_tv;
    r2g_adam_opts adam;
    float *image, *dimage;                      /* device [H][W] */
    float *vol, *dvol;                          /* device [D^3] */
    float* loss;                                /* device [2]: projection loss, TV loss */
    void* raster_ws;
    size_t raster_ws_bytes;
    void* voxel_ws;
    size_t voxel_ws_bytes;
    void* loss_ws;
    size_t loss_ws_bytes;
    void* tv_ws;
    size_t tv_ws_bytes;
    /* adaptive-control statistics (optional, device [M] each, or NULL): every step adds,
     * per Gaussian whose projection received a gradient, |dL/dp^| in normalised device
     * coordinates (the pixel-space gradient of its projected mean times (W/2, H/2)) to
     * dens_grad and 1 to dens_count; r2g_densify reads them. */
    float* dens_grad;
    float* dens_count;
    /* TV form of the step: <= 0 the anisotropic TV of r2g_tv3d (the default), > 0 the
     * isotropic TV of r2g_tv3d_iso with this eps */
    float tv_eps;
    /* ---- batch form of the step (all zero / NULL: the one-view, one-patch step above).
     * views_per_step: 0 or 1 = the round entry's view; V = every view of the scan in one
     *   rasterizer launch (entry->view ignored): image and dimage are [V][H][W], the
     *   projection loss is Eq. 8's over the V views (L1 over all their pixels, SSIM
     *   averaged over the views), raster_ws and loss_ws are sized for V views.
     * n_patches: TV patches per step, 0 or 1 = one at entry->origin; 2..64 = patches
     *   whose origins are read from patch_origins (device [n_patches][3]) when the step
     *   runs; vol and dvol hold n_patches D^3 volumes, voxel_ws and tv_ws are sized for
     *   n_patches grids; the TV loss is the sum over the patches.
     * full_vol (optional, device [Z][Y][X] of full_grid): the forward voxelization (Eq. 4)
     *   of full_grid with the step's parameters before its update, on the TV branch,
     *   through its own workspace full_ws of full_ws_bytes (r2g_voxel_workspace_size for
     *   1 grid); it takes no part in the loss. */
    int32_t views_per_step;
    int32_t n_patches;
    const float* patch_origins;
    float* full_vol;
    r2g_grid full_grid;
    void* full_ws;
    size_t full_ws_bytes;
} r2g_job;

/* Numeric guard: when either loss of the step is not finite (a NaN or an infinity in
 * the measured projections, say), the step takes no update -- the parameters, both
 * Adam moments and the adaptive-control statistics stay as they were -- and the raster
 * workspace's status reads R2G_E_NUMERIC (r2g_poll) until the next step on it. */
r2g_status r2g_train_step(const r2g_job* job, const r2g_round_entry* entry, r2g_stream stream);

/* Staging slots of r2g_train_step_host (all caller-owned): n_slots in 1..16.  Vs =
 * the views a step rasterizes (1, or V with job->views_per_step = V), NP = the job's
 * TV patches per step. */
typedef struct {
    int32_t n_slots;
    float* meas;                      /* device [n_slots][Vs][H][W] */
    float* views;                     /* device [n_slots][Vs][12] */
    r2g_round_entry* entries;         /* device [n_slots] */
    r2g_round_entry* entries_host;    /* pinned host [n_slots]; written by the call */
    float* loss;                      /* device [n_slots][2]: the step's losses (instead of job->loss) */
    float* patch_origins;             /* device [n_slots][NP][3] when NP > 1 (else unused) */
} r2g_staging;

/* One training iteration fed from HOST memory: the step's measured projection
 * meas_host[H][W], its geometry row view_host[12] and its round entry (host
 * memory, read during the call; its view field is ignored) are copied into staging slot step % n_slots on a copy stream
 * owned by the library (one per caller stream, created by the first call), the
 * iteration of r2g_train_step runs on `stream` once they have arrived (with the
 * job's view table, measurements and loss buffer replaced by the slot's), and its
 * two losses are copied to loss_host[2] on a second library stream, so that no copy
 * sits between two steps on `stream`.  meas_host, view_host and loss_host should be pinned for
 * the copies to overlap; step counts the caller's calls from 0.  Before rewriting
 * a slot the call BLOCKS until the step that used it last (step - n_slots) has
 * finished, so at most n_slots steps are in flight.  loss_host of a step is valid
 * once r2g_train_step_host_wait(stg, step, stream) has returned; the caller must not
 * reuse it for another step before then.  Not capturable (host waits). */
r2g_status r2g_train_step_host(const r2g_job* job, const r2g_staging* stg, int64_t step, const float* meas_host,
                               const float* view_host, const r2g_round_entry* entry_host, float* loss_host,
                               r2g_stream stream);
/* r2g_train_step_host for the batch form of the step: meas_host [Vs][H][W] and
 * views_host [Vs][12] are the step's measured projections and their geometry rows (Vs
 * = 1, or V when job->views_per_step = V), patch_origins_host [NP][3] the origins of
 * its TV patches when the job has NP = n_patches > 1 (else NULL; the entry's origin
 * is used); all host memory, read during the call.  Everything else as
 * r2g_train_step_host, which is this call with patch_origins_host = NULL. */
r2g_status r2g_train_step_host_batch(const r2g_job* job, const r2g_staging* stg, int64_t step, const float* meas_host,
                                     const float* views_host, const float* patch_origins_host,
                                     const r2g_round_entry* entry_host, float* loss_host, r2g_stream stream);

/* Blocks until step `step` of r2g_train_step_host on `stream` has finished (its
 * loss_host filled); returns at once for a slot that never ran. */
r2g_status r2g_train_step_host_wait(const r2g_staging* stg, int64_t step, r2g_stream stream);

/* Copy n round entries from PAGE-LOCKED host memory `src` to device `dst` on
 * `stream` (an asynchronous copy; inside a captured graph the copy reads `src`
 * each time the graph runs, so the host rewrites it between replays). */
r2g_status r2g_upload_round(r2g_round_entry* dst, const r2g_round_entry* src, int32_t n, r2g_stream stream);

/* ---------------------------------------------------------------- FDK initialisation (Sec. 4.1)
 *
 * The preliminary reconstruction that the Gaussians start from: Feldkamp-Davis-
 * Kress filtered back-projection for a circular orbit and a flat detector (cone
 * beam), or plain filtered back-projection (parallel beam), then M positions drawn
 * among the voxels above a density threshold.  Projections are the log
 * projections of Eq. 1 on the camera's detector, [V][H][W] row-major. */

/* Pre-weighting and ramp filtering of every detector row: filt[v][r][c] =
 * (1 / pitch_u) sum_n c_(c-n) R'[v][r][n], R' = proj * L_SD / sqrt(L_SD^2 + xi^2 +
 * eta^2) (cone; parallel: R' = proj), c_0 = 1/8, c_m = -1/(2 pi^2 m^2) for odd m
 * and 0 for even m != 0 -- the band-limited (Ram-Lak) ramp at the detector
 * spacing with the factor 1/2 of a full-circle scan; the row is zero outside the
 * detector.  proj, filt: device [V][H][W], not aliased.  W <= 8192. */
r2g_status r2g_fdk_filter(int32_t V, const r2g_camera* cam, const float* proj, float* filt, r2g_stream stream);

/* Back-projection of filtered projections onto one grid: vol[z][y][x] (device,
 * written) = dbeta * sum_v w_v F_v(xi, eta) at the voxel centre p, u = W_v p + t_v;
 * cone: (xi, eta) = L_SD (u0, u1) / u2, w_v = t_v[2] L_SD / u2^2 (views with u2 <=
 * near_plane skip the voxel); parallel: (xi, eta) = (u0, u1), w_v = 1.  F_v is
 * read by bilinear interpolation between pixel centres; samples outside the
 * detector count as zero.  dbeta = angular step of the views (2 pi / V for V
 * evenly spaced views on a full circle).  views: device [V][12] as for the
 * rasterizer; filt: device [V][H][W]. */
r2g_status r2g_fdk_backproject(int32_t V, const float* views, const r2g_camera* cam, const float* filt,
                               const r2g_grid* grid, float dbeta, float* vol, r2g_stream stream);

/* Workspace bytes of r2g_init_gaussians for this grid and M (0 for bad arguments). */
size_t r2g_init_workspace_size(const r2g_grid* grid, int64_t M);

/* Sec. 4.1's initialisation from a volume vol[z][y][x] (device) on `grid`:
 * candidates are the voxels with vol > tau (FP32 comparison); candidate j (flat
 * index) gets the key SplitMix64(seed + (j + 1) * 0x9E3779B97F4A7C15) (Steele, Lea
 * & Flood 2014), and the M candidates with the smallest (key, j) are chosen (all
 * of them when there are at most M).  The chosen voxels, in increasing index
 * order, become Gaussians: mean = voxel centre, quat = (1, 0, 0, 0), rho = k *
 * vol, and an isotropic scale = the mean distance to the three nearest other
 * chosen centres (fewer when fewer exist; the smallest voxel edge for a lone one).
 * mean[M][3], scale[M][3], quat[M][4] (16-byte aligned), rho[M]: device, the
 * first *n_out rows written; n_out: device int64 (number chosen).  ws: device,
 * r2g_init_workspace_size bytes.  The grid has fewer than 2^31 voxels. */
r2g_status r2g_init_gaussians(const float* vol, const r2g_grid* grid, float tau, int64_t M, uint64_t seed, float k,
                              float* mean, float* scale, float* quat, float* rho, int64_t* n_out, void* ws,
                              size_t ws_bytes, r2g_stream stream);

/* ---------------------------------------------------------------- adaptive density control (Sec. 4.2.3)
 *
 * Between training steps (Sec. 5.1: every 100 iterations from 500 to 15k), empty
 * Gaussians are removed and those whose projected means received large gradients
 * are cloned or split, the density of the original and of every copy halved. */
typedef struct {
    float grad_threshold;  /* densify where the mean |dL/dp^| (NDC, see r2g_job.dens_grad) >= this (5e-5) */
    float min_density;     /* remove where rho < this; no size-based removal */
    float split_scale;     /* a densified Gaussian whose largest scale exceeds this is split, else cloned */
    float split_factor;    /* a split's two children have scales / split_factor (1.6) */
    uint64_t seed;         /* counter for the children's offsets (see below) */
} r2g_densify_opts;

size_t r2g_densify_workspace_size(void);
/* In: the training state of M Gaussians (device raw, act, m, v in the flat layout
 * [quat 4M | mean 3M | scale 3M | rho M]) and the accumulated statistics dens_grad[M],
 * dens_count[M].  Out: the new state in raw_out, act_out, m_out, v_out (device, each
 * holding 11 * max_gaussians floats, not aliasing the inputs), flat layout with the
 * new count M' = *m_new (device int64): the survivors in index order (Adam moments
 * kept; a clone's original with rho / 2), then the copies in the order of their
 * originals with zero moments -- a clone's copy (rho / 2), a split's two children
 * (means p + R(q)(s * z), scales s / split_factor, rho / 2; the split original is
 * removed).  z: child c of Gaussian i, component k, uses u_j, u_(j+1) with j =
 * ((2 i + c) 3 + k) 2, u_j = ((SplitMix64(seed + (j + 1) 0x9E3779B97F4A7C15) >> 40)
 * + 1/2) / 2^24, z = sqrt(-2 ln u_j) cos(2 pi u_(j+1)) (Box-Muller).  Densify
 * candidates beyond max_gaussians (>= M) are left as they are, in index order.
 * The activated values of the copies are written and the raw ones derived from them
 * (scale: log, rho: inverse softplus). */
r2g_status r2g_densify(int64_t M, const float* raw, const float* act, const float* m, const float* v,
                       const float* dens_grad, const float* dens_count, const r2g_densify_opts* opts,
                       int64_t max_gaussians, float* raw_out, float* act_out, float* m_out, float* v_out,
                       int64_t* m_new, void* ws, size_t ws_bytes, r2g_stream stream);

/* ---------------------------------------------------------------- volume metrics (Sec. 5.1)
 *
 * The scores the paper reports for a reconstruction: PSNR over the whole volume and
 * SSIM averaged over the 2D slices in the axial, coronal and sagittal directions.
 * For vol[Z][Y][X] (z the rotation axis): axial slices are z = const (rows y,
 * columns x), coronal y = const (rows z, columns x), sagittal x = const (rows z,
 * columns y).  Slice SSIM: Wang et al. 2004 with an 11 x 11 Gaussian window (sigma
 * 1.5), zero-padded "same" filtering, C1 = 1e-4, C2 = 9e-4 (data range 1), the mean
 * of the SSIM map over the slice; per orientation the mean over its slices; SSIM =
 * the mean of the three.  PSNR = 10 log10(1 / MSE) (data range 1). */
size_t r2g_metrics_workspace_size(int32_t X, int32_t Y, int32_t Z);
/* vol, ref: device [Z][Y][X]; out: device double[6] = {MSE, PSNR, SSIM, axial,
 * coronal, sagittal}, written; ws: device, 256-byte aligned,
 * r2g_metrics_workspace_size bytes (it holds transposed copies of both volumes).
 * Deterministic (fixed summation order). */
r2g_status r2g_volume_metrics(int32_t X, int32_t Y, int32_t Z, const float* vol, const float* ref, double* out,
                              void* ws, size_t ws_bytes, r2g_stream stream);

/* ---------------------------------------------------------------- measurement
 *
 * Optional timing of the library's own kernels: when enabled, every call records
 * a CUDA event pair on its stream around each hot kernel (or kernel group):
 * 0 project, 1 emit (tile entries: count + emit), 2 sort (tile lists: offsets +
 * scatter, or the radix passes), 3 ranges (radix path only), 4 splat_fwd,
 * 5 splat_bwd, 6 project_bwd, 7 vox_project, 8 vox_fwd, 9 vox_bwd, 10 vox_chain,
 * 11 loss, 12 tv, 13 adam, 14-16 the same three list stages for the brick lists,
 * 17 fdk_filter, 18 fdk_bp, 19 init_select (the selection passes and the writes
 * of r2g_init_gaussians), 20 init_knn, 21 metrics (r2g_volume_metrics), 22 densify.
 * Not for use inside stream capture.
 * max_spans bounds the recorded pairs (events are created once, here). */
r2g_status r2g_profile_enable(int32_t on, int32_t max_spans);
/* Restrict recording to the kernel ids whose bit is set in kernel_mask (bit k =
 * id k; all bits set by default), so that a timed run can bracket only the
 * kernel it reports without event records around every other one. */
r2g_status r2g_profile_select(uint32_t kernel_mask);
r2g_status r2g_profile_reset(void);
/* Launch count and summed device time (ms) of one kernel id since the last reset;
 * waits for the recorded events. */
r2g_status r2g_profile_read(int32_t kernel, int64_t* launches, double* total_ms);
const char* r2g_profile_name(int32_t kernel);
/* Total number of CUDA kernels this library has launched in this process. */
int64_t r2g_launch_count(void);

/* Thread-local description of the last error returned on this thread. */
const char* r2g_last_error(void);

/* Library version string. */
const char* r2g_version(void);

#ifdef __cplusplus
}
#endif
#endif /* R2G_H */
