// train.cu -- one training iteration of one scan (Eq. 8, Sec. 4.2) as a single C
// call, with every per-iteration choice read from a device-resident round entry,
// so that a round over many scans can be captured once as a CUDA graph and
// replayed: rasterize the selected view, L1 + D-SSIM against its measurement,
// voxelize the TV patch at the selected origin, TV, both backward passes, Adam.
#include "r2g_internal.cuh"

using namespace r2g;

R2G_API r2g_status r2g_train_step(const r2g_job* job, const r2g_round_entry* entry, r2g_stream stream) {
    if (!job || !entry) return fail(R2G_E_INVAL, "r2g_train_step: NULL job or round entry");
    const r2g_job& J = *job;
    if (J.M < 1 || !J.raw || !J.act || !J.grad || !J.adam_m || !J.adam_v || !J.views || !J.meas || !J.image ||
        !J.dimage || !J.vol || !J.dvol || !J.loss || !J.raster_ws || !J.voxel_ws || !J.loss_ws || !J.tv_ws)
        return fail(R2G_E_INVAL, "r2g_train_step: NULL pointer in the job");
    if (J.D < 2 || !(J.voxel > 0.f)) return fail(R2G_E_INVAL, "r2g_train_step: bad TV patch");
    const int64_t M = J.M;
    // activated parameters [quat 4M | mean 3M | scale 3M | rho M]
    const float* quat = J.act;
    const float* mean = J.act + 4 * M;
    const float* scale = J.act + 7 * M;
    const float* rho = J.act + 10 * M;
    float* dquat = J.grad;
    float* dmean = J.grad + 4 * M;
    float* dscale = J.grad + 7 * M;
    float* drho = J.grad + 10 * M;
    const int* view_sel = &entry->view;
    r2g_grid grid;
    for (int k = 0; k < 3; ++k) {
        grid.origin[k] = 0.f;  // replaced on the device by entry->origin
        grid.voxel[k] = J.voxel;
        grid.dims[k] = J.D;
    }
    r2g_status e;
    if ((e = rasterize_impl(M, mean, scale, quat, rho, 1, J.views, view_sel, &J.cam, &J.ropts, J.image, J.raster_ws,
                            J.raster_ws_bytes, stream)))
        return e;
    if ((e = projection_loss_impl(1, J.cam.H, J.cam.W, J.image, J.meas, view_sel, J.lambda_ssim, J.loss, J.dimage,
                                  J.loss_ws, J.loss_ws_bytes, stream)))
        return e;
    if ((e = voxelize_impl(M, mean, scale, quat, rho, 1, &grid, entry->origin, J.Q3, J.vol, J.voxel_ws,
                           J.voxel_ws_bytes, stream, false)))
        return e;
    if ((e = r2g_tv3d(1, J.D, J.vol, J.lambda_tv, J.loss + 1, J.dvol, J.tv_ws, J.tv_ws_bytes, stream))) return e;
    if ((e = rasterize_backward_impl(M, mean, scale, quat, rho, 1, J.views, view_sel, &J.cam, &J.ropts, J.dimage,
                                     dmean, dscale, dquat, drho, J.raster_ws, J.raster_ws_bytes, stream)))
        return e;
    if ((e = r2g_voxelize_backward(M, mean, scale, quat, rho, 1, &grid, J.Q3, J.dvol, dmean, dscale, dquat, drho,
                                   J.voxel_ws, J.voxel_ws_bytes, stream)))
        return e;
    return adam_impl(M, J.raw, J.act, J.grad, J.adam_m, J.adam_v, 0, &entry->it, &J.adam, stream);
}

R2G_API r2g_status r2g_upload_round(r2g_round_entry* dst, const r2g_round_entry* src, int32_t n, r2g_stream stream) {
    if (!dst || !src || n < 1) return fail(R2G_E_INVAL, "r2g_upload_round: bad arguments");
    if (cudaMemcpyAsync(dst, src, sizeof(r2g_round_entry) * (size_t)n, cudaMemcpyHostToDevice, stream) != cudaSuccess)
        return fail(R2G_E_CUDA, "r2g_upload_round: %s", cudaGetErrorString(cudaGetLastError()));
    return R2G_OK;
}
