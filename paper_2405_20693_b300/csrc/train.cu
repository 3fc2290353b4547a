// train.cu -- one training iteration of one scan (Eq. 8, Sec. 4.2) as a single C
// call, with every per-iteration choice read from a device-resident round entry,
// so that a round over many scans can be captured once as a CUDA graph and
// replayed: rasterize the selected view, L1 + D-SSIM against its measurement,
// voxelize the TV patch at the selected origin, TV, both backward passes, Adam.
// The batch form of the same call rasterizes every view of the scan in one launch
// (the loss over all of them), takes several TV patches whose origins are read on
// the device, and can voxelize the full output volume alongside (forward only).
//
// The projection branch (rasterize, loss, raster moments) and the TV branch
// (voxelize, TV, voxel moments and chain rule) share nothing until the gradients
// are summed, so the TV branch runs on a side stream forked from the caller's
// stream; it writes its gradient (assigning, so nothing needs clearing) and is
// joined before the raster chain rule, which adds its own gradient in registers
// and takes the Adam step of each Gaussian in the same kernel.  The two
// branches' latency-bound kernels overlap.  Each caller stream gets its own side
// stream and event pair (created on first use, kept for the process), so calls
// on different streams -- the branches of a batched round -- stay independent.
#include <map>
#include <mutex>
#include <utility>

#include "adam_math.cuh"
#include "r2g_internal.cuh"

using namespace r2g;

namespace {

struct SideStream {
    cudaStream_t s;
    cudaEvent_t fork, join;
};

std::mutex g_side_mu;
std::map<std::pair<int, cudaStream_t>, SideStream> g_side;

// Copy stream and per-slot events of r2g_train_step_host, per (device, caller stream).
constexpr int kMaxSlots = 16;
// `in` carries the host -> device copies, `out` the loss read-back (kept off the
// caller's stream, where a copy between two steps would hold the next step back).
struct HostStage {
    cudaStream_t in_s, out_s;
    cudaEvent_t in[kMaxSlots], step[kMaxSlots], done[kMaxSlots];
};

std::map<std::pair<int, cudaStream_t>, HostStage> g_stage;

r2g_status host_stage_for(cudaStream_t caller, HostStage** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(R2G_E_CUDA, "r2g_train_step_host: no current device");
    std::lock_guard<std::mutex> lk(g_side_mu);
    const auto key = std::make_pair(dev, caller);
    auto it = g_stage.find(key);
    if (it == g_stage.end()) {
        HostStage hs{};
        bool ok = cudaStreamCreateWithFlags(&hs.in_s, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&hs.out_s, cudaStreamNonBlocking) == cudaSuccess;
        for (int k = 0; ok && k < kMaxSlots; ++k)
            ok = cudaEventCreateWithFlags(&hs.in[k], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&hs.step[k], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&hs.done[k], cudaEventDisableTiming) == cudaSuccess;
        if (!ok)
            return fail(R2G_E_CUDA, "r2g_train_step_host: creating the copy stream failed (%s)",
                        cudaGetErrorString(cudaGetLastError()));
        it = g_stage.emplace(key, hs).first;
    }
    *out = &it->second;
    return R2G_OK;
}

r2g_status side_stream_for(cudaStream_t caller, SideStream** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(R2G_E_CUDA, "r2g_train_step: no current device");
    std::lock_guard<std::mutex> lk(g_side_mu);
    const auto key = std::make_pair(dev, caller);
    auto it = g_side.find(key);
    if (it == g_side.end()) {
        SideStream sd{};
        if (cudaStreamCreateWithFlags(&sd.s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sd.fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&sd.join, cudaEventDisableTiming) != cudaSuccess)
            return fail(R2G_E_CUDA, "r2g_train_step: creating the side stream failed (%s)",
                        cudaGetErrorString(cudaGetLastError()));
        it = g_side.emplace(key, sd).first;
    }
    *out = &it->second;
    return R2G_OK;
}

}  // namespace

R2G_API r2g_status r2g_train_step(const r2g_job* job, const r2g_round_entry* entry, r2g_stream stream) {
    if (!job || !entry) return fail(R2G_E_INVAL, "r2g_train_step: NULL job or round entry");
    const r2g_job& J = *job;
    if (J.M < 1 || !J.raw || !J.act || !J.grad || !J.adam_m || !J.adam_v || !J.views || !J.meas || !J.image ||
        !J.dimage || !J.vol || !J.dvol || !J.loss || !J.raster_ws || !J.voxel_ws || !J.loss_ws || !J.tv_ws)
        return fail(R2G_E_INVAL, "r2g_train_step: NULL pointer in the job");
    if (J.D < 2 || !(J.voxel > 0.f)) return fail(R2G_E_INVAL, "r2g_train_step: bad TV patch");
    // batch form: every view per step, several TV patches, the full volume
    if (J.views_per_step < 0 || (J.views_per_step > 1 && J.views_per_step != J.V))
        return fail(R2G_E_INVAL, "r2g_train_step: views_per_step %d must be 0, 1 or V = %d", J.views_per_step, J.V);
    const int Vs = J.views_per_step > 1 ? J.V : 1;
    const int NP = J.n_patches > 1 ? J.n_patches : 1;
    if (J.n_patches < 0 || NP > 64) return fail(R2G_E_INVAL, "r2g_train_step: n_patches %d out of range", J.n_patches);
    if (NP > 1 && !J.patch_origins) return fail(R2G_E_INVAL, "r2g_train_step: n_patches > 1 needs patch_origins");
    if (J.full_vol && !J.full_ws) return fail(R2G_E_INVAL, "r2g_train_step: full_vol needs full_ws");
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
    // one view picked by the entry (on the device), or all V views in order
    const int* view_sel = Vs == 1 ? &entry->view : nullptr;
    const float* origin_dev = NP > 1 ? J.patch_origins : entry->origin;
    r2g_grid grids[64];
    for (int g = 0; g < NP; ++g)
        for (int k = 0; k < 3; ++k) {
            grids[g].origin[k] = 0.f;  // replaced on the device by the patch origins
            grids[g].voxel[k] = J.voxel;
            grids[g].dims[k] = J.D;
        }
    SideStream* side = nullptr;
    r2g_status e = side_stream_for(stream, &side);
    if (e) return e;
    const cudaStream_t tv = side->s;
    // fork: the TV branch starts after everything already queued on the caller's
    // stream (the previous iteration's Adam step)
    if (cudaEventRecord(side->fork, stream) != cudaSuccess || cudaStreamWaitEvent(tv, side->fork, 0) != cudaSuccess)
        return fail(R2G_E_CUDA, "r2g_train_step: fork failed (%s)", cudaGetErrorString(cudaGetLastError()));
    r2g_status e_tv = voxelize_impl(M, mean, scale, quat, rho, NP, grids, origin_dev, J.Q3, J.vol, J.voxel_ws,
                                    J.voxel_ws_bytes, tv, false, J.ropts.separate_lists != 0);
    if (!e_tv)
        e_tv = J.tv_eps > 0.f
                   ? r2g_tv3d_iso(NP, J.D, J.vol, J.lambda_tv, J.tv_eps, J.loss + 1, J.dvol, J.tv_ws, J.tv_ws_bytes, tv)
                   : r2g_tv3d(NP, J.D, J.vol, J.lambda_tv, J.loss + 1, J.dvol, J.tv_ws, J.tv_ws_bytes, tv);
    if (!e_tv)
        e_tv = voxelize_backward_impl(M, mean, scale, quat, rho, NP, grids, J.Q3, J.dvol, dmean, dscale, dquat, drho,
                                      J.voxel_ws, J.voxel_ws_bytes, tv,
                                      kVoxBwdMoments | kVoxBwdChain | kVoxBwdAssign);
    // the full volume: forward only, with the parameters this step started from
    if (!e_tv && J.full_vol)
        e_tv = voxelize_impl(M, mean, scale, quat, rho, 1, &J.full_grid, nullptr, J.Q3, J.full_vol, J.full_ws,
                             J.full_ws_bytes, tv, false, J.ropts.separate_lists != 0);
    // the loss's arrival counter is cleared first, so that no copy sits between the
    // rasterizer and the loss kernel (which then takes a programmatic dependent launch)
    r2g_status e_px = projection_loss_clear(Vs, J.cam.H, J.cam.W, J.loss_ws, J.loss_ws_bytes, stream);
    if (!e_px)
        e_px = rasterize_impl(M, mean, scale, quat, rho, Vs, J.views, view_sel, &J.cam, &J.ropts, J.image,
                              J.raster_ws, J.raster_ws_bytes, stream);
    if (!e_px)
        e_px = projection_loss_impl(Vs, J.cam.H, J.cam.W, J.image, J.meas, view_sel, J.lambda_ssim, J.loss, J.dimage,
                                    J.loss_ws, J.loss_ws_bytes, stream, false);
    // a view-chunked rasterizer rebuilds each chunk's lists in its backward and takes
    // the moments and the chain rule together, after the join
    const bool chunked = J.ropts.view_chunk > 0 && J.ropts.view_chunk < Vs;
    if (!e_px && !chunked)
        e_px = rasterize_backward_impl(M, mean, scale, quat, rho, Vs, J.views, view_sel, &J.cam, &J.ropts, J.dimage,
                                       dmean, dscale, dquat, drho, J.raster_ws, J.raster_ws_bytes, stream,
                                       kRasterBwdMoments);
    // join (also on error, so that no captured branch is left open)
    if (cudaEventRecord(side->join, tv) != cudaSuccess || cudaStreamWaitEvent(stream, side->join, 0) != cudaSuccess)
        return fail(R2G_E_CUDA, "r2g_train_step: join failed (%s)", cudaGetErrorString(cudaGetLastError()));
    if (e_tv) return e_tv;
    if (e_px) return e_px;
    if (J.adam.total_iters < 1 || !(J.adam.final_factor > 0.f))
        return fail(R2G_E_INVAL, "r2g_train_step: bad Adam options");
    // the update is skipped (and R2G_E_NUMERIC reported in the raster workspace's
    // status) when the step's loss is not finite, so one bad step cannot poison the state
    const AdamState adam{J.raw,       J.act,        J.adam_m, J.adam_v, J.grad, adam_args(M, &J.adam, 0, &entry->it),
                         J.dens_grad, J.dens_count, J.loss,   reinterpret_cast<WsStatus*>(J.raster_ws)};
    return rasterize_backward_impl(M, mean, scale, quat, rho, Vs, J.views, view_sel, &J.cam, &J.ropts, J.dimage,
                                   dmean, dscale, dquat, drho, J.raster_ws, J.raster_ws_bytes, stream,
                                   chunked ? (kRasterBwdMoments | kRasterBwdChain) : kRasterBwdChain, &adam);
}

R2G_API r2g_status r2g_train_step_host_batch(const r2g_job* job, const r2g_staging* stg, int64_t step,
                                             const float* meas_host, const float* views_host,
                                             const float* patch_origins_host, const r2g_round_entry* entry_host,
                                             float* loss_host, r2g_stream stream) {
    if (!job || !stg || !meas_host || !views_host || !entry_host || !loss_host)
        return fail(R2G_E_INVAL, "r2g_train_step_host: NULL argument");
    if (stg->n_slots < 1 || stg->n_slots > kMaxSlots || !stg->meas || !stg->views || !stg->entries ||
        !stg->entries_host || !stg->loss || step < 0)
        return fail(R2G_E_INVAL, "r2g_train_step_host: bad staging (n_slots %d, step %lld)", stg->n_slots,
                    (long long)step);
    if (job->cam.H < 1 || job->cam.W < 1 || !job->loss) return fail(R2G_E_INVAL, "r2g_train_step_host: bad job");
    const int Vs = job->views_per_step > 1 ? job->V : 1;
    const int NP = job->n_patches > 1 ? job->n_patches : 1;
    if (NP > 1 && (!patch_origins_host || !stg->patch_origins))
        return fail(R2G_E_INVAL, "r2g_train_step_host: the job's %d TV patches need their origins", NP);
    HostStage* hs = nullptr;
    r2g_status e = host_stage_for(stream, &hs);
    if (e) return e;
    const int slot = (int)(step % stg->n_slots);
    const size_t img = (size_t)Vs * (size_t)job->cam.H * (size_t)job->cam.W;
    // the step that used this slot last (step - n_slots) must be done, its losses
    // read back, before the slot's pinned entry, device inputs and losses are
    // rewritten (no wait if it never ran)
    if (cudaEventSynchronize(hs->done[slot]) != cudaSuccess)
        return fail(R2G_E_CUDA, "r2g_train_step_host: waiting for slot %d (%s)", slot,
                    cudaGetErrorString(cudaGetLastError()));
    stg->entries_host[slot] = *entry_host;
    stg->entries_host[slot].view = Vs == 1 ? slot : 0;  // the slot holds the step's views and measurements
    float* pdev = NP > 1 ? stg->patch_origins + (size_t)slot * 3 * NP : nullptr;
    if (cudaMemcpyAsync(stg->meas + slot * img, meas_host, img * sizeof(float), cudaMemcpyHostToDevice, hs->in_s) !=
            cudaSuccess ||
        cudaMemcpyAsync(stg->views + 12 * (size_t)Vs * slot, views_host, 12 * sizeof(float) * Vs,
                        cudaMemcpyHostToDevice, hs->in_s) != cudaSuccess ||
        (pdev && cudaMemcpyAsync(pdev, patch_origins_host, 3 * sizeof(float) * NP, cudaMemcpyHostToDevice,
                                 hs->in_s) != cudaSuccess) ||
        cudaMemcpyAsync(stg->entries + slot, stg->entries_host + slot, sizeof(r2g_round_entry),
                        cudaMemcpyHostToDevice, hs->in_s) != cudaSuccess ||
        cudaEventRecord(hs->in[slot], hs->in_s) != cudaSuccess || cudaStreamWaitEvent(stream, hs->in[slot], 0) != cudaSuccess)
        return fail(R2G_E_CUDA, "r2g_train_step_host: staging copy failed (%s)", cudaGetErrorString(cudaGetLastError()));
    r2g_job J = *job;
    if (Vs == 1) {
        J.V = stg->n_slots;  // the slots' views, picked by the entry
        J.views = stg->views;
        J.meas = stg->meas;
    } else {
        J.views = stg->views + 12 * (size_t)Vs * slot;
        J.meas = stg->meas + slot * img;
    }
    if (pdev) J.patch_origins = pdev;
    J.loss = stg->loss + 2 * (size_t)slot;
    e = r2g_train_step(&J, stg->entries + slot, stream);
    if (e) return e;
    if (cudaEventRecord(hs->step[slot], stream) != cudaSuccess ||
        cudaStreamWaitEvent(hs->out_s, hs->step[slot], 0) != cudaSuccess ||
        cudaMemcpyAsync(loss_host, J.loss, 2 * sizeof(float), cudaMemcpyDeviceToHost, hs->out_s) != cudaSuccess ||
        cudaEventRecord(hs->done[slot], hs->out_s) != cudaSuccess)
        return fail(R2G_E_CUDA, "r2g_train_step_host: loss read-back failed (%s)",
                    cudaGetErrorString(cudaGetLastError()));
    return R2G_OK;
}

R2G_API r2g_status r2g_train_step_host(const r2g_job* job, const r2g_staging* stg, int64_t step,
                                       const float* meas_host, const float* view_host,
                                       const r2g_round_entry* entry_host, float* loss_host, r2g_stream stream) {
    return r2g_train_step_host_batch(job, stg, step, meas_host, view_host, nullptr, entry_host, loss_host, stream);
}

R2G_API r2g_status r2g_train_step_host_wait(const r2g_staging* stg, int64_t step, r2g_stream stream) {
    if (!stg || stg->n_slots < 1 || stg->n_slots > kMaxSlots || step < 0)
        return fail(R2G_E_INVAL, "r2g_train_step_host_wait: bad arguments");
    HostStage* hs = nullptr;
    r2g_status e = host_stage_for(stream, &hs);
    if (e) return e;
    if (cudaEventSynchronize(hs->done[step % stg->n_slots]) != cudaSuccess)
        return fail(R2G_E_CUDA, "r2g_train_step_host_wait: %s", cudaGetErrorString(cudaGetLastError()));
    return R2G_OK;
}

R2G_API r2g_status r2g_upload_round(r2g_round_entry* dst, const r2g_round_entry* src, int32_t n, r2g_stream stream) {
    if (!dst || !src || n < 1) return fail(R2G_E_INVAL, "r2g_upload_round: bad arguments");
    if (cudaMemcpyAsync(dst, src, sizeof(r2g_round_entry) * (size_t)n, cudaMemcpyHostToDevice, stream) != cudaSuccess)
        return fail(R2G_E_CUDA, "r2g_upload_round: %s", cudaGetErrorString(cudaGetLastError()));
    return R2G_OK;
}
