// adam_math.cuh -- the per-parameter Adam arithmetic (Sec. 5.1), shared by the
// standalone fused Adam kernel and the training step's fused chain-rule + Adam
// kernel.  Parameter layout [quat 4M | mean 3M | scale 3M | rho M]; groups index
// the learning rates as mean, scale, quat, rho; activations: scale = exp(raw),
// rho = softplus(raw), mean and quat as is.
#pragma once

#include <math.h>

#include "r2g_internal.cuh"

namespace r2g {

struct AdamArgs {
    long long M;
    float lr[4];        // mean, scale, quat, rho at this iteration
    float b1, b2, eps;
    float bc1, bc2;     // 1 - beta^(it+1)
    // with it_dev: the iteration is read on the device and the schedule formed there
    // as lr0 * 2^(t log2 final_factor) and 1 - 2^((it + 1) log2 beta)
    const int* it_dev;
    float lr0[4], log2_final, log2_b1, log2_b2;
    int total;
};

// Host: the arguments for iteration `it` (or it_dev, read on the device).
inline AdamArgs adam_args(long long M, const r2g_adam_opts* opts, int it, const int* it_dev) {
    AdamArgs a;
    a.M = M;
    const double t = fmin(fmax((double)it / opts->total_iters, 0.0), 1.0);
    for (int g = 0; g < 4; ++g) a.lr[g] = (float)(opts->lr0[g] * pow((double)opts->final_factor, t));
    a.b1 = opts->beta1;
    a.b2 = opts->beta2;
    a.eps = opts->eps;
    a.bc1 = (float)(1.0 - pow((double)opts->beta1, it + 1.0));
    a.bc2 = (float)(1.0 - pow((double)opts->beta2, it + 1.0));
    a.it_dev = it_dev;
    for (int g = 0; g < 4; ++g) a.lr0[g] = opts->lr0[g];
    a.log2_final = (float)log2((double)opts->final_factor);
    a.log2_b1 = (float)log2((double)opts->beta1);
    a.log2_b2 = (float)log2((double)opts->beta2);
    a.total = opts->total_iters;
    return a;
}

// Device: this iteration's learning rates and bias corrections.
__device__ __forceinline__ void adam_schedule(const AdamArgs& a, float lr[4], float& bc1, float& bc2) {
#pragma unroll
    for (int g = 0; g < 4; ++g) lr[g] = a.lr[g];
    bc1 = a.bc1;
    bc2 = a.bc2;
    if (a.it_dev) {
        const int it = __ldg(a.it_dev);
        const float t = fminf(fmaxf((float)it / (float)a.total, 0.0f), 1.0f);
        const float f = exp2f(t * a.log2_final);
#pragma unroll
        for (int g = 0; g < 4; ++g) lr[g] = a.lr0[g] * f;
        bc1 = 1.0f - exp2f((float)(it + 1) * a.log2_b1);
        bc2 = 1.0f - exp2f((float)(it + 1) * a.log2_b2);
    }
}

// Device: one parameter of group grp (0 mean, 1 scale, 2 quat, 3 rho): the
// gradient g with respect to the activated value (act = the current activated
// value) is chained to the raw value r, both moments are updated in place, and
// the new raw value rn and its activation out are returned.
__device__ __forceinline__ void adam_elem(const AdamArgs& a, int grp, float lr, float bc1, float bc2, float r,
                                          float g, float act, float& mk, float& vk, float& rn, float& out) {
    if (grp == 1) g *= act;                          // d exp(r)/dr = exp(r)
    if (grp == 3) g *= 1.0f / (1.0f + expf(-r));     // d softplus(r)/dr = sigmoid(r)
    mk = a.b1 * mk + (1.0f - a.b1) * g;
    vk = a.b2 * vk + (1.0f - a.b2) * g * g;
    rn = r - lr * (mk / bc1) / (sqrtf(vk / bc2) + a.eps);
    out = rn;
    if (grp == 1) out = expf(rn);
    if (grp == 3) out = fmaxf(rn, 0.0f) + log1pf(expf(-fabsf(rn)));
}

// The optimizer state one fused update touches.
struct AdamState {
    float* raw;
    float* act;
    float* m;
    float* v;
    const float* grad;  // gradient already accumulated by other kernels (added to this kernel's own)
    AdamArgs a;
    // adaptive-control statistics (optional): per Gaussian, the sum over its records
    // with a gradient of |dL/dp^| in normalised device coordinates, and their count
    float* dens_grad;
    float* dens_count;
    // numeric guard (optional): when the step's losses loss_guard[0..1] are not both
    // finite, the kernel takes no step at all (parameters, moments and statistics
    // unchanged) and writes R2G_E_NUMERIC into *guard_status
    const float* loss_guard;
    WsStatus* guard_status;
};

// Device: whether the step's losses allow an update (true without a guard).
__device__ __forceinline__ bool adam_loss_ok(const AdamState& st) {
    if (!st.loss_guard) return true;
    return isfinite(st.loss_guard[0]) && isfinite(st.loss_guard[1]);
}

// Device: one parameter at flat index e of group grp with this kernel's own
// gradient contribution g_own (added to st.grad[e]).
__device__ __forceinline__ void adam_param(const AdamState& st, const float lr[4], float bc1, float bc2, int grp,
                                           long long e, float g_own) {
    float mk = st.m[e], vk = st.v[e], rn, out;
    adam_elem(st.a, grp, lr[grp], bc1, bc2, st.raw[e], st.grad[e] + g_own, st.act[e], mk, vk, rn, out);
    st.m[e] = mk;
    st.v[e] = vk;
    st.raw[e] = rn;
    st.act[e] = out;
}

// Device: the Adam step of Gaussian i's eleven parameters, given this kernel's own
// gradient contributions.
__device__ __forceinline__ void adam_gaussian(const AdamState& st, long long i, const float gq[4],
                                              const float gp[3], const float gs[3], float grho) {
    const long long M = st.a.M;
    float lr[4], bc1, bc2;
    adam_schedule(st.a, lr, bc1, bc2);
#pragma unroll
    for (int k = 0; k < 4; ++k) adam_param(st, lr, bc1, bc2, 2, 4 * i + k, gq[k]);
#pragma unroll
    for (int k = 0; k < 3; ++k) adam_param(st, lr, bc1, bc2, 0, 4 * M + 3 * i + k, gp[k]);
#pragma unroll
    for (int k = 0; k < 3; ++k) adam_param(st, lr, bc1, bc2, 1, 7 * M + 3 * i + k, gs[k]);
    adam_param(st, lr, bc1, bc2, 3, 10 * M + i, grho);
}

// The Adam state of one Gaussian's eleven parameters, loaded ahead of the
// arithmetic that produces its gradient (so the loads' latency overlaps it), in
// the order quat (4), mean (3), scale (3), rho.
struct AdamPre {
    float raw[11], m[11], v[11], g[11];
};

__device__ __forceinline__ long long adam_index(long long M, long long i, int e) {
    return e < 4 ? 4 * i + e : (e < 7 ? 4 * M + 3 * i + (e - 4) : (e < 10 ? 7 * M + 3 * i + (e - 7) : 10 * M + i));
}

__device__ __forceinline__ void adam_prefetch_state(const AdamState& st, long long i, AdamPre& p) {
    const long long M = st.a.M;
#pragma unroll
    for (int e = 0; e < 11; ++e) {
        const long long x = adam_index(M, i, e);
        p.raw[e] = st.raw[x];
        p.m[e] = st.m[x];
        p.v[e] = st.v[x];
    }
}
__device__ __forceinline__ void adam_prefetch_grad(const AdamState& st, long long i, AdamPre& p) {
    const long long M = st.a.M;
#pragma unroll
    for (int e = 0; e < 11; ++e) p.g[e] = st.grad[adam_index(M, i, e)];
}

// adam_gaussian with the state prefetched; act: the activated values (the
// Gaussian's parameters as the kernel loaded them), same order.
__device__ __forceinline__ void adam_gaussian_pre(const AdamState& st, long long i, const AdamPre& p,
                                                  const float act[11], const float gq[4], const float gp[3],
                                                  const float gs[3], float grho) {
    const long long M = st.a.M;
    float lr[4], bc1, bc2;
    adam_schedule(st.a, lr, bc1, bc2);
    const float own[11] = {gq[0], gq[1], gq[2], gq[3], gp[0], gp[1], gp[2], gs[0], gs[1], gs[2], grho};
#pragma unroll
    for (int e = 0; e < 11; ++e) {
        const int grp = e < 4 ? 2 : (e < 7 ? 0 : (e < 10 ? 1 : 3));
        float mk = p.m[e], vk = p.v[e], rn, out;
        adam_elem(st.a, grp, lr[grp], bc1, bc2, p.raw[e], p.g[e] + own[e], act[e], mk, vk, rn, out);
        const long long x = adam_index(M, i, e);
        st.m[x] = mk;
        st.v[x] = vk;
        st.raw[x] = rn;
        st.act[x] = out;
    }
}

}  // namespace r2g
