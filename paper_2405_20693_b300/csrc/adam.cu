// adam.cu -- one fused Adam step over all parameter groups (Sec. 5.1): gradient
// chain rule to the raw parameters, both moment updates, the bias-corrected step
// with the group's exponentially decayed learning rate, the activated copy for
// the next iteration, and clearing of the gradient -- one pass over memory.
#include <math.h>

#include "r2g_internal.cuh"

namespace r2g {
namespace {

struct AdamArgs {
    long long M;
    float lr[4];        // mean, scale, quat, rho at this iteration
    float b1, b2, eps;
    float bc1, bc2;     // 1 - beta^(it+1)
    // with it_dev: the iteration is read on the device and the schedule formed there
    const int* it_dev;
    float lr0[4], final_factor;
    int total;
};

__global__ void __launch_bounds__(256) k_adam(AdamArgs a, float* __restrict__ raw, float* __restrict__ act,
                                              float* __restrict__ grad, float* __restrict__ m,
                                              float* __restrict__ v) {
    const long long n = 11 * a.M;
    if (a.it_dev) {
        const int it = *a.it_dev;
        const float t = fminf(fmaxf((float)it / (float)a.total, 0.0f), 1.0f);
        const float f = powf(a.final_factor, t);
#pragma unroll
        for (int g = 0; g < 4; ++g) a.lr[g] = a.lr0[g] * f;
        a.bc1 = 1.0f - powf(a.b1, (float)(it + 1));
        a.bc2 = 1.0f - powf(a.b2, (float)(it + 1));
    }
    for (long long k = (long long)blockIdx.x * 256 + threadIdx.x; k < n; k += (long long)gridDim.x * 256) {
        // layout: quat [0, 4M), mean [4M, 7M), scale [7M, 10M), rho [10M, 11M)
        // (quat first keeps it 16-byte aligned); grp indexes lr as mean, scale, quat, rho
        const int grp = k < 4 * a.M ? 2 : (k < 7 * a.M ? 0 : (k < 10 * a.M ? 1 : 3));
        const float r = raw[k];
        float g = grad[k];
        if (grp == 1) g *= act[k];                       // d exp(r)/dr = exp(r)
        if (grp == 3) g *= 1.0f / (1.0f + expf(-r));     // d softplus(r)/dr = sigmoid(r)
        const float mk = a.b1 * m[k] + (1.0f - a.b1) * g;
        const float vk = a.b2 * v[k] + (1.0f - a.b2) * g * g;
        m[k] = mk;
        v[k] = vk;
        const float rn = r - a.lr[grp] * (mk / a.bc1) / (sqrtf(vk / a.bc2) + a.eps);
        raw[k] = rn;
        float out = rn;
        if (grp == 1) out = expf(rn);
        if (grp == 3) out = fmaxf(rn, 0.0f) + log1pf(expf(-fabsf(rn)));
        act[k] = out;
        grad[k] = 0.0f;
    }
}

}  // namespace
}  // namespace r2g

using namespace r2g;

r2g_status r2g::adam_impl(int64_t M, float* raw, float* act, float* grad, float* m, float* v, int32_t it,
                          const int* it_dev, const r2g_adam_opts* opts, cudaStream_t stream) {
    if (M < 1 || !raw || !act || !grad || !m || !v || !opts) return fail(R2G_E_INVAL, "bad Adam arguments");
    if (it < 0 || opts->total_iters < 1) return fail(R2G_E_INVAL, "bad iteration counter");
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
    a.final_factor = opts->final_factor;
    a.total = opts->total_iters;
    const long long n = 11 * (long long)M;
    long long blocks = (n + 255) / 256;
    if (blocks > 148 * 16) blocks = 148 * 16;
    prof_begin(P_ADAM, stream);
    k_adam<<<(unsigned)blocks, 256, 0, stream>>>(a, raw, act, grad, m, v);
    prof_end(P_ADAM, stream);
    note_launches(1);
    return check_launch("r2g_adam_step");
}

R2G_API r2g_status r2g_adam_step(int64_t M, float* raw, float* act, float* grad, float* m, float* v, int32_t it,
                                 const r2g_adam_opts* opts, r2g_stream stream) {
    return adam_impl(M, raw, act, grad, m, v, it, nullptr, opts, stream);
}
