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
    // as lr0 * 2^(t log2 final_factor) and 1 - 2^((it + 1) log2 beta)
    const int* it_dev;
    float lr0[4], log2_final, log2_b1, log2_b2;
    int total;
};

__device__ __forceinline__ void adam_one(const AdamArgs& a, const float lr[4], float bc1, float bc2, long long k,
                                         float r, float g, float ac, float& mk, float& vk, float& rn, float& out) {
    // layout: quat [0, 4M), mean [4M, 7M), scale [7M, 10M), rho [10M, 11M)
    // (quat first keeps it 16-byte aligned); grp indexes lr as mean, scale, quat, rho
    const int grp = k < 4 * a.M ? 2 : (k < 7 * a.M ? 0 : (k < 10 * a.M ? 1 : 3));
    if (grp == 1) g *= ac;                          // d exp(r)/dr = exp(r)
    if (grp == 3) g *= 1.0f / (1.0f + expf(-r));    // d softplus(r)/dr = sigmoid(r)
    mk = a.b1 * mk + (1.0f - a.b1) * g;
    vk = a.b2 * vk + (1.0f - a.b2) * g * g;
    rn = r - lr[grp] * (mk / bc1) / (sqrtf(vk / bc2) + a.eps);
    out = rn;
    if (grp == 1) out = expf(rn);
    if (grp == 3) out = fmaxf(rn, 0.0f) + log1pf(expf(-fabsf(rn)));
}

// VEC: all five arrays are 16-byte aligned and each thread takes groups of four
// consecutive elements with vector loads and stores (the < 4 trailing elements
// go one by one).
template <bool VEC>
__global__ void __launch_bounds__(256) k_adam(AdamArgs a, float* __restrict__ raw, float* __restrict__ act,
                                              float* __restrict__ grad, float* __restrict__ m,
                                              float* __restrict__ v) {
    const long long n = 11 * a.M;
    float lr[4] = {a.lr[0], a.lr[1], a.lr[2], a.lr[3]};
    float bc1 = a.bc1, bc2 = a.bc2;
    if (a.it_dev) {
        const int it = __ldg(a.it_dev);
        const float t = fminf(fmaxf((float)it / (float)a.total, 0.0f), 1.0f);
        const float f = exp2f(t * a.log2_final);
#pragma unroll
        for (int g = 0; g < 4; ++g) lr[g] = a.lr0[g] * f;
        bc1 = 1.0f - exp2f((float)(it + 1) * a.log2_b1);
        bc2 = 1.0f - exp2f((float)(it + 1) * a.log2_b2);
    }
    const long long stride = (long long)gridDim.x * 256;
    long long k0 = 0;
    if (VEC) {
        const long long n4 = n / 4;
        for (long long q = (long long)blockIdx.x * 256 + threadIdx.x; q < n4; q += stride) {
            const float4 r = reinterpret_cast<const float4*>(raw)[q];
            const float4 g = reinterpret_cast<const float4*>(grad)[q];
            const float4 ac = reinterpret_cast<const float4*>(act)[q];
            float4 mm = reinterpret_cast<const float4*>(m)[q];
            float4 vv = reinterpret_cast<const float4*>(v)[q];
            float4 rn, out;
            adam_one(a, lr, bc1, bc2, 4 * q + 0, r.x, g.x, ac.x, mm.x, vv.x, rn.x, out.x);
            adam_one(a, lr, bc1, bc2, 4 * q + 1, r.y, g.y, ac.y, mm.y, vv.y, rn.y, out.y);
            adam_one(a, lr, bc1, bc2, 4 * q + 2, r.z, g.z, ac.z, mm.z, vv.z, rn.z, out.z);
            adam_one(a, lr, bc1, bc2, 4 * q + 3, r.w, g.w, ac.w, mm.w, vv.w, rn.w, out.w);
            reinterpret_cast<float4*>(m)[q] = mm;
            reinterpret_cast<float4*>(v)[q] = vv;
            reinterpret_cast<float4*>(raw)[q] = rn;
            reinterpret_cast<float4*>(act)[q] = out;
            reinterpret_cast<float4*>(grad)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        k0 = 4 * n4;
    }
    for (long long k = k0 + (long long)blockIdx.x * 256 + threadIdx.x; k < n; k += stride) {
        float mk = m[k], vk = v[k], rn, out;
        adam_one(a, lr, bc1, bc2, k, raw[k], grad[k], act[k], mk, vk, rn, out);
        m[k] = mk;
        v[k] = vk;
        raw[k] = rn;
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
    if (!(opts->final_factor > 0.f)) return fail(R2G_E_INVAL, "final_factor must be > 0");
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
    const long long n = 11 * (long long)M;
    const bool vec = ((reinterpret_cast<uintptr_t>(raw) | reinterpret_cast<uintptr_t>(act) |
                       reinterpret_cast<uintptr_t>(grad) | reinterpret_cast<uintptr_t>(m) |
                       reinterpret_cast<uintptr_t>(v)) & 15) == 0;
    long long blocks = ((vec ? n / 4 : n) + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 148 * 16) blocks = 148 * 16;
    prof_begin(P_ADAM, stream);
    if (vec)
        k_adam<true><<<(unsigned)blocks, 256, 0, stream>>>(a, raw, act, grad, m, v);
    else
        k_adam<false><<<(unsigned)blocks, 256, 0, stream>>>(a, raw, act, grad, m, v);
    prof_end(P_ADAM, stream);
    note_launches(1);
    return check_launch("r2g_adam_step");
}

R2G_API r2g_status r2g_adam_step(int64_t M, float* raw, float* act, float* grad, float* m, float* v, int32_t it,
                                 const r2g_adam_opts* opts, r2g_stream stream) {
    return adam_impl(M, raw, act, grad, m, v, it, nullptr, opts, stream);
}
