// adam.cu -- one fused Adam step over all parameter groups (Sec. 5.1): gradient
// chain rule to the raw parameters, both moment updates, the bias-corrected step
// with the group's exponentially decayed learning rate, the activated copy for
// the next iteration, and clearing of the gradient -- one pass over memory.
#include <math.h>

#include "adam_math.cuh"
#include "r2g_internal.cuh"

namespace r2g {
namespace {

// Element k of the flat layout: its group, then the shared update.
__device__ __forceinline__ void adam_at(const AdamArgs& a, const float lr[4], float bc1, float bc2, long long k,
                                        float r, float g, float ac, float& mk, float& vk, float& rn, float& out) {
    const int grp = k < 4 * a.M ? 2 : (k < 7 * a.M ? 0 : (k < 10 * a.M ? 1 : 3));
    adam_elem(a, grp, lr[grp], bc1, bc2, r, g, ac, mk, vk, rn, out);
}

// VEC: all five arrays are 16-byte aligned and each thread takes groups of four
// consecutive elements with vector loads and stores (the < 4 trailing elements
// go one by one).
template <bool VEC>
__global__ void __launch_bounds__(256) k_adam(AdamArgs a, float* __restrict__ raw, float* __restrict__ act,
                                              float* __restrict__ grad, float* __restrict__ m,
                                              float* __restrict__ v) {
    const long long n = 11 * a.M;
    float lr[4], bc1, bc2;
    adam_schedule(a, lr, bc1, bc2);
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
            adam_at(a, lr, bc1, bc2, 4 * q + 0, r.x, g.x, ac.x, mm.x, vv.x, rn.x, out.x);
            adam_at(a, lr, bc1, bc2, 4 * q + 1, r.y, g.y, ac.y, mm.y, vv.y, rn.y, out.y);
            adam_at(a, lr, bc1, bc2, 4 * q + 2, r.z, g.z, ac.z, mm.z, vv.z, rn.z, out.z);
            adam_at(a, lr, bc1, bc2, 4 * q + 3, r.w, g.w, ac.w, mm.w, vv.w, rn.w, out.w);
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
        adam_at(a, lr, bc1, bc2, k, raw[k], grad[k], act[k], mk, vk, rn, out);
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
    const AdamArgs a = adam_args(M, opts, it, it_dev);
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
