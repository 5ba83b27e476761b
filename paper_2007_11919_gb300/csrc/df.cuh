// Double-FP32 arithmetic shared by the kernels (device functions): a value is
// an unevaluated sum hi + lo of two floats, about 48 significant bits, built
// from error-free transformations (Dekker 1971, "A floating-point technique
// for extending the available precision"; Knuth's TwoSum).  It runs on the
// FP32 pipe, which GB300 issues at 64x its FP64 rate.  __fmul_rn / __fadd_rn
// / __fsub_rn keep the compiler from contracting the transformations into FMAs.
#pragma once
#include <cuda_runtime.h>

namespace gbmds {

// sh + sl += (qh + ql) * (vh + vl).
static __device__ __forceinline__ void df_madd(float& sh, float& sl, float qh, float ql, float vh,
                                               float vl) {
    const float p = __fmul_rn(qh, vh);
    float e = fmaf(qh, vh, -p);          // exact rounding error of qh * vh
    e = fmaf(qh, vl, e);
    e = fmaf(ql, vh, e);
    const float s = __fadd_rn(sh, p);    // TwoSum(sh, p) = s + t exactly
    const float z = __fsub_rn(s, sh);
    const float t = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, z)), __fsub_rn(p, z));
    sl = __fadd_rn(sl, __fadd_rn(t, e));
    sh = s;
}

// sh + sl += q * (vh + vl) for an FP32 entry q (the product q * vh is split
// exactly by the FMA; q * vl only needs FP32).
static __device__ __forceinline__ void df_madd1(float& sh, float& sl, float q, float vh, float vl) {
    const float p = __fmul_rn(q, vh);
    float e = fmaf(q, vh, -p);
    e = fmaf(q, vl, e);
    const float s = __fadd_rn(sh, p);
    const float z = __fsub_rn(s, sh);
    const float t = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, z)), __fsub_rn(p, z));
    sl = __fadd_rn(sl, __fadd_rn(t, e));
    sh = s;
}

static __device__ __forceinline__ void df_add(float& sh, float& sl, float oh, float ol) {
    const float s = __fadd_rn(sh, oh);
    const float z = __fsub_rn(s, sh);
    const float t = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, z)), __fsub_rn(oh, z));
    sl = __fadd_rn(sl, __fadd_rn(t, ol));
    sh = s;
}


// Renormalised double-FP32 helpers (values as float2 {hi, lo}).
static __device__ __forceinline__ float2 df_of(double x) {
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
}
static __device__ __forceinline__ float2 df_norm(float sh, float sl) {
    const float h = __fadd_rn(sh, sl);
    return make_float2(h, __fsub_rn(sl, __fsub_rn(h, sh)));
}
// a * s
static __device__ __forceinline__ float2 df_mul(float2 a, float2 s) {
    const float p = __fmul_rn(a.x, s.x);
    float e = fmaf(a.x, s.x, -p);
    e = fmaf(a.x, s.y, e);
    e = fmaf(a.y, s.x, e);
    return df_norm(p, e);
}
// Warp sum of a double-FP32 accumulator (fixed butterfly order).
static __device__ __forceinline__ void df_warp_sum(float& sh, float& sl) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, sh, o);
        const float ol = __shfl_xor_sync(0xffffffffu, sl, o);
        df_add(sh, sl, oh, ol);
    }
}

// x - y, x * y and 1 / x for renormalised double-FP32 values.
static __device__ __forceinline__ float2 df_sub2(float2 x, float2 y) {
    const float s = __fsub_rn(x.x, y.x);
    const float z = __fsub_rn(s, x.x);
    float e = __fadd_rn(__fsub_rn(x.x, __fsub_rn(s, z)), __fsub_rn(-y.x, z));   // TwoSum error
    e = __fadd_rn(e, __fsub_rn(x.y, y.y));
    return df_norm(s, e);
}
static __device__ __forceinline__ float2 df_mul2(float2 x, float2 y) {
    const float p = __fmul_rn(x.x, y.x);
    float e = fmaf(x.x, y.x, -p);
    e = fmaf(x.x, y.y, e);
    e = fmaf(x.y, y.x, e);
    return df_norm(p, e);
}
static __device__ __forceinline__ float2 df_rcp2(float2 x) {
    const float y0 = __frcp_rn(x.x);
    const float2 r = df_sub2(make_float2(1.f, 0.f), df_mul2(x, make_float2(y0, 0.f)));   // 1 - x y0
    return df_norm(y0, __fmul_rn(y0, r.x));                                           // y0 (1 + r)
}
static __device__ __forceinline__ float2 df_scale(float2 x, float s) { return make_float2(x.x * s, x.y * s); }

}  // namespace gbmds
