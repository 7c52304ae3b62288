// Double-word arithmetic for the FP64-grade kernels (pd_step_dw.cu,
// pd_adjoint_dw.cu), device code only.
//
// A double-word is an unevaluated sum h + l of two FP32 numbers (Dekker 1971;
// Knuth's two-sum; the products and error bounds of Joldes, Muller & Popescu,
// ACM TOMS 2017), about 48 significant bits.  The operations below leave their
// result unnormalised (|l| up to a few ulp(h)) wherever the next operation
// takes that, which keeps ~46-bit accuracy for far fewer FP32 operations than
// renormalising after each step.  GB300's FP32 pipe is the limit of these
// kernels, so the code is scalar: negated operands cost nothing.
#pragma once

#include <cuda_runtime.h>

namespace pd {
namespace dwa {

__device__ __forceinline__ void ld_rec(const float4* p, float4& a, float4& b)
{
    asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z),
                   "=f"(b.w)
                 : "l"(p));
}

__device__ __forceinline__ void st_rec(float4* p, const float4& a, const float4& b)
{
    asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(a.x),
                 "f"(a.y), "f"(a.z), "f"(a.w), "f"(b.x), "f"(b.y), "f"(b.z), "f"(b.w)
                 : "memory");
}

// hardware approximations, used only as seeds that are refined below
__device__ __forceinline__ float rsqrt_seed(float x)
{
    float r;
    asm("rsqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_seed(float x)
{
    float r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

struct Dw {
    float h, l;
};

// exact sum (Knuth)
__device__ __forceinline__ Dw two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}

// a + b: the leading words summed exactly, everything else in FP32
__device__ __forceinline__ Dw dw_add(Dw a, Dw b)
{
    Dw t = two_sum(a.h, b.h);
    t.l += a.l + b.l;
    return t;
}

// a * b: the exact product of the leading words plus the cross terms
// (Joldes, Muller & Popescu's DWTimesDW without the final renormalisation)
__device__ __forceinline__ Dw dw_mul(Dw a, Dw b)
{
    const float p = a.h * b.h;
    return {p, fmaf(a.h, b.l, fmaf(a.l, b.h, fmaf(a.h, b.h, -p)))};
}

// |y| and 1/|y| from |y|^2: an FP32 reciprocal-square-root seed refined once
// by Newton's iteration, then both corrected to double-word accuracy from
// their residuals
__device__ __forceinline__ void dw_norm(Dw y2, Dw& r, Dw& ir)
{
    float r0 = rsqrt_seed(y2.h);
    r0 = r0 * fmaf(-(0.5f * y2.h) * r0, r0, 1.5f);
    const float rh = y2.h * r0;
    r = Dw{rh, (fmaf(-rh, rh, y2.h) + y2.l) * r0 * 0.5f};
    ir = Dw{r0, r0 * fmaf(-r.l, r0, fmaf(-r.h, r0, 1.0f))};
}

// num / den: an FP32 quotient from a refined reciprocal seed, plus the
// remainder's quotient
__device__ __forceinline__ Dw dw_div(Dw num, Dw den)
{
    float q = rcp_seed(den.h);
    q = fmaf(q, fmaf(-den.h, q, 1.0f), q);
    const float q0 = num.h * q;
    const float ph = den.h * q0;
    const float pl = fmaf(den.l, q0, fmaf(den.h, q0, -ph));
    return Dw{q0, (((num.h - ph) - pl) + num.l) * q};
}

// 1/a: an FP32 reciprocal seed refined once, corrected from the residual
__device__ __forceinline__ Dw dw_rcp(Dw a)
{
    float q = rcp_seed(a.h);
    q = fmaf(q, fmaf(-a.h, q, 1.0f), q);
    return Dw{q, q * fmaf(-a.l, q, fmaf(-a.h, q, 1.0f))};
}

// The lane's own record (double-word position and displacement).
struct OwnDw {
    float xh[3], xl[3], uh[3], ul[3];
};

// One neighbour's record as the two 256-bit loads deliver it.
struct Rec {
    float4 a0, a1, b0, b1;
};

__device__ __forceinline__ OwnDw own_of(const Rec& r)
{
    OwnDw o;
    o.xh[0] = r.a0.x; o.xh[1] = r.a0.y; o.xh[2] = r.a0.z;
    o.uh[0] = r.a0.w; o.uh[1] = r.a1.x; o.uh[2] = r.a1.y;
    o.xl[0] = r.b0.x; o.xl[1] = r.b0.y; o.xl[2] = r.b0.z;
    o.ul[0] = r.b0.w; o.ul[1] = r.b1.x; o.ul[2] = r.b1.y;
    return o;
}

}  // namespace dwa
}  // namespace pd
