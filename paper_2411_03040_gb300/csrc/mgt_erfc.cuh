// FP32 complementary error function shared by the formal-solution and image
// kernels (internal, not part of the C-ABI).
#pragma once

namespace mgt {

// FP32 complementary error function from a fitted scaled form (coefficients
// from fit_erfcx.py, max relative error 3.3e-7 on [0, 9.5] in FP32):
// erfc(|x|) = exp(-x^2) t P(2t - 1), t = 1/(1 + 0.4|x|); erfc(-x) = 2 - erfc(x).
__device__ __forceinline__ float erfc_fit(float x)
{
    const float ax = fabsf(x);
    float t;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(fmaf(0.4f, ax, 1.0f)));
    const float s = fmaf(2.0f, t, -1.0f);
    float p = -2.942456576e-05f;
    p = fmaf(p, s, -1.129791453e-05f);
    p = fmaf(p, s, 2.668800640e-04f);
    p = fmaf(p, s, 1.665944132e-04f);
    p = fmaf(p, s, -1.921493629e-03f);
    p = fmaf(p, s, -3.353950657e-03f);
    p = fmaf(p, s, 1.134349779e-02f);
    p = fmaf(p, s, 6.849996818e-02f);
    p = fmaf(p, s, 1.815657182e-01f);
    p = fmaf(p, s, 3.218607602e-01f);
    p = fmaf(p, s, 4.216127275e-01f);
    // explicit roundings: no context may contract these into its own FMAs
    const float r = __fmul_rn(__fmul_rn(t, p), __expf(-__fmul_rn(ax, ax)));
    return x < 0.0f ? __fsub_rn(2.0f, r) : r;
}

}  // namespace mgt
