// FP32 complementary error function shared by the formal-solution and image
// kernels (internal, not part of the C-ABI).
#pragma once

namespace mgt {

// FP32 complementary error function from a fitted scaled form (coefficients
// from fit_erfcx.py, max relative error 3.3e-7 on [0, 9.5] in FP32):
// erfc(|x|) = exp(-x^2) t P(2t - 1), t = 1/(1 + 0.4|x|); erfc(-x) = 2 - erfc(x).
// The coefficients of P, highest degree first:
static __constant__ float kErfcP[11] = {-2.942456576e-05f, -1.129791453e-05f, 2.668800640e-04f, 1.665944132e-04f,
                              -1.921493629e-03f, -3.353950657e-03f, 1.134349779e-02f,  6.849996818e-02f,
                              1.815657182e-01f,  3.218607602e-01f,  4.216127275e-01f};
constexpr float kLog2E = 1.44269504088896341f;   // exp(y) = 2^(y log2 e)

__device__ __forceinline__ float rcp_mufu(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float ex2_mufu(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Every operation explicitly rounded, so that erfc_fit and each lane of
// erfc_fit2 give the same bits in any context.
__device__ __forceinline__ float erfc_fit(float x)
{
    const float ax = fabsf(x);
    const float t = rcp_mufu(fmaf(0.4f, ax, 1.0f));
    const float s = fmaf(2.0f, t, -1.0f);
    float p = kErfcP[0];
#pragma unroll
    for (int i = 1; i < 11; ++i) p = fmaf(p, s, kErfcP[i]);
    const float e = ex2_mufu(__fmul_rn(__fmul_rn(ax, ax), -kLog2E));
    const float r = __fmul_rn(__fmul_rn(t, p), e);
    return x < 0.0f ? __fsub_rn(2.0f, r) : r;
}

// erfc_fit of two independent arguments on packed FP32 (Blackwell's two-lane
// FFMA2 / FMUL2: one issue slot per pair), lane for lane the same arithmetic.
__device__ __forceinline__ float2 erfc_fit2(float x0, float x1)
{
    const float2 ax = make_float2(fabsf(x0), fabsf(x1));
    const float2 u = __ffma2_rn(make_float2(0.4f, 0.4f), ax, make_float2(1.0f, 1.0f));
    const float2 t = make_float2(rcp_mufu(u.x), rcp_mufu(u.y));
    const float2 s = __ffma2_rn(make_float2(2.0f, 2.0f), t, make_float2(-1.0f, -1.0f));
    float2 p = make_float2(kErfcP[0], kErfcP[0]);
#pragma unroll
    for (int i = 1; i < 11; ++i) p = __ffma2_rn(p, s, make_float2(kErfcP[i], kErfcP[i]));
    const float2 y = __fmul2_rn(__fmul2_rn(ax, ax), make_float2(-kLog2E, -kLog2E));
    const float2 e = make_float2(ex2_mufu(y.x), ex2_mufu(y.y));
    const float2 r = __fmul2_rn(__fmul2_rn(t, p), e);
    return make_float2(x0 < 0.0f ? __fsub_rn(2.0f, r.x) : r.x, x1 < 0.0f ? __fsub_rn(2.0f, r.y) : r.y);
}

}  // namespace mgt
