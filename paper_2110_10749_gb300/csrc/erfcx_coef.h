// Generated by gen_erfcx.py: erfcx(rho) ~ sum_k kErfcx[k] w^k on [0.5, 5.5], with
// w = kErfcxA / (1 + rho) - kErfcxB.  Do not edit.
#pragma once
#define SSD_ERFCX_DEG 7
static constexpr float kErfcxA = 3.900000000e+00f;
static constexpr float kErfcxB = 1.600000000e+00f;
static constexpr float kErfcx0 = 3.321175619e-01f;
static constexpr float kErfcx1 = 2.643791630e-01f;
static constexpr float kErfcx2 = 2.658716093e-02f;
static constexpr float kErfcx3 = -7.505408731e-03f;
static constexpr float kErfcx4 = -2.841155446e-04f;
static constexpr float kErfcx5 = 5.038700072e-04f;
static constexpr float kErfcx6 = -1.169991738e-04f;
static constexpr float kErfcx7 = 9.110261344e-06f;
// Horner evaluation for a packed pair of arguments
static __device__ __forceinline__ float2 erfcx_fit2(float2 w) {
    float2 p = make_float2(kErfcx7, kErfcx7);
    p = __ffma2_rn(p, w, make_float2(kErfcx6, kErfcx6));
    p = __ffma2_rn(p, w, make_float2(kErfcx5, kErfcx5));
    p = __ffma2_rn(p, w, make_float2(kErfcx4, kErfcx4));
    p = __ffma2_rn(p, w, make_float2(kErfcx3, kErfcx3));
    p = __ffma2_rn(p, w, make_float2(kErfcx2, kErfcx2));
    p = __ffma2_rn(p, w, make_float2(kErfcx1, kErfcx1));
    p = __ffma2_rn(p, w, make_float2(kErfcx0, kErfcx0));
    return p;
}
