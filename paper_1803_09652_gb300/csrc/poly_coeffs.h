/* Generated by gen_poly.py: far-field HCT polynomials, see that script. */
#pragma once
#define GB_POLY_YMAX 0.36000000f
#define GB_POLY_YFAR 0.10000000f
/* g(y) on [0, 0.36], degree 8, max relative error in FP32 Horner 1.23e-07 */
__device__ __forceinline__ float gb_poly_g(float y) {
    return fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(6.372991085e+00f, y, -3.979435205e+00f), y, 3.000669241e+00f), y, 4.458978176e-01f), y, 9.718360901e-01f), y, 8.843408227e-01f), y, 8.573058248e-01f), y, 7.999977469e-01f), y, 6.666666865e-01f);
}
__device__ __forceinline__ float2 gb_poly_g2(float2 y) {
    return __ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(make_float2(6.372991085e+00f, 6.372991085e+00f), y, make_float2(-3.979435205e+00f, -3.979435205e+00f)), y, make_float2(3.000669241e+00f, 3.000669241e+00f)), y, make_float2(4.458978176e-01f, 4.458978176e-01f)), y, make_float2(9.718360901e-01f, 9.718360901e-01f)), y, make_float2(8.843408227e-01f, 8.843408227e-01f)), y, make_float2(8.573058248e-01f, 8.573058248e-01f)), y, make_float2(7.999977469e-01f, 7.999977469e-01f)), y, make_float2(6.666666865e-01f, 6.666666865e-01f));
}
/* h(y) on [0, 0.36], degree 10, max relative error in FP32 Horner 1.47e-07 */
__device__ __forceinline__ float gb_poly_h(float y) {
    return fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(2.890447998e+02f, y, -3.036016235e+02f), y, 2.056483459e+02f), y, -4.527267456e+01f), y, 2.778405762e+01f), y, 1.125458431e+01f), y, 1.104221439e+01f), y, 8.882757187e+00f), y, 6.857286453e+00f), y, 4.799998760e+00f), y, 2.666666746e+00f);
}
__device__ __forceinline__ float2 gb_poly_h2(float2 y) {
    return __ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(make_float2(2.890447998e+02f, 2.890447998e+02f), y, make_float2(-3.036016235e+02f, -3.036016235e+02f)), y, make_float2(2.056483459e+02f, 2.056483459e+02f)), y, make_float2(-4.527267456e+01f, -4.527267456e+01f)), y, make_float2(2.778405762e+01f, 2.778405762e+01f)), y, make_float2(1.125458431e+01f, 1.125458431e+01f)), y, make_float2(1.104221439e+01f, 1.104221439e+01f)), y, make_float2(8.882757187e+00f, 8.882757187e+00f)), y, make_float2(6.857286453e+00f, 6.857286453e+00f)), y, make_float2(4.799998760e+00f, 4.799998760e+00f)), y, make_float2(2.666666746e+00f, 2.666666746e+00f));
}
/* gf(y) on [0, 0.1], degree 4, max relative error in FP32 Horner 8.50e-08 */
__device__ __forceinline__ float gb_poly_gf(float y) {
    return fmaf(fmaf(fmaf(fmaf(1.183633924e+00f, y, 8.635628223e-01f), y, 8.580689430e-01f), y, 7.999883294e-01f), y, 6.666666865e-01f);
}
__device__ __forceinline__ float2 gb_poly_gf2(float2 y) {
    return __ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(make_float2(1.183633924e+00f, 1.183633924e+00f), y, make_float2(8.635628223e-01f, 8.635628223e-01f)), y, make_float2(8.580689430e-01f, 8.580689430e-01f)), y, make_float2(7.999883294e-01f, 7.999883294e-01f)), y, make_float2(6.666666865e-01f, 6.666666865e-01f));
}
/* hf(y) on [0, 0.1], degree 5, max relative error in FP32 Horner 8.21e-08 */
__device__ __forceinline__ float gb_poly_hf(float y) {
    return fmaf(fmaf(fmaf(fmaf(fmaf(1.854454994e+01f, y, 1.023153305e+01f), y, 8.925169945e+00f), y, 6.856277943e+00f), y, 4.800007343e+00f), y, 2.666666746e+00f);
}
__device__ __forceinline__ float2 gb_poly_hf2(float2 y) {
    return __ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(make_float2(1.854454994e+01f, 1.854454994e+01f), y, make_float2(1.023153305e+01f, 1.023153305e+01f)), y, make_float2(8.925169945e+00f, 8.925169945e+00f)), y, make_float2(6.856277943e+00f, 6.856277943e+00f)), y, make_float2(4.800007343e+00f, 4.800007343e+00f)), y, make_float2(2.666666746e+00f, 2.666666746e+00f));
}
#define GB_POLY_ZJ 0.50000000f
/* q(y) on [0, 0.5], degree 9, max relative error in FP32 Horner 1.19e-07 */
__device__ __forceinline__ float gb_poly_q(float y) {
    return fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(1.507509708e+00f, y, -2.156293154e+00f), y, 1.706731677e+00f), y, -5.312927365e-01f), y, 2.776696980e-01f), y, 1.213092506e-01f), y, 1.683840305e-01f), y, 1.999313831e-01f), y, 2.500010431e-01f), y, 3.333333433e-01f);
}
__device__ __forceinline__ float2 gb_poly_q2(float2 y) {
    return __ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(make_float2(1.507509708e+00f, 1.507509708e+00f), y, make_float2(-2.156293154e+00f, -2.156293154e+00f)), y, make_float2(1.706731677e+00f, 1.706731677e+00f)), y, make_float2(-5.312927365e-01f, -5.312927365e-01f)), y, make_float2(2.776696980e-01f, 2.776696980e-01f)), y, make_float2(1.213092506e-01f, 1.213092506e-01f)), y, make_float2(1.683840305e-01f, 1.683840305e-01f)), y, make_float2(1.999313831e-01f, 1.999313831e-01f)), y, make_float2(2.500010431e-01f, 2.500010431e-01f)), y, make_float2(3.333333433e-01f, 3.333333433e-01f));
}
#define GB_POLY_ZJ2 0.75000000f
#define GB_POLY_ZMID 0.62500000f
/* q(z) on [0.5, 0.75] as a polynomial in y = z - 0.625: */
/* q_hi(y) on [-0.125, 0.125], degree 8, max relative error in FP32 Horner 1.29e-07 */
__device__ __forceinline__ float gb_poly_q_hi(float y) {
    return fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(3.442066040e+02f, y, 1.440139923e+02f), y, 4.896784210e+01f), y, 2.128055954e+01f), y, 9.618304253e+00f), y, 4.423333168e+00f), y, 2.134392262e+00f), y, 1.110777140e+00f), y, 6.574766040e-01f);
}
__device__ __forceinline__ float2 gb_poly_q_hi2(float2 y) {
    return __ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(make_float2(3.442066040e+02f, 3.442066040e+02f), y, make_float2(1.440139923e+02f, 1.440139923e+02f)), y, make_float2(4.896784210e+01f, 4.896784210e+01f)), y, make_float2(2.128055954e+01f, 2.128055954e+01f)), y, make_float2(9.618304253e+00f, 9.618304253e+00f)), y, make_float2(4.423333168e+00f, 4.423333168e+00f)), y, make_float2(2.134392262e+00f, 2.134392262e+00f)), y, make_float2(1.110777140e+00f, 1.110777140e+00f)), y, make_float2(6.574766040e-01f, 6.574766040e-01f));
}
