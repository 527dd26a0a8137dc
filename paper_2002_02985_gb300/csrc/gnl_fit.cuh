// Generated by gen_gnl_fit.py (do not edit): polynomial forms of the kernel G_NL of
// Sec. 2.3 for the FP32-mixed kernels.  eta <= 1/2: G_NL = y S(y), y = eta^2; eta >= 2:
// G_NL = L(x), x = 1/eta^2; S (degree 6) and L (degree 6) are Chebyshev
// interpolants on [0, 1/4] of the closed form (largest relative error 1.8e-10 and 1.3e-10,
// below FP32 rounding), evaluated by Horner's rule.
#pragma once

namespace ofdft {
__device__ __forceinline__ float gnl_small_s(float y) {
    return fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(6.242049043e-02f, y, 2.573520713e-02f), y, 5.482175907e-02f), y, 7.371785135e-02f), y, 1.100620656e-01f), y, 1.777776332e-01f), y, -2.666666666e+00f);
}
__device__ __forceinline__ float gnl_large_l(float x) {
    return fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(-2.905759356e-02f, x, -1.199505511e-02f), x, -2.629342381e-02f), x, -3.768162710e-02f), x, -6.400429678e-02f), x, -1.371427893e-01f), x, -1.600000000e+00f);
}
}  // namespace ofdft
