// cg_device.cuh -- device helpers of the finite-difference flow-map gradient and the
// largest eigenvalue of the Cauchy-Green tensor (Eq. 1; Sec. 2 "Cauchy-Green"), shared by
// the regular pass (cg_ftle.cu) and the early evaluation (early_cg.cu).
#pragma once
#include "lcs_internal.cuh"

#include <math.h>

__device__ __forceinline__ long long lattice_nbr(const CgLaunch &L, const long long *idx, int b, int off, int *wrap)
{
    long long c[3] = {idx[0], idx[1], idx[2]};
    long long v = c[b] + off;
    *wrap = 0;
    int nb = L.n[b];
    if (L.periodic[b]) {
        if (v < 0) {
            v += nb;
            *wrap = -1;
        } else if (v >= nb) {
            v -= nb;
            *wrap = 1;
        }
    } else if (v < 0 || v >= nb) {
        return -1;
    }
    c[b] = v;
    return c[0] + (long long)L.n[0] * (c[1] + (long long)L.n[1] * c[2]);
}

// RN(x / d) for a fixed divisor d with y = RN(1 / d): q = RN(x y) is within about one
// ulp of x / d, one FMA-corrected step q1 = RN(q + RN(x - q d) y) makes it faithful, so
// the remainder x - q1 d is exact, and then RN(q1 + (x - q1 d) y) is the correctly
// rounded quotient (Markstein 1990, Theorem 8: a faithful quotient corrected with the
// correctly rounded reciprocal).  No overflow or underflow occurs for lattice spacings
// and flow-map differences.
__device__ __forceinline__ double div_fixed(double x, double d, double y)
{
    const double q = __dmul_rn(x, y);
    const double q1 = __fma_rn(__fma_rn(-q, d, x), y, q);
    return __fma_rn(__fma_rn(-q1, d, x), y, q1);
}

// neighbour position with the periodic shift of axis b (a == b only; w in {-1, 0, 1})
__device__ __forceinline__ double nbr_pos(float x, int w, double sh, bool shifted)
{
    double v = (double)x;
    if (shifted && w != 0) v = __dadd_rn(v, w > 0 ? sh : -sh);
    return v;
}

__device__ __forceinline__ double eig_max2(const double *C)
{
    // C = [[a, b], [b, c]]: lambda_max = (a + c)/2 + sqrt(((a - c)/2)^2 + b^2)
    double a = C[0], b = C[1], c = C[2];
    double m = __dmul_rn(0.5, __dadd_rn(a, c));
    double d = __dmul_rn(0.5, __dsub_rn(a, c));
    return __dadd_rn(m, sqrt(__dadd_rn(__dmul_rn(d, d), __dmul_rn(b, b))));
}

// trigonometric form in FP64 throughout (kept for matrices outside the scaled range)
static __device__ __noinline__ double eig_max3_slow(double a00, double a01, double a02, double a11, double a12,
                                             double a22)
{
    double p1 = a01 * a01 + a02 * a02 + a12 * a12;
    double q = (a00 + a11 + a22) / 3.0;
    double b00 = a00 - q, b11 = a11 - q, b22 = a22 - q;
    double p2 = b00 * b00 + b11 * b11 + b22 * b22 + 2.0 * p1;
    if (!(p2 > 0.0)) return q;
    double p = sqrt(p2 / 6.0);
    double ip = 1.0 / p;
    double c00 = b00 * ip, c11 = b11 * ip, c22 = b22 * ip, c01 = a01 * ip, c02 = a02 * ip, c12 = a12 * ip;
    double det = c00 * (c11 * c22 - c12 * c12) - c01 * (c01 * c22 - c12 * c02) + c02 * (c01 * c12 - c11 * c02);
    double r = fmin(fmax(0.5 * det, -1.0), 1.0);
    return q + 2.0 * p * cos(acos(r) / 3.0);
}

__device__ __forceinline__ double eig_max3(const double *C)
{
    const double dmax = fmax(C[0], fmax(C[3], C[5]));
    const double p1 = C[1] * C[1] + C[2] * C[2] + C[4] * C[4];
    if (p1 == 0.0) return dmax;  // diagonal (or NaN, which fmax passes on only if all are NaN)
    // scale by a power of two s so that the largest diagonal entry lies in [1, 2): exact, and it
    // keeps the FP32 steps below in range.  C is positive semidefinite, so dmax > 0 here.
    const int hi = __double2hiint(dmax);
    const int ex = ((hi >> 20) & 0x7ff) - 1023;
    if (!(dmax > 0.0) || ex < -1000 || ex > 1000) return eig_max3_slow(C[0], C[1], C[2], C[3], C[4], C[5]);
    const double s = __hiloint2double((1023 - ex) << 20, 0), is = __hiloint2double((1023 + ex) << 20, 0);
    const double a00 = C[0] * s, a01 = C[1] * s, a02 = C[2] * s, a11 = C[3] * s, a12 = C[4] * s, a22 = C[5] * s;
    const double q = (a00 + a11 + a22) * (1.0 / 3.0);
    const double b00 = a00 - q, b11 = a11 - q, b22 = a22 - q;
    const double p2 = (b00 * b00 + b11 * b11 + b22 * b22 + 2.0 * (p1 * s * s)) * (1.0 / 6.0);
    // eigenvalues are q + 2 p cos(.), p = sqrt(p2) and q >= 1/3: below 1e-28, lambda_max = q to 1e-13
    if (!(p2 >= 1e-28)) return p2 < 1e-28 ? q * is : eig_max3_slow(C[0], C[1], C[2], C[3], C[4], C[5]);
    // y = 1/sqrt(p2): FP32 estimate, two FP64 Newton steps (relative error 1e-7 -> 1e-14 -> 1e-16)
    double y = (double)rsqrtf((float)p2);
    y = y * (1.5 - 0.5 * p2 * y * y);
    y = y * (1.5 - 0.5 * p2 * y * y);
    const double p = p2 * y;
    // r = det((C - qI) / p) / 2 in [-1, 1]; beta = 2 cos(acos(r) / 3) is the largest root of
    // beta^3 - 3 beta - 2 r = 0
    const double det = b00 * (b11 * b22 - a12 * a12) - a01 * (a01 * b22 - a12 * a02) + a02 * (a01 * a12 - b11 * a02);
    const double r = fmin(fmax(0.5 * det * (y * y * y), -1.0), 1.0);
    double beta = (double)(2.0f * cosf(acosf((float)r) * (1.0f / 3.0f)));
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const double f = fma(beta, fma(beta, beta, -3.0), -2.0 * r);
        const double fp = 3.0 * fma(beta, beta, -1.0);
        if (fp > 1e-6) beta -= f * (double)__frcp_rn((float)fp);
    }
    return (q + p * beta) * is;
}

