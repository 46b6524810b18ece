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

// ln(lambda_max) in FP32 from the FP64 eigenvalue, for sigma = ln(sqrt(lambda_max)) / |T|: near
// lambda_max = 1 as log1p of the FP64 difference lambda_max - 1 (which keeps its relative
// accuracy where sigma is near 0), elsewhere as log of the rounded eigenvalue (log1p of a
// rounded lambda_max - 1 close to -1 would lose digits: a contracting map, lambda_max << 1)
__device__ __forceinline__ float log_lambda(double lm)
{
    const double d = lm - 1.0;
    return fabs(d) < 0.5 ? log1pf((float)d) : logf((float)lm);
}

// All eigenpairs of the packed symmetric C by cyclic Jacobi rotations in FP64.  Each
// rotation zeroes a_pq with t = tan(theta) the smaller root of t^2 + 2 tau t - 1 = 0,
// tau = (a_qq - a_pp) / (2 a_pq), updates the diagonal as a_pp - t a_pq and a_qq + t a_pq
// (Rutishauser's form), rotates the other row of the pair and accumulates V <- V J.  A pair
// counts as converged when |a_pq| <= 1e-18 sqrt(|a_pp a_qq|), a relative test that keeps
// the small eigenvalues of a graded C accurate; at most 16 sweeps.  Ascending order, each
// eigenvector with its largest-magnitude component positive.
template <int DIM>
__device__ __forceinline__ void eig_jacobi(const double *Cp, double *ev, double *V)
{
    double A[DIM][DIM];
    int o = 0;
#pragma unroll
    for (int i = 0; i < DIM; ++i)
#pragma unroll
        for (int j = i; j < DIM; ++j) {
            A[i][j] = Cp[o];
            A[j][i] = Cp[o];
            ++o;
        }
    double W[DIM][DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i)
#pragma unroll
        for (int j = 0; j < DIM; ++j) W[i][j] = i == j ? 1.0 : 0.0;
    bool bad = false;
#pragma unroll
    for (int i = 0; i < DIM * (DIM + 1) / 2; ++i) bad |= isnan(Cp[i]);
    for (int sweep = 0; sweep < 16 && !bad; ++sweep) {
        bool rotated = false;
#pragma unroll
        for (int p = 0; p < DIM - 1; ++p)
#pragma unroll
            for (int q = p + 1; q < DIM; ++q) {
                const double apq = A[p][q];
                if (!(fabs(apq) > 1e-18 * sqrt(fabs(A[p][p] * A[q][q])))) continue;
                rotated = true;
                const double tau = (A[q][q] - A[p][p]) / (2.0 * apq);
                const double t = copysign(1.0, tau) / (fabs(tau) + sqrt(fma(tau, tau, 1.0)));
                const double c = rsqrt(fma(t, t, 1.0)), s = t * c;
                A[p][p] = fma(-t, apq, A[p][p]);
                A[q][q] = fma(t, apq, A[q][q]);
                A[p][q] = A[q][p] = 0.0;
#pragma unroll
                for (int r = 0; r < DIM; ++r) {
                    if (r == p || r == q) continue;
                    const double arp = A[r][p], arq = A[r][q];
                    A[r][p] = A[p][r] = c * arp - s * arq;
                    A[r][q] = A[q][r] = s * arp + c * arq;
                }
#pragma unroll
                for (int r = 0; r < DIM; ++r) {
                    const double wp = W[r][p], wq = W[r][q];
                    W[r][p] = c * wp - s * wq;
                    W[r][q] = s * wp + c * wq;
                }
            }
        if (!rotated) break;
    }
    int ord[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) ord[i] = i;
#pragma unroll
    for (int i = 0; i < DIM; ++i)
#pragma unroll
        for (int j = i + 1; j < DIM; ++j)
            if (A[ord[j]][ord[j]] < A[ord[i]][ord[i]]) {
                const int t = ord[i];
                ord[i] = ord[j];
                ord[j] = t;
            }
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        int m = 0;
#pragma unroll
        for (int r = 1; r < DIM; ++r)
            if (fabs(W[r][ord[k]]) > fabs(W[m][ord[k]])) m = r;
        const double sg = W[m][ord[k]] < 0.0 ? -1.0 : 1.0;
        ev[k] = bad ? nan : A[ord[k]][ord[k]];
#pragma unroll
        for (int r = 0; r < DIM; ++r) V[k * DIM + r] = bad ? nan : sg * W[r][ord[k]];
    }
}

// lambda_max by the Jacobi rotations above: matrices outside the scaled range of eig_max3, and
// those whose two largest eigenvalues (nearly) coincide, where no root of the characteristic
// cubic is accurate in FP64 (see eig_max3).  Out of line: rare, and it keeps eig_max3 small.
static __device__ __noinline__ double eig_max3_jacobi(const double *C)
{
    double ev[3], V[9];
    eig_jacobi<3>(C, ev, V);
    return ev[2];
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
    if (!(dmax > 0.0) || ex < -1000 || ex > 1000) return eig_max3_jacobi(C);
    const double s = __hiloint2double((1023 - ex) << 20, 0), is = __hiloint2double((1023 + ex) << 20, 0);
    const double a00 = C[0] * s, a01 = C[1] * s, a02 = C[2] * s, a11 = C[3] * s, a12 = C[4] * s, a22 = C[5] * s;
    const double q = (a00 + a11 + a22) * (1.0 / 3.0);
    const double b00 = a00 - q, b11 = a11 - q, b22 = a22 - q;
    const double p2 = (b00 * b00 + b11 * b11 + b22 * b22 + 2.0 * (p1 * s * s)) * (1.0 / 6.0);
    // eigenvalues are q + 2 p cos(.), p = sqrt(p2) and q >= 1/3: below 1e-28, lambda_max = q to 1e-13
    if (!(p2 >= 1e-28)) return p2 < 1e-28 ? q * is : eig_max3_jacobi(C);
    // y = 1/sqrt(p2): FP32 estimate, two FP64 Newton steps (relative error 1e-7 -> 1e-14 -> 1e-16)
    double y = (double)rsqrtf((float)p2);
    y = y * (1.5 - 0.5 * p2 * y * y);
    y = y * (1.5 - 0.5 * p2 * y * y);
    const double p = p2 * y;
    // r = det((C - qI) / p) / 2 in [-1, 1]; beta = 2 cos(acos(r) / 3) is the largest root of
    // beta^3 - 3 beta - 2 r = 0
    const double det = b00 * (b11 * b22 - a12 * a12) - a01 * (a01 * b22 - a12 * a02) + a02 * (a01 * a12 - b11 * a02);
    const double r = fmin(fmax(0.5 * det * (y * y * y), -1.0), 1.0);
    // r = -1 is a double largest root (beta = 1, lambda_1 = lambda_2).  Near it, with r = -1 + d,
    // the root sits at 1 + sqrt(2 d / 3) + ..., so an error of one ulp in r or in the cubic's value
    // moves it by about the square root of an ulp (1e-8 relative to lambda_max) whatever the
    // polish.  Below 1 + r = 1e-3 (a gap lambda_1 - lambda_2 under about 5% of p) the Jacobi
    // rotations, which are backward stable, give lambda_max instead; above it two Newton steps
    // from the FP32 root reach ~1e-14 relative (f' = 3 (beta^2 - 1) >= 0.15 there).  NaN
    // entries also end up here (fmax and fmin pass -1), and Jacobi returns NaN for them.
    if (!(r >= -1.0 + 1e-3)) return eig_max3_jacobi(C);
    double beta = (double)(2.0f * cosf(acosf((float)r) * (1.0f / 3.0f)));
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const double f = fma(beta, fma(beta, beta, -3.0), -2.0 * r);
        const double fp = 3.0 * fma(beta, beta, -1.0);
        beta -= f * (double)__frcp_rn((float)fp);
    }
    return (q + p * beta) * is;
}
