// cg_ftle.cu -- flow-map gradient, Cauchy-Green tensor, largest eigenvalue, FTLE.
//
// Paper: Eq. 1, C = grad(F)^T grad(F); Sec. 2 "Cauchy-Green": grad F from
// central differences of the final seed positions over the seed lattice, then
// the eigenvalues of C; Sec. 1: the FTLE is derived from the largest one,
// sigma = ln(sqrt(lambda_max)) / |T|.
//
// One thread per seed, FP64 from the FP32 flow map.  Every difference, product
// and sum uses round-to-nearest operations without contraction, so grad F and C
// equal the plain FP64 definition bit for bit on the same positions.
// lambda_max is closed-form: 2x2 from the quadratic formula, 3x3 from the
// trigonometric solution of the characteristic cubic (Smith 1961).
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

template <int DIM>
__device__ __forceinline__ double eig_max(const double *C)
{
    if (DIM == 2) {
        // C = [[a, b], [b, c]]: lambda_max = (a + c)/2 + sqrt(((a - c)/2)^2 + b^2)
        double a = C[0], b = C[1], c = C[2];
        double m = __dmul_rn(0.5, __dadd_rn(a, c));
        double d = __dmul_rn(0.5, __dsub_rn(a, c));
        return __dadd_rn(m, sqrt(__dadd_rn(__dmul_rn(d, d), __dmul_rn(b, b))));
    } else {
        double a00 = C[0], a01 = C[1], a02 = C[2], a11 = C[3], a12 = C[4], a22 = C[5];
        double p1 = a01 * a01 + a02 * a02 + a12 * a12;
        if (p1 == 0.0) return fmax(a00, fmax(a11, a22));
        double q = (a00 + a11 + a22) / 3.0;
        double b00 = a00 - q, b11 = a11 - q, b22 = a22 - q;
        double p2 = b00 * b00 + b11 * b11 + b22 * b22 + 2.0 * p1;
        double p = sqrt(p2 / 6.0);
        double ip = 1.0 / p;
        // det((C - qI) / p) / 2
        double c00 = b00 * ip, c11 = b11 * ip, c22 = b22 * ip, c01 = a01 * ip, c02 = a02 * ip, c12 = a12 * ip;
        double det = c00 * (c11 * c22 - c12 * c12) - c01 * (c01 * c22 - c12 * c02) + c02 * (c01 * c12 - c11 * c02);
        double r = 0.5 * det;
        double phi;
        if (r <= -1.0)
            phi = M_PI / 3.0;
        else if (r >= 1.0)
            phi = 0.0;
        else
            phi = acos(r) / 3.0;
        return q + 2.0 * p * cos(phi);
    }
}

template <int DIM>
__global__ void __launch_bounds__(256) cg_ftle_kernel(CgLaunch L)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int jr = blockIdx.y;        // job relative to job0
    const int job = L.job0 + jr;
    const long long N = L.N;
    if (p >= N) return;
    constexpr int NP = DIM == 2 ? 3 : 6;
    const float *X = L.xyz + (size_t)job * DIM * N;
    const unsigned char *S = L.status + (size_t)job * N;
    const long long idx[3] = {p % L.n[0], (p / L.n[0]) % L.n[1], DIM == 3 ? p / ((long long)L.n[0] * L.n[1]) : 0};
    double G[DIM][DIM];
    bool valid = S[p] == LCS_TRACER_OK;
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
        int wp1, wm1, wp2, wm2;
        long long qp1 = lattice_nbr(L, idx, b, 1, &wp1);
        long long qm1 = lattice_nbr(L, idx, b, -1, &wm1);
        long long qp2 = lattice_nbr(L, idx, b, 2, &wp2);
        long long qm2 = lattice_nbr(L, idx, b, -2, &wm2);
        bool okp1 = qp1 >= 0 && S[qp1] == LCS_TRACER_OK;
        bool okm1 = qm1 >= 0 && S[qm1] == LCS_TRACER_OK;
        bool okp2 = qp2 >= 0 && S[qp2] == LCS_TRACER_OK;
        bool okm2 = qm2 >= 0 && S[qm2] == LCS_TRACER_OK;
        int mode = !valid ? 0 : (okp1 && okm1) ? 1 : (okp1 && okp2) ? 2 : (okm1 && okm2) ? 3 : 0;
        const double h2 = __dmul_rn(2.0, L.h[b]);
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            const double sh = (a == b) ? L.period[b] : 0.0;
            const float *Xa = X + (size_t)a * N;
            double d;
            if (mode == 1) {
                double Fp1 = __dadd_rn((double)Xa[qp1], __dmul_rn((double)wp1, sh));
                double Fm1 = __dadd_rn((double)Xa[qm1], __dmul_rn((double)wm1, sh));
                d = __ddiv_rn(__dsub_rn(Fp1, Fm1), h2);
            } else if (mode == 2) {
                double F0 = (double)Xa[p];
                double Fp1 = __dadd_rn((double)Xa[qp1], __dmul_rn((double)wp1, sh));
                double Fp2 = __dadd_rn((double)Xa[qp2], __dmul_rn((double)wp2, sh));
                d = __ddiv_rn(__dsub_rn(__dadd_rn(__dmul_rn(-3.0, F0), __dmul_rn(4.0, Fp1)), Fp2), h2);
            } else if (mode == 3) {
                double F0 = (double)Xa[p];
                double Fm1 = __dadd_rn((double)Xa[qm1], __dmul_rn((double)wm1, sh));
                double Fm2 = __dadd_rn((double)Xa[qm2], __dmul_rn((double)wm2, sh));
                d = __ddiv_rn(__dadd_rn(__dsub_rn(__dmul_rn(3.0, F0), __dmul_rn(4.0, Fm1)), Fm2), h2);
            } else {
                d = __longlong_as_double(0x7ff8000000000000LL);  // NaN
            }
            G[a][b] = d;
        }
    }
    // Eq. 1: C_ij = sum_a G_ai G_aj, packed upper triangle row by row
    double C[NP];
    int o = 0;
#pragma unroll
    for (int i = 0; i < DIM; ++i)
#pragma unroll
        for (int j = i; j < DIM; ++j) {
            double s = 0.0;
#pragma unroll
            for (int a = 0; a < DIM; ++a) s = __dadd_rn(s, __dmul_rn(G[a][i], G[a][j]));
            C[o++] = s;
        }
    const size_t out = (size_t)jr * N + p;
    if (L.C) {
#pragma unroll
        for (int q = 0; q < NP; ++q) L.C[out * NP + q] = C[q];
    }
    if (L.lam || L.ftle) {
        double lm = eig_max<DIM>(C);
        if (L.lam) L.lam[out] = lm;
        if (L.ftle) L.ftle[out] = __double2float_rn(log(sqrt(lm)) / L.absT[job]);
    }
}

cudaError_t launch_cg_ftle(const CgLaunch &L, cudaStream_t s)
{
    if (L.N == 0 || L.njobs == 0) return cudaSuccess;
    int bt = 256;
    dim3 grid((unsigned)((L.N + bt - 1) / bt), (unsigned)L.njobs);
    if (L.dim == 2)
        cg_ftle_kernel<2><<<grid, bt, 0, s>>>(L);
    else
        cg_ftle_kernel<3><<<grid, bt, 0, s>>>(L);
    return cudaGetLastError();
}
