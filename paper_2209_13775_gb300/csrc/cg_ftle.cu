// cg_ftle.cu -- flow-map gradient, Cauchy-Green tensor, largest eigenvalue, FTLE.
//
// Paper: Eq. 1, C = grad(F)^T grad(F); Sec. 2 "Cauchy-Green": grad F from
// central differences of the final seed positions over the seed lattice, then
// the eigenvalues of C; Sec. 1: the FTLE is derived from the largest one,
// sigma = ln(sqrt(lambda_max)) / |T|.
//
// One thread per seed, FP64 from the FP32 flow map.  FP64 issue is the limit of this
// kernel on GB300, so the FP64 work is kept to what the results need:
//  * grad F and C: every difference, product and sum is a round-to-nearest operation
//    without contraction, and the division by 2h is correctly rounded (Markstein's
//    method below), so both equal the plain FP64 definition bit for bit;
//  * lambda_max: 2x2 from the quadratic formula; 3x3 from the characteristic cubic of
//    the shifted, scaled matrix (Smith 1961), whose trigonometric root is taken in FP32
//    and polished by two FP64 Newton steps (relative error ~1e-15 for a simple root),
//    and by Jacobi rotations where the two largest eigenvalues (nearly) coincide;
//  * FTLE = ln(lambda_max) / (2 |T|) in FP32: log1p of the FP64 difference lambda_max - 1
//    near 1, which keeps its relative accuracy (a few FP32 ulps) where sigma is near 0, and
//    log of lambda_max elsewhere (log_lambda).
#include "lcs_internal.cuh"

#include <math.h>

#include "cg_device.cuh"

// grad F of lattice seed p from its 2 DIM auxiliary points (lcs_seed_aux): per axis b the
// difference of the two points' final positions over that of their FP32 starting points,
// RN operations in FP64; NaN unless every point is OK
template <int DIM>
__device__ __forceinline__ void aux_gradient(const CgLaunch &L, int job, long long p, double (*G)[DIM])
{
    const long long M = L.npts;
    const float *X = L.xyz + (size_t)job * DIM * M;
    const unsigned char *S = L.status + (size_t)job * M;
    bool ok = true;
#pragma unroll
    for (int q = 0; q < 2 * DIM; ++q) ok &= S[p * 2 * DIM + q] == LCS_TRACER_OK;
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
        const long long i0 = (p * DIM + b) * 2, i1 = i0 + 1;
        const double den = __dsub_rn((double)L.x0aux[b * M + i0], (double)L.x0aux[b * M + i1]);
#pragma unroll
        for (int a = 0; a < DIM; ++a)
            G[a][b] = ok ? __ddiv_rn(__dsub_rn((double)X[a * M + i0], (double)X[a * M + i1]), den) : nan;
    }
}

// gradient sources: finite differences over the lattice, over auxiliary points, or the
// variational grad F integrated with the flow map
enum { GM_LATTICE = 0, GM_AUX = 1, GM_VAR = 2 };

template <int DIM, bool EIG, int GM>
__global__ void __launch_bounds__(256) cg_ftle_kernel(CgLaunch L)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int jr = blockIdx.y;        // job relative to job0
    const int job = L.job0 + jr;
    const long long N = L.N;
    if (p >= N) return;
    constexpr int NP = DIM == 2 ? 3 : 6;
    double G[DIM][DIM];
    if constexpr (GM == GM_AUX) {
        aux_gradient<DIM>(L, job, p, G);
    } else if constexpr (GM == GM_VAR) {
        const bool ok = L.status[(size_t)job * N + p] == LCS_TRACER_OK;
        const float *Mp = L.grad + ((size_t)job * N + p) * DIM * DIM;
#pragma unroll
        for (int a = 0; a < DIM; ++a)
#pragma unroll
            for (int b = 0; b < DIM; ++b)
                G[a][b] = ok ? (double)Mp[a * DIM + b] : __longlong_as_double(0x7ff8000000000000LL);
    } else {
    const float *X = L.xyz + (size_t)job * DIM * N;
    const unsigned char *S = L.status + (size_t)job * N;
    const long long idx[3] = {p % L.n[0], (p / L.n[0]) % L.n[1], DIM == 3 ? p / ((long long)L.n[0] * L.n[1]) : 0};
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
        const double h2 = L.h2[b], rh2 = L.rh2[b], sh = L.period[b];
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            const bool on = a == b;
            const float *Xa = X + (size_t)a * N;
            double d;
            if (mode == 1) {
                const double Fp1 = nbr_pos(Xa[qp1], wp1, sh, on), Fm1 = nbr_pos(Xa[qm1], wm1, sh, on);
                d = div_fixed(__dsub_rn(Fp1, Fm1), h2, rh2);
            } else if (mode == 2) {
                const double F0 = (double)Xa[p];
                const double Fp1 = nbr_pos(Xa[qp1], wp1, sh, on), Fp2 = nbr_pos(Xa[qp2], wp2, sh, on);
                d = div_fixed(__dsub_rn(__dadd_rn(__dmul_rn(-3.0, F0), __dmul_rn(4.0, Fp1)), Fp2), h2, rh2);
            } else if (mode == 3) {
                const double F0 = (double)Xa[p];
                const double Fm1 = nbr_pos(Xa[qm1], wm1, sh, on), Fm2 = nbr_pos(Xa[qm2], wm2, sh, on);
                d = div_fixed(__dadd_rn(__dsub_rn(__dmul_rn(3.0, F0), __dmul_rn(4.0, Fm1)), Fm2), h2, rh2);
            } else {
                d = __longlong_as_double(0x7ff8000000000000LL);  // NaN
            }
            G[a][b] = d;
        }
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
    if constexpr (EIG) {   // lcs_cg_eigen
        double ev[DIM], V[DIM * DIM];
        eig_jacobi<DIM>(C, ev, V);
        if (L.eigval) {
#pragma unroll
            for (int k = 0; k < DIM; ++k) L.eigval[out * DIM + k] = ev[k];
        }
        if (L.eigvec) {
#pragma unroll
            for (int k = 0; k < DIM * DIM; ++k) L.eigvec[out * DIM * DIM + k] = V[k];
        }
        return;
    }
    if (L.lam || L.ftle) {
        const double lm = DIM == 2 ? eig_max2(C) : eig_max3(C);
        if (L.lam) L.lam[out] = lm;
        // sigma = ln(sqrt(lm)) / |T| = ln(lm) / (2 |T|)
        if (L.ftle) L.ftle[out] = log_lambda(lm) * (0.5f / (float)L.absT[job]);
    }
}

cudaError_t launch_cg_ftle(const CgLaunch &L0, cudaStream_t s)
{
    if (L0.N == 0 || L0.njobs == 0) return cudaSuccess;
    CgLaunch L = L0;
    for (int b = 0; b < 3; ++b) {
        L.h2[b] = 2.0 * L.h[b];  // exact
        L.rh2[b] = 1.0 / L.h2[b];
    }
    int bt = 256;
    dim3 grid((unsigned)((L.N + bt - 1) / bt), (unsigned)L.njobs);
    const bool eig = L.eigval || L.eigvec;
    const int gm = L.grad ? GM_VAR : (L.x0aux ? GM_AUX : GM_LATTICE);
#define CG_LAUNCH(D, G) (eig ? cg_ftle_kernel<D, true, G><<<grid, bt, 0, s>>>(L) \
                             : cg_ftle_kernel<D, false, G><<<grid, bt, 0, s>>>(L))
    if (L.dim == 2) {
        if (gm == GM_VAR) CG_LAUNCH(2, GM_VAR);
        else if (gm == GM_AUX) CG_LAUNCH(2, GM_AUX);
        else CG_LAUNCH(2, GM_LATTICE);
    } else {
        if (gm == GM_VAR) CG_LAUNCH(3, GM_VAR);
        else if (gm == GM_AUX) CG_LAUNCH(3, GM_AUX);
        else CG_LAUNCH(3, GM_LATTICE);
    }
#undef CG_LAUNCH
    return cudaGetLastError();
}
