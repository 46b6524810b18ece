// early_cg.cu -- early Cauchy-Green evaluation where a stencil leaves the domain.
//
// Paper: Sec. 2 "Flow Map" names, for trajectories that exit the velocity data, forming the
// CG tensor ahead of the horizon for every seed whose differences use such a trajectory (and
// Sec. 3.1 notes that synchronous updates make the CG tensor available at any step).
//
// After a fixed-step RK4 integration over (t0, t0 + T) (lcs_advect), each seed's finite
// differences use a fixed set of lattice neighbours (central, or one-sided at a lattice
// edge).  m(p) = the fewest steps that the seed or one of those neighbours stayed in the
// domain: ns for a tracer still OK at the end, one less than the step it left in (its exit
// time t0 + (n + 1) h) otherwise.  Seeds with m = ns keep the regular FTLE over |T|; seeds
// with 0 < m < ns get the flow map of their stencil re-integrated over m steps (the same
// arithmetic as the integration, so the positions are those the tracers had after step m),
// grad F, C, lambda_max and sigma = ln sqrt(lambda_max) / (m |h|); m = 0 gives NaN.
//
// Three launches: a scan that finds m and lists the early seeds (one thread per seed), the
// re-integration (one thread per listed seed and stencil member), the differences (one
// thread per listed seed).  The list is short where few tracers leave.
#include "cg_device.cuh"
#include "rect_device.cuh"
#include "tri_device.cuh"

namespace {

// a lattice seed that is valid at the start: all of them on rectilinear fields, those inside
// the mesh (cell >= 0) on mesh fields
__device__ __forceinline__ bool valid0(const int *cells0, long long q) { return q >= 0 && (!cells0 || cells0[q] >= 0); }

// the difference rule along axis b, chosen as the regular pass chooses it from the seeds valid at
// the start: 1 central (+1, -1), 2 forward (+1, +2), 3 backward (-1, -2), 0 none.  On a lattice of
// valid seeds: central on periodic axes and inside, forward at the low edge, backward at the high.
__device__ __forceinline__ int axis_mode(const CgLaunch &L, const long long *idx, int b, const int *cells0)
{
    int w;
    const bool p1 = valid0(cells0, lattice_nbr(L, idx, b, 1, &w)), m1 = valid0(cells0, lattice_nbr(L, idx, b, -1, &w));
    if (p1 && m1) return 1;
    if (p1 && valid0(cells0, lattice_nbr(L, idx, b, 2, &w))) return 2;
    if (m1 && valid0(cells0, lattice_nbr(L, idx, b, -2, &w))) return 3;
    return 0;
}

// stencil member s (0: the seed, then two per axis) of seed idx for the rule `mode` of its axis.
// Returns the id (-1 when the axis has no rule); *wrap = periods crossed.
__device__ __forceinline__ long long member(const CgLaunch &L, const long long *idx, int s, int mode, int *wrap)
{
    *wrap = 0;
    if (s == 0) return idx[0] + (long long)L.n[0] * (idx[1] + (long long)L.n[1] * idx[2]);
    const int b = (s - 1) >> 1, second = (s - 1) & 1;
    if (mode == 0) return -1;
    const int off = mode == 1 ? (second ? -1 : 1) : mode == 2 ? (second ? 2 : 1) : (second ? -2 : -1);
    return lattice_nbr(L, idx, b, off, wrap);
}

// steps a tracer of this slot stayed in the domain: a rectilinear tracer leaves at the end of a
// step (the one before it counts), a mesh tracer at the start of the step it failed in
__device__ __forceinline__ int in_steps(unsigned char st, float te, int ns, double t0, double adt, bool mesh)
{
    if (st == LCS_TRACER_OK) return ns;
    if (st != LCS_TRACER_LEFT) return 0;
    const int n1 = (int)rint(fabs((double)te - t0) / adt);
    return mesh ? n1 : max(n1 - 1, 0);
}

template <int DIM>
__global__ void early_scan_kernel(CgLaunch L, int job, int ns, double t0, double adt, float absT,
                                  const int *__restrict__ cells0, unsigned *__restrict__ count,
                                  int2 *__restrict__ list, float *__restrict__ t_eval)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= L.N) return;
    const unsigned char *S = L.status + (size_t)job * L.N;
    const float *TE = L.texit + (size_t)job * L.N;
    const long long idx[3] = {p % L.n[0], (p / L.n[0]) % L.n[1], DIM == 3 ? p / ((long long)L.n[0] * L.n[1]) : 0};
    const bool mesh = cells0 != nullptr;
    int m = ns;
#pragma unroll
    for (int s = 0; s < 2 * DIM + 1; ++s) {
        int w;
        const int mode = s == 0 ? 1 : axis_mode(L, idx, (s - 1) >> 1, cells0);
        const long long q = member(L, idx, s, mode, &w);
        m = min(m, q < 0 ? 0 : in_steps(S[q], TE[q], ns, t0, adt, mesh));
    }
    if (m >= ns) {
        if (t_eval) t_eval[p] = absT;
        return;
    }
    if (t_eval) t_eval[p] = (float)((double)m * adt);
    if (m > 0) {
        const unsigned e = atomicAdd(count, 1u);
        list[e] = make_int2((int)p, m);
    }
}

// re-integration of member (e % (2 DIM + 1)) of listed seed e / (2 DIM + 1) over m steps,
// with the one-pass kernel's arithmetic; the unwrapped FP32 position goes to pos
template <int DIM, int ST>
__global__ void early_advect_kernel(CgLaunch L, RectParams P, const char *__restrict__ frames, size_t fstride,
                                    Rk4Args A, int job, const unsigned *__restrict__ count,
                                    const int2 *__restrict__ list, float *__restrict__ pos)
{
    constexpr int NM = 2 * DIM + 1;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long e = t / NM;
    const int s = (int)(t % NM);
    if (e >= (long long)*count) return;
    const int2 it = list[e];
    const long long p = it.x;
    const long long idx[3] = {p % L.n[0], (p / L.n[0]) % L.n[1], DIM == 3 ? p / ((long long)L.n[0] * L.n[1]) : 0};
    int w;
    const long long q = member(L, idx, s, s == 0 ? 1 : axis_mode(L, idx, (s - 1) >> 1, nullptr), &w);
    float x[DIM], cx[DIM];
    int img[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        x[d] = A.seeds[d * A.N + q];
        cx[d] = 0.0f;
        img[d] = 0;
    }
    wrap_periodic<DIM>(P, x, cx, img);
    const SchedEntry *sc = A.sched + (size_t)job * A.nsteps_max * 3;
    const float h = A.job_h[job];
    for (int n = 0; n < it.y; ++n) {
        SchedEntry e0 = load_sched(sc + 3 * n), e1 = load_sched(sc + 3 * n + 1), e2 = load_sched(sc + 3 * n + 2);
        if constexpr (DIM == 2)
            rk4_step<2, ST, SRC_GLOBAL>(P, x, cx, h, frames + (size_t)e0.k * fstride,
                                        frames + (size_t)(e0.k + 1) * fstride, e0.a, frames + (size_t)e1.k * fstride,
                                        frames + (size_t)(e1.k + 1) * fstride, e1.a, frames + (size_t)e2.k * fstride,
                                        frames + (size_t)(e2.k + 1) * fstride, e2.a);
        else
            rk4_step3p<ST>(P, x, cx, h, frames + (size_t)e0.k * fstride, e0.a, frames + (size_t)e1.k * fstride,
                           e1.a, frames + (size_t)e2.k * fstride, e2.a);
        wrap_periodic<DIM>(P, x, cx, img);
    }
    float *o = pos + (size_t)t * DIM;
#pragma unroll
    for (int d = 0; d < DIM; ++d) o[d] = out_coord(P, d, x[d], cx[d], img[d]);
}

// the same on a tet (DIM 3, MD = TetDev) or triangle (DIM 2, TriDev) field: member q from its seed
// and start cell with the plain mesh kernels' arithmetic (the listed members stayed inside for m steps)
template <int DIM, int ST, class MD>
__global__ void early_advect_mesh_kernel(CgLaunch L, MD T, Rk4Args A, const int *__restrict__ cells0, int job,
                                         const unsigned *__restrict__ count, const int2 *__restrict__ list,
                                         float *__restrict__ pos)
{
    constexpr int NM = 2 * DIM + 1;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long e = t / NM;
    const int s = (int)(t % NM);
    if (e >= (long long)*count) return;
    const int2 it = list[e];
    const long long p = it.x;
    const long long idx[3] = {p % L.n[0], (p / L.n[0]) % L.n[1], DIM == 3 ? p / ((long long)L.n[0] * L.n[1]) : 0};
    int w;
    const long long q = member(L, idx, s, s == 0 ? 1 : axis_mode(L, idx, (s - 1) >> 1, cells0), &w);
    float x[DIM], cx[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        x[d] = A.seeds[d * A.N + q];
        cx[d] = 0.0f;
    }
    int cell = cells0[q];
    const SchedEntry *sc = A.sched + (size_t)job * A.nsteps_max * 3;
    const float h = A.job_h[job], hh = 0.5f * h;
    for (int n = 0; n < it.y; ++n) {
        const SchedEntry es3[3] = {load_sched(sc + 3 * n), load_sched(sc + 3 * n + 1), load_sched(sc + 3 * n + 2)};
        float k[4][DIM], y[DIM], lam[DIM + 1];
#pragma unroll
        for (int st = 0; st < 4; ++st) {
            const float c = st == 0 ? 0.0f : (st == 3 ? h : hh);
#pragma unroll
            for (int d = 0; d < DIM; ++d) y[d] = st == 0 ? x[d] : fmaf(c, k[st - 1][d], x[d]);
            const SchedEntry &es = es3[st == 0 ? 0 : (st == 3 ? 2 : 1)];
            const char *fp = T.pairs + (size_t)es.k * T.fstride;
            if constexpr (DIM == 3) {
                tet_locate(T, y, &cell, lam);
                tet_interp<ST>(T, cell, lam, fp, es.a, k[st]);
            } else {
                tri_locate(T, y, &cell, lam);
                tri_interp<ST>(T, cell, lam, fp, es.a, k[st]);
            }
        }
        const float h6 = h * (1.0f / 6.0f);
#pragma unroll
        for (int d = 0; d < DIM; ++d) rk4_advance(x[d], cx[d], h6, k[0][d], k[1][d], k[2][d], k[3][d]);
    }
    float *o = pos + (size_t)t * DIM;
#pragma unroll
    for (int d = 0; d < DIM; ++d) o[d] = x[d] + cx[d];
}

// grad F from the re-integrated stencil (the regular pass's formulas), C, lambda_max, FTLE
template <int DIM>
__global__ void early_fd_kernel(CgLaunch L, const int *__restrict__ cells0, const unsigned *__restrict__ count,
                                const int2 *__restrict__ list, const float *__restrict__ pos, double adt,
                                float *__restrict__ ftle)
{
    constexpr int NM = 2 * DIM + 1;
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)*count) return;
    const int2 it = list[e];
    const long long p = it.x;
    const long long idx[3] = {p % L.n[0], (p / L.n[0]) % L.n[1], DIM == 3 ? p / ((long long)L.n[0] * L.n[1]) : 0};
    const float *X = pos + (size_t)e * NM * DIM;
    double G[DIM][DIM];
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
        int w1, w2;
        const int mode = axis_mode(L, idx, b, cells0);
        member(L, idx, 1 + 2 * b, mode, &w1);
        member(L, idx, 2 + 2 * b, mode, &w2);
        const double h2 = L.h2[b], rh2 = L.rh2[b], sh = L.period[b];
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            const bool on = a == b;
            const double F0 = (double)X[a];
            const double F1 = nbr_pos(X[(1 + 2 * b) * DIM + a], w1, sh, on);
            const double F2 = nbr_pos(X[(2 + 2 * b) * DIM + a], w2, sh, on);
            double d;
            if (mode == 1)
                d = div_fixed(__dsub_rn(F1, F2), h2, rh2);
            else if (mode == 2)
                d = div_fixed(__dsub_rn(__dadd_rn(__dmul_rn(-3.0, F0), __dmul_rn(4.0, F1)), F2), h2, rh2);
            else
                d = div_fixed(__dadd_rn(__dsub_rn(__dmul_rn(3.0, F0), __dmul_rn(4.0, F1)), F2), h2, rh2);
            G[a][b] = d;
        }
    }
    constexpr int NP = DIM == 2 ? 3 : 6;
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
    const double lm = DIM == 2 ? eig_max2(C) : eig_max3(C);
    // sigma = ln(sqrt(lm)) / (m |h|), as the regular pass forms it
    ftle[p] = log_lambda(lm) * (0.5f / (float)((double)it.y * adt));
}

}  // namespace

cudaError_t launch_early_cg(const EarlyLaunch &E, cudaStream_t s)
{
    CgLaunch L = E.cg;
    for (int b = 0; b < 3; ++b) {
        L.h2[b] = 2.0 * L.h[b];
        L.rh2[b] = 1.0 / L.h2[b];
    }
    const int bt = 256;
    const unsigned grid = (unsigned)((L.N + bt - 1) / bt);
    if (E.phase == 0) {
        if (L.dim == 2)
            early_scan_kernel<2><<<grid, bt, 0, s>>>(L, E.job, E.ns, E.t0, E.adt, E.absT, E.cells0, E.count, E.list,
                                                      E.t_eval);
        else
            early_scan_kernel<3><<<grid, bt, 0, s>>>(L, E.job, E.ns, E.t0, E.adt, E.absT, E.cells0, E.count, E.list,
                                                      E.t_eval);
        return cudaGetLastError();
    }
    if (E.nlisted == 0) return cudaSuccess;
    const lcs_field *f = E.field;
    const RectParams P = make_rect_params(f);
    Rk4Args A;
    A.seeds = E.seeds;
    A.N = L.N;
    A.nsteps_max = E.nsteps_max;
    A.sched = E.sched;
    A.job_nsteps = nullptr;
    A.job_h = E.job_h;
    A.job_t0 = nullptr;
    A.job_tend = nullptr;
    A.out_xyz = nullptr;
    A.out_status = nullptr;
    A.out_texit = nullptr;
    const int nm = 2 * L.dim + 1;
    const unsigned ga = (unsigned)((E.nlisted * nm + bt - 1) / bt);
    const char *fr = (const char *)f->d_frames;
    if (lcs_is_mesh(f)) {
#define EARLY_MESH(D, ST, MD, T) early_advect_mesh_kernel<D, ST, MD><<<ga, bt, 0, s>>>(L, T, A, E.cells0, E.job, E.count, E.list, E.pos)
        if (f->kind == LCS_TRI) {
            const TriDev T = tri_dev(f, E.walk_limit);
            if (f->storage == LCS_F32) EARLY_MESH(2, LCS_F32, TriDev, T);
            else if (f->storage == LCS_F16) EARLY_MESH(2, LCS_F16, TriDev, T);
            else EARLY_MESH(2, LCS_BF16, TriDev, T);
        } else {
            const TetDev T = tet_dev(f, E.walk_limit);
            if (f->storage == LCS_F32) EARLY_MESH(3, LCS_F32, TetDev, T);
            else if (f->storage == LCS_F16) EARLY_MESH(3, LCS_F16, TetDev, T);
            else EARLY_MESH(3, LCS_BF16, TetDev, T);
        }
#undef EARLY_MESH
    } else {
#define EARLY_ADVECT(D, ST) early_advect_kernel<D, ST><<<ga, bt, 0, s>>>(L, P, fr, f->frame_stride, A, E.job, E.count, E.list, E.pos)
    if (L.dim == 2) {
        if (f->storage == LCS_F32) EARLY_ADVECT(2, LCS_F32);
        else if (f->storage == LCS_F16) EARLY_ADVECT(2, LCS_F16);
        else EARLY_ADVECT(2, LCS_BF16);
    } else {
        if (f->storage == LCS_F32) EARLY_ADVECT(3, LCS_F32);
        else if (f->storage == LCS_F16) EARLY_ADVECT(3, LCS_F16);
        else EARLY_ADVECT(3, LCS_BF16);
    }
#undef EARLY_ADVECT
    }
    const unsigned gf = (unsigned)((E.nlisted + bt - 1) / bt);
    if (L.dim == 2)
        early_fd_kernel<2><<<gf, bt, 0, s>>>(L, E.cells0, E.count, E.list, E.pos, E.adt, E.ftle);
    else
        early_fd_kernel<3><<<gf, bt, 0, s>>>(L, E.cells0, E.count, E.list, E.pos, E.adt, E.ftle);
    return cudaGetLastError();
}
