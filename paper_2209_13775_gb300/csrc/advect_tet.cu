// advect_tet.cu -- advection on tetrahedral and triangle meshes (RK4) and adaptive
// Dormand-Prince 5(4) with one step size per warp (meshes and rectilinear fields).
//
// Paper: Eq. 2 integrated with a Runge-Kutta method (Sec. 2 "Flow Map"); on
// unstructured data every stage evaluation needs a cell search (Sec. 3.1: local
// search on tetrahedra) before the interpolation.  The paper launches a search
// kernel and an interpolation kernel per stage; here one thread walks from the cell
// of its previous stage and interpolates in the same pass.
//
// The adaptive integrator keeps one step size per warp of 32 consecutive seeds: a
// step is accepted only when every live lane's error norm is at most 1 (__all_sync),
// and the next step size is the smallest lane proposal (__reduce_min_sync), so the
// warp's lanes never diverge in time.  Tracers whose stage point leaves the mesh stop
// (status LEFT, frozen at the start of that step) and stop voting.
#include "rect_device.cuh"
#include "tri_device.cuh"
#include "dp45_args.cuh"

#include <math.h>

// ------------------------------------------------------------------ RK4 on tets

// tracer state into flow-map slot `slot` (mesh fields: no periodic images): x + c rounded once
template <int DIM>
__device__ __forceinline__ void mesh_store(const Rk4Args &A, int slot, long long i, const float *x, const float *c,
                                           unsigned char st, float te)
{
    float *o = A.out_xyz + (size_t)slot * DIM * A.N;
#pragma unroll
    for (int d = 0; d < DIM; ++d) o[d * A.N + i] = x[d] + c[d];
    A.out_status[(size_t)slot * A.N + i] = st;
    A.out_texit[(size_t)slot * A.N + i] = te;
}

template <int ST>
__global__ void __launch_bounds__(256) rk4_tet_kernel(TetDev T, Rk4Args A, const int *__restrict__ cells0,
                                                      unsigned *errword)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int job = blockIdx.y;
    if (i >= A.N) return;
    float x[3] = {A.seeds[i], A.seeds[A.N + i], A.seeds[2 * A.N + i]}, cx[3] = {0.0f, 0.0f, 0.0f};
    int cell = cells0[i];
    unsigned char st = LCS_TRACER_OK;
    float te = A.job_tend[job];
    if (cell < 0) {
        st = LCS_TRACER_OUTSIDE;
        te = A.job_t0[job];
    }
    const SchedEntry *sc = A.sched + (size_t)job * A.nsteps_max * 3;
    const int ns = A.job_nsteps[job];
    const float h = A.job_h[job], hh = 0.5f * h;
    int si = 0;   // next snapshot
    for (int n = 0; n < ns && st == LCS_TRACER_OK; ++n) {
        const SchedEntry e[3] = {load_sched(sc + 3 * n), load_sched(sc + 3 * n + 1), load_sched(sc + 3 * n + 2)};
        float k[4][3], y[3], lam[4];
        int r = TET_INSIDE;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const float c = s == 0 ? 0.0f : (s == 3 ? h : hh);
#pragma unroll
            for (int q = 0; q < 3; ++q) y[q] = s == 0 ? x[q] : fmaf(c, k[s - 1][q], x[q]);
            const SchedEntry &es = e[s == 0 ? 0 : (s == 3 ? 2 : 1)];
            r = tet_locate(T, y, &cell, lam);
            if (r != TET_INSIDE) break;
            tet_interp<ST>(T, cell, lam, T.pairs + (size_t)es.k * T.fstride, es.a, k[s]);
        }
        if (r != TET_INSIDE) {  // a stage point left the mesh: freeze at the start of the step
            st = r == TET_OUTSIDE ? LCS_TRACER_LEFT : LCS_TRACER_WALKFAIL;
            if (r == TET_WALKFAIL) atomicOr(errword, LCS_ERRBIT_WALK);
            te = fmaf((float)n, h, A.job_t0[job]);
            break;
        }
        const float h6 = h * (1.0f / 6.0f);
#pragma unroll
        for (int q = 0; q < 3; ++q) rk4_advance(x[q], cx[q], h6, k[0][q], k[1][q], k[2][q], k[3][q]);
        for (; si < A.nsnap && snap_step(A, si, ns) == n + 1; ++si)
            mesh_store<3>(A, snap_slot(A, job, si), i, x, cx, st, snap_exit(A, job, si, st, te));
    }
    for (; si < A.nsnap; ++si)  // snapshots after the tracer stopped
        mesh_store<3>(A, snap_slot(A, job, si), i, x, cx, st, snap_exit(A, job, si, st, te));
    mesh_store<3>(A, job, i, x, cx, st, te);
}

// ------------------------------------------------------------- RK4 on triangles

template <int ST>
__global__ void __launch_bounds__(256) rk4_tri_kernel(TriDev T, Rk4Args A, const int *__restrict__ cells0,
                                                      unsigned *errword)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int job = blockIdx.y;
    if (i >= A.N) return;
    float x[2] = {A.seeds[i], A.seeds[A.N + i]}, cx[2] = {0.0f, 0.0f};
    int cell = cells0[i];
    unsigned char st = LCS_TRACER_OK;
    float te = A.job_tend[job];
    if (cell < 0) {
        st = LCS_TRACER_OUTSIDE;
        te = A.job_t0[job];
    }
    const SchedEntry *sc = A.sched + (size_t)job * A.nsteps_max * 3;
    const int ns = A.job_nsteps[job];
    const float h = A.job_h[job], hh = 0.5f * h;
    int si = 0;   // next snapshot
    TriCache cc;
    tri_cache_init(cc);
    for (int n = 0; n < ns && st == LCS_TRACER_OK; ++n) {
        const SchedEntry e[3] = {load_sched(sc + 3 * n), load_sched(sc + 3 * n + 1), load_sched(sc + 3 * n + 2)};
        float k[4][2], y[2], lam[3];
        int r = TET_INSIDE;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const float c = s == 0 ? 0.0f : (s == 3 ? h : hh);
#pragma unroll
            for (int q = 0; q < 2; ++q) y[q] = s == 0 ? x[q] : fmaf(c, k[s - 1][q], x[q]);
            const SchedEntry &es = e[s == 0 ? 0 : (s == 3 ? 2 : 1)];
            r = tri_locate_cached(T, y, &cell, lam, cc);
            if (r != TET_INSIDE) break;
            tri_interp_cached<ST>(T, cell, es.k, lam, T.pairs + (size_t)es.k * T.fstride, es.a, k[s], cc);
        }
        if (r != TET_INSIDE) {  // a stage point left the mesh: freeze at the start of the step
            st = r == TET_OUTSIDE ? LCS_TRACER_LEFT : LCS_TRACER_WALKFAIL;
            if (r == TET_WALKFAIL) atomicOr(errword, LCS_ERRBIT_WALK);
            te = fmaf((float)n, h, A.job_t0[job]);
            break;
        }
        const float h6 = h * (1.0f / 6.0f);
#pragma unroll
        for (int q = 0; q < 2; ++q) rk4_advance(x[q], cx[q], h6, k[0][q], k[1][q], k[2][q], k[3][q]);
        for (; si < A.nsnap && snap_step(A, si, ns) == n + 1; ++si)
            mesh_store<2>(A, snap_slot(A, job, si), i, x, cx, st, snap_exit(A, job, si, st, te));
    }
    for (; si < A.nsnap; ++si)  // snapshots after the tracer stopped
        mesh_store<2>(A, snap_slot(A, job, si), i, x, cx, st, snap_exit(A, job, si, st, te));
    mesh_store<2>(A, job, i, x, cx, st, te);
}

// ------------------------------------------------ variational equations on meshes

// RK4 with dM/dt = J M on tets (DIM 3, MD = TetDev) or triangles (DIM 2, TriDev): the position
// follows the plain mesh kernels' arithmetic (so x, status and exit time equal theirs), M the
// rectilinear variational kernel's, with the cell's constant P1 gradient as J
template <int DIM, int ST, class MD>
__global__ void __launch_bounds__(256) rk4_mesh_var_kernel(MD T, Rk4Args A, const int *__restrict__ cells0,
                                                           unsigned *errword)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int job = blockIdx.y;
    if (i >= A.N) return;
    float x[DIM], cx[DIM], M[DIM][DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        x[d] = A.seeds[d * A.N + i];
        cx[d] = 0.0f;
#pragma unroll
        for (int e = 0; e < DIM; ++e) M[d][e] = d == e ? 1.0f : 0.0f;
    }
    int cell = cells0[i];
    unsigned char st = LCS_TRACER_OK;
    float te = A.job_tend[job];
    if (cell < 0) {
        st = LCS_TRACER_OUTSIDE;
        te = A.job_t0[job];
    }
    TriCache tc;   // triangles only, and only its map (the tet branch never touches it)
    tri_cache_init(tc);
    const SchedEntry *sc = A.sched + (size_t)job * A.nsteps_max * 3;
    const int ns = A.job_nsteps[job];
    const float h = A.job_h[job], hh = 0.5f * h, h6 = h * (1.0f / 6.0f);
    for (int n = 0; n < ns && st == LCS_TRACER_OK; ++n) {
        const SchedEntry e[3] = {load_sched(sc + 3 * n), load_sched(sc + 3 * n + 1), load_sched(sc + 3 * n + 2)};
        float k[4][DIM], K[4][DIM][DIM], y[DIM], Y[DIM][DIM], lam[DIM + 1], J[DIM][DIM];
        int r = TET_INSIDE;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float c = q == 0 ? 0.0f : (q == 3 ? h : hh);
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                y[a] = q == 0 ? x[a] : fmaf(c, k[q - 1][a], x[a]);
#pragma unroll
                for (int b = 0; b < DIM; ++b) Y[a][b] = q == 0 ? M[a][b] : fmaf(c, K[q - 1][a][b], M[a][b]);
            }
            const SchedEntry &es = e[q == 0 ? 0 : (q == 3 ? 2 : 1)];
            const char *fp = T.pairs + (size_t)es.k * T.fstride;
            if constexpr (DIM == 3) {
                r = tet_locate(T, y, &cell, lam);
                if (r != TET_INSIDE) break;
                tet_interp_grad<ST>(T, cell, lam, fp, es.a, k[q], J);
            } else {
                r = tri_locate_cached(T, y, &cell, lam, tc);
                if (r != TET_INSIDE) break;
                tri_interp_grad<ST>(T, cell, tc.m, lam, fp, es.a, k[q], J);
            }
#pragma unroll
            for (int a = 0; a < DIM; ++a)
#pragma unroll
                for (int b = 0; b < DIM; ++b) {
                    float acc = 0.0f;
#pragma unroll
                    for (int cc = 0; cc < DIM; ++cc) acc = fmaf(J[a][cc], Y[cc][b], acc);
                    K[q][a][b] = acc;
                }
        }
        if (r != TET_INSIDE) {  // a stage point left the mesh: freeze at the start of the step
            st = r == TET_OUTSIDE ? LCS_TRACER_LEFT : LCS_TRACER_WALKFAIL;
            if (r == TET_WALKFAIL) atomicOr(errword, LCS_ERRBIT_WALK);
            te = fmaf((float)n, h, A.job_t0[job]);
            break;
        }
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            rk4_advance(x[a], cx[a], h6, k[0][a], k[1][a], k[2][a], k[3][a]);
#pragma unroll
            for (int b = 0; b < DIM; ++b)
                M[a][b] = fmaf(h6, (K[0][a][b] + K[3][a][b]) + 2.0f * (K[1][a][b] + K[2][a][b]), M[a][b]);
        }
    }
    mesh_store<DIM>(A, job, i, x, cx, st, te);
    float *o = A.out_grad + ((size_t)job * A.N + i) * DIM * DIM;
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
        for (int b = 0; b < DIM; ++b) o[a * DIM + b] = M[a][b];
}

// ------------------------------------------------------- time bracket (FP32)

// largest k with t_k <= t (after the periodic wrap), clamped to [0, nf-2]; the weight of
// frame k+1, clamped to [0, 1] unless time is periodic.  times: FP32 copy in shared memory
__device__ __forceinline__ void bracket_f32(const float *times, int nf, int tp, float period, float t, int &k,
                                            float &a)
{
    if (nf <= 1) {
        k = 0;
        a = 0.0f;
        return;
    }
    float tt = t;
    if (tp) tt = t - period * floorf((t - times[0]) / period);
    int lo = 0, hi = nf - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (times[mid] <= tt)
            lo = mid;
        else
            hi = mid - 1;
    }
    k = lo < nf - 2 ? lo : nf - 2;
    a = (tt - times[k]) / (times[k + 1] - times[k]);
    if (!tp) a = fminf(fmaxf(a, 0.0f), 1.0f);
}

// ------------------------------------------------------------ field evaluators

// per-thread state an evaluator keeps between its calls (none, or the triangle register cache)
struct NoEvalState {};
__device__ __forceinline__ void eval_state_init(NoEvalState &) {}
__device__ __forceinline__ void eval_state_init(TriCache &cc) { tri_cache_init(cc); }

// velocity at (x, t) on a tet mesh; walks from *cell.  Returns TET_INSIDE / OUTSIDE / WALKFAIL
template <int ST>
struct TetEval {
    static constexpr int DIM = 3;
    using State = NoEvalState;
    TetDev T;
    __device__ __forceinline__ int eval(const float *x, int k, float a, int *cell, float *u, State &) const
    {
        float lam[4];
        int r = tet_locate(T, x, cell, lam);
        if (r == TET_INSIDE) tet_interp<ST>(T, *cell, lam, T.pairs + (size_t)k * T.fstride, a, u);
        return r;
    }
};

// velocity at (x, t) on a triangle mesh; walks from *cell (the bin lists settle boundary edges)
template <int ST>
struct TriEval {
    static constexpr int DIM = 2;
    using State = TriCache;   // the seven stage points of a step mostly share a cell and an interval
    TriDev T;
    __device__ __forceinline__ int eval(const float *x, int k, float a, int *cell, float *u, State &cc) const
    {
        float lam[3];
        int r = tri_locate_cached<true>(T, x, cell, lam, cc);   // adaptive steps span many cells
        if (r == TET_INSIDE) tri_interp_cached<ST>(T, *cell, k, lam, T.pairs + (size_t)k * T.fstride, a, u, cc);
        return r;
    }
};

// velocity at (x, t) on a 2D rectilinear field of per-frame slabs (queries clamped into the box)
template <int ST>
struct Rect2Eval {
    static constexpr int DIM = 2;
    using State = NoEvalState;
    RectParams P;
    const char *frames;
    size_t fstride;
    __device__ __forceinline__ int eval(const float *x, int k, float a, int *cell, float *u, State &) const
    {
        Stencil<2> S;
        make_stencil<2>(P, x, S);
        interp<2, ST, SRC_GLOBAL>(S, frames + (size_t)k * fstride, frames + (size_t)(k + 1) * fstride, a, u);
        return TET_INSIDE;
    }
};

// velocity at (x, t) on a 3D rectilinear field of interval pairs (queries clamped into the box)
template <int ST>
struct Rect3Eval {
    static constexpr int DIM = 3;
    using State = NoEvalState;
    RectParams P;
    const char *pairs;
    size_t fstride;
    __device__ __forceinline__ int eval(const float *x, int k, float a, int *cell, float *u, State &) const
    {
        Stencil<3> S;
        make_stencil<3>(P, x, S);
        interp3p<ST>(S, pairs + (size_t)k * fstride, a, u);
        return TET_INSIDE;
    }
};

// ----------------------------------------------------------------- DP5(4)

// Dormand & Prince (1980) tableau
__constant__ float DPC[7] = {0.0f, 1.0f / 5.0f, 3.0f / 10.0f, 4.0f / 5.0f, 8.0f / 9.0f, 1.0f, 1.0f};
__constant__ float DPA[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0f / 5.0f, 0, 0, 0, 0, 0},
    {3.0f / 40.0f, 9.0f / 40.0f, 0, 0, 0, 0},
    {44.0f / 45.0f, -56.0f / 15.0f, 32.0f / 9.0f, 0, 0, 0},
    {19372.0f / 6561.0f, -25360.0f / 2187.0f, 64448.0f / 6561.0f, -212.0f / 729.0f, 0, 0},
    {9017.0f / 3168.0f, -355.0f / 33.0f, 46732.0f / 5247.0f, 49.0f / 176.0f, -5103.0f / 18656.0f, 0},
    {35.0f / 384.0f, 0.0f, 500.0f / 1113.0f, 125.0f / 192.0f, -2187.0f / 6784.0f, 11.0f / 84.0f}};
// b - b*: 5th-order weights minus embedded 4th-order weights
__constant__ float DPE[7] = {35.0f / 384.0f - 5179.0f / 57600.0f,
                             0.0f,
                             500.0f / 1113.0f - 7571.0f / 16695.0f,
                             125.0f / 192.0f - 393.0f / 640.0f,
                             -2187.0f / 6784.0f + 92097.0f / 339200.0f,
                             11.0f / 84.0f - 187.0f / 2100.0f,
                             -1.0f / 40.0f};

template <class EV>
__device__ __forceinline__ int dp_eval(const EV &E, const Dp45Args &A, const float *times, const float *x, float t,
                                       int *cell, float *u, typename EV::State &cs)
{
    int k;
    float a;
    bracket_f32(times, A.nf, A.tp, A.period, t, k, a);
    return E.eval(x, k, a, cell, u, cs);
}

template <class EV>
__global__ void __launch_bounds__(256, 4) dp45_kernel(EV E, Dp45Args A, RectParams P)
{
    extern __shared__ float s_times[];
    for (int q = threadIdx.x; q < A.nf; q += blockDim.x) s_times[q] = (float)A.times[q];
    __syncthreads();
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int job = blockIdx.y;
    const bool active = i < A.N;
    const unsigned FULL = 0xffffffffu;
    constexpr int D = EV::DIM;
    float x[D], k1[D];
#pragma unroll
    for (int q = 0; q < D; ++q) x[q] = k1[q] = 0.0f;
    int cell = 0, steps = 0;
    bool have_k1 = false;
    typename EV::State cs;
    eval_state_init(cs);
    unsigned char st = active ? LCS_TRACER_OK : LCS_TRACER_OUTSIDE;
    const float t0 = (float)A.job_t0[job];
    const float tend = (float)(A.job_t0[job] + A.job_T[job]);
    const float dir = A.job_T[job] < 0.0 ? -1.0f : 1.0f;
    float te = tend;
    if (active) {
#pragma unroll
        for (int q = 0; q < D; ++q) x[q] = A.seeds[q * A.N + i];
        if (A.cells0) {
            cell = A.cells0[i];
            if (cell < 0) {
                st = LCS_TRACER_OUTSIDE;
                te = t0;
            }
        }
    }
    float t = t0, h = dir * fabsf(A.h0);
    long long attempts = 0;
    for (;;) {
        bool live = st == LCS_TRACER_OK;
        if (!__any_sync(FULL, live)) break;
        if (dir * (tend - t) <= 0.0f) break;
        if (attempts >= A.max_steps) {
            if (live) {
                st = LCS_TRACER_MAXSTEPS;
                te = t;
                atomicOr(A.errword, LCS_ERRBIT_MAXSTEPS);
            }
            break;
        }
        const bool last = dir * (t + h - tend) >= 0.0f;
        const float hs = last ? tend - t : h;
        ++attempts;
        float err = 0.0f, xn[D], kk[7][D];
        int r = TET_INSIDE;
        if (live) {
            if (!have_k1) {
                r = dp_eval(E, A, s_times, x, t, &cell, k1, cs);
                if (r == TET_INSIDE) have_k1 = true;
            }
#pragma unroll
            for (int q = 0; q < D; ++q) kk[0][q] = k1[q];
#pragma unroll
            for (int s = 1; s < 7; ++s) {
                if (r != TET_INSIDE) break;
                float y[D];
#pragma unroll
                for (int q = 0; q < D; ++q) {
                    float acc = 0.0f;
#pragma unroll
                    for (int j = 0; j < 6; ++j)
                        if (j < s) acc = fmaf(DPA[s][j], kk[j][q], acc);
                    y[q] = fmaf(hs, acc, x[q]);
                }
                r = dp_eval(E, A, s_times, y, fmaf(DPC[s], hs, t), &cell, kk[s], cs);
            }
            if (r == TET_INSIDE) {
#pragma unroll
                for (int q = 0; q < D; ++q) {
                    float acc = 0.0f, ea = 0.0f;
#pragma unroll
                    for (int j = 0; j < 6; ++j) acc = fmaf(DPA[6][j], kk[j][q], acc);
#pragma unroll
                    for (int s = 0; s < 7; ++s) ea = fmaf(DPE[s], kk[s][q], ea);
                    xn[q] = fmaf(hs, acc, x[q]);
                    const float sc = A.atol + A.rtol * fmaxf(fabsf(x[q]), fabsf(xn[q]));
                    err = fmaxf(err, fabsf(hs * ea) / sc);
                }
            } else {  // a stage point left the mesh: freeze at the start of the step, stop voting
                st = r == TET_OUTSIDE ? LCS_TRACER_LEFT : LCS_TRACER_WALKFAIL;
                if (r == TET_WALKFAIL) atomicOr(A.errword, LCS_ERRBIT_WALK);
                te = t;
                live = false;
            }
        }
        const bool all_ok = __all_sync(FULL, !live || err <= 1.0f);
        float prop = INFINITY;
        if (live) {
            float f = err == 0.0f ? 5.0f : fminf(5.0f, fmaxf(0.2f, 0.9f * __powf(err, -0.2f)));
            prop = fabsf(hs * f);
        }
        const unsigned pm = __reduce_min_sync(FULL, __float_as_uint(prop));
        if (all_ok) {
            if (live) {
#pragma unroll
                for (int q = 0; q < D; ++q) {
                    x[q] = xn[q];
                    k1[q] = kk[6][q];
                }
                ++steps;
                if (A.rect_left && rect_left<D>(P, x)) {
                    st = LCS_TRACER_LEFT;
                    te = last ? tend : t + hs;
                }
            }
            t = last ? tend : t + hs;
        }
        if (pm != __float_as_uint(INFINITY)) h = dir * __uint_as_float(pm);
    }
    if (!active) return;
    float *o = A.out_xyz + (size_t)job * D * A.N;
#pragma unroll
    for (int q = 0; q < D; ++q) o[q * A.N + i] = x[q];
    A.out_status[(size_t)job * A.N + i] = st;
    A.out_texit[(size_t)job * A.N + i] = te;
    if (A.out_steps) A.out_steps[(size_t)job * A.N + i] = steps;
}

// ------------------------------------------------------------------ launchers

cudaError_t launch_rk4_tet(lcs_ctx *ctx, const Rk4Launch &L, const int *cells0, int walk_limit, cudaStream_t s)
{
    const lcs_field *f = L.field;
    Rk4Args A;
    A.seeds = L.seeds;
    A.N = L.N;
    A.nsteps_max = L.nsteps_max;
    A.sched = L.sched;
    A.job_nsteps = L.job_nsteps;
    A.job_h = L.job_h;
    A.job_t0 = L.job_t0;
    A.job_tend = L.job_tend;
    A.out_xyz = L.out_xyz;
    A.out_status = L.out_status;
    A.out_texit = L.out_texit;
    A.njobs = L.njobs;
    A.nsnap = L.nsnap;
    A.snap_n = L.snap_n;
    A.snap_te = L.snap_te;
    A.out_grad = L.out_grad;
    if (L.N == 0) return cudaSuccess;
    const int bt = L.block_threads > 0 && L.block_threads <= 256 ? L.block_threads : 128;
    dim3 grid((unsigned)((L.N + bt - 1) / bt), (unsigned)L.njobs);
    if (A.out_grad) {   // the variational equations
        lcs_tm_begin(ctx, 0, s);
        if (f->kind == LCS_TRI) {
            const TriDev T = tri_dev(f, walk_limit);
            if (f->storage == LCS_F32)
                rk4_mesh_var_kernel<2, LCS_F32><<<grid, bt, 0, s>>>(T, A, cells0, ctx->d_errword);
            else if (f->storage == LCS_F16)
                rk4_mesh_var_kernel<2, LCS_F16><<<grid, bt, 0, s>>>(T, A, cells0, ctx->d_errword);
            else
                rk4_mesh_var_kernel<2, LCS_BF16><<<grid, bt, 0, s>>>(T, A, cells0, ctx->d_errword);
        } else {
            const TetDev T = tet_dev(f, walk_limit);
            if (f->storage == LCS_F32)
                rk4_mesh_var_kernel<3, LCS_F32><<<grid, bt, 0, s>>>(T, A, cells0, ctx->d_errword);
            else if (f->storage == LCS_F16)
                rk4_mesh_var_kernel<3, LCS_F16><<<grid, bt, 0, s>>>(T, A, cells0, ctx->d_errword);
            else
                rk4_mesh_var_kernel<3, LCS_BF16><<<grid, bt, 0, s>>>(T, A, cells0, ctx->d_errword);
        }
        lcs_tm_end(ctx, 0, s);
        return cudaGetLastError();
    }
    if (f->kind == LCS_TRI) {
        const TriDev T = tri_dev(f, walk_limit);
        lcs_tm_begin(ctx, 0, s);
        if (f->storage == LCS_F32)
            rk4_tri_kernel<LCS_F32><<<grid, bt, 0, s>>>(T, A, cells0, ctx->d_errword);
        else if (f->storage == LCS_F16)
            rk4_tri_kernel<LCS_F16><<<grid, bt, 0, s>>>(T, A, cells0, ctx->d_errword);
        else
            rk4_tri_kernel<LCS_BF16><<<grid, bt, 0, s>>>(T, A, cells0, ctx->d_errword);
        lcs_tm_end(ctx, 0, s);
        return cudaGetLastError();
    }
    const TetDev T = tet_dev(f, walk_limit);
    lcs_tm_begin(ctx, 0, s);
    if (f->storage == LCS_F32)
        rk4_tet_kernel<LCS_F32><<<grid, bt, 0, s>>>(T, A, cells0, ctx->d_errword);
    else if (f->storage == LCS_F16)
        rk4_tet_kernel<LCS_F16><<<grid, bt, 0, s>>>(T, A, cells0, ctx->d_errword);
    else
        rk4_tet_kernel<LCS_BF16><<<grid, bt, 0, s>>>(T, A, cells0, ctx->d_errword);
    lcs_tm_end(ctx, 0, s);
    return cudaGetLastError();
}

template <class EV>
static cudaError_t dp45_go(const EV &E, const Dp45Args &A, const RectParams &P, int njobs, int bt, cudaStream_t s)
{
    dim3 grid((unsigned)((A.N + bt - 1) / bt), (unsigned)njobs);
    size_t smem = sizeof(float) * (size_t)(A.nf > 0 ? A.nf : 1);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(dp45_kernel<EV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dp45_kernel<EV><<<grid, bt, smem, s>>>(E, A, P);
    return cudaGetLastError();
}

cudaError_t launch_dp45(lcs_ctx *ctx, const lcs_field *f, const Dp45Args &A0, int njobs, int block_threads,
                        int walk_limit, cudaStream_t s)
{
    if (A0.N == 0 || njobs == 0) return cudaSuccess;
    Dp45Args A = A0;
    A.errword = ctx->d_errword;
    A.times = f->d_times;
    A.nf = f->nframes;
    A.tp = f->time_periodic;
    A.period = (float)f->period;
    int bt = block_threads > 0 && block_threads <= 256 ? (block_threads / 32) * 32 : 128;
    if (bt < 32) bt = 32;
    cudaError_t e;
    lcs_tm_begin(ctx, 0, s);
    RectParams P = make_rect_params(f);
    if (f->kind == LCS_TRI) {
        A.rect_left = 0;
        const TriDev T = tri_dev(f, walk_limit);
        if (f->storage == LCS_F32)
            e = dp45_go(TriEval<LCS_F32>{T}, A, P, njobs, bt, s);
        else if (f->storage == LCS_F16)
            e = dp45_go(TriEval<LCS_F16>{T}, A, P, njobs, bt, s);
        else
            e = dp45_go(TriEval<LCS_BF16>{T}, A, P, njobs, bt, s);
    } else if (f->kind == LCS_TET) {
        A.rect_left = 0;
        const TetDev T = tet_dev(f, walk_limit);
        if (f->storage == LCS_F32)
            e = dp45_go(TetEval<LCS_F32>{T}, A, P, njobs, bt, s);
        else if (f->storage == LCS_F16)
            e = dp45_go(TetEval<LCS_F16>{T}, A, P, njobs, bt, s);
        else
            e = dp45_go(TetEval<LCS_BF16>{T}, A, P, njobs, bt, s);
    } else if (f->dim == 2) {
        A.rect_left = 1;
        const char *fr = (const char *)f->d_frames;
        if (f->storage == LCS_F32)
            e = dp45_go(Rect2Eval<LCS_F32>{P, fr, f->frame_stride}, A, P, njobs, bt, s);
        else if (f->storage == LCS_F16)
            e = dp45_go(Rect2Eval<LCS_F16>{P, fr, f->frame_stride}, A, P, njobs, bt, s);
        else
            e = dp45_go(Rect2Eval<LCS_BF16>{P, fr, f->frame_stride}, A, P, njobs, bt, s);
    } else {
        A.rect_left = 1;
        if (f->storage == LCS_F32)
            e = dp45_go(Rect3Eval<LCS_F32>{P, (const char *)f->d_frames, f->frame_stride}, A, P, njobs, bt, s);
        else if (f->storage == LCS_F16)
            e = dp45_go(Rect3Eval<LCS_F16>{P, (const char *)f->d_frames, f->frame_stride}, A, P, njobs, bt, s);
        else
            e = dp45_go(Rect3Eval<LCS_BF16>{P, (const char *)f->d_frames, f->frame_stride}, A, P, njobs, bt, s);
    }
    lcs_tm_end(ctx, 0, s);
    return e;
}
