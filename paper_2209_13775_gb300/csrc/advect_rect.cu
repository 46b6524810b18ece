// advect_rect.cu -- fixed-step RK4 advection through rectilinear velocity frames.
//
// Paper: Eq. 2 integrated over (t0, t0 + T) from a structured seed grid with
// the classical 4th-order Runge-Kutta method (Sec. 2 "Flow Map", Sec. 3.1),
// velocity interpolated bilinearly / trilinearly in space and linearly in time
// between two frames (Sec. 2 "Interpolator").
//
// Design (differs from the paper's split kernels, Sec. 3.1): one thread owns one
// tracer for the whole integration, with its state in registers; a step is
// four fused stage evaluations.  All tracers of a launch share the time
// schedule, so the frame bracket (k, alpha) of every stage is computed once
// per (job, step, stage) in FP64 by a small kernel and read as a warp-uniform
// broadcast.  Two kernels:
//   * gather: nodes read through L1/L2 (any field size, 2D and 3D);
//   * ring (2D): a block keeps three whole frames in shared memory, staged by
//     bulk asynchronous copies (cp.async.bulk + mbarrier) and prefetched one
//     step ahead, so the stage evaluations read shared memory only.
#include "rect_device.cuh"

#include <math.h>

// ===================================================================== schedule

// Stage time of (step n, stage s): t_n = t0 + n h; s = 0: t_n, 1: t_n + h/2, 2: t_n + h.
// Round-to-nearest FP64 operations, no fused multiply-add.
__device__ __forceinline__ double stage_time(double t0, double h, int n, int s)
{
    double t = __dadd_rn(t0, __dmul_rn((double)n, h));
    if (s == 1) t = __dadd_rn(t, __dmul_rn(0.5, h));
    if (s == 2) t = __dadd_rn(t, h);
    return t;
}

// frame bracket: largest k with t_k <= t (after the periodic wrap), clamped to [0, nf-2];
// alpha = (t - t_k) / (t_{k+1} - t_k), clamped to [0, 1] unless time is periodic
__device__ void frame_bracket(const double *__restrict__ times, int nf, int tp, double period, double t,
                              int *k, double *alpha)
{
    if (nf <= 1) {
        *k = 0;
        *alpha = 0.0;
        return;
    }
    double tt = t;
    if (tp) tt = __dsub_rn(t, __dmul_rn(period, floor(__ddiv_rn(__dsub_rn(t, times[0]), period))));
    int lo = 0, hi = nf - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (times[mid] <= tt)
            lo = mid;
        else
            hi = mid - 1;
    }
    int kk = lo < nf - 2 ? lo : nf - 2;
    double a = __ddiv_rn(__dsub_rn(tt, times[kk]), __dsub_rn(times[kk + 1], times[kk]));
    if (!tp) a = fmin(fmax(a, 0.0), 1.0);
    *k = kk;
    *alpha = a;
}

__global__ void rk4_schedule_kernel(const double *__restrict__ times, int nf, int tp, double period,
                                    const JobTable J, JobDev D, SchedEntry *__restrict__ sched)
{
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int nsm = J.nsteps_max;
    long long total = (long long)J.njobs * nsm * 3;
    if (idx < J.njobs) {
        int j = (int)idx;
        D.nsteps[j] = J.nsteps[j];
        D.h[j] = __double2float_rn(J.h[j]);
        D.t0[j] = __double2float_rn(J.t0[j]);
        D.tend[j] = __double2float_rn(__dadd_rn(J.t0[j], J.T[j]));
        D.absT[j] = fabs(J.T[j]);
        for (int q = 0; q < J.nsnap; ++q)   // snapshot slots: |T| of the horizon they hold
            D.absT[J.njobs + j * J.nsnap + q] = fmin(J.snap_T[q], fabs(J.T[j]));
        if (j == 0 && D.snap_n)
            for (int q = 0; q < J.nsnap; ++q) D.snap_n[q] = J.snap_n[q];
        if (D.snap_te)   // t0 + T of the horizon a snapshot holds, as a run with that horizon computes it
            for (int q = 0; q < J.nsnap; ++q) {
                const double a = fmin(J.snap_T[q], fabs(J.T[j]));
                D.snap_te[j * J.nsnap + q] = __double2float_rn(__dadd_rn(J.t0[j], J.T[j] < 0.0 ? -a : a));
            }
        if (D.order) D.order[j] = J.order[j];
        if (D.t0d) D.t0d[j] = J.t0[j];
        if (D.Td) D.Td[j] = J.T[j];
    }
    if (idx >= total || !sched) return;
    int s = (int)(idx % 3);
    int n = (int)((idx / 3) % nsm);
    int job = (int)(idx / (3LL * nsm));
    SchedEntry e = {0, 0.0f};
    if (n < J.nsteps[job]) {
        int k;
        double a;
        frame_bracket(times, nf, tp, period, stage_time(J.t0[job], J.h[job], n, s), &k, &a);
        e.k = k;
        e.a = __double2float_rn(a);
    }
    sched[idx] = e;
}

cudaError_t launch_rk4_schedule(const double *d_times, int nframes, int time_periodic, double period,
                                const JobTable &J, JobDev D, SchedEntry *d_sched, cudaStream_t s)
{
    long long total = (long long)J.njobs * J.nsteps_max * 3;
    if (total < J.njobs) total = J.njobs;
    if (total == 0) return cudaSuccess;
    int bt = 256;
    unsigned grid = (unsigned)((total + bt - 1) / bt);
    rk4_schedule_kernel<<<grid, bt, 0, s>>>(d_times, nframes, time_periodic, period, J, D, d_sched);
    return cudaGetLastError();
}

// ============================================================ gather kernel

template <int DIM, int ST>
__global__ void __launch_bounds__(256) rk4_gather_kernel(RectParams P, const char *__restrict__ frames,
                                                         size_t fstride, Rk4Args A)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    int job = blockIdx.y;
    if (i >= A.N) return;
    float x[DIM], cx[DIM];
    int img[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        x[d] = A.seeds[d * A.N + i];
        cx[d] = 0.0f;
        img[d] = 0;
    }
    wrap_periodic<DIM>(P, x, cx, img);
    const SchedEntry *sc = A.sched + (size_t)job * A.nsteps_max * 3;
    const int ns = A.job_nsteps[job];
    const float h = A.job_h[job];
    unsigned char st = LCS_TRACER_OK;
    float te = A.job_tend[job];
    int si = 0;   // next snapshot
    for (int n = 0; n < ns; ++n) {
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
        if (rect_left<DIM>(P, x)) {
            st = LCS_TRACER_LEFT;
            te = fmaf((float)(n + 1), h, A.job_t0[job]);
            break;
        }
        for (; si < A.nsnap && snap_step(A, si, ns) == n + 1; ++si)
            store_tracer<DIM>(P, A, snap_slot(A, job, si), i, x, cx, img, st, snap_exit(A, job, si, st, te));
    }
    for (; si < A.nsnap; ++si)  // snapshots after the tracer stopped (or of a zero-step job)
        store_tracer<DIM>(P, A, snap_slot(A, job, si), i, x, cx, img, st, snap_exit(A, job, si, st, te));
    store_tracer<DIM>(P, A, job, i, x, cx, img, st, te);
}

// ============================================================ variational

// u and its spatial Jacobian J[c][d] at x, linear in time between two frames: u with
// interp's arithmetic (node blends first, then make_stencil's weights in order), J from the
// same blended corner values and the derivatives of the weights inside the cell; a
// non-periodic axis on which x lies outside the box gives a zero column (the clamped query
// does not move with x).
template <int DIM, int ST>
__device__ __forceinline__ void interp_grad(const RectParams &P, const float *x, const char *fa, const char *fb,
                                            float a, float *u, float (*J)[DIM])
{
    Stencil<DIM> S;
    make_stencil<DIM>(P, x, S);
    float f[DIM], on[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        int i0, i1;
        axis_cell<-1>(P, d, x[d], i0, i1, f[d]);
        on[d] = (P.periodic[d] || (x[d] >= P.origin[d] && x[d] <= P.hi_node[d])) ? P.inv_h[d] : 0.0f;
    }
    float uq[1 << DIM][DIM], va[DIM], vb[DIM];
    const float g = 1.0f - a;
#pragma unroll
    for (int q = 0; q < (1 << DIM); ++q) {
        if constexpr (DIM == 2) {   // frames: fa = frame k, fb = frame k + 1 (read only when a != 0)
            node_load<2, ST, SRC_GLOBAL>(fa, S.v[q], va);
            if (a != 0.0f) node_load<2, ST, SRC_GLOBAL>(fb, S.v[q], vb);
        } else {                    // interval pairs: fa = pair k holds both frames of a node
            Pair3<ST>::ld(fa, S.v[q], va, vb);
        }
#pragma unroll
        for (int c = 0; c < DIM; ++c) uq[q][c] = a == 0.0f ? va[c] : tblend(va[c], vb[c], a, g);
    }
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        float acc = 0.0f;
#pragma unroll
        for (int q = 0; q < (1 << DIM); ++q) acc = fmaf(S.w[q], uq[q][c], acc);
        u[c] = acc;
    }
    // corner q has offsets (q & 1, (q >> 1) & 1, (q >> 2) & 1); d w_q / d x_d = +-(product of the
    // other axes' weights) / h_d
#pragma unroll
    for (int c = 0; c < DIM; ++c)
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            float acc = 0.0f;
#pragma unroll
            for (int q = 0; q < (1 << DIM); ++q) {
                float w = ((q >> d) & 1) ? 1.0f : -1.0f;
#pragma unroll
                for (int e = 0; e < DIM; ++e)
                    if (e != d) w *= ((q >> e) & 1) ? f[e] : 1.0f - f[e];
                acc = fmaf(w, uq[q][c], acc);
            }
            J[c][d] = acc * on[d];
        }
}

// RK4 with the variational equations dM/dt = J M: the position follows rk4_step's arithmetic
// exactly (so x(T) equals the other kernels'), M the same stages in FP32
template <int DIM, int ST>
__global__ void __launch_bounds__(256) rk4_var_kernel(RectParams P, const char *__restrict__ frames, size_t fstride,
                                                      Rk4Args A)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int job = blockIdx.y;
    if (i >= A.N) return;
    float x[DIM], cx[DIM], M[DIM][DIM];
    int img[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        x[d] = A.seeds[d * A.N + i];
        cx[d] = 0.0f;
        img[d] = 0;
#pragma unroll
        for (int e = 0; e < DIM; ++e) M[d][e] = d == e ? 1.0f : 0.0f;
    }
    wrap_periodic<DIM>(P, x, cx, img);
    const SchedEntry *sc = A.sched + (size_t)job * A.nsteps_max * 3;
    const int ns = A.job_nsteps[job];
    const float h = A.job_h[job], hh = 0.5f * h, h6 = h * (1.0f / 6.0f);
    unsigned char st = LCS_TRACER_OK;
    float te = A.job_tend[job];
    for (int n = 0; n < ns; ++n) {
        const SchedEntry es[3] = {load_sched(sc + 3 * n), load_sched(sc + 3 * n + 1), load_sched(sc + 3 * n + 2)};
        float k[4][DIM], K[4][DIM][DIM], y[DIM], Y[DIM][DIM], J[DIM][DIM];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const SchedEntry e = es[q == 0 ? 0 : (q == 3 ? 2 : 1)];
            const float c = q == 0 ? 0.0f : (q == 3 ? h : hh);
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                y[a] = q == 0 ? x[a] : fmaf(c, k[q - 1][a], x[a]);
#pragma unroll
                for (int b = 0; b < DIM; ++b) Y[a][b] = q == 0 ? M[a][b] : fmaf(c, K[q - 1][a][b], M[a][b]);
            }
            const char *fa = frames + (size_t)e.k * fstride;
            interp_grad<DIM, ST>(P, y, fa, DIM == 2 ? fa + fstride : fa, e.a, k[q], J);
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
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            rk4_advance(x[a], cx[a], h6, k[0][a], k[1][a], k[2][a], k[3][a]);
#pragma unroll
            for (int b = 0; b < DIM; ++b)
                M[a][b] = fmaf(h6, (K[0][a][b] + K[3][a][b]) + 2.0f * (K[1][a][b] + K[2][a][b]), M[a][b]);
        }
        wrap_periodic<DIM>(P, x, cx, img);
        if (rect_left<DIM>(P, x)) {
            st = LCS_TRACER_LEFT;
            te = fmaf((float)(n + 1), h, A.job_t0[job]);
            break;
        }
    }
    store_tracer<DIM>(P, A, job, i, x, cx, img, st, te);
    float *o = A.out_grad + ((size_t)job * A.N + i) * DIM * DIM;
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
        for (int b = 0; b < DIM; ++b) o[a * DIM + b] = M[a][b];
}

// ============================================================== ring kernel

// Three frame slots in shared memory, tagged with the frame they hold.  Thread 0
// makes the frames of step n resident (bulk copies into slots no stage of step n
// needs), prefetches those of step n + 1 into a free slot, and publishes the
// slot of every stage frame; a frame that cannot get a slot is read from global
// memory for that step.
#define RING_SLOTS 3
#define RING_GLOBAL (-2)
#define RING_NONE (-1)

struct RingState {
    uint64_t bar[RING_SLOTS];
    int tag[RING_SLOTS];
    unsigned nload[RING_SLOTS];
    int slot[6];   // per stage (0..2): slot of frame k, slot of frame k + 1 (or NONE / GLOBAL)
    int kf[6];     // frame ids for the GLOBAL case
    int abort;     // a wait timed out: the block stops issuing copies and computing
};

struct RingWork {
    int persistent;        // 0: block (x, y) = tile x of job y; 1: items pulled from *queue
    unsigned *queue;       // persistent: item counter, zero at launch
    long long nitems;      // persistent: tiles_per_job * njobs
    int tiles_per_job;
    const int *jorder;     // persistent: job of rank r, longest first
};

__device__ __forceinline__ int ring_find(const RingState &R, int f)
{
    for (int s = 0; s < RING_SLOTS; ++s)
        if (R.tag[s] == f) return s;
    return -1;
}

// frames a step reads: k of each stage, and k + 1 where alpha != 0
__device__ __forceinline__ int step_frames(const SchedEntry *e, int *F)
{
    int m = 0;
    for (int s = 0; s < 3; ++s) {
        int c[2] = {e[s].k, e[s].a != 0.0f ? e[s].k + 1 : -1};
        for (int q = 0; q < 2; ++q) {
            if (c[q] < 0) continue;
            bool dup = false;
            for (int r = 0; r < m; ++r) dup |= (F[r] == c[q]);
            if (!dup) F[m++] = c[q];
        }
    }
    return m;
}

__device__ __forceinline__ bool in_list(const int *F, int m, int f)
{
    for (int r = 0; r < m; ++r)
        if (F[r] == f) return true;
    return false;
}

// thread 0: load frame f into a slot that holds none of the protected frames
__device__ int ring_load(RingState &R, char *slots, const char *frames, size_t fstride, int f, const int *keep,
                         int nkeep, unsigned *errword, uint64_t wait_ns)
{
    int v = -1;
    for (int s = 0; s < RING_SLOTS && v < 0; ++s)
        if (R.tag[s] < 0) v = s;
    for (int s = 0; s < RING_SLOTS && v < 0; ++s)
        if (!in_list(keep, nkeep, R.tag[s])) v = s;
    if (v < 0) return RING_GLOBAL;
    if (R.nload[v] > 0 && !mbar_wait_limit(&R.bar[v], (R.nload[v] - 1) & 1, wait_ns)) {  // previous copy into v
        atomicOr(errword, LCS_ERRBIT_TIMEOUT);
        R.abort = 1;
        return RING_GLOBAL;
    }
    R.tag[v] = f;
    R.nload[v] += 1;
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&R.bar[v], (unsigned)fstride);
    bulk_g2s(slots + (size_t)v * fstride, frames + (size_t)f * fstride, (unsigned)fstride, &R.bar[v]);
    return v;
}

// Work of one block: the tracers [tile * TPT * bt, (tile + 1) * TPT * bt) of one job, each
// thread holding TPT tracers (sub-tiles of bt consecutive seeds, so loads stay coalesced).
template <int ST, int TPT>
__device__ __forceinline__ void ring_tile(const RectParams &P, const char *__restrict__ frames, size_t fstride,
                                          const Rk4Args &A, unsigned *errword, char *slots, RingState &R, int job,
                                          long long tile)
{
    const int tid = threadIdx.x, bt = blockDim.x;
    long long idx[TPT];
    bool active[TPT], live[TPT];
    float x[TPT][2], cx[TPT][2];
    int img[TPT][2];
    unsigned char st[TPT];
    float te[TPT];
    const float tend = A.job_tend[job];
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        idx[t] = (tile * TPT + t) * bt + tid;
        active[t] = idx[t] < A.N;
        live[t] = active[t];
        x[t][0] = active[t] ? A.seeds[idx[t]] : 0.0f;
        x[t][1] = active[t] ? A.seeds[A.N + idx[t]] : 0.0f;
        cx[t][0] = cx[t][1] = 0.0f;
        img[t][0] = img[t][1] = 0;
        wrap_periodic<2>(P, x[t], cx[t], img[t]);
        st[t] = LCS_TRACER_OK;
        te[t] = tend;
    }
    const SchedEntry *sc = A.sched + (size_t)job * A.nsteps_max * 3;
    const int ns = A.job_nsteps[job];
    const float h = A.job_h[job];
    int si = 0;   // next snapshot
    for (int n = 0; n < ns; ++n) {
        __syncthreads();  // every thread is done with the previous step's slots
        if (R.abort) break;
        if (tid == 0) {
            SchedEntry e[3] = {sc[3 * n], sc[3 * n + 1], sc[3 * n + 2]};
            int F[6], Fn[6];
            int m = step_frames(e, F);
            for (int r = 0; r < m; ++r)
                if (ring_find(R, F[r]) < 0) ring_load(R, slots, frames, fstride, F[r], F, m, errword, A.wait_ns);
            for (int s = 0; s < 3; ++s) {
                int fa = e[s].k, fb = e[s].k + 1;
                int sa = ring_find(R, fa);
                R.slot[2 * s] = sa >= 0 ? sa : RING_GLOBAL;
                R.kf[2 * s] = fa;
                if (e[s].a != 0.0f) {
                    int sb = ring_find(R, fb);
                    R.slot[2 * s + 1] = sb >= 0 ? sb : RING_GLOBAL;
                } else {
                    R.slot[2 * s + 1] = RING_NONE;
                }
                R.kf[2 * s + 1] = fb;
            }
            if (n + 1 < ns) {  // prefetch the next step's frames into slots this step leaves alone
                SchedEntry en[3] = {sc[3 * n + 3], sc[3 * n + 4], sc[3 * n + 5]};
                int mn = step_frames(en, Fn);
                int keep[12];
                int nk = 0;
                for (int r = 0; r < m; ++r) keep[nk++] = F[r];
                for (int r = 0; r < mn; ++r) keep[nk++] = Fn[r];
                for (int r = 0; r < mn; ++r)
                    if (ring_find(R, Fn[r]) < 0) ring_load(R, slots, frames, fstride, Fn[r], keep, nk, errword, A.wait_ns);
            }
        }
        __syncthreads();
        // wait for the copies this step reads
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            int s = R.slot[q];
            if (s >= 0 && !R.abort && !mbar_wait_limit(&R.bar[s], (R.nload[s] - 1) & 1, A.wait_ns)) {
                atomicOr(errword, LCS_ERRBIT_TIMEOUT);
                R.abort = 1;
            }
        }
        if (R.abort) continue;
        const char *p[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            int s = R.slot[q];
            if (s >= 0)
                p[q] = slots + (size_t)s * fstride;
            else if (s == RING_NONE)
                p[q] = p[q - 1];  // alpha == 0: frame k + 1 is never read; keep a pointer of the same space
            else
                p[q] = frames + (size_t)R.kf[q] * fstride;
        }
        const SchedEntry e0 = load_sched(sc + 3 * n), e1 = load_sched(sc + 3 * n + 1), e2 = load_sched(sc + 3 * n + 2);
        const bool all_smem = (R.slot[0] != RING_GLOBAL) && (R.slot[1] != RING_GLOBAL) &&
                              (R.slot[2] != RING_GLOBAL) && (R.slot[3] != RING_GLOBAL) &&
                              (R.slot[4] != RING_GLOBAL) && (R.slot[5] != RING_GLOBAL);
#pragma unroll
        for (int t = 0; t < TPT; ++t) {
            if (!live[t]) continue;
            // a step whose frames did not all get a slot (e.g. one straddling the periodic wrap, which
            // reads four frames) mixes shared and global pointers: generic loads serve both
            if (all_smem)
                rk4_step<2, ST, SRC_SHARED>(P, x[t], cx[t], h, p[0], p[1], e0.a, p[2], p[3], e1.a, p[4], p[5],
                                            e2.a);
            else
                rk4_step<2, ST, SRC_GENERIC>(P, x[t], cx[t], h, p[0], p[1], e0.a, p[2], p[3], e1.a, p[4], p[5],
                                             e2.a);
            wrap_periodic<2>(P, x[t], cx[t], img[t]);
            if (rect_left<2>(P, x[t])) {
                st[t] = LCS_TRACER_LEFT;
                te[t] = fmaf((float)(n + 1), h, A.job_t0[job]);
                live[t] = false;
            }
        }
        for (; si < A.nsnap && snap_step(A, si, ns) == n + 1; ++si)
#pragma unroll
            for (int t = 0; t < TPT; ++t)
                if (active[t])
                    store_tracer<2>(P, A, snap_slot(A, job, si), idx[t], x[t], cx[t], img[t], st[t],
                                    snap_exit(A, job, si, st[t], te[t]));
    }
    for (; si < A.nsnap; ++si)  // a zero-step job, or a block that stopped on a copy timeout
#pragma unroll
        for (int t = 0; t < TPT; ++t)
            if (active[t])
                store_tracer<2>(P, A, snap_slot(A, job, si), idx[t], x[t], cx[t], img[t], st[t],
                                snap_exit(A, job, si, st[t], te[t]));
#pragma unroll
    for (int t = 0; t < TPT; ++t)
        if (active[t]) store_tracer<2>(P, A, job, idx[t], x[t], cx[t], img[t], st[t], te[t]);
}

// Ring kernel.  Non-persistent: block (x, y) is tile x of job y.  Persistent: the grid
// fills the GPU once and every block pulls (job, tile) items from an atomic counter in
// the order of W.jorder (longest jobs first), keeping its frame ring across items.
template <int ST, int TPT>
__global__ void __launch_bounds__(512, 1) rk4_ring2d_kernel(RectParams P, const char *__restrict__ frames,
                                                         size_t fstride, Rk4Args A, unsigned *errword, RingWork W)
{
    extern __shared__ __align__(128) char slots[];
    __shared__ RingState R;
    __shared__ long long s_item;
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < RING_SLOTS; ++s) {
            mbar_init(&R.bar[s], 1);
            R.tag[s] = -1;
            R.nload[s] = 0;
        }
        R.abort = 0;
        mbar_fence_init();
    }
    __syncthreads();
    if (!W.persistent) {
        ring_tile<ST, TPT>(P, frames, fstride, A, errword, slots, R, blockIdx.y, blockIdx.x);
    } else {
        for (;;) {
            if (tid == 0) s_item = (long long)atomicAdd(W.queue, 1u);
            __syncthreads();
            const long long item = s_item;
            __syncthreads();
            if (item >= W.nitems || R.abort) break;
            const int job = W.jorder[item / W.tiles_per_job];
            ring_tile<ST, TPT>(P, frames, fstride, A, errword, slots, R, job, item % W.tiles_per_job);
        }
    }
    // drain copies still in flight (prefetches nobody read, or copies a shortened wait gave up on)
    // before the block exits, with the full bound whatever the call's wait limit
    __syncthreads();
    if (tid == 0)
        for (int s = 0; s < RING_SLOTS; ++s)
            if (R.nload[s] > 0 && !mbar_wait_bounded(&R.bar[s], (R.nload[s] - 1) & 1))
                atomicOr(errword, LCS_ERRBIT_TIMEOUT);
    __syncthreads();
}

// ========================================================== 2D time slices

// Variant 5 (2D): every stage time of every job gets its own time slice, the field blended
// to that time once (interp's node-first arithmetic, FP32), stored per node as two float4
// quads (u(i,j), u(i1,j), u(i,j1), u(i1,j1)) and the same for v, with i1, j1 the next node
// (wrapped on a periodic axis, clamped on a closed one).  A stage evaluation is then the
// cell and weights of make_stencil and two 16-byte loads, with the products of interp in
// interp's order: bit-identical to the other variants.  Slice (job, n, stage) is number
// off[job] + 3 n + stage, each 2 * nodes float4.
struct Slice2dOffsets {
    long long off[LCS_MAX_JOBS];
};

__global__ void slice2d_fill_kernel(RectParams P, const char *__restrict__ frames, size_t fstride, int storage,
                                    const SchedEntry *__restrict__ sched, int nsteps_max,
                                    const int *__restrict__ job_nsteps, Slice2dOffsets O, long long nodes,
                                    float4 *__restrict__ slices)
{
    const int job = blockIdx.y;
    const long long per_job = 3LL * job_nsteps[job] * nodes;
    const SchedEntry *sc = sched + (size_t)job * nsteps_max * 3;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < per_job;
         t += (long long)gridDim.x * blockDim.x) {
        const long long l = t / nodes, v = t % nodes;
        const SchedEntry e = load_sched(sc + l);   // slice l of the job = schedule entry l (= 3 n + stage)
        const int i = (int)(v % P.n[0]), j = (int)(v / P.n[0]);
        const int i1 = P.periodic[0] ? (i + 1 == P.n[0] ? 0 : i + 1) : min(i + 1, P.n[0] - 1);
        const int j1 = P.periodic[1] ? (j + 1 == P.n[1] ? 0 : j + 1) : min(j + 1, P.n[1] - 1);
        const int corner[4] = {(int)(i + j * P.sy), (int)(i1 + j * P.sy), (int)(i + j1 * P.sy),
                               (int)(i1 + j1 * P.sy)};
        const char *fa = frames + (size_t)e.k * fstride;
        float u[4][2];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float va[2], vb[2];
            if (storage == LCS_F32)
                Node<2, LCS_F32>::ld(fa, corner[q], va);
            else if (storage == LCS_F16)
                Node<2, LCS_F16>::ld(fa, corner[q], va);
            else
                Node<2, LCS_BF16>::ld(fa, corner[q], va);
            if (e.a == 0.0f) {   // frame k + 1 is not read (it may not exist)
                u[q][0] = va[0];
                u[q][1] = va[1];
                continue;
            }
            const char *fb = fa + fstride;
            if (storage == LCS_F32)
                Node<2, LCS_F32>::ld(fb, corner[q], vb);
            else if (storage == LCS_F16)
                Node<2, LCS_F16>::ld(fb, corner[q], vb);
            else
                Node<2, LCS_BF16>::ld(fb, corner[q], vb);
            const float g = 1.0f - e.a;
            u[q][0] = tblend(va[0], vb[0], e.a, g);
            u[q][1] = tblend(va[1], vb[1], e.a, g);
        }
        float4 *o = slices + (O.off[job] + l) * 2 * nodes + 2 * v;
        o[0] = make_float4(u[0][0], u[1][0], u[2][0], u[3][0]);
        o[1] = make_float4(u[0][1], u[1][1], u[2][1], u[3][1]);
    }
}

// u(x) from a 2D slice: make_stencil's cell and weights, interp's products and order
template <int PM>
__device__ __forceinline__ void interp2s(const RectParams &P, const float *x, const float4 *__restrict__ sl, float *u)
{
    Stencil<2> S;
    make_stencil<2, PM>(P, x, S);
    const float4 qu = __ldg(sl + 2 * S.v[0]), qv = __ldg(sl + 2 * S.v[0] + 1);
    u[0] = fmaf(S.w[3], qu.w, fmaf(S.w[2], qu.z, fmaf(S.w[1], qu.y, fmaf(S.w[0], qu.x, 0.0f))));
    u[1] = fmaf(S.w[3], qv.w, fmaf(S.w[2], qv.z, fmaf(S.w[1], qv.y, fmaf(S.w[0], qv.x, 0.0f))));
}

// PM: compile-time periodicity (bit d: axis d periodic; -1: read from P)
template <int PM>
__global__ void __launch_bounds__(256) rk4_slice2d_kernel(RectParams P, const float4 *__restrict__ slices,
                                                          long long nodes, Slice2dOffsets O, Rk4Args A)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int job = blockIdx.y;
    if (i >= A.N) return;
    float x[2] = {A.seeds[i], A.seeds[A.N + i]}, cx[2] = {0.0f, 0.0f};
    int img[2] = {0, 0};
    wrap_periodic<2, PM>(P, x, cx, img);
    const int ns = A.job_nsteps[job];
    const float h = A.job_h[job];
    const float4 *sj = slices + O.off[job] * 2 * nodes;
    const size_t ss = 2 * (size_t)nodes;
    unsigned char st = LCS_TRACER_OK;
    float te = A.job_tend[job];
    int si = 0;   // next snapshot
    for (int n = 0; n < ns; ++n) {
        const float4 *s0 = sj + (size_t)(3 * n) * ss;
        float k1[2], k2[2], k3[2], k4[2], y[2];
        const float hh = 0.5f * h;
        interp2s<PM>(P, x, s0, k1);
#pragma unroll
        for (int c = 0; c < 2; ++c) y[c] = fmaf(hh, k1[c], x[c]);
        interp2s<PM>(P, y, s0 + ss, k2);
#pragma unroll
        for (int c = 0; c < 2; ++c) y[c] = fmaf(hh, k2[c], x[c]);
        interp2s<PM>(P, y, s0 + ss, k3);
#pragma unroll
        for (int c = 0; c < 2; ++c) y[c] = fmaf(h, k3[c], x[c]);
        interp2s<PM>(P, y, s0 + 2 * ss, k4);
        const float h6 = h * (1.0f / 6.0f);
#pragma unroll
        for (int c = 0; c < 2; ++c) rk4_advance(x[c], cx[c], h6, k1[c], k2[c], k3[c], k4[c]);
        wrap_periodic<2, PM>(P, x, cx, img);
        if (rect_left<2, PM>(P, x)) {
            st = LCS_TRACER_LEFT;
            te = fmaf((float)(n + 1), h, A.job_t0[job]);
            break;
        }
        for (; si < A.nsnap && snap_step(A, si, ns) == n + 1; ++si)
            store_tracer<2>(P, A, snap_slot(A, job, si), i, x, cx, img, st, snap_exit(A, job, si, st, te));
    }
    for (; si < A.nsnap; ++si)
        store_tracer<2>(P, A, snap_slot(A, job, si), i, x, cx, img, st, snap_exit(A, job, si, st, te));
    store_tracer<2>(P, A, job, i, x, cx, img, st, te);
}

size_t rk4_slice2d_bytes(const lcs_field *f, int njobs, const int *host_nsteps)
{
    long long n = 0;
    for (int j = 0; j < njobs; ++j) n += 3LL * host_nsteps[j];
    return (size_t)n * 2 * (size_t)f->nodes * sizeof(float4);
}

static cudaError_t launch_slice2d(const RectParams &P, const lcs_field *f, const Rk4Args &A, const Rk4Launch &L,
                                  int bt, cudaStream_t s)
{
    Slice2dOffsets O;
    long long acc = 0;
    for (int j = 0; j < L.njobs; ++j) {
        O.off[j] = acc;
        acc += 3LL * L.host_nsteps[j];
    }
    float4 *slices = (float4 *)L.work;
    const long long nodes = f->nodes;
    lcs_tm_begin(L.ctx, 2, s);
    slice2d_fill_kernel<<<dim3(1024, (unsigned)L.njobs), 256, 0, s>>>(P, (const char *)f->d_frames, f->frame_stride,
                                                                      f->storage, A.sched, A.nsteps_max,
                                                                      A.job_nsteps, O, nodes, slices);
    lcs_tm_end(L.ctx, 2, s);
    lcs_tm_begin(L.ctx, 0, s);
    dim3 grid((unsigned)((A.N + bt - 1) / bt), (unsigned)L.njobs);
    const int pm = P.periodic[0] | (P.periodic[1] << 1);
    if (pm == 0)
        rk4_slice2d_kernel<0><<<grid, bt, 0, s>>>(P, slices, nodes, O, A);
    else if (pm == 3)
        rk4_slice2d_kernel<3><<<grid, bt, 0, s>>>(P, slices, nodes, O, A);
    else
        rk4_slice2d_kernel<-1><<<grid, bt, 0, s>>>(P, slices, nodes, O, A);
    lcs_tm_end(L.ctx, 0, s);
    return cudaGetLastError();
}

// ================================================================ dispatch

RectParams make_rect_params(const lcs_field *f)
{
    RectParams P;
    for (int d = 0; d < 3; ++d) {
        int dd = d < f->dim ? d : 0;
        P.n[d] = f->n[dd];
        P.periodic[d] = d < f->dim ? f->periodic[d] : 0;
        P.origin[d] = (float)f->origin[dd];
        P.inv_h[d] = (float)(1.0 / f->spacing[dd]);
        P.hi_node[d] = (float)(f->origin[dd] + (f->n[dd] - 1) * f->spacing[dd]);
        P.left_lo[d] = (float)(f->origin[dd] - f->spacing[dd]);
        P.left_hi[d] = (float)(f->origin[dd] + f->n[dd] * f->spacing[dd]);
        P.L[d] = (float)(f->n[dd] * f->spacing[dd]);
    }
    P.sy = f->n[0];
    P.sz = (long long)f->n[0] * f->n[1];
    P.fstride = (long long)(f->frame_stride / (f->vec * f->elem_bytes));
    return P;
}

template <int DIM, int ST>
static cudaError_t launch_gather(const RectParams &P, const lcs_field *f, const Rk4Args &A, int njobs, int bt,
                                 cudaStream_t s)
{
    dim3 grid((unsigned)((A.N + bt - 1) / bt), (unsigned)njobs);
    rk4_gather_kernel<DIM, ST><<<grid, bt, 0, s>>>(P, (const char *)f->d_frames, f->frame_stride, A);
    return cudaGetLastError();
}

template <int ST, int TPT>
static cudaError_t launch_ring(lcs_ctx *ctx, const RectParams &P, const lcs_field *f, const Rk4Args &A,
                               const Rk4Launch &L, int bt, bool persistent, cudaStream_t s)
{
    size_t smem = RING_SLOTS * f->frame_stride;
    cudaError_t e = cudaFuncSetAttribute(rk4_ring2d_kernel<ST, TPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const long long tiles = (A.N + (long long)bt * TPT - 1) / ((long long)bt * TPT);
    RingWork W;
    W.persistent = persistent ? 1 : 0;
    W.queue = L.queue;
    W.tiles_per_job = (int)tiles;
    W.nitems = tiles * L.njobs;
    W.jorder = L.job_order;
    if (!persistent) {
        dim3 grid((unsigned)tiles, (unsigned)L.njobs);
        rk4_ring2d_kernel<ST, TPT><<<grid, bt, smem, s>>>(P, (const char *)f->d_frames, f->frame_stride, A,
                                                           ctx->d_errword, W);
        return cudaGetLastError();
    }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rk4_ring2d_kernel<ST, TPT>, bt, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    long long blocks = (long long)per_sm * ctx->num_sms;
    if (blocks > W.nitems) blocks = W.nitems;
    if (blocks < 1) blocks = 1;
    e = cudaMemsetAsync(L.queue, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    rk4_ring2d_kernel<ST, TPT><<<(unsigned)blocks, bt, smem, s>>>(P, (const char *)f->d_frames, f->frame_stride, A,
                                                                   ctx->d_errword, W);
    return cudaGetLastError();
}

template <int ST>
static cudaError_t launch_ring_tpt(lcs_ctx *ctx, const RectParams &P, const lcs_field *f, const Rk4Args &A,
                                   const Rk4Launch &L, int bt, bool persistent, cudaStream_t s)
{
    if (L.tracers_per_thread >= 2) return launch_ring<ST, 2>(ctx, P, f, A, L, bt, persistent, s);
    return launch_ring<ST, 1>(ctx, P, f, A, L, bt, persistent, s);
}

int launch_rk4_rect(lcs_ctx *ctx, const Rk4Launch &L, cudaStream_t s)
{
    const lcs_field *f = L.field;
    RectParams P = make_rect_params(f);
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
    A.out_grad = L.out_grad;
    A.njobs = L.njobs;
    A.nsnap = L.nsnap;
    A.snap_n = L.snap_n;
    A.snap_te = L.snap_te;
    A.wait_ns = L.wait_ns;
    if (L.N == 0 || L.njobs == 0) return 1;
    bool ring_fits = f->dim == 2 && RING_SLOTS * f->frame_stride <= ctx->smem_optin;
    bool sorted_ok = f->dim == 3 && L.work != nullptr;
    bool queue_ok = L.queue != nullptr && L.job_order != nullptr;
    int variant = L.variant;
    // default: 2D time slices when lcs_advect reserved them (at most 2 GiB; the autotuner's choice on
    // GB300 for the sliding-window batches), else the cached gather in 2D (the shared-memory ring's
    // per-step block barriers cost more than the loads they save while the field stays in L2);
    // re-bundled episodes for large 3D lattices
    if (variant == 0) variant = sorted_ok && L.N >= LCS_SORTED_MIN_SEEDS ? 3 : (f->dim == 2 && L.work ? 5 : 1);
    if ((variant == 2 || variant == 4) && !ring_fits) variant = 1;
    if (variant == 4 && !queue_ok) variant = 2;
    if (variant == 3 && !sorted_ok) variant = 1;
    cudaError_t e;
    if (A.out_grad && variant == 3) {   // the variational equations in the re-bundled episodes
        e = launch_rk4_episodes(P, f, A, L, s);
        return e == cudaSuccess ? variant : -1;
    }
    if (A.out_grad) {   // the variational equations elsewhere: their own one-pass kernel
        const int bt = L.block_threads > 0 && L.block_threads <= 256 ? L.block_threads : 256;
        dim3 grid((unsigned)((A.N + bt - 1) / bt), (unsigned)L.njobs);
        const char *fr = (const char *)f->d_frames;
        lcs_tm_begin(ctx, 0, s);
#define VAR_LAUNCH(D, ST) rk4_var_kernel<D, ST><<<grid, bt, 0, s>>>(P, fr, f->frame_stride, A)
        if (f->dim == 2) {
            if (f->storage == LCS_F32) VAR_LAUNCH(2, LCS_F32);
            else if (f->storage == LCS_F16) VAR_LAUNCH(2, LCS_F16);
            else VAR_LAUNCH(2, LCS_BF16);
        } else {
            if (f->storage == LCS_F32) VAR_LAUNCH(3, LCS_F32);
            else if (f->storage == LCS_F16) VAR_LAUNCH(3, LCS_F16);
            else VAR_LAUNCH(3, LCS_BF16);
        }
#undef VAR_LAUNCH
        lcs_tm_end(ctx, 0, s);
        return cudaGetLastError() == cudaSuccess ? 6 : -1;
    }
    if (variant == 5 && !(f->dim == 2 && L.work != nullptr)) variant = 1;
    if (variant == 3) {
        e = launch_rk4_episodes(P, f, A, L, s);
        return e == cudaSuccess ? variant : -1;
    }
    if (variant == 5) {
        int bt = L.block_threads > 0 && L.block_threads <= 256 ? L.block_threads : 256;
        e = launch_slice2d(P, f, A, L, bt, s);
        return e == cudaSuccess ? variant : -1;
    }
    lcs_tm_begin(ctx, 0, s);
    if (variant == 2 || variant == 4) {
        int bt = L.block_threads > 0 ? L.block_threads : 512;
        if (bt > 512) bt = 512;
        const bool pers = variant == 4;
        if (f->storage == LCS_F32)
            e = launch_ring_tpt<LCS_F32>(ctx, P, f, A, L, bt, pers, s);
        else if (f->storage == LCS_F16)
            e = launch_ring_tpt<LCS_F16>(ctx, P, f, A, L, bt, pers, s);
        else
            e = launch_ring_tpt<LCS_BF16>(ctx, P, f, A, L, bt, pers, s);
    } else {
        int bt = L.block_threads > 0 ? L.block_threads : 256;
        if (bt > 256) bt = 256;
        if (f->dim == 2) {
            if (f->storage == LCS_F32)
                e = launch_gather<2, LCS_F32>(P, f, A, L.njobs, bt, s);
            else if (f->storage == LCS_F16)
                e = launch_gather<2, LCS_F16>(P, f, A, L.njobs, bt, s);
            else
                e = launch_gather<2, LCS_BF16>(P, f, A, L.njobs, bt, s);
        } else {
            if (f->storage == LCS_F32)
                e = launch_gather<3, LCS_F32>(P, f, A, L.njobs, bt, s);
            else if (f->storage == LCS_F16)
                e = launch_gather<3, LCS_F16>(P, f, A, L.njobs, bt, s);
            else
                e = launch_gather<3, LCS_BF16>(P, f, A, L.njobs, bt, s);
        }
    }
    lcs_tm_end(ctx, 0, s);
    return e == cudaSuccess ? variant : -1;
}
