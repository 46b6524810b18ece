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
#include "lcs_internal.cuh"

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
    }
    if (idx >= total) return;
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

// ================================================================ node loads

// Node v of a frame -> FP32 components.  Storage: 2D = 2 components, 3D = 4
// (the 4th is padding); FP16/BF16 are widened to FP32.
template <int DIM, int ST>
struct Node;

// ld: global memory (read-only path); lds: generic address (shared or global);
// lss: shared memory only (explicit shared-space load)
__device__ __forceinline__ unsigned ld_shared_u32(const char *f, int v)
{
    unsigned r;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(r) : "r"(smem_u32(f) + 4u * (unsigned)v));
    return r;
}

template <>
struct Node<2, LCS_F32> {
    static __device__ __forceinline__ void ld(const char *f, int v, float *u)
    {
        float2 t = __ldg(reinterpret_cast<const float2 *>(f) + v);
        u[0] = t.x;
        u[1] = t.y;
    }
    static __device__ __forceinline__ void lds(const char *f, int v, float *u)
    {
        float2 t = reinterpret_cast<const float2 *>(f)[v];
        u[0] = t.x;
        u[1] = t.y;
    }
    static __device__ __forceinline__ void lss(const char *f, int v, float *u)
    {
        asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(u[0]), "=f"(u[1]) : "r"(smem_u32(f) + 8u * (unsigned)v));
    }
};

__device__ __forceinline__ float2 h2f(unsigned r)
{
    __half2 h = *reinterpret_cast<__half2 *>(&r);
    return __half22float2(h);
}

__device__ __forceinline__ float2 b2f(unsigned r)
{
    __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162 *>(&r);
    return __bfloat1622float2(h);
}

template <>
struct Node<2, LCS_F16> {
    static __device__ __forceinline__ void ld(const char *f, int v, float *u)
    {
        float2 t = h2f(__ldg(reinterpret_cast<const unsigned *>(f) + v));
        u[0] = t.x;
        u[1] = t.y;
    }
    static __device__ __forceinline__ void lds(const char *f, int v, float *u)
    {
        float2 t = h2f(reinterpret_cast<const unsigned *>(f)[v]);
        u[0] = t.x;
        u[1] = t.y;
    }
    static __device__ __forceinline__ void lss(const char *f, int v, float *u)
    {
        float2 t = h2f(ld_shared_u32(f, v));
        u[0] = t.x;
        u[1] = t.y;
    }
};

template <>
struct Node<2, LCS_BF16> {
    static __device__ __forceinline__ void ld(const char *f, int v, float *u)
    {
        float2 t = b2f(__ldg(reinterpret_cast<const unsigned *>(f) + v));
        u[0] = t.x;
        u[1] = t.y;
    }
    static __device__ __forceinline__ void lds(const char *f, int v, float *u)
    {
        float2 t = b2f(reinterpret_cast<const unsigned *>(f)[v]);
        u[0] = t.x;
        u[1] = t.y;
    }
    static __device__ __forceinline__ void lss(const char *f, int v, float *u)
    {
        float2 t = b2f(ld_shared_u32(f, v));
        u[0] = t.x;
        u[1] = t.y;
    }
};

// 3D nodes are stored as interval pairs: node v of pair k holds (u_k, 0, u_{k+1}, 0),
// so one 32-byte (FP32) or 16-byte (FP16/BF16) load brings both frames of a corner.
template <int ST>
struct Pair3;

template <>
struct Pair3<LCS_F32> {
    static __device__ __forceinline__ void ld(const char *f, int v, float *ua, float *ub)
    {
        float t[8];
        asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=f"(t[0]), "=f"(t[1]), "=f"(t[2]), "=f"(t[3]), "=f"(t[4]), "=f"(t[5]), "=f"(t[6]), "=f"(t[7])
            : "l"(f + 32 * (size_t)v));
        ua[0] = t[0];
        ua[1] = t[1];
        ua[2] = t[2];
        ub[0] = t[4];
        ub[1] = t[5];
        ub[2] = t[6];
    }
};

template <>
struct Pair3<LCS_F16> {
    static __device__ __forceinline__ void ld(const char *f, int v, float *ua, float *ub)
    {
        uint4 r = __ldg(reinterpret_cast<const uint4 *>(f) + v);
        float2 a = h2f(r.x), b = h2f(r.y), c = h2f(r.z), d = h2f(r.w);
        ua[0] = a.x;
        ua[1] = a.y;
        ua[2] = b.x;
        ub[0] = c.x;
        ub[1] = c.y;
        ub[2] = d.x;
    }
};

template <>
struct Pair3<LCS_BF16> {
    static __device__ __forceinline__ void ld(const char *f, int v, float *ua, float *ub)
    {
        uint4 r = __ldg(reinterpret_cast<const uint4 *>(f) + v);
        float2 a = b2f(r.x), b = b2f(r.y), c = b2f(r.z), d = b2f(r.w);
        ua[0] = a.x;
        ua[1] = a.y;
        ua[2] = b.x;
        ub[0] = c.x;
        ub[1] = c.y;
        ub[2] = d.x;
    }
};

// ============================================================ interpolation

// Cell along axis d.  Non-periodic: clamp the query into the box, cell i with
// node_i <= x < node_{i+1}, the last cell closed.  Periodic: wrap the index.
__device__ __forceinline__ void axis_cell(const RectParams &P, int d, float x, int &i0, int &i1, float &f)
{
    if (P.periodic[d]) {
        float s = (x - P.origin[d]) * P.inv_h[d];
        float fl = floorf(s);
        int i = (int)fl;
        f = s - fl;
        int n = P.n[d];
        if (i < 0 || i >= n) {
            i %= n;
            if (i < 0) i += n;
        }
        i0 = i;
        i1 = (i + 1 == n) ? 0 : i + 1;
    } else {
        float xc = fminf(fmaxf(x, P.origin[d]), P.hi_node[d]);
        float s = (xc - P.origin[d]) * P.inv_h[d];
        int i = min((int)s, P.n[d] - 2);
        f = s - (float)i;
        i0 = i;
        i1 = i + 1;
    }
}

// Spatial corners and weights of x (bilinear: 4, trilinear: 8).
template <int DIM>
struct Stencil {
    int v[1 << DIM];
    float w[1 << DIM];
};

template <int DIM>
__device__ __forceinline__ void make_stencil(const RectParams &P, const float *x, Stencil<DIM> &S)
{
    int i0, i1, j0, j1;
    float fx, fy;
    axis_cell(P, 0, x[0], i0, i1, fx);
    axis_cell(P, 1, x[1], j0, j1, fy);
    float gx = 1.0f - fx, gy = 1.0f - fy;
    int r0 = j0 * (int)P.sy, r1 = j1 * (int)P.sy;
    if constexpr (DIM == 2) {
        S.v[0] = i0 + r0;
        S.v[1] = i1 + r0;
        S.v[2] = i0 + r1;
        S.v[3] = i1 + r1;
        S.w[0] = gx * gy;
        S.w[1] = fx * gy;
        S.w[2] = gx * fy;
        S.w[3] = fx * fy;
    } else {
        int k0, k1;
        float fz;
        axis_cell(P, 2, x[2], k0, k1, fz);
        float gz = 1.0f - fz;
        int p0 = k0 * (int)P.sz, p1 = k1 * (int)P.sz;
        S.v[0] = i0 + r0 + p0;
        S.v[1] = i1 + r0 + p0;
        S.v[2] = i0 + r1 + p0;
        S.v[3] = i1 + r1 + p0;
        S.v[4] = i0 + r0 + p1;
        S.v[5] = i1 + r0 + p1;
        S.v[6] = i0 + r1 + p1;
        S.v[7] = i1 + r1 + p1;
        float a = gy * gz, b = fy * gz, c = gy * fz, d = fy * fz;
        S.w[0] = gx * a;
        S.w[1] = fx * a;
        S.w[2] = gx * b;
        S.w[3] = fx * b;
        S.w[4] = gx * c;
        S.w[5] = fx * c;
        S.w[6] = gx * d;
        S.w[7] = fx * d;
    }
}

// where stage frames live: global memory, any (generic address), shared memory
enum { SRC_GLOBAL = 0, SRC_GENERIC = 1, SRC_SHARED = 2 };

template <int DIM, int ST, int SRC>
__device__ __forceinline__ void node_load(const char *f, int v, float *u)
{
    if constexpr (SRC == SRC_GLOBAL)
        Node<DIM, ST>::ld(f, v, u);
    else if constexpr (SRC == SRC_GENERIC)
        Node<DIM, ST>::lds(f, v, u);
    else
        Node<DIM, ST>::lss(f, v, u);
}

// u = (1 - a) I[frame fa](x) + a I[frame fb](x); frame fb is not read when a == 0
template <int DIM, int ST, int SRC>
__device__ __forceinline__ void interp(const Stencil<DIM> &S, const char *fa, const char *fb, float a, float *u)
{
    float ua[DIM], ub[DIM], v[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) ua[c] = 0.0f;
#pragma unroll
    for (int q = 0; q < (1 << DIM); ++q) {
        node_load<DIM, ST, SRC>(fa, S.v[q], v);
#pragma unroll
        for (int c = 0; c < DIM; ++c) ua[c] = fmaf(S.w[q], v[c], ua[c]);
    }
    if (a == 0.0f) {
#pragma unroll
        for (int c = 0; c < DIM; ++c) u[c] = ua[c];
        return;
    }
#pragma unroll
    for (int c = 0; c < DIM; ++c) ub[c] = 0.0f;
#pragma unroll
    for (int q = 0; q < (1 << DIM); ++q) {
        node_load<DIM, ST, SRC>(fb, S.v[q], v);
#pragma unroll
        for (int c = 0; c < DIM; ++c) ub[c] = fmaf(S.w[q], v[c], ub[c]);
    }
    float g = 1.0f - a;
#pragma unroll
    for (int c = 0; c < DIM; ++c) u[c] = fmaf(a, ub[c], g * ua[c]);
}

// Time blend of one node, FP32: u = (1 - a) u_k + a u_{k+1} (exactly u_k when a == 0).
// 3D fields blend at the nodes first, then interpolate in space; both orders are the
// same linear map, and every 3D kernel uses this one so that they agree bit for bit.
__device__ __forceinline__ float tblend(float ua, float ub, float a, float g)
{
    return fmaf(a, ub, g * ua);
}

// 3D: u(x, t) from the interval pair k with weight a of frame k + 1
template <int ST>
__device__ __forceinline__ void interp3p(const Stencil<3> &S, const char *fp, float a, float *u)
{
    float acc[3] = {0.0f, 0.0f, 0.0f}, va[3], vb[3];
    const float g = 1.0f - a;
    if (a == 0.0f) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            Pair3<ST>::ld(fp, S.v[q], va, vb);
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[c] = fmaf(S.w[q], va[c], acc[c]);
        }
    } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            Pair3<ST>::ld(fp, S.v[q], va, vb);
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[c] = fmaf(S.w[q], tblend(va[c], vb[c], a, g), acc[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) u[c] = acc[c];
}

// 3D: u(x, t) from a time slice (nodes already blended to the stage time), float4 per node
__device__ __forceinline__ void interp3s(const Stencil<3> &S, const float4 *__restrict__ sl, float *u)
{
    float acc[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        float4 v = __ldg(sl + S.v[q]);
        acc[0] = fmaf(S.w[q], v.x, acc[0]);
        acc[1] = fmaf(S.w[q], v.y, acc[1]);
        acc[2] = fmaf(S.w[q], v.z, acc[2]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) u[c] = acc[c];
}

struct Rk4Args {
    const float *seeds;
    long long N;
    int nsteps_max;
    const SchedEntry *sched;
    const int *job_nsteps;
    const float *job_h;
    const float *job_t0;
    const float *job_tend;
    float *out_xyz;
    unsigned char *out_status;
    float *out_texit;
};

__device__ __forceinline__ SchedEntry load_sched(const SchedEntry *p)
{
    int2 r = __ldg(reinterpret_cast<const int2 *>(p));
    SchedEntry e;
    e.k = r.x;
    e.a = __int_as_float(r.y);
    return e;
}

// periodic axes: keep x in [origin, origin + L) with an integer count of periods
template <int DIM>
__device__ __forceinline__ void wrap_periodic(const RectParams &P, float *x, int *img)
{
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        if (!P.periodic[d]) continue;
        float hiL = P.origin[d] + P.L[d];
        if (x[d] >= hiL) {
            x[d] -= P.L[d];
            img[d] += 1;
        } else if (x[d] < P.origin[d]) {
            x[d] += P.L[d];
            img[d] -= 1;
        }
        if (!(x[d] >= P.origin[d] && x[d] < hiL) && isfinite(x[d])) {  // far outside: full reduction
            float m = floorf((x[d] - P.origin[d]) / P.L[d]);
            x[d] -= m * P.L[d];
            img[d] += (int)m;
            if (x[d] >= hiL) x[d] = P.origin[d];
        }
    }
}

template <int DIM>
__device__ __forceinline__ bool rect_left(const RectParams &P, const float *x)
{
    bool out = false;
#pragma unroll
    for (int d = 0; d < DIM; ++d)
        if (!P.periodic[d]) out |= (x[d] < P.left_lo[d]) || (x[d] > P.left_hi[d]);
    return out;
}

template <int DIM>
__device__ __forceinline__ void store_tracer(const RectParams &P, const Rk4Args &A, int job, long long i,
                                             const float *x, const int *img, unsigned char st, float te)
{
    float *o = A.out_xyz + (size_t)job * DIM * A.N;
#pragma unroll
    for (int d = 0; d < DIM; ++d) o[d * A.N + i] = P.periodic[d] ? fmaf((float)img[d], P.L[d], x[d]) : x[d];
    A.out_status[(size_t)job * A.N + i] = st;
    A.out_texit[(size_t)job * A.N + i] = te;
}

// one RK4 step; stage frames given by (fa, fb, a) triples
template <int DIM, int ST, int SRC>
__device__ __forceinline__ void rk4_step(const RectParams &P, float *x, float h, const char *fa0, const char *fb0,
                                         float a0, const char *fa1, const char *fb1, float a1, const char *fa2,
                                         const char *fb2, float a2)
{
    float k1[DIM], k2[DIM], k3[DIM], k4[DIM], y[DIM];
    Stencil<DIM> S;
    const float hh = 0.5f * h;
    make_stencil<DIM>(P, x, S);
    interp<DIM, ST, SRC>(S, fa0, fb0, a0, k1);
#pragma unroll
    for (int c = 0; c < DIM; ++c) y[c] = fmaf(hh, k1[c], x[c]);
    make_stencil<DIM>(P, y, S);
    interp<DIM, ST, SRC>(S, fa1, fb1, a1, k2);
#pragma unroll
    for (int c = 0; c < DIM; ++c) y[c] = fmaf(hh, k2[c], x[c]);
    make_stencil<DIM>(P, y, S);
    interp<DIM, ST, SRC>(S, fa1, fb1, a1, k3);
#pragma unroll
    for (int c = 0; c < DIM; ++c) y[c] = fmaf(h, k3[c], x[c]);
    make_stencil<DIM>(P, y, S);
    interp<DIM, ST, SRC>(S, fa2, fb2, a2, k4);
    const float h6 = h * (1.0f / 6.0f);
#pragma unroll
    for (int c = 0; c < DIM; ++c) x[c] = fmaf(h6, (k1[c] + k4[c]) + 2.0f * (k2[c] + k3[c]), x[c]);
}

// one RK4 step in 3D; stage s reads interval pair ps with weight as
template <int ST>
__device__ __forceinline__ void rk4_step3p(const RectParams &P, float *x, float h, const char *p0, float a0,
                                           const char *p1, float a1, const char *p2, float a2)
{
    float k1[3], k2[3], k3[3], k4[3], y[3];
    Stencil<3> S;
    const float hh = 0.5f * h;
    make_stencil<3>(P, x, S);
    interp3p<ST>(S, p0, a0, k1);
#pragma unroll
    for (int c = 0; c < 3; ++c) y[c] = fmaf(hh, k1[c], x[c]);
    make_stencil<3>(P, y, S);
    interp3p<ST>(S, p1, a1, k2);
#pragma unroll
    for (int c = 0; c < 3; ++c) y[c] = fmaf(hh, k2[c], x[c]);
    make_stencil<3>(P, y, S);
    interp3p<ST>(S, p1, a1, k3);
#pragma unroll
    for (int c = 0; c < 3; ++c) y[c] = fmaf(h, k3[c], x[c]);
    make_stencil<3>(P, y, S);
    interp3p<ST>(S, p2, a2, k4);
    const float h6 = h * (1.0f / 6.0f);
#pragma unroll
    for (int c = 0; c < 3; ++c) x[c] = fmaf(h6, (k1[c] + k4[c]) + 2.0f * (k2[c] + k3[c]), x[c]);
}

// one RK4 step in 3D from three time slices (stage times t_n, t_n + h/2, t_n + h)
__device__ __forceinline__ void rk4_step3s(const RectParams &P, float *x, float h, const float4 *s0,
                                           const float4 *s1, const float4 *s2)
{
    float k1[3], k2[3], k3[3], k4[3], y[3];
    Stencil<3> S;
    const float hh = 0.5f * h;
    make_stencil<3>(P, x, S);
    interp3s(S, s0, k1);
#pragma unroll
    for (int c = 0; c < 3; ++c) y[c] = fmaf(hh, k1[c], x[c]);
    make_stencil<3>(P, y, S);
    interp3s(S, s1, k2);
#pragma unroll
    for (int c = 0; c < 3; ++c) y[c] = fmaf(hh, k2[c], x[c]);
    make_stencil<3>(P, y, S);
    interp3s(S, s1, k3);
#pragma unroll
    for (int c = 0; c < 3; ++c) y[c] = fmaf(h, k3[c], x[c]);
    make_stencil<3>(P, y, S);
    interp3s(S, s2, k4);
    const float h6 = h * (1.0f / 6.0f);
#pragma unroll
    for (int c = 0; c < 3; ++c) x[c] = fmaf(h6, (k1[c] + k4[c]) + 2.0f * (k2[c] + k3[c]), x[c]);
}

// ============================================================ gather kernel

template <int DIM, int ST>
__global__ void __launch_bounds__(256) rk4_gather_kernel(RectParams P, const char *__restrict__ frames,
                                                         size_t fstride, Rk4Args A)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    int job = blockIdx.y;
    if (i >= A.N) return;
    float x[DIM];
    int img[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        x[d] = A.seeds[d * A.N + i];
        img[d] = 0;
    }
    wrap_periodic<DIM>(P, x, img);
    const SchedEntry *sc = A.sched + (size_t)job * A.nsteps_max * 3;
    const int ns = A.job_nsteps[job];
    const float h = A.job_h[job];
    unsigned char st = LCS_TRACER_OK;
    float te = A.job_tend[job];
    for (int n = 0; n < ns; ++n) {
        SchedEntry e0 = load_sched(sc + 3 * n), e1 = load_sched(sc + 3 * n + 1), e2 = load_sched(sc + 3 * n + 2);
        if constexpr (DIM == 2)
            rk4_step<2, ST, SRC_GLOBAL>(P, x, h, frames + (size_t)e0.k * fstride,
                                        frames + (size_t)(e0.k + 1) * fstride, e0.a, frames + (size_t)e1.k * fstride,
                                        frames + (size_t)(e1.k + 1) * fstride, e1.a, frames + (size_t)e2.k * fstride,
                                        frames + (size_t)(e2.k + 1) * fstride, e2.a);
        else
            rk4_step3p<ST>(P, x, h, frames + (size_t)e0.k * fstride, e0.a, frames + (size_t)e1.k * fstride, e1.a,
                           frames + (size_t)e2.k * fstride, e2.a);
        wrap_periodic<DIM>(P, x, img);
        if (rect_left<DIM>(P, x)) {
            st = LCS_TRACER_LEFT;
            te = fmaf((float)(n + 1), h, A.job_t0[job]);
            break;
        }
    }
    store_tracer<DIM>(P, A, job, i, x, img, st, te);
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
                         int nkeep, unsigned *errword)
{
    int v = -1;
    for (int s = 0; s < RING_SLOTS && v < 0; ++s)
        if (R.tag[s] < 0) v = s;
    for (int s = 0; s < RING_SLOTS && v < 0; ++s)
        if (!in_list(keep, nkeep, R.tag[s])) v = s;
    if (v < 0) return RING_GLOBAL;
    if (R.nload[v] > 0 && !mbar_wait_bounded(&R.bar[v], (R.nload[v] - 1) & 1)) {  // previous copy into v
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

template <int ST>
__global__ void __launch_bounds__(512) rk4_ring2d_kernel(RectParams P, const char *__restrict__ frames,
                                                         size_t fstride, Rk4Args A, unsigned *errword)
{
    extern __shared__ __align__(128) char slots[];
    __shared__ RingState R;
    const int tid = threadIdx.x;
    const long long i = blockIdx.x * (long long)blockDim.x + tid;
    const int job = blockIdx.y;
    const bool active = i < A.N;
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
    float x[2] = {0.0f, 0.0f};
    int img[2] = {0, 0};
    if (active) {
        x[0] = A.seeds[i];
        x[1] = A.seeds[A.N + i];
    }
    wrap_periodic<2>(P, x, img);
    const SchedEntry *sc = A.sched + (size_t)job * A.nsteps_max * 3;
    const int ns = A.job_nsteps[job];
    const float h = A.job_h[job];
    unsigned char st = LCS_TRACER_OK;
    float te = A.job_tend[job];
    bool live = active;
    for (int n = 0; n < ns; ++n) {
        __syncthreads();  // every thread is done with the previous step's slots
        if (R.abort) break;
        if (tid == 0) {
            SchedEntry e[3] = {sc[3 * n], sc[3 * n + 1], sc[3 * n + 2]};
            int F[6], Fn[6];
            int m = step_frames(e, F);
            for (int r = 0; r < m; ++r)
                if (ring_find(R, F[r]) < 0) ring_load(R, slots, frames, fstride, F[r], F, m, errword);
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
                    if (ring_find(R, Fn[r]) < 0) ring_load(R, slots, frames, fstride, Fn[r], keep, nk, errword);
            }
        }
        __syncthreads();
        // wait for the copies this step reads
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            int s = R.slot[q];
            if (s >= 0 && !R.abort && !mbar_wait_bounded(&R.bar[s], (R.nload[s] - 1) & 1)) {
                atomicOr(errword, LCS_ERRBIT_TIMEOUT);
                R.abort = 1;
            }
        }
        if (!live || R.abort) continue;
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
        bool all_smem = (R.slot[0] != RING_GLOBAL) && (R.slot[1] != RING_GLOBAL) && (R.slot[2] != RING_GLOBAL) &&
                        (R.slot[3] != RING_GLOBAL) && (R.slot[4] != RING_GLOBAL) && (R.slot[5] != RING_GLOBAL);
        // a step whose frames did not all get a slot (e.g. one straddling the periodic wrap, which
        // reads four frames) mixes shared and global pointers: generic loads serve both
        if (all_smem)
            rk4_step<2, ST, SRC_SHARED>(P, x, h, p[0], p[1], e0.a, p[2], p[3], e1.a, p[4], p[5], e2.a);
        else
            rk4_step<2, ST, SRC_GENERIC>(P, x, h, p[0], p[1], e0.a, p[2], p[3], e1.a, p[4], p[5], e2.a);
        wrap_periodic<2>(P, x, img);
        if (rect_left<2>(P, x)) {
            st = LCS_TRACER_LEFT;
            te = fmaf((float)(n + 1), h, A.job_t0[job]);
            live = false;
        }
    }
    // drain copies still in flight (prefetches nobody read) before the block exits
    __syncthreads();
    if (tid == 0)
        for (int s = 0; s < RING_SLOTS; ++s)
            if (R.nload[s] > 0 && !mbar_wait_bounded(&R.bar[s], (R.nload[s] - 1) & 1))
                atomicOr(errword, LCS_ERRBIT_TIMEOUT);
    __syncthreads();
    if (active) store_tracer<2>(P, A, job, i, x, img, st, te);
}

// ======================================================= re-bundled episodes (3D)
//
// Tracers of one warp drift apart in a mixing flow, so after a few hundred steps
// the 32 lanes of a warp read 32 unrelated cells and every load turns into ~30 L1
// wavefronts.  The integration is therefore cut into episodes of E steps; before
// each episode the tracer states are re-bundled by the cell they sit in (a
// counting sort on the x-fastest cell index), so that consecutive threads sit in
// the same rows of cells again (the spatial re-bundling the paper cites, Sec. 3.2).
// Each tracer's arithmetic does not depend on where it sits, so the result is
// bit-identical to the unsorted kernel.

struct TState {
    float *x, *y, *z;      // positions, wrapped into [origin, origin + L) on periodic axes
    short *ix, *iy, *iz;   // periods crossed per axis
    int *id;               // seed index
    unsigned char *st;     // tracer status
    float *te;             // exit time
};

__global__ void ep_init_kernel(RectParams P, const float *__restrict__ seeds, long long N, TState S,
                               const float *__restrict__ job_tend, int job)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    float x[3] = {seeds[i], seeds[N + i], seeds[2 * N + i]};
    int img[3] = {0, 0, 0};
    wrap_periodic<3>(P, x, img);
    S.x[i] = x[0];
    S.y[i] = x[1];
    S.z[i] = x[2];
    S.ix[i] = (short)img[0];
    S.iy[i] = (short)img[1];
    S.iz[i] = (short)img[2];
    S.id[i] = (int)i;
    S.st[i] = LCS_TRACER_OK;
    S.te[i] = job_tend[job];
}

// key = x-fastest index of the cell holding the tracer (coarsened by `shift` bits)
__global__ void ep_key_kernel(RectParams P, TState S, long long N, int shift, unsigned *__restrict__ keys,
                              unsigned *__restrict__ hist)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    float x[3] = {S.x[i], S.y[i], S.z[i]};
    int c[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float sd = (x[d] - P.origin[d]) * P.inv_h[d];
        int v = isfinite(sd) ? (int)floorf(fminf(fmaxf(sd, 0.0f), (float)P.n[d])) : 0;
        int hi = P.periodic[d] ? P.n[d] - 1 : P.n[d] - 2;
        c[d] = min(max(v, 0), hi);
    }
    unsigned key = (unsigned)((c[0] + P.sy * (long long)c[1] + P.sz * (long long)c[2]) >> shift);
    keys[i] = key;
    atomicAdd(hist + key, 1u);
}

// exclusive scan of a 1024-thread block (one value per thread)
__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned *total)
{
    __shared__ unsigned wsum[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned t = lane < nw ? wsum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        wsum[lane] = t;
    }
    __syncthreads();
    unsigned pre = (w > 0 ? wsum[w - 1] : 0u) + x - v;
    *total = wsum[nw - 1];
    __syncthreads();
    return pre;
}

#define SCAN_ITEMS 4
#define SCAN_TILE (1024 * SCAN_ITEMS)

__global__ void __launch_bounds__(1024) scan_reduce_kernel(const unsigned *__restrict__ in, long long n,
                                                           unsigned *__restrict__ bsum)
{
    long long base = (long long)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    unsigned t = 0;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q)
        if (base + q < n) t += in[base + q];
    unsigned tot;
    block_excl_scan(t, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// one block: exclusive scan of up to 1024 * SCAN_ITEMS block sums, in place
__global__ void __launch_bounds__(1024) scan_top_kernel(unsigned *__restrict__ bsum, int nb)
{
    int base = threadIdx.x * SCAN_ITEMS;
    unsigned v[SCAN_ITEMS], t = 0;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        v[q] = base + q < nb ? bsum[base + q] : 0u;
        t += v[q];
    }
    unsigned tot;
    unsigned pre = block_excl_scan(t, &tot);
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        if (base + q < nb) bsum[base + q] = pre;
        pre += v[q];
    }
}

__global__ void __launch_bounds__(1024) scan_down_kernel(const unsigned *__restrict__ in, long long n,
                                                         const unsigned *__restrict__ bsum,
                                                         unsigned *__restrict__ out)
{
    long long base = (long long)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    unsigned v[SCAN_ITEMS], t = 0;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        v[q] = base + q < n ? in[base + q] : 0u;
        t += v[q];
    }
    unsigned tot;
    unsigned pre = block_excl_scan(t, &tot) + bsum[blockIdx.x];
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        if (base + q < n) out[base + q] = pre;
        pre += v[q];
    }
}

__global__ void ep_scatter_kernel(TState A, TState B, long long N, const unsigned *__restrict__ keys,
                                  unsigned *__restrict__ cursor)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    unsigned p = atomicAdd(cursor + keys[i], 1u);
    B.x[p] = A.x[i];
    B.y[p] = A.y[i];
    B.z[p] = A.z[i];
    B.ix[p] = A.ix[i];
    B.iy[p] = A.iy[i];
    B.iz[p] = A.iz[i];
    B.id[p] = A.id[i];
    B.st[p] = A.st[i];
    B.te[p] = A.te[i];
}

template <int ST>
__global__ void __launch_bounds__(256) ep_advect3_kernel(RectParams P, const char *__restrict__ pairs, size_t fstride,
                                                         Rk4Args A, TState S, int job, int s0, int s1)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= A.N) return;
    if (S.st[i] != LCS_TRACER_OK) return;
    float x[3] = {S.x[i], S.y[i], S.z[i]};
    int img[3] = {S.ix[i], S.iy[i], S.iz[i]};
    const SchedEntry *sc = A.sched + (size_t)job * A.nsteps_max * 3;
    const int ns = A.job_nsteps[job];
    const float h = A.job_h[job];
    const int e = min(s1, ns);
    unsigned char st = LCS_TRACER_OK;
    float te = 0.0f;
    for (int n = s0; n < e; ++n) {
        SchedEntry e0 = load_sched(sc + 3 * n), e1 = load_sched(sc + 3 * n + 1), e2 = load_sched(sc + 3 * n + 2);
        rk4_step3p<ST>(P, x, h, pairs + (size_t)e0.k * fstride, e0.a, pairs + (size_t)e1.k * fstride, e1.a,
                       pairs + (size_t)e2.k * fstride, e2.a);
        wrap_periodic<3>(P, x, img);
        if (rect_left<3>(P, x)) {
            st = LCS_TRACER_LEFT;
            te = fmaf((float)(n + 1), h, A.job_t0[job]);
            break;
        }
    }
    S.x[i] = x[0];
    S.y[i] = x[1];
    S.z[i] = x[2];
    S.ix[i] = (short)img[0];
    S.iy[i] = (short)img[1];
    S.iz[i] = (short)img[2];
    if (st != LCS_TRACER_OK) {
        S.st[i] = st;
        S.te[i] = te;
    }
}

__global__ void ep_finalize_kernel(RectParams P, TState S, long long N, float *__restrict__ out_xyz,
                                   unsigned char *__restrict__ out_st, float *__restrict__ out_te)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    long long id = S.id[i];
    float x[3] = {S.x[i], S.y[i], S.z[i]};
    int img[3] = {S.ix[i], S.iy[i], S.iz[i]};
#pragma unroll
    for (int d = 0; d < 3; ++d) out_xyz[d * N + id] = P.periodic[d] ? fmaf((float)img[d], P.L[d], x[d]) : x[d];
    out_st[id] = S.st[i];
    out_te[id] = S.te[i];
}

// Time slices of one episode: every distinct stage time of steps [s0, s1) gets the
// field blended to it at every node (consecutive equal schedule entries -- the end of
// step n and the start of step n + 1 -- share one slice).  One thread builds the
// table: smap[3 (n - s0) + stage] = slice, stab[slice] = (k, alpha), count in *nsl.
__global__ void ep_slice_table_kernel(const SchedEntry *__restrict__ sched, int nsteps_max, int job, int s0,
                                      int s1, int *__restrict__ smap, SchedEntry *__restrict__ stab,
                                      int *__restrict__ nsl)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const SchedEntry *sc = sched + (size_t)job * nsteps_max * 3;
    int m = 0;
    SchedEntry last = {-1, 0.0f};
    for (int n = s0; n < s1; ++n)
        for (int st = 0; st < 3; ++st) {
            SchedEntry e = sc[3 * n + st];
            bool same = m > 0 && e.k == last.k && __float_as_int(e.a) == __float_as_int(last.a);
            if (!same) {
                stab[m++] = e;
                last = e;
            }
            smap[3 * (n - s0) + st] = m - 1;
        }
    *nsl = m;
}

// slice j, node v = blend of interval pair stab[j].k at weight stab[j].a (same arithmetic as interp3p)
__global__ void ep_slice_fill_kernel(const char *__restrict__ pairs, size_t fstride, long long nodes,
                                     const SchedEntry *__restrict__ stab, const int *__restrict__ nsl,
                                     float4 *__restrict__ slices, size_t slice_stride)
{
    const int j = blockIdx.y;
    if (j >= *nsl) return;
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= nodes) return;
    const SchedEntry e = stab[j];
    float va[3], vb[3];
    Pair3<LCS_F32>::ld(pairs + (size_t)e.k * fstride, (int)v, va, vb);
    const float g = 1.0f - e.a;
    float4 o;
    if (e.a == 0.0f) {
        o = make_float4(va[0], va[1], va[2], 0.0f);
    } else {
        o = make_float4(tblend(va[0], vb[0], e.a, g), tblend(va[1], vb[1], e.a, g), tblend(va[2], vb[2], e.a, g),
                        0.0f);
    }
    slices[(size_t)j * slice_stride + v] = o;
}

__global__ void __launch_bounds__(256) ep_advect3s_kernel(RectParams P, const float4 *__restrict__ slices,
                                                          size_t slice_stride, const int *__restrict__ smap, Rk4Args A,
                                                          TState S, int job, int s0, int s1)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= A.N) return;
    if (S.st[i] != LCS_TRACER_OK) return;
    float x[3] = {S.x[i], S.y[i], S.z[i]};
    int img[3] = {S.ix[i], S.iy[i], S.iz[i]};
    const int ns = A.job_nsteps[job];
    const float h = A.job_h[job];
    const int e = min(s1, ns);
    unsigned char st = LCS_TRACER_OK;
    float te = 0.0f;
    for (int n = s0; n < e; ++n) {
        const int *m = smap + 3 * (n - s0);
        rk4_step3s(P, x, h, slices + (size_t)__ldg(m) * slice_stride, slices + (size_t)__ldg(m + 1) * slice_stride,
                   slices + (size_t)__ldg(m + 2) * slice_stride);
        wrap_periodic<3>(P, x, img);
        if (rect_left<3>(P, x)) {
            st = LCS_TRACER_LEFT;
            te = fmaf((float)(n + 1), h, A.job_t0[job]);
            break;
        }
    }
    S.x[i] = x[0];
    S.y[i] = x[1];
    S.z[i] = x[2];
    S.ix[i] = (short)img[0];
    S.iy[i] = (short)img[1];
    S.iz[i] = (short)img[2];
    if (st != LCS_TRACER_OK) {
        S.st[i] = st;
        S.te[i] = te;
    }
}

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// coarsen cell keys so that at most 2^24 bins exist (the scan handles 4096 tiles of 4096)
static int sort_shift(long long nodes)
{
    int shift = 0;
    while (((nodes - 1) >> shift) + 1 > (1LL << 24)) ++shift;
    return shift;
}

static size_t slice_bytes(long long nodes, int E)
{
    return al256(16 * (size_t)nodes) * 3 * E + al256(sizeof(int) * 3 * E) + al256(sizeof(SchedEntry) * 3 * E) + 256;
}

size_t rk4_sorted_scratch_bytes(long long N, long long nodes, int storage, int E)
{
    long long nbins = ((nodes - 1) >> sort_shift(nodes)) + 1;
    size_t per = al256(4 * N) * 3 + al256(2 * N) * 3 + al256(4 * N) + al256(N) + al256(4 * N);
    long long nb = (nbins + SCAN_TILE - 1) / SCAN_TILE;
    size_t b = 2 * per + al256(4 * N) + 2 * al256(4 * nbins) + al256(4 * nb);
    if (storage == LCS_F32) b += slice_bytes(nodes, E);
    return b;
}

static TState carve_state(char *&p, long long N)
{
    TState S;
    S.x = (float *)p;
    p += al256(4 * N);
    S.y = (float *)p;
    p += al256(4 * N);
    S.z = (float *)p;
    p += al256(4 * N);
    S.ix = (short *)p;
    p += al256(2 * N);
    S.iy = (short *)p;
    p += al256(2 * N);
    S.iz = (short *)p;
    p += al256(2 * N);
    S.id = (int *)p;
    p += al256(4 * N);
    S.st = (unsigned char *)p;
    p += al256(N);
    S.te = (float *)p;
    p += al256(4 * N);
    return S;
}

template <int ST>
static cudaError_t launch_sorted3(const RectParams &P, const lcs_field *f, const Rk4Args &A, const Rk4Launch &L,
                                  cudaStream_t s)
{
    const long long N = A.N;
    const int shift = sort_shift(f->nodes);
    const long long nbins = ((f->nodes - 1) >> shift) + 1;
    const long long nb = (nbins + SCAN_TILE - 1) / SCAN_TILE;
    if (nb > 1024 * SCAN_ITEMS) return cudaErrorInvalidValue;
    char *p = (char *)L.work;
    TState SA = carve_state(p, N), SB = carve_state(p, N);
    unsigned *keys = (unsigned *)p;
    p += al256(4 * N);
    unsigned *hist = (unsigned *)p;
    p += al256(4 * nbins);
    unsigned *cursor = (unsigned *)p;
    p += al256(4 * nbins);
    unsigned *bsum = (unsigned *)p;
    p += al256(4 * nb);
    const int bt = 256;
    const unsigned grid = (unsigned)((N + bt - 1) / bt);
    const int E = L.episode_steps > 0 ? L.episode_steps : LCS_EPISODE_STEPS;
    // FP32 storage: time slices (16-byte nodes) instead of 32-byte interval pairs per corner
    const bool use_slices = ST == LCS_F32;
    const size_t slice_stride = al256(16 * (size_t)f->nodes) / 16;
    float4 *slices = nullptr;
    int *smap = nullptr, *nsl = nullptr;
    SchedEntry *stab = nullptr;
    if (use_slices) {
        slices = (float4 *)p;
        p += al256(16 * (size_t)f->nodes) * 3 * E;
        smap = (int *)p;
        p += al256(sizeof(int) * 3 * E);
        stab = (SchedEntry *)p;
        p += al256(sizeof(SchedEntry) * 3 * E);
        nsl = (int *)p;
    }
    for (int job = 0; job < L.njobs; ++job) {
        ep_init_kernel<<<grid, bt, 0, s>>>(P, A.seeds, N, SA, A.job_tend, job);
        const int ns = L.host_nsteps[job];
        for (int s0 = 0; s0 < ns; s0 += E) {
            cudaMemsetAsync(hist, 0, 4 * nbins, s);
            ep_key_kernel<<<grid, bt, 0, s>>>(P, SA, N, shift, keys, hist);
            scan_reduce_kernel<<<(unsigned)nb, 1024, 0, s>>>(hist, nbins, bsum);
            scan_top_kernel<<<1, 1024, 0, s>>>(bsum, (int)nb);
            scan_down_kernel<<<(unsigned)nb, 1024, 0, s>>>(hist, nbins, bsum, cursor);
            ep_scatter_kernel<<<grid, bt, 0, s>>>(SA, SB, N, keys, cursor);
            const int s1 = s0 + E < ns ? s0 + E : ns;
            if (use_slices) {
                ep_slice_table_kernel<<<1, 32, 0, s>>>(A.sched, A.nsteps_max, job, s0, s1, smap, stab, nsl);
                dim3 fg((unsigned)((f->nodes + 255) / 256), (unsigned)(3 * (s1 - s0)));
                ep_slice_fill_kernel<<<fg, 256, 0, s>>>((const char *)f->d_frames, f->frame_stride, f->nodes, stab,
                                                         nsl, slices, slice_stride);
                ep_advect3s_kernel<<<grid, bt, 0, s>>>(P, slices, slice_stride, smap, A, SB, job, s0, s1);
            } else {
                ep_advect3_kernel<ST><<<grid, bt, 0, s>>>(P, (const char *)f->d_frames, f->frame_stride, A, SB, job,
                                                          s0, s1);
            }
            TState t = SA;
            SA = SB;
            SB = t;
        }
        ep_finalize_kernel<<<grid, bt, 0, s>>>(P, SA, N, A.out_xyz + (size_t)job * 3 * N, A.out_status + (size_t)job * N,
                                               A.out_texit + (size_t)job * N);
    }
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

template <int ST>
static cudaError_t launch_ring(lcs_ctx *ctx, const RectParams &P, const lcs_field *f, const Rk4Args &A, int njobs,
                               int bt, cudaStream_t s)
{
    size_t smem = RING_SLOTS * f->frame_stride;
    cudaError_t e = cudaFuncSetAttribute(rk4_ring2d_kernel<ST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((A.N + bt - 1) / bt), (unsigned)njobs);
    rk4_ring2d_kernel<ST><<<grid, bt, smem, s>>>(P, (const char *)f->d_frames, f->frame_stride, A, ctx->d_errword);
    return cudaGetLastError();
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
    if (L.N == 0 || L.njobs == 0) return 1;
    bool ring_fits = f->dim == 2 && RING_SLOTS * f->frame_stride <= ctx->smem_optin;
    bool sorted_ok = f->dim == 3 && L.work != nullptr;
    int variant = L.variant;
    if (variant == 0) variant = ring_fits ? 2 : (sorted_ok && L.N >= LCS_SORTED_MIN_SEEDS ? 3 : 1);
    if (variant == 2 && !ring_fits) variant = 1;
    if (variant == 3 && !sorted_ok) variant = 1;
    cudaError_t e;
    if (variant == 3) {
        if (f->storage == LCS_F32)
            e = launch_sorted3<LCS_F32>(P, f, A, L, s);
        else if (f->storage == LCS_F16)
            e = launch_sorted3<LCS_F16>(P, f, A, L, s);
        else
            e = launch_sorted3<LCS_BF16>(P, f, A, L, s);
    } else if (variant == 2) {
        int bt = L.block_threads > 0 ? L.block_threads : 512;
        if (bt > 512) bt = 512;
        if (f->storage == LCS_F32)
            e = launch_ring<LCS_F32>(ctx, P, f, A, L.njobs, bt, s);
        else if (f->storage == LCS_F16)
            e = launch_ring<LCS_F16>(ctx, P, f, A, L.njobs, bt, s);
        else
            e = launch_ring<LCS_BF16>(ctx, P, f, A, L.njobs, bt, s);
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
    return e == cudaSuccess ? variant : -1;
}
