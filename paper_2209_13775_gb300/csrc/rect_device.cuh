// rect_device.cuh -- device building blocks of the rectilinear advection kernels:
// storage loads, cell location, (bi/tri)linear stencils, time blending, one RK4
// step, periodic wrapping and the domain-exit test.  Included by advect_rect.cu
// and advect_episodes.cu.
#pragma once

#include "lcs_internal.cuh"

#include <math.h>

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

// Periodicity of axis d: from the compile-time mask PM when PM >= 0 (bit d set =
// periodic), else from the run-time parameters.
template <int PM>
__device__ __forceinline__ bool per_axis(const RectParams &P, int d)
{
    if constexpr (PM >= 0)
        return (PM >> d) & 1;
    else
        return P.periodic[d] != 0;
}

static __device__ __noinline__ int wrap_index_slow(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

// Cell along axis d.  Non-periodic: clamp the query into the box, cell i with
// node_i <= x < node_{i+1}, the last cell closed.  Periodic: wrap the index (one
// period up or down inline; farther only through the slow path).
template <int PM>
__device__ __forceinline__ void axis_cell(const RectParams &P, int d, float x, int &i0, int &i1, float &f)
{
    if (per_axis<PM>(P, d)) {
        float s = (x - P.origin[d]) * P.inv_h[d];
        float fl = floorf(s);
        int i = (int)fl;
        f = s - fl;
        const int n = P.n[d];
        i = i < 0 ? i + n : (i >= n ? i - n : i);
        if ((unsigned)i >= (unsigned)n) i = wrap_index_slow(i, n);
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

template <int DIM, int PM = -1>
__device__ __forceinline__ void make_stencil(const RectParams &P, const float *x, Stencil<DIM> &S)
{
    int i0, i1, j0, j1;
    float fx, fy;
    axis_cell<PM>(P, 0, x[0], i0, i1, fx);
    axis_cell<PM>(P, 1, x[1], j0, j1, fy);
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
        axis_cell<PM>(P, 2, x[2], k0, k1, fz);
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

// Time blend of one node, FP32: u = (1 - a) u_k + a u_{k+1} (exactly u_k when a == 0).
// Every kernel blends at the nodes first, then interpolates in space: both orders are the
// same linear map, and one order everywhere makes the kernels agree bit for bit (and lets
// a whole field be blended to a stage time once, as a time slice, with the same result).
__device__ __forceinline__ float tblend(float ua, float ub, float a, float g)
{
    return fmaf(a, ub, g * ua);
}

// u = I[(1 - a) frame fa + a frame fb](x), node blends first; frame fb is not read when a == 0
template <int DIM, int ST, int SRC>
__device__ __forceinline__ void interp(const Stencil<DIM> &S, const char *fa, const char *fb, float a, float *u)
{
    float acc[DIM], va[DIM], vb[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) acc[c] = 0.0f;
    if (a == 0.0f) {
#pragma unroll
        for (int q = 0; q < (1 << DIM); ++q) {
            node_load<DIM, ST, SRC>(fa, S.v[q], va);
#pragma unroll
            for (int c = 0; c < DIM; ++c) acc[c] = fmaf(S.w[q], va[c], acc[c]);
        }
    } else {
        const float g = 1.0f - a;
#pragma unroll
        for (int q = 0; q < (1 << DIM); ++q) {
            node_load<DIM, ST, SRC>(fa, S.v[q], va);
            node_load<DIM, ST, SRC>(fb, S.v[q], vb);
#pragma unroll
            for (int c = 0; c < DIM; ++c) acc[c] = fmaf(S.w[q], tblend(va[c], vb[c], a, g), acc[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < DIM; ++c) u[c] = acc[c];
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
    float *out_grad = nullptr;       // variational grad F [njobs][N][dim][dim], or null
    int njobs = 0;                   // jobs of the call: snapshot s of job j goes to slot njobs + j nsnap + s
    int nsnap = 0;
    const int *snap_n = nullptr;     // [nsnap] snapshot step counts (device; capped per job at use)
    const float *snap_te = nullptr;  // [njobs][nsnap] snapshot end times, the exit time of a tracer OK there
    unsigned long long wait_ns = LCS_WAIT_LIMIT_NS;  // ring kernels: bound on a wait for a frame copy
};

// Step after which snapshot s of a job with ns steps is taken.
__device__ __forceinline__ int snap_step(const Rk4Args &A, int s, int ns) { return min(__ldg(A.snap_n + s), ns); }

__device__ __forceinline__ int snap_slot(const Rk4Args &A, int job, int s) { return A.njobs + job * A.nsnap + s; }

// exit time recorded in snapshot s of a tracer with status st and exit time te
__device__ __forceinline__ float snap_exit(const Rk4Args &A, int job, int s, unsigned char st, float te)
{
    return st == LCS_TRACER_OK ? __ldg(A.snap_te + job * A.nsnap + s) : te;
}

__device__ __forceinline__ SchedEntry load_sched(const SchedEntry *p)
{
    int2 r = __ldg(reinterpret_cast<const int2 *>(p));
    SchedEntry e;
    e.k = r.x;
    e.a = __int_as_float(r.y);
    return e;
}

// periodic axes: keep x in [origin, origin + L) with an integer count of periods; c is the
// coordinate's carried rounding (rk4_advance), which the shift's own rounding joins
template <int DIM, int PM = -1>
__device__ __forceinline__ void wrap_periodic(const RectParams &P, float *x, float *c, int *img)
{
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        if (!per_axis<PM>(P, d)) continue;
        float hiL = P.origin[d] + P.L[d];
        if (x[d] >= hiL) {
            add_carried(x[d], c[d], -P.L[d]);
            img[d] += 1;
        } else if (x[d] < P.origin[d]) {
            add_carried(x[d], c[d], P.L[d]);
            img[d] -= 1;
        }
        if (!(x[d] >= P.origin[d] && x[d] < hiL) && isfinite(x[d])) {  // far outside: full reduction
            float m = floorf((x[d] - P.origin[d]) / P.L[d]);
            add_carried(x[d], c[d], -m * P.L[d]);
            img[d] += (int)m;
            if (x[d] >= hiL) {
                x[d] = P.origin[d];
                c[d] = 0.0f;
            }
        }
    }
}

template <int DIM, int PM = -1>
__device__ __forceinline__ bool rect_left(const RectParams &P, const float *x)
{
    bool out = false;
#pragma unroll
    for (int d = 0; d < DIM; ++d)
        if (!per_axis<PM>(P, d)) out |= (x[d] < P.left_lo[d]) || (x[d] > P.left_hi[d]);
    return out;
}

// the flow-map coordinate of a tracer: x + c rounded once, unwrapped on periodic axes
__device__ __forceinline__ float out_coord(const RectParams &P, int d, float x, float c, int img)
{
    const float v = x + c;
    return P.periodic[d] ? fmaf((float)img, P.L[d], v) : v;
}

template <int DIM>
__device__ __forceinline__ void store_tracer(const RectParams &P, const Rk4Args &A, int job, long long i,
                                             const float *x, const float *c, const int *img, unsigned char st,
                                             float te)
{
    float *o = A.out_xyz + (size_t)job * DIM * A.N;
#pragma unroll
    for (int d = 0; d < DIM; ++d) o[d * A.N + i] = out_coord(P, d, x[d], c[d], img[d]);
    A.out_status[(size_t)job * A.N + i] = st;
    A.out_texit[(size_t)job * A.N + i] = te;
}

// one RK4 step of x (+ its carried rounding c); stage frames given by (fa, fb, a) triples
template <int DIM, int ST, int SRC>
__device__ __forceinline__ void rk4_step(const RectParams &P, float *x, float *cx, float h, const char *fa0,
                                         const char *fb0,
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
    for (int c = 0; c < DIM; ++c) rk4_advance(x[c], cx[c], h6, k1[c], k2[c], k3[c], k4[c]);
}

// one RK4 step in 3D; stage s reads interval pair ps with weight as
template <int ST, int PM = -1>
__device__ __forceinline__ void rk4_step3p(const RectParams &P, float *x, float *cx, float h, const char *p0, float a0,
                                           const char *p1, float a1, const char *p2, float a2)
{
    float k1[3], k2[3], k3[3], k4[3], y[3];
    Stencil<3> S;
    const float hh = 0.5f * h;
    make_stencil<3, PM>(P, x, S);
    interp3p<ST>(S, p0, a0, k1);
#pragma unroll
    for (int c = 0; c < 3; ++c) y[c] = fmaf(hh, k1[c], x[c]);
    make_stencil<3, PM>(P, y, S);
    interp3p<ST>(S, p1, a1, k2);
#pragma unroll
    for (int c = 0; c < 3; ++c) y[c] = fmaf(hh, k2[c], x[c]);
    make_stencil<3, PM>(P, y, S);
    interp3p<ST>(S, p1, a1, k3);
#pragma unroll
    for (int c = 0; c < 3; ++c) y[c] = fmaf(h, k3[c], x[c]);
    make_stencil<3, PM>(P, y, S);
    interp3p<ST>(S, p2, a2, k4);
    const float h6 = h * (1.0f / 6.0f);
#pragma unroll
    for (int c = 0; c < 3; ++c) rk4_advance(x[c], cx[c], h6, k1[c], k2[c], k3[c], k4[c]);
}

// 3D RK4 with tracers re-bundled by cell between episodes (advect_episodes.cu)
cudaError_t launch_rk4_episodes(const RectParams &P, const lcs_field *f, const Rk4Args &A, const Rk4Launch &L,
                                cudaStream_t s);
