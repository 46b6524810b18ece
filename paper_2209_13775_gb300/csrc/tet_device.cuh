// tet_device.cuh -- device building blocks for velocity data on tetrahedral meshes
// (Sec. 3.1: data tetrahedralized so that one local cell search serves every mesh).
//
//  * tet_locate: the local walk of the hot loop, FP32 barycentric coordinates from a
//    per-tet inverse affine map: stop when no coordinate is below -tol, else cross the
//    face of the most negative one.  A walk that meets a boundary face means the point is
//    outside when the mesh is convex (checked at load time); otherwise the tets listed for
//    the point's bin (every tet whose bounding box meets the bin) decide, so the mesh need
//    not be convex.  A walk past its step limit reports WALKFAIL.
//  * tet_interp: piecewise-linear (P1) interpolation of the frame pair k, blended in
//    time at the four vertices.
//  * orient3d_sign: exact orientation of four FP32 points (filtered FP64 evaluation,
//    exact expansion arithmetic when the filter cannot decide), for the exact seed
//    location of lcs_seed_grid.
#pragma once

#include "lcs_internal.cuh"

#include <math.h>

struct TetDev {
    const float4 *xyz;    // [nnodes]
    const int4 *tets;     // [ncells] node ids
    const int4 *nbrs;     // [ncells] tet across the face opposite vertex j, -1 boundary
    const float4 *tmap;   // [ncells][4]: row r < 3 = (M_r0, M_r1, M_r2, v0_r), lambda_{r+1} = M_r . (x - v0);
                          // row 3 = the cell's nbrs entry (int bits), so a walk step is two 32-byte loads
    const int *bstart;    // [nbins + 1] CSR of the tets whose bounding box meets a bin
    const int *blist;     //   (ids increasing within a bin)
    float blo[3], binv[3];
    int bn[3];
    const char *pairs;    // [nslabs][nnodes] (u_k, 0, u_{k+1}, 0) in storage precision
    size_t fstride;       // bytes per slab
    long long ncells;
    int walk_limit;
    float tol;            // barycentric tolerance of the FP32 walk
    int convex;           // the mesh is convex: a boundary face separates the point from the mesh
};

enum { TET_INSIDE = 0, TET_OUTSIDE = 1, TET_WALKFAIL = 2 };

TetDev tet_dev(const lcs_field *f, int walk_limit);  // tet_store.cu

// bin of a coordinate: floor((x - lo) * inv) clamped to the grid (monotone in x, so a cell's
// bounding-box bins always include the bin of every point it holds)
__device__ __forceinline__ int mesh_bin_axis(float x, float lo, float inv, int n)
{
    const float s = (x - lo) * inv;
    return isfinite(s) ? (int)fminf(fmaxf(floorf(s), 0.0f), (float)(n - 1)) : 0;
}

__device__ __forceinline__ int tet_bin(const TetDev &T, const float *x)
{
    return mesh_bin_axis(x[0], T.blo[0], T.binv[0], T.bn[0]) +
           T.bn[0] * (mesh_bin_axis(x[1], T.blo[1], T.binv[1], T.bn[1]) +
                      T.bn[1] * mesh_bin_axis(x[2], T.blo[2], T.binv[2], T.bn[2]));
}

// the 64-byte record of tet c: map rows r0..r2 and the neighbours, as two 32-byte loads (lanes
// gathering 32 bytes each cost the L1 data stage fewer wavefronts per byte than 16-byte gathers)
__device__ __forceinline__ void tet_record(const TetDev &T, int c, float4 &r0, float4 &r1, float4 &r2, int4 &nb)
{
    const float4 *p = T.tmap + 4 * (size_t)c;
    float a[8], b[8];
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a[0]), "=f"(a[1]), "=f"(a[2]), "=f"(a[3]), "=f"(a[4]), "=f"(a[5]), "=f"(a[6]), "=f"(a[7])
        : "l"(p));
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(b[0]), "=f"(b[1]), "=f"(b[2]), "=f"(b[3]), "=f"(b[4]), "=f"(b[5]), "=f"(b[6]), "=f"(b[7])
        : "l"(p + 2));
    r0 = make_float4(a[0], a[1], a[2], a[3]);
    r1 = make_float4(a[4], a[5], a[6], a[7]);
    r2 = make_float4(b[0], b[1], b[2], b[3]);
    nb = make_int4(__float_as_int(b[4]), __float_as_int(b[5]), __float_as_int(b[6]), __float_as_int(b[7]));
}

// barycentric coordinates of x in the tet with map rows r0..r2 (FP32)
__device__ __forceinline__ void tet_bary_rows(const float4 &r0, const float4 &r1, const float4 &r2, const float *x,
                                              float *lam)
{
    const float dx = x[0] - r0.w, dy = x[1] - r1.w, dz = x[2] - r2.w;
    lam[1] = fmaf(r0.x, dx, fmaf(r0.y, dy, r0.z * dz));
    lam[2] = fmaf(r1.x, dx, fmaf(r1.y, dy, r1.z * dz));
    lam[3] = fmaf(r2.x, dx, fmaf(r2.y, dy, r2.z * dz));
    lam[0] = 1.0f - lam[1] - lam[2] - lam[3];
}

// barycentric coordinates of x in tet c (FP32).  Plain 16-byte loads: the out-of-line bin scan
// calls this, and with tet_record's 32-byte loads there the CUDA 13.0 ptxas crashed on this file.
__device__ __forceinline__ void tet_bary(const TetDev &T, int c, const float *x, float *lam)
{
    const float4 *p = T.tmap + 4 * (size_t)c;
    tet_bary_rows(__ldg(p), __ldg(p + 1), __ldg(p + 2), x, lam);
}

// the tets listed for x's bin, in id order: the first whose coordinates all reach -tol
static __device__ __noinline__ int tet_bin_scan(const TetDev &T, const float *x, int *cell, float *lam)
{
    if (!(isfinite(x[0]) && isfinite(x[1]) && isfinite(x[2]))) return TET_OUTSIDE;
    const int b = tet_bin(T, x);
    const int q1 = __ldg(T.bstart + b + 1);
    for (int q = __ldg(T.bstart + b); q < q1; ++q) {
        const int c = __ldg(T.blist + q);
        tet_bary(T, c, x, lam);
        if (fminf(fminf(lam[0], lam[1]), fminf(lam[2], lam[3])) >= -T.tol) {
            *cell = c;
            return TET_INSIDE;
        }
    }
    return TET_OUTSIDE;
}

// walk from *cell to the tet holding x; lam receives its barycentric coordinates
__device__ __forceinline__ int tet_locate(const TetDev &T, const float *x, int *cell, float *lam)
{
    int c = *cell;
    if (c < 0 || c >= T.ncells) c = 0;
    for (int it = 0; it < T.walk_limit; ++it) {
        float4 r0, r1, r2;
        int4 nb;
        tet_record(T, c, r0, r1, r2, nb);
        tet_bary_rows(r0, r1, r2, x, lam);
        int jm = 0;
        float lm = lam[0];
#pragma unroll
        for (int j = 1; j < 4; ++j)
            if (lam[j] < lm) {
                lm = lam[j];
                jm = j;
            }
        if (lm >= -T.tol) {
            *cell = c;
            return TET_INSIDE;
        }
        const int n = jm == 0 ? nb.x : jm == 1 ? nb.y : jm == 2 ? nb.z : nb.w;
        if (n < 0) {
            *cell = c;
            return T.convex ? TET_OUTSIDE : tet_bin_scan(T, x, cell, lam);
        }
        c = n;
    }
    *cell = c;
    return TET_WALKFAIL;
}

template <int ST>
struct TetPair;

template <>
struct TetPair<LCS_F32> {
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

__device__ __forceinline__ float2 tet_h2f(unsigned r)
{
    __half2 h = *reinterpret_cast<__half2 *>(&r);
    return __half22float2(h);
}

__device__ __forceinline__ float2 tet_b2f(unsigned r)
{
    __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162 *>(&r);
    return __bfloat1622float2(h);
}

template <>
struct TetPair<LCS_F16> {
    static __device__ __forceinline__ void ld(const char *f, int v, float *ua, float *ub)
    {
        uint4 r = __ldg(reinterpret_cast<const uint4 *>(f) + v);
        float2 a = tet_h2f(r.x), b = tet_h2f(r.y), c = tet_h2f(r.z), d = tet_h2f(r.w);
        ua[0] = a.x;
        ua[1] = a.y;
        ua[2] = b.x;
        ub[0] = c.x;
        ub[1] = c.y;
        ub[2] = d.x;
    }
};

template <>
struct TetPair<LCS_BF16> {
    static __device__ __forceinline__ void ld(const char *f, int v, float *ua, float *ub)
    {
        uint4 r = __ldg(reinterpret_cast<const uint4 *>(f) + v);
        float2 a = tet_b2f(r.x), b = tet_b2f(r.y), c = tet_b2f(r.z), d = tet_b2f(r.w);
        ua[0] = a.x;
        ua[1] = a.y;
        ua[2] = b.x;
        ub[0] = c.x;
        ub[1] = c.y;
        ub[2] = d.x;
    }
};

// u = sum_i lam_i [(1 - a) u_k + a u_{k+1}](vertex i) from the interval pair at fp
template <int ST>
__device__ __forceinline__ void tet_interp(const TetDev &T, int c, const float *lam, const char *fp, float a, float *u)
{
    const int4 t = __ldg(T.tets + c);
    const int vs[4] = {t.x, t.y, t.z, t.w};
    const float g = 1.0f - a;
    float acc[3] = {0.0f, 0.0f, 0.0f}, va[3], vb[3];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        TetPair<ST>::ld(fp, vs[i], va, vb);
#pragma unroll
        for (int q = 0; q < 3; ++q) acc[q] = fmaf(lam[i], a == 0.0f ? va[q] : fmaf(a, vb[q], g * va[q]), acc[q]);
    }
    u[0] = acc[0];
    u[1] = acc[1];
    u[2] = acc[2];
}

// tet_interp's u plus the Jacobian of the P1 interpolant, constant in the tet:
// J[c][d] = sum_i u_i[c] d lambda_i / d x_d, the lambda gradients being the inverse map's rows
// (lambda_0's their negated sum)
template <int ST>
__device__ __forceinline__ void tet_interp_grad(const TetDev &T, int c, const float *lam, const char *fp, float a,
                                                float *u, float (*J)[3])
{
    const int4 t = __ldg(T.tets + c);
    const int vs[4] = {t.x, t.y, t.z, t.w};
    const float4 r0 = __ldg(T.tmap + 4 * (size_t)c), r1 = __ldg(T.tmap + 4 * (size_t)c + 1),
                 r2 = __ldg(T.tmap + 4 * (size_t)c + 2);
    const float gr[4][3] = {{-(r0.x + r1.x + r2.x), -(r0.y + r1.y + r2.y), -(r0.z + r1.z + r2.z)},
                            {r0.x, r0.y, r0.z},
                            {r1.x, r1.y, r1.z},
                            {r2.x, r2.y, r2.z}};
    const float g = 1.0f - a;
    float acc[3] = {0.0f, 0.0f, 0.0f}, va[3], vb[3];
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int d = 0; d < 3; ++d) J[q][d] = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        TetPair<ST>::ld(fp, vs[i], va, vb);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float ub = a == 0.0f ? va[q] : fmaf(a, vb[q], g * va[q]);
            acc[q] = fmaf(lam[i], ub, acc[q]);
#pragma unroll
            for (int d = 0; d < 3; ++d) J[q][d] = fmaf(gr[i][d], ub, J[q][d]);
        }
    }
    u[0] = acc[0];
    u[1] = acc[1];
    u[2] = acc[2];
}

// ------------------------------------------------------------ exact orientation

// error-free transformations (Knuth's TwoSum; the FMA residual of a product)
__device__ __forceinline__ void e_two_sum(double a, double b, double &s, double &e)
{
    s = __dadd_rn(a, b);
    double bv = __dsub_rn(s, a);
    double av = __dsub_rn(s, bv);
    e = __dadd_rn(__dsub_rn(a, av), __dsub_rn(b, bv));
}

// add b into the nonoverlapping expansion h[0..n) (increasing magnitude); returns the new length
__device__ __forceinline__ int e_grow(double *h, int n, double b)
{
    double q = b;
    int m = 0;
    for (int i = 0; i < n; ++i) {
        double qn, hn;
        e_two_sum(q, h[i], qn, hn);
        q = qn;
        if (hn != 0.0) h[m++] = hn;
    }
    h[m++] = q;
    return m;
}

// adds s * p q r exactly: p q is exact in FP64 (two FP32 factors), its product with r splits
// into a rounded part and the FMA residual
__device__ __forceinline__ int e_add_triple(double *h, int n, double s, float p, float q, float r)
{
    double pq = __dmul_rn((double)p, (double)q);
    double hi = __dmul_rn(pq, (double)r);
    double lo = fma(pq, (double)r, -hi);
    n = e_grow(h, n, s * hi);
    return e_grow(h, n, s * lo);
}

__device__ __forceinline__ int e_add_det3(double *h, int n, double s, const float *p, const float *q, const float *r)
{
    n = e_add_triple(h, n, s, p[0], q[1], r[2]);
    n = e_add_triple(h, n, -s, p[0], q[2], r[1]);
    n = e_add_triple(h, n, -s, p[1], q[0], r[2]);
    n = e_add_triple(h, n, s, p[1], q[2], r[0]);
    n = e_add_triple(h, n, s, p[2], q[0], r[1]);
    return e_add_triple(h, n, -s, p[2], q[1], r[0]);
}

// sign of ((b - a) x (c - a)) . (d - a) for FP32 points, exactly
static __device__ __noinline__ int orient3d_sign(const float *a, const float *b, const float *c, const float *d)
{
    // filter: FP64 evaluation on differences; its error is below 16 ulp of the permanent
    const double ux = (double)b[0] - a[0], uy = (double)b[1] - a[1], uz = (double)b[2] - a[2];
    const double vx = (double)c[0] - a[0], vy = (double)c[1] - a[1], vz = (double)c[2] - a[2];
    const double wx = (double)d[0] - a[0], wy = (double)d[1] - a[1], wz = (double)d[2] - a[2];
    const double det = ux * (vy * wz - vz * wy) + uy * (vz * wx - vx * wz) + uz * (vx * wy - vy * wx);
    const double perm = fabs(ux) * (fabs(vy * wz) + fabs(vz * wy)) + fabs(uy) * (fabs(vz * wx) + fabs(vx * wz)) +
                        fabs(uz) * (fabs(vx * wy) + fabs(vy * wx));
    if (fabs(det) > 1e-14 * perm) return det > 0.0 ? 1 : -1;
    // exact: det3(b,c,d) - det3(a,c,d) + det3(a,b,d) - det3(a,b,c) on raw coordinates
    double h[100];
    int n = 0;
    n = e_add_det3(h, n, 1.0, b, c, d);
    n = e_add_det3(h, n, -1.0, a, c, d);
    n = e_add_det3(h, n, 1.0, a, b, d);
    n = e_add_det3(h, n, -1.0, a, b, c);
    for (int i = n - 1; i >= 0; --i) {
        if (h[i] > 0.0) return 1;
        if (h[i] < 0.0) return -1;
    }
    return 0;
}
