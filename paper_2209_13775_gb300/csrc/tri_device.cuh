// tri_device.cuh -- device building blocks for velocity data on triangle meshes (2D
// unstructured data such as the stenosis geometries of Sec. 4; Sec. 3.1: the local cell
// search of tetrahedral grids, triangles in 2D).
//
//  * tri_locate: the hot loop's local walk on FP32 barycentric coordinates from a per-
//    triangle inverse affine map (stop when no coordinate is below -tol, else cross the
//    edge of the most negative one).  A walk that meets a boundary edge is settled by the
//    triangles listed for the point's bin, so meshes need not be convex (a channel with a
//    constriction is not); a walk past its step limit reports WALKFAIL.
//  * tri_interp: P1 interpolation of the frame pair k, blended in time at the vertices.
//  * TriCache: a tracer's registers holding the last cell's map and vertex pairs (RK4 and
//    DP5(4) use both; the variational kernel only the map).
//  * orient2d_sign: exact orientation of three FP32 points (FP64 filter, exact expansion
//    sum of the six two-factor products when the filter cannot decide).
#pragma once

#include "tet_device.cuh"

struct TriDev {
    const float2 *xy;     // [nnodes]
    const int4 *tris;     // [ncells] (a, b, c, 0)
    const int4 *nbrs;     // [ncells] (across the edge opposite vertex 0, 1, 2; -1 boundary)
    const float4 *tmap;   // [ncells] (M00, M01, M10, M11): lambda_{r+1} = M_r . (x - v0)
    const float2 *tv0;    // [ncells] vertex 0
    const int *bstart;    // [nbins + 1] CSR of the triangles whose bounding box meets a bin
    const int *blist;     //   (ids increasing within a bin)
    float blo[2], binv[2];
    int bn[2];
    const char *pairs;    // [nslabs][nnodes] (u_k, v_k, u_{k+1}, v_{k+1}) in storage precision
    size_t fstride;
    long long ncells;
    int walk_limit;
    float tol;
    int convex;           // the mesh is convex: a boundary edge separates the point from the mesh
};

TriDev tri_dev(const lcs_field *f, int walk_limit);  // tri_store.cu

// barycentric coordinates of x from a triangle's map m and vertex 0
__device__ __forceinline__ void tri_bary_mv(const float4 m, const float2 v, const float *x, float *lam)
{
    const float dx = x[0] - v.x, dy = x[1] - v.y;
    lam[1] = fmaf(m.x, dx, m.y * dy);
    lam[2] = fmaf(m.z, dx, m.w * dy);
    lam[0] = 1.0f - lam[1] - lam[2];
}

__device__ __forceinline__ void tri_bary(const TriDev &T, int c, const float *x, float *lam)
{
    tri_bary_mv(__ldg(T.tmap + c), __ldg(T.tv0 + c), x, lam);
}

// the triangles listed for x's bin, in id order: the first whose coordinates all reach -tol
__device__ __forceinline__ int tri_bin_scan(const TriDev &T, const float *x, int *cell, float *lam)
{
    if (!(isfinite(x[0]) && isfinite(x[1]))) return TET_OUTSIDE;
    const int b = mesh_bin_axis(x[0], T.blo[0], T.binv[0], T.bn[0]) +
                  T.bn[0] * mesh_bin_axis(x[1], T.blo[1], T.binv[1], T.bn[1]);
    const int q1 = __ldg(T.bstart + b + 1);
    for (int q = __ldg(T.bstart + b); q < q1; ++q) {
        const int c = __ldg(T.blist + q);
        tri_bary(T, c, x, lam);
        if (fminf(lam[0], fminf(lam[1], lam[2])) >= -T.tol) {
            *cell = c;
            return TET_INSIDE;
        }
    }
    return TET_OUTSIDE;
}

__device__ __forceinline__ int tri_locate(const TriDev &T, const float *x, int *cell, float *lam)
{
    int c = *cell;
    if (c < 0 || c >= T.ncells) c = 0;
    for (int it = 0; it < T.walk_limit; ++it) {
        tri_bary(T, c, x, lam);
        int jm = 0;
        float lm = lam[0];
        if (lam[1] < lm) {
            lm = lam[1];
            jm = 1;
        }
        if (lam[2] < lm) {
            lm = lam[2];
            jm = 2;
        }
        if (lm >= -T.tol) {
            *cell = c;
            return TET_INSIDE;
        }
        const int4 nb = __ldg(T.nbrs + c);
        const int n = jm == 0 ? nb.x : jm == 1 ? nb.y : nb.z;
        if (n < 0) return T.convex ? TET_OUTSIDE : tri_bin_scan(T, x, cell, lam);
        c = n;
    }
    *cell = c;
    return TET_WALKFAIL;
}

// A tracer's register cache: the map of the cell its last walk ended in, and the vertex
// pairs of the cell and frame interval it last interpolated.  Consecutive stage points of a
// tracer mostly share a cell and an interval (steps are short against cells and frame gaps), so
// a walk that starts in the held cell and stays there, and an interpolation in the held cell
// and interval, issue no loads.  A hit reuses exactly the values a reload would read: results
// are bit-identical to the uncached walk and interpolation.
struct TriCache {
    float4 m;
    float2 v;
    int mc;        // cell of m, v (-1: none)
    int pc, pk;    // cell and interval of ua, ub (-1: none)
    float ua[3][2], ub[3][2];
};

__device__ __forceinline__ void tri_cache_init(TriCache &cc)
{
    cc.mc = -1;
    cc.pc = -1;
    cc.pk = -1;
}

// tri_locate with the map of each visited cell taken from, or put into, the cache.  The two
// walks are kept apart: the uncached one serves the seed location and the surrogate gate,
// which make one walk per tracer and would gain nothing from the cache's registers.
// LONG_WALKS loads a cell's neighbours together with its map (when the map is not held), so
// that a walk that goes on waits for one round trip per cell instead of two.  It pays where
// walks are long (DP5(4) on the stenosis: about 8 cells per stage point, 10% faster) and costs
// where most walks end in their first cell (RK4 at dt = 0.002: 1.2 cells, 5% slower).
template <bool LONG_WALKS = false>
__device__ __forceinline__ int tri_locate_cached(const TriDev &T, const float *x, int *cell, float *lam, TriCache &cc)
{
    int c = *cell;
    if ((unsigned)c >= (unsigned)T.ncells) c = 0;   // one unsigned compare (cell ids fit in an int)
    for (int it = 0; it < T.walk_limit; ++it) {
        int4 nb = make_int4(-1, -1, -1, 0);
        bool have_nb = false;
        if (c != cc.mc) {
            cc.m = __ldg(T.tmap + c);
            cc.v = __ldg(T.tv0 + c);
            cc.mc = c;
            if (LONG_WALKS) {
                nb = __ldg(T.nbrs + c);
                have_nb = true;
            }
        }
        tri_bary_mv(cc.m, cc.v, x, lam);
        // the inside test on the smallest coordinate (lam is finite for a finite x) and the face
        // to cross, the first smallest coordinate: for short walks the face is found only when the
        // walk goes on (RK4 2.8% faster); long walks find both in one pass (DP5(4) 1.6% faster)
        int jm = 0;
        float lm = lam[0];
        if (LONG_WALKS) {
            if (lam[1] < lm) {
                lm = lam[1];
                jm = 1;
            }
            if (lam[2] < lm) {
                lm = lam[2];
                jm = 2;
            }
        } else {
            lm = fminf(lam[0], fminf(lam[1], lam[2]));
        }
        if (lm >= -T.tol) {
            *cell = c;
            return TET_INSIDE;
        }
        if (!LONG_WALKS) {
            float lo = lam[0];
            if (lam[1] < lo) {
                lo = lam[1];
                jm = 1;
            }
            if (lam[2] < lo) jm = 2;
        }
        if (!have_nb) nb = __ldg(T.nbrs + c);
        const int n = jm == 0 ? nb.x : jm == 1 ? nb.y : nb.z;
        if (n < 0) return T.convex ? TET_OUTSIDE : tri_bin_scan(T, x, cell, lam);
        c = n;
    }
    *cell = c;
    return TET_WALKFAIL;
}

template <int ST>
struct TriPair;

template <>
struct TriPair<LCS_F32> {
    static __device__ __forceinline__ void ld(const char *f, int v, float *ua, float *ub)
    {
        const float4 r = __ldg(reinterpret_cast<const float4 *>(f) + v);
        ua[0] = r.x;
        ua[1] = r.y;
        ub[0] = r.z;
        ub[1] = r.w;
    }
};

template <>
struct TriPair<LCS_F16> {
    static __device__ __forceinline__ void ld(const char *f, int v, float *ua, float *ub)
    {
        const uint2 r = __ldg(reinterpret_cast<const uint2 *>(f) + v);
        const float2 a = tet_h2f(r.x), b = tet_h2f(r.y);
        ua[0] = a.x;
        ua[1] = a.y;
        ub[0] = b.x;
        ub[1] = b.y;
    }
};

template <>
struct TriPair<LCS_BF16> {
    static __device__ __forceinline__ void ld(const char *f, int v, float *ua, float *ub)
    {
        const uint2 r = __ldg(reinterpret_cast<const uint2 *>(f) + v);
        const float2 a = tet_b2f(r.x), b = tet_b2f(r.y);
        ua[0] = a.x;
        ua[1] = a.y;
        ub[0] = b.x;
        ub[1] = b.y;
    }
};

// u = sum_i lam_i [(1 - a) u_k + a u_{k+1}](vertex i) from the vertices' pairs (u_k, u_{k+1}).
// Every pair holds finite values (a single frame is paired with itself), so a = 0 gives u_k
// exactly without a select: 0 * u_{k+1} + 1 * u_k.
__device__ __forceinline__ void tri_blend(const float *lam, const float (*ua)[2], const float (*ub)[2], float a,
                                          float *u)
{
    const float g = 1.0f - a;
    float acc[2] = {0.0f, 0.0f};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int q = 0; q < 2; ++q)
            acc[q] = fmaf(lam[i], fmaf(a, ub[i][q], g * ua[i][q]), acc[q]);
    u[0] = acc[0];
    u[1] = acc[1];
}

// tri_blend of cell c's vertices from the interval pair at fp
template <int ST>
__device__ __forceinline__ void tri_interp(const TriDev &T, int c, const float *lam, const char *fp, float a, float *u)
{
    const int4 t = __ldg(T.tris + c);
    float ua[3][2], ub[3][2];
    TriPair<ST>::ld(fp, t.x, ua[0], ub[0]);
    TriPair<ST>::ld(fp, t.y, ua[1], ub[1]);
    TriPair<ST>::ld(fp, t.z, ua[2], ub[2]);
    tri_blend(lam, ua, ub, a, u);
}

// tri_interp in interval k (pairs at fp) with the vertex pairs taken from, or put into, the cache
template <int ST>
__device__ __forceinline__ void tri_interp_cached(const TriDev &T, int c, int k, const float *lam, const char *fp,
                                                  float a, float *u, TriCache &cc)
{
    if (c != cc.pc || k != cc.pk) {
        const int4 t = __ldg(T.tris + c);
        TriPair<ST>::ld(fp, t.x, cc.ua[0], cc.ub[0]);
        TriPair<ST>::ld(fp, t.y, cc.ua[1], cc.ub[1]);
        TriPair<ST>::ld(fp, t.z, cc.ua[2], cc.ub[2]);
        cc.pc = c;
        cc.pk = k;
    }
    tri_blend(lam, cc.ua, cc.ub, a, u);
}

// tri_interp's u plus the Jacobian of the P1 interpolant, constant in the triangle, with c's map m
// passed in (tri_locate_cached leaves it in TriCache::m).  The vertex pairs are loaded, not cached:
// in the variational kernel, whose 2x2 M, its four stage slopes and J already hold many registers,
// keeping the pairs too took it from 62 to 80 registers a thread and made it slower than reloading.
template <int ST>
__device__ __forceinline__ void tri_interp_grad(const TriDev &T, int c, const float4 &m, const float *lam,
                                                const char *fp, float a, float *u, float (*J)[2])
{
    const int4 t = __ldg(T.tris + c);
    float ua[3][2], ub[3][2];
    TriPair<ST>::ld(fp, t.x, ua[0], ub[0]);
    TriPair<ST>::ld(fp, t.y, ua[1], ub[1]);
    TriPair<ST>::ld(fp, t.z, ua[2], ub[2]);
    const float gr[3][2] = {{-(m.x + m.z), -(m.y + m.w)}, {m.x, m.y}, {m.z, m.w}};
    const float g = 1.0f - a;
    float acc[2] = {0.0f, 0.0f};
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int d = 0; d < 2; ++d) J[q][d] = 0.0f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const float v = fmaf(a, ub[i][q], g * ua[i][q]);
            acc[q] = fmaf(lam[i], v, acc[q]);
#pragma unroll
            for (int d = 0; d < 2; ++d) J[q][d] = fmaf(gr[i][d], v, J[q][d]);
        }
    }
    u[0] = acc[0];
    u[1] = acc[1];
}

// sign of (b - a) x (c - a) for FP32 points, exactly
static __device__ __noinline__ int orient2d_sign(const float *a, const float *b, const float *c)
{
    // filter: FP64 on differences (each difference of FP32 values is exact unless their
    // exponents are far apart; the bound covers the rounding of both products and the sum)
    const double ux = (double)b[0] - a[0], uy = (double)b[1] - a[1];
    const double vx = (double)c[0] - a[0], vy = (double)c[1] - a[1];
    const double det = ux * vy - uy * vx;
    const double perm = fabs(ux * vy) + fabs(uy * vx);
    if (fabs(det) > 1e-14 * perm) return det > 0.0 ? 1 : -1;
    // exact: bx cy - by cx - ax cy + ay cx + ax by - ay bx, each product exact in FP64
    const double terms[6] = {__dmul_rn(b[0], c[1]), -__dmul_rn(b[1], c[0]), -__dmul_rn(a[0], c[1]),
                             __dmul_rn(a[1], c[0]),  __dmul_rn(a[0], b[1]), -__dmul_rn(a[1], b[0])};
    double h[8];
    int n = 0;
    for (int i = 0; i < 6; ++i) n = e_grow(h, n, terms[i]);
    for (int i = n - 1; i >= 0; --i) {
        if (h[i] > 0.0) return 1;
        if (h[i] < 0.0) return -1;
    }
    return 0;
}
