/*
 * lcs_oracle.c -- plain FP64 CPU oracle for the LCS flow-map / FTLE hot path.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark, never by the library.  It is the slow,
 * literal statement of what the GPU path computes, written from the paper
 * (Ameli, Desai, Shadden, arXiv 2209.13775) and the textbook definitions it
 * names.  Every routine follows the paper's order of operations; nothing is
 * blocked, fused or reordered.  Compiled with -ffp-contract=off.
 *
 * Parity status of each part is pinned by tests/test_oracle_*.py.
 */
#include "lcs_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_PI 3.14159265358979323846

int ora_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ====================================================================
 * Time bracket (Sec. 2 "Interpolator": a window of two frames, linear in
 * time between them).
 * ==================================================================== */
void ora_time_locate(const double *times, int nframes, int time_periodic,
                     double period, double t, int *k, double *alpha)
{
    double tt = t;
    if (nframes <= 1) {
        *k = 0;
        *alpha = 0.0;
        return;
    }
    if (time_periodic) tt = t - period * floor((t - times[0]) / period);
    int kk = 0;
    for (int i = 0; i < nframes; ++i)
        if (times[i] <= tt) kk = i;
    if (kk > nframes - 2) kk = nframes - 2;
    double a = (tt - times[kk]) / (times[kk + 1] - times[kk]);
    if (!time_periodic) {
        if (a < 0.0) a = 0.0;
        if (a > 1.0) a = 1.0;
    }
    *k = kk;
    *alpha = a;
}

/* ====================================================================
 * Rectilinear interpolation: bilinear (2D) / trilinear (3D) in space,
 * u = (1 - alpha) I[u_k](x) + alpha I[u_{k+1}](x) in time (Sec. 2).
 * ==================================================================== */

/* Cell along one axis.  Non-periodic: clamp x into the box, cell i with
 * node_i <= x < node_{i+1}, last cell closed.  Periodic: wrap the index.   */
static void axis_cell(double x, double o, double h, int n, int periodic,
                      int *i0, int *i1, double *frac)
{
    if (periodic) {
        double s = (x - o) / h;
        double fl = floor(s);
        long long i = (long long)fl;
        long long m = i % n;
        if (m < 0) m += n;
        *i0 = (int)m;
        *i1 = (int)((m + 1) % n);
        *frac = s - fl;
    } else {
        double hi = o + (double)(n - 1) * h;
        double xc = x;
        if (xc < o) xc = o;
        if (xc > hi) xc = hi;
        double s = (xc - o) / h;
        int i = (int)floor(s);
        if (i > n - 2) i = n - 2;
        if (i < 0) i = 0;
        *i0 = i;
        *i1 = i + 1;
        *frac = s - (double)i;
    }
}

static double rect_node(const ora_rect_field *f, int frame, int i, int j, int k, int c)
{
    long long node = (long long)i + (long long)f->n[0] * ((long long)j + (long long)f->n[1] * (long long)k);
    long long nn = (long long)f->n[0] * f->n[1] * (f->dim == 3 ? f->n[2] : 1);
    return (double)f->frames[((long long)frame * nn + node) * f->dim + c];
}

/* spatial interpolation of one frame */
static void rect_frame_interp(const ora_rect_field *f, int frame, const double *x, double *u)
{
    int i0, i1, j0, j1, k0 = 0, k1 = 0;
    double fx, fy, fz = 0.0;
    axis_cell(x[0], f->origin[0], f->spacing[0], f->n[0], f->periodic[0], &i0, &i1, &fx);
    axis_cell(x[1], f->origin[1], f->spacing[1], f->n[1], f->periodic[1], &j0, &j1, &fy);
    if (f->dim == 3)
        axis_cell(x[2], f->origin[2], f->spacing[2], f->n[2], f->periodic[2], &k0, &k1, &fz);
    for (int c = 0; c < f->dim; ++c) {
        if (f->dim == 2) {
            u[c] = (1.0 - fx) * (1.0 - fy) * rect_node(f, frame, i0, j0, 0, c)
                 + fx * (1.0 - fy) * rect_node(f, frame, i1, j0, 0, c)
                 + (1.0 - fx) * fy * rect_node(f, frame, i0, j1, 0, c)
                 + fx * fy * rect_node(f, frame, i1, j1, 0, c);
        } else {
            u[c] = (1.0 - fx) * (1.0 - fy) * (1.0 - fz) * rect_node(f, frame, i0, j0, k0, c)
                 + fx * (1.0 - fy) * (1.0 - fz) * rect_node(f, frame, i1, j0, k0, c)
                 + (1.0 - fx) * fy * (1.0 - fz) * rect_node(f, frame, i0, j1, k0, c)
                 + fx * fy * (1.0 - fz) * rect_node(f, frame, i1, j1, k0, c)
                 + (1.0 - fx) * (1.0 - fy) * fz * rect_node(f, frame, i0, j0, k1, c)
                 + fx * (1.0 - fy) * fz * rect_node(f, frame, i1, j0, k1, c)
                 + (1.0 - fx) * fy * fz * rect_node(f, frame, i0, j1, k1, c)
                 + fx * fy * fz * rect_node(f, frame, i1, j1, k1, c);
        }
    }
}

int ora_rect_velocity(const ora_rect_field *f, const double *x, double t, double *u)
{
    int k;
    double a;
    double ua[3], ub[3];
    ora_time_locate(f->times, f->nframes, f->time_periodic, f->period, t, &k, &a);
    int k1 = (f->nframes > 1) ? k + 1 : k;
    rect_frame_interp(f, k, x, ua);
    rect_frame_interp(f, k1, x, ub);
    for (int c = 0; c < f->dim; ++c) u[c] = (1.0 - a) * ua[c] + a * ub[c];
    return 0;
}

/* Spatial Jacobian of the bilinear / trilinear interpolant of one frame at x:
 * J[c][d] = d u_c / d x_d inside the cell of x (the derivative of the weights times the node
 * values); along a non-periodic axis where x lies outside the box the clamped field is
 * constant, so that column is zero.                                                       */
static void rect_frame_grad(const ora_rect_field *f, int frame, const double *x, double J[3][3])
{
    int i0, i1, j0, j1, k0 = 0, k1 = 0;
    double fx, fy, fz = 0.0;
    axis_cell(x[0], f->origin[0], f->spacing[0], f->n[0], f->periodic[0], &i0, &i1, &fx);
    axis_cell(x[1], f->origin[1], f->spacing[1], f->n[1], f->periodic[1], &j0, &j1, &fy);
    if (f->dim == 3)
        axis_cell(x[2], f->origin[2], f->spacing[2], f->n[2], f->periodic[2], &k0, &k1, &fz);
    double on[3];
    for (int d = 0; d < f->dim; ++d) {
        double hi = f->origin[d] + (double)(f->n[d] - 1) * f->spacing[d];
        on[d] = (f->periodic[d] || (x[d] >= f->origin[d] && x[d] <= hi)) ? 1.0 : 0.0;
    }
    for (int c = 0; c < f->dim; ++c) {
        if (f->dim == 2) {
            double u00 = rect_node(f, frame, i0, j0, 0, c), u10 = rect_node(f, frame, i1, j0, 0, c);
            double u01 = rect_node(f, frame, i0, j1, 0, c), u11 = rect_node(f, frame, i1, j1, 0, c);
            J[c][0] = on[0] * ((1.0 - fy) * (u10 - u00) + fy * (u11 - u01)) / f->spacing[0];
            J[c][1] = on[1] * ((1.0 - fx) * (u01 - u00) + fx * (u11 - u10)) / f->spacing[1];
        } else {
            double v[2][2][2];
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b)
                    for (int e = 0; e < 2; ++e)
                        v[a][b][e] = rect_node(f, frame, a ? i1 : i0, b ? j1 : j0, e ? k1 : k0, c);
            double dx = 0.0, dy = 0.0, dz = 0.0;
            for (int b = 0; b < 2; ++b)
                for (int e = 0; e < 2; ++e) {
                    double wy = b ? fy : 1.0 - fy, wz = e ? fz : 1.0 - fz;
                    dx += wy * wz * (v[1][b][e] - v[0][b][e]);
                }
            for (int a = 0; a < 2; ++a)
                for (int e = 0; e < 2; ++e) {
                    double wx = a ? fx : 1.0 - fx, wz = e ? fz : 1.0 - fz;
                    dy += wx * wz * (v[a][1][e] - v[a][0][e]);
                }
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) {
                    double wx = a ? fx : 1.0 - fx, wy = b ? fy : 1.0 - fy;
                    dz += wx * wy * (v[a][b][1] - v[a][b][0]);
                }
            J[c][0] = on[0] * dx / f->spacing[0];
            J[c][1] = on[1] * dy / f->spacing[1];
            J[c][2] = on[2] * dz / f->spacing[2];
        }
    }
}

/* u(x, t) and its spatial Jacobian, both linear in time between the bracketing frames */
int ora_rect_velocity_grad(const ora_rect_field *f, const double *x, double t, double *u, double *Jflat)
{
    int k;
    double a;
    double ua[3], ub[3], Ja[3][3], Jb[3][3];
    ora_time_locate(f->times, f->nframes, f->time_periodic, f->period, t, &k, &a);
    int k1 = (f->nframes > 1) ? k + 1 : k;
    rect_frame_interp(f, k, x, ua);
    rect_frame_interp(f, k1, x, ub);
    rect_frame_grad(f, k, x, Ja);
    rect_frame_grad(f, k1, x, Jb);
    for (int c = 0; c < f->dim; ++c) {
        u[c] = (1.0 - a) * ua[c] + a * ub[c];
        for (int d = 0; d < f->dim; ++d) Jflat[c * f->dim + d] = (1.0 - a) * Ja[c][d] + a * Jb[c][d];
    }
    return 0;
}

/* rectilinear tracer has left: more than one cell outside a non-periodic axis */
static int rect_left(const ora_rect_field *f, const double *x)
{
    for (int a = 0; a < f->dim; ++a) {
        if (f->periodic[a]) continue;
        double lo = f->origin[a] - f->spacing[a];
        double hi = f->origin[a] + (double)f->n[a] * f->spacing[a];
        if (x[a] < lo || x[a] > hi) return 1;
    }
    return 0;
}

/* ====================================================================
 * Analytic fields (pins only).
 * Double gyre: Shadden, Lekien, Marsden 2005 (the paper's 2D Cartesian case,
 * Sec. 3.2).  ABC: Arnold-Beltrami-Childress flow with a time-modulated A.
 * Pipe: Poiseuille profile with pulsatile amplitude plus an azimuthal swirl.
 * ==================================================================== */
int ora_analytic_velocity(const ora_analytic_field *f, const double *x, double t, double *u)
{
    const double *p = f->p;
    if (f->kind == ORA_AN_GYRE) {
        double A = p[0], eps = p[1], om = p[2];
        double a = eps * sin(om * t);
        double b = 1.0 - 2.0 * eps * sin(om * t);
        double fx = a * x[0] * x[0] + b * x[0];
        double dfdx = 2.0 * a * x[0] + b;
        u[0] = -ORA_PI * A * sin(ORA_PI * fx) * cos(ORA_PI * x[1]);
        u[1] = ORA_PI * A * cos(ORA_PI * fx) * sin(ORA_PI * x[1]) * dfdx;
    } else if (f->kind == ORA_AN_ABC) {
        double At = p[0] + p[3] * t * sin(ORA_PI * t);
        double B = p[1], C = p[2];
        u[0] = At * sin(x[2]) + C * cos(x[1]);
        u[1] = B * sin(x[0]) + At * cos(x[2]);
        u[2] = C * sin(x[1]) + B * cos(x[0]);
    } else if (f->kind == ORA_AN_AFFINE) {
        int d = f->dim;
        for (int r = 0; r < d; ++r) {
            double s = p[18 + r] + t * p[21 + r];
            for (int c = 0; c < d; ++c) s += (p[r * 3 + c] + t * p[9 + r * 3 + c]) * x[c];
            u[r] = s;
        }
    } else if (f->kind == ORA_AN_PIPE) {
        double R = p[0], L = p[1], amp = p[2];
        double r2 = (x[0] * x[0] + x[1] * x[1]) / (R * R);
        double prof = 1.0 - r2;
        double sw = 0.0;
        for (int m = 1; m <= 4; ++m)
            sw += sin(2.0 * ORA_PI * m * x[2] / L + p[2 + m] + 2.0 * ORA_PI * t) / (double)m;
        double s = amp * prof * sw;
        u[0] = -s * x[1];
        u[1] = s * x[0];
        u[2] = prof * (1.0 + 0.5 * sin(2.0 * ORA_PI * t));
    } else {
        return 1;
    }
    return 0;
}

/* ====================================================================
 * Tetrahedral meshes (Sec. 3.1: a single cell search for tetrahedralized
 * data; local walk of Shadden, Astorino, Gerbeau 2010).
 *
 * Exact orientation: the 4x4 determinant with a column of ones expands
 * into 24 products of three FP32 coordinates.  A product of two FP32 values
 * is exact in FP64; the third factor is applied with an error-free product
 * (FMA residual, Ogita-Rump-Oishi 2005).  The 48 doubles are summed exactly
 * into a nonoverlapping expansion with Knuth's TwoSum (Shewchuk 1997,
 * grow-expansion); the sign is that of its largest nonzero component.
 * ==================================================================== */
static void two_sum(double a, double b, double *s, double *e)
{
    double x = a + b;
    double bv = x - a;
    double av = x - bv;
    double br = b - bv;
    double ar = a - av;
    *s = x;
    *e = ar + br;
}

static int grow_expansion(int elen, const double *e, double b, double *h)
{
    double q = b;
    int hi = 0;
    for (int i = 0; i < elen; ++i) {
        double qn, hn;
        two_sum(q, e[i], &qn, &hn);
        q = qn;
        if (hn != 0.0) h[hi++] = hn;
    }
    h[hi++] = q;
    return hi;
}

/* adds s * p*q*r exactly into the expansion (e, *len) */
static void add_triple(double *e, int *len, double s, float p, float q, float r)
{
    double pq = (double)p * (double)q;   /* exact: 48 significant bits */
    double hi = pq * (double)r;
    double lo = fma(pq, (double)r, -hi); /* exact residual */
    double tmp[128];
    int n = grow_expansion(*len, e, s * hi, tmp);
    n = grow_expansion(n, tmp, s * lo, e);
    *len = n;
}

/* det of rows (p, q, r), 6 signed triple products */
static void add_det3(double *e, int *len, double s, const float *p, const float *q, const float *r)
{
    add_triple(e, len, s, p[0], q[1], r[2]);
    add_triple(e, len, -s, p[0], q[2], r[1]);
    add_triple(e, len, -s, p[1], q[0], r[2]);
    add_triple(e, len, s, p[1], q[2], r[0]);
    add_triple(e, len, s, p[2], q[0], r[1]);
    add_triple(e, len, -s, p[2], q[1], r[0]);
}

int ora_orient3d_exact(const float *a, const float *b, const float *c, const float *d)
{
    /* ((b-a) x (c-a)) . (d-a) = det3(b,c,d) - det3(a,c,d) + det3(a,b,d) - det3(a,b,c) */
    double e[128];
    int len = 0;
    add_det3(e, &len, 1.0, b, c, d);
    add_det3(e, &len, -1.0, a, c, d);
    add_det3(e, &len, 1.0, a, b, d);
    add_det3(e, &len, -1.0, a, b, c);
    for (int i = len - 1; i >= 0; --i) {
        if (e[i] > 0.0) return 1;
        if (e[i] < 0.0) return -1;
    }
    return 0;
}

static const float *tet_vertex(const ora_tet_field *f, long long t, int v)
{
    return f->xyz + 3LL * f->tets[4 * t + v];
}

/* signs of the barycentric coordinates of p in tet t: lam_sign[i] =
 * sign(orient with vertex i replaced by p) * sign(orient of the tet).       */
static void tet_bary_signs(const ora_tet_field *f, long long t, const float *p, int *sg)
{
    const float *v[4];
    for (int i = 0; i < 4; ++i) v[i] = tet_vertex(f, t, i);
    int D = ora_orient3d_exact(v[0], v[1], v[2], v[3]);
    for (int i = 0; i < 4; ++i) {
        const float *w[4] = {v[0], v[1], v[2], v[3]};
        w[i] = p;
        sg[i] = D * ora_orient3d_exact(w[0], w[1], w[2], w[3]);
    }
}

int ora_tet_contains(const ora_tet_field *f, long long t, const float *p, int *on_boundary)
{
    int sg[4];
    tet_bary_signs(f, t, p, sg);
    int inside = 1, onb = 0;
    for (int i = 0; i < 4; ++i) {
        if (sg[i] < 0) inside = 0;
        if (sg[i] == 0) onb = 1;
    }
    if (on_boundary) *on_boundary = inside && onb;
    return inside;
}

/* a closed tet lies inside the bounding box of its vertices */
static int tet_bbox_holds(const ora_tet_field *f, long long t, const float *p)
{
    for (int c = 0; c < 3; ++c) {
        float lo = tet_vertex(f, t, 0)[c], hi = lo;
        for (int v = 1; v < 4; ++v) {
            float q = tet_vertex(f, t, v)[c];
            if (q < lo) lo = q;
            if (q > hi) hi = q;
        }
        if (p[c] < lo || p[c] > hi) return 0;
    }
    return 1;
}

long long ora_tet_locate_brute(const ora_tet_field *f, const float *p)
{
    for (long long t = 0; t < f->ncells; ++t)
        if (tet_bbox_holds(f, t, p) && ora_tet_contains(f, t, p, NULL)) return t;
    return -1;
}

/* FP64 barycentric coordinates of x in tet t (Cramer's rule on differences) */
static double det3d(const double *a, const double *b, const double *c)
{
    return a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0])
         + a[2] * (b[0] * c[1] - b[1] * c[0]);
}

static void tet_bary(const ora_tet_field *f, long long t, const double *x, double *lam)
{
    double v[4][3];
    for (int i = 0; i < 4; ++i) {
        const float *q = tet_vertex(f, t, i);
        v[i][0] = q[0];
        v[i][1] = q[1];
        v[i][2] = q[2];
    }
    double e1[3], e2[3], e3[3], r[3];
    for (int c = 0; c < 3; ++c) {
        e1[c] = v[1][c] - v[0][c];
        e2[c] = v[2][c] - v[0][c];
        e3[c] = v[3][c] - v[0][c];
        r[c] = x[c] - v[0][c];
    }
    double D = det3d(e1, e2, e3);
    lam[1] = det3d(r, e2, e3) / D;
    lam[2] = det3d(e1, r, e3) / D;
    lam[3] = det3d(e1, e2, r) / D;
    lam[0] = 1.0 - lam[1] - lam[2] - lam[3];
}

long long ora_tet_locate_walk(const ora_tet_field *f, long long start, const float *p)
{
    long long t = (start >= 0 && start < f->ncells) ? start : 0;
    int found = 0;
    int limit = f->walk_limit > 0 ? f->walk_limit : 100000;
    double xp[3] = {p[0], p[1], p[2]};
    for (int step = 0; step < limit; ++step) {
        int sg[4];
        tet_bary_signs(f, t, p, sg);
        int best = -1;
        double bestv = 0.0;
        double lam[4];
        tet_bary(f, t, xp, lam);
        for (int i = 0; i < 4; ++i) {
            if (sg[i] < 0 && (best < 0 || lam[i] < bestv)) {
                best = i;
                bestv = lam[i];
            }
        }
        if (best < 0) {
            found = 1;
            break;
        }
        long long nb = f->nbrs[4 * t + best];
        /* a boundary face separates p from this tet: outside a convex mesh, but a non-convex
         * one (a curved vessel, an aneurysm) may still hold p elsewhere */
        if (nb < 0) return ora_tet_locate_brute(f, p);
        t = nb;
    }
    if (!found) return ora_tet_locate_brute(f, p);
    int onb = 0;
    ora_tet_contains(f, t, p, &onb);
    if (!onb) return t;
    /* tie-break: lowest id among the closed tets holding p, collected across
     * faces that contain p (a face, edge or vertex star is face-connected)  */
    long long stack[1024], seen[1024];
    int ns = 0, nseen = 0;
    stack[ns++] = t;
    seen[nseen++] = t;
    long long best = t;
    while (ns > 0) {
        long long c = stack[--ns];
        if (c < best) best = c;
        int sg[4];
        tet_bary_signs(f, c, p, sg);
        for (int i = 0; i < 4; ++i) {
            if (sg[i] != 0) continue;
            long long nb = f->nbrs[4 * c + i];
            if (nb < 0) continue;
            int dup = 0;
            for (int s = 0; s < nseen; ++s)
                if (seen[s] == nb) dup = 1;
            if (dup) continue;
            if (!ora_tet_contains(f, nb, p, NULL)) continue;
            if (nseen >= 1024 || ns >= 1024) return ora_tet_locate_brute(f, p);
            seen[nseen++] = nb;
            stack[ns++] = nb;
        }
    }
    return best;
}

/* Interpolation-time location of an FP64 point: walk on FP64 barycentric
 * coordinates (P1 interpolation is continuous across faces, so which of two
 * face-sharing tets is found does not change u beyond rounding).          */
/* x within the vertices' bounding box widened by 1e-9 (1 + extent) per axis: a cell whose
 * barycentric coordinates of x are all >= -1e-12 always passes, so the test only skips work */
static int near_bbox(const float *pts, const int *cell, int nv, int dim, const double *x)
{
    for (int c = 0; c < dim; ++c) {
        double lo = pts[(long long)dim * cell[0] + c], hi = lo;
        for (int v = 1; v < nv; ++v) {
            double q = pts[(long long)dim * cell[v] + c];
            if (q < lo) lo = q;
            if (q > hi) hi = q;
        }
        double m = 1e-9 * (1.0 + hi - lo);
        if (x[c] < lo - m || x[c] > hi + m) return 0;
    }
    return 1;
}

static long long tet_locate_fp64(const ora_tet_field *f, long long start, const double *x, double *lam)
{
    const double tol = 1e-12;
    long long t = (start >= 0 && start < f->ncells) ? start : 0;
    int limit = f->walk_limit > 0 ? f->walk_limit : 100000;
    for (int step = 0; step < limit; ++step) {
        tet_bary(f, t, x, lam);
        int best = -1;
        double bestv = -tol;
        for (int i = 0; i < 4; ++i)
            if (lam[i] < bestv) {
                best = i;
                bestv = lam[i];
            }
        if (best < 0) return t;
        long long nb = f->nbrs[4 * t + best];
        if (nb < 0) break; /* across a boundary face: settled by testing every tet */
        t = nb;
    }
    for (long long c = 0; c < f->ncells; ++c) {
        if (!near_bbox(f->xyz, f->tets + 4 * c, 4, 3, x)) continue;
        tet_bary(f, c, x, lam);
        if (lam[0] >= -tol && lam[1] >= -tol && lam[2] >= -tol && lam[3] >= -tol) return c;
    }
    return -1;
}

int ora_tet_velocity(const ora_tet_field *f, const double *x, double t, int *cell, double *u)
{
    double lam[4];
    long long c = tet_locate_fp64(f, *cell, x, lam);
    if (c < 0) return 1;
    *cell = (int)c;
    int k;
    double a;
    ora_time_locate(f->times, f->nframes, f->time_periodic, f->period, t, &k, &a);
    int k1 = (f->nframes > 1) ? k + 1 : k;
    const float *fa = f->frames + 3LL * f->nnodes * k;
    const float *fb = f->frames + 3LL * f->nnodes * k1;
    for (int comp = 0; comp < 3; ++comp) {
        double sa = 0.0, sb = 0.0;
        for (int v = 0; v < 4; ++v) {
            long long node = f->tets[4 * c + v];
            sa += lam[v] * (double)fa[3 * node + comp];
            sb += lam[v] * (double)fb[3 * node + comp];
        }
        u[comp] = (1.0 - a) * sa + a * sb;
    }
    return 0;
}

/* ====================================================================
 * Triangle meshes (2D unstructured velocity data, e.g. the stenosis
 * geometries of Sec. 4): the same exact predicates, walk, tie-break and P1
 * interpolation as the tets, one dimension lower.  orient2d sums six
 * products of two FP32 coordinates, each exact in FP64, into a
 * nonoverlapping expansion (Shewchuk 1997).
 * ==================================================================== */
int ora_orient2d_exact(const float *a, const float *b, const float *c)
{
    /* (b-a) x (c-a) = bx cy - by cx - ax cy + ay cx + ax by - ay bx */
    const double terms[6] = {(double)b[0] * (double)c[1], -((double)b[1] * (double)c[0]),
                             -((double)a[0] * (double)c[1]), (double)a[1] * (double)c[0],
                             (double)a[0] * (double)b[1], -((double)a[1] * (double)b[0])};
    double e[16], h[16];
    int len = 0;
    for (int i = 0; i < 6; ++i) {
        int n = grow_expansion(len, e, terms[i], h);
        for (int k = 0; k < n; ++k) e[k] = h[k];
        len = n;
    }
    for (int i = len - 1; i >= 0; --i) {
        if (e[i] > 0.0) return 1;
        if (e[i] < 0.0) return -1;
    }
    return 0;
}

static const float *tri_vertex(const ora_tri_field *f, long long t, int v)
{
    return f->xy + 2LL * f->tris[3 * t + v];
}

static void tri_bary_signs(const ora_tri_field *f, long long t, const float *p, int *sg)
{
    const float *v[3];
    for (int i = 0; i < 3; ++i) v[i] = tri_vertex(f, t, i);
    int D = ora_orient2d_exact(v[0], v[1], v[2]);
    for (int i = 0; i < 3; ++i) {
        const float *w[3] = {v[0], v[1], v[2]};
        w[i] = p;
        sg[i] = D * ora_orient2d_exact(w[0], w[1], w[2]);
    }
}

int ora_tri_contains(const ora_tri_field *f, long long t, const float *p, int *on_boundary)
{
    int sg[3];
    tri_bary_signs(f, t, p, sg);
    int inside = 1, onb = 0;
    for (int i = 0; i < 3; ++i) {
        if (sg[i] < 0) inside = 0;
        if (sg[i] == 0) onb = 1;
    }
    if (on_boundary) *on_boundary = inside && onb;
    return inside;
}

/* a closed triangle lies inside the bounding box of its vertices */
static int tri_bbox_holds(const ora_tri_field *f, long long t, const float *p)
{
    for (int c = 0; c < 2; ++c) {
        float lo = tri_vertex(f, t, 0)[c], hi = lo;
        for (int v = 1; v < 3; ++v) {
            float q = tri_vertex(f, t, v)[c];
            if (q < lo) lo = q;
            if (q > hi) hi = q;
        }
        if (p[c] < lo || p[c] > hi) return 0;
    }
    return 1;
}

long long ora_tri_locate_brute(const ora_tri_field *f, const float *p)
{
    for (long long t = 0; t < f->ncells; ++t)
        if (tri_bbox_holds(f, t, p) && ora_tri_contains(f, t, p, NULL)) return t;
    return -1;
}

/* FP64 barycentric coordinates of x in triangle t (Cramer's rule on differences) */
static void tri_bary(const ora_tri_field *f, long long t, const double *x, double *lam)
{
    const float *a = tri_vertex(f, t, 0), *b = tri_vertex(f, t, 1), *c = tri_vertex(f, t, 2);
    double e1[2] = {(double)b[0] - a[0], (double)b[1] - a[1]};
    double e2[2] = {(double)c[0] - a[0], (double)c[1] - a[1]};
    double r[2] = {x[0] - a[0], x[1] - a[1]};
    double D = e1[0] * e2[1] - e1[1] * e2[0];
    lam[1] = (r[0] * e2[1] - r[1] * e2[0]) / D;
    lam[2] = (e1[0] * r[1] - e1[1] * r[0]) / D;
    lam[0] = 1.0 - lam[1] - lam[2];
}

long long ora_tri_locate_walk(const ora_tri_field *f, long long start, const float *p)
{
    long long t = (start >= 0 && start < f->ncells) ? start : 0;
    int found = 0;
    int limit = f->walk_limit > 0 ? f->walk_limit : 100000;
    double xp[2] = {p[0], p[1]};
    for (int step = 0; step < limit; ++step) {
        int sg[3];
        tri_bary_signs(f, t, p, sg);
        int best = -1;
        double bestv = 0.0, lam[3];
        tri_bary(f, t, xp, lam);
        for (int i = 0; i < 3; ++i)
            if (sg[i] < 0 && (best < 0 || lam[i] < bestv)) {
                best = i;
                bestv = lam[i];
            }
        if (best < 0) {
            found = 1;
            break;
        }
        long long nb = f->nbrs[3 * t + best];
        /* a boundary edge separates p from this triangle: outside a convex mesh, but a
         * non-convex one (a channel with a constriction) may still hold p elsewhere */
        if (nb < 0) return ora_tri_locate_brute(f, p);
        t = nb;
    }
    if (!found) return ora_tri_locate_brute(f, p);
    int onb = 0;
    ora_tri_contains(f, t, p, &onb);
    if (!onb) return t;
    /* p on an edge or a vertex: lowest id among the closed triangles holding p,
     * collected across edges that contain p                                  */
    long long stack[1024], seen[1024];
    int ns = 0, nseen = 0;
    stack[ns++] = t;
    seen[nseen++] = t;
    long long best = t;
    while (ns > 0) {
        long long c = stack[--ns];
        if (c < best) best = c;
        int sg[3];
        tri_bary_signs(f, c, p, sg);
        for (int i = 0; i < 3; ++i) {
            if (sg[i] != 0) continue;
            long long nb = f->nbrs[3 * c + i];
            if (nb < 0) continue;
            int dup = 0;
            for (int s = 0; s < nseen; ++s)
                if (seen[s] == nb) dup = 1;
            if (dup) continue;
            if (!ora_tri_contains(f, nb, p, NULL)) continue;
            if (nseen >= 1024 || ns >= 1024) return ora_tri_locate_brute(f, p);
            seen[nseen++] = nb;
            stack[ns++] = nb;
        }
    }
    return best;
}

static long long tri_locate_fp64(const ora_tri_field *f, long long start, const double *x, double *lam)
{
    const double tol = 1e-12;
    long long t = (start >= 0 && start < f->ncells) ? start : 0;
    int limit = f->walk_limit > 0 ? f->walk_limit : 100000;
    for (int step = 0; step < limit; ++step) {
        tri_bary(f, t, x, lam);
        int best = -1;
        double bestv = -tol;
        for (int i = 0; i < 3; ++i)
            if (lam[i] < bestv) {
                best = i;
                bestv = lam[i];
            }
        if (best < 0) return t;
        long long nb = f->nbrs[3 * t + best];
        if (nb < 0) break; /* across a boundary edge: settled by testing every triangle */
        t = nb;
    }
    for (long long c = 0; c < f->ncells; ++c) {
        if (!near_bbox(f->xy, f->tris + 3 * c, 3, 2, x)) continue;
        tri_bary(f, c, x, lam);
        if (lam[0] >= -tol && lam[1] >= -tol && lam[2] >= -tol) return c;
    }
    return -1;
}

int ora_tri_velocity(const ora_tri_field *f, const double *x, double t, int *cell, double *u)
{
    double lam[3];
    long long c = tri_locate_fp64(f, *cell, x, lam);
    if (c < 0) return 1;
    *cell = (int)c;
    int k;
    double a;
    ora_time_locate(f->times, f->nframes, f->time_periodic, f->period, t, &k, &a);
    int k1 = (f->nframes > 1) ? k + 1 : k;
    const float *fa = f->frames + 2LL * f->nnodes * k;
    const float *fb = f->frames + 2LL * f->nnodes * k1;
    for (int comp = 0; comp < 2; ++comp) {
        double sa = 0.0, sb = 0.0;
        for (int v = 0; v < 3; ++v) {
            long long node = f->tris[3 * c + v];
            sa += lam[v] * (double)fa[2 * node + comp];
            sb += lam[v] * (double)fb[2 * node + comp];
        }
        u[comp] = (1.0 - a) * sa + a * sb;
    }
    return 0;
}

/* u(x, t) and its spatial Jacobian on meshes: P1 is affine inside a cell, so J is constant
 * there, J[c][d] = sum_v u_v[c] d lambda_v / d x_d with the lambda gradients from Cramer's
 * rule (lambda_1 = (x - v0) . (e2 x e3) / D and cyclically; lambda_0 = 1 - the others).  */
int ora_tet_velocity_grad(const ora_tet_field *f, const double *x, double t, int *cell, double *u, double *J)
{
    double lam[4];
    long long c = tet_locate_fp64(f, *cell, x, lam);
    if (c < 0) return 1;
    *cell = (int)c;
    double v[4][3], e[3][3], g[4][3];
    for (int i = 0; i < 4; ++i)
        for (int d = 0; d < 3; ++d) v[i][d] = tet_vertex(f, c, i)[d];
    for (int r = 0; r < 3; ++r)
        for (int d = 0; d < 3; ++d) e[r][d] = v[r + 1][d] - v[0][d];
    const double D = det3d(e[0], e[1], e[2]);
    for (int r = 0; r < 3; ++r) {   /* gradient of lambda_{r+1}: e_{r+1} x e_{r+2} / D */
        const double *a = e[(r + 1) % 3], *b = e[(r + 2) % 3];
        g[r + 1][0] = (a[1] * b[2] - a[2] * b[1]) / D;
        g[r + 1][1] = (a[2] * b[0] - a[0] * b[2]) / D;
        g[r + 1][2] = (a[0] * b[1] - a[1] * b[0]) / D;
    }
    for (int d = 0; d < 3; ++d) g[0][d] = -(g[1][d] + g[2][d] + g[3][d]);
    int k;
    double a;
    ora_time_locate(f->times, f->nframes, f->time_periodic, f->period, t, &k, &a);
    int k1 = (f->nframes > 1) ? k + 1 : k;
    const float *fa = f->frames + 3LL * f->nnodes * k;
    const float *fb = f->frames + 3LL * f->nnodes * k1;
    for (int comp = 0; comp < 3; ++comp) {
        double sa = 0.0, sb = 0.0, ja[3] = {0, 0, 0}, jb[3] = {0, 0, 0};
        for (int i = 0; i < 4; ++i) {
            long long node = f->tets[4 * c + i];
            const double ua = fa[3 * node + comp], ub = fb[3 * node + comp];
            sa += lam[i] * ua;
            sb += lam[i] * ub;
            for (int d = 0; d < 3; ++d) {
                ja[d] += g[i][d] * ua;
                jb[d] += g[i][d] * ub;
            }
        }
        u[comp] = (1.0 - a) * sa + a * sb;
        for (int d = 0; d < 3; ++d) J[comp * 3 + d] = (1.0 - a) * ja[d] + a * jb[d];
    }
    return 0;
}

int ora_tri_velocity_grad(const ora_tri_field *f, const double *x, double t, int *cell, double *u, double *J)
{
    double lam[3];
    long long c = tri_locate_fp64(f, *cell, x, lam);
    if (c < 0) return 1;
    *cell = (int)c;
    const float *p0 = tri_vertex(f, c, 0), *p1 = tri_vertex(f, c, 1), *p2 = tri_vertex(f, c, 2);
    const double e1[2] = {(double)p1[0] - p0[0], (double)p1[1] - p0[1]};
    const double e2[2] = {(double)p2[0] - p0[0], (double)p2[1] - p0[1]};
    const double D = e1[0] * e2[1] - e1[1] * e2[0];
    double g[3][2];
    g[1][0] = e2[1] / D;        /* lambda_1 = (r0 e2_1 - r1 e2_0) / D */
    g[1][1] = -e2[0] / D;
    g[2][0] = -e1[1] / D;       /* lambda_2 = (e1_0 r1 - e1_1 r0) / D */
    g[2][1] = e1[0] / D;
    g[0][0] = -(g[1][0] + g[2][0]);
    g[0][1] = -(g[1][1] + g[2][1]);
    int k;
    double a;
    ora_time_locate(f->times, f->nframes, f->time_periodic, f->period, t, &k, &a);
    int k1 = (f->nframes > 1) ? k + 1 : k;
    const float *fa = f->frames + 2LL * f->nnodes * k;
    const float *fb = f->frames + 2LL * f->nnodes * k1;
    for (int comp = 0; comp < 2; ++comp) {
        double sa = 0.0, sb = 0.0, ja[2] = {0, 0}, jb[2] = {0, 0};
        for (int i = 0; i < 3; ++i) {
            long long node = f->tris[3 * c + i];
            const double ua = fa[2 * node + comp], ub = fb[2 * node + comp];
            sa += lam[i] * ua;
            sb += lam[i] * ub;
            for (int d = 0; d < 2; ++d) {
                ja[d] += g[i][d] * ua;
                jb[d] += g[i][d] * ub;
            }
        }
        u[comp] = (1.0 - a) * sa + a * sb;
        for (int d = 0; d < 2; ++d) J[comp * 2 + d] = (1.0 - a) * ja[d] + a * jb[d];
    }
    return 0;
}

/* ====================================================================
 * Seed lattice (Sec. 2 "Seed": structured grid of seed points).
 * ==================================================================== */
void ora_seed_grid(int dim, const int n[3], const double lo[3], const double hi[3],
                   const int endpoint[3], float *out)
{
    long long nx = n[0], ny = n[1], nz = (dim == 3) ? n[2] : 1;
    long long N = nx * ny * nz;
    double step[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < dim; ++a) {
        if (endpoint[a])
            step[a] = (n[a] > 1) ? (hi[a] - lo[a]) / (double)(n[a] - 1) : 0.0;
        else
            step[a] = (hi[a] - lo[a]) / (double)n[a];
    }
    for (long long k = 0; k < nz; ++k)
        for (long long j = 0; j < ny; ++j)
            for (long long i = 0; i < nx; ++i) {
                long long id = i + nx * (j + ny * k);
                long long idx[3] = {i, j, k};
                for (int a = 0; a < dim; ++a) {
                    double xa = lo[a] + (double)idx[a] * step[a];
                    out[a * N + id] = (float)xa;
                }
            }
}

/* ====================================================================
 * Integrators of Eq. 2 (Sec. 2 "Flow Map").
 * ==================================================================== */
typedef struct {
    int kind;
    const void *field;
    int dim;
} vel_src;

/* returns 0 inside, 1 outside (only meshes can be outside) */
static int eval_u(const vel_src *s, const double *x, double t, int *cell, double *u)
{
    if (s->kind == 0) return ora_rect_velocity((const ora_rect_field *)s->field, x, t, u);
    if (s->kind == 1) return ora_analytic_velocity((const ora_analytic_field *)s->field, x, t, u);
    if (s->kind == 3) return ora_tri_velocity((const ora_tri_field *)s->field, x, t, cell, u);
    return ora_tet_velocity((const ora_tet_field *)s->field, x, t, cell, u);
}

/* distance of x to the mesh boundary, capped at rmax (defined with the boundary index below) */
static double boundary_dist(const ora_bindex *bi, const double *x, double rmax);

/* RK4 as ora_rk4; with bi, margin[p] = the smallest distance (capped at rmax) from the mesh
 * boundary of any stage point the tracer evaluated, the failing one included */
static long long rk4_impl(int field_kind, const void *field, int dim, long long n,
                          const double *x0, const int *cells, double t0, double T, double dt,
                          double *xT, unsigned char *status, double *t_exit,
                          const ora_bindex *bi, double rmax, double *margin)
{
    vel_src src = {field_kind, field, dim};
    double adt = fabs(dt);
    long long nsteps = (long long)floor(fabs(T) / adt + 0.5);
    double h = (T < 0.0) ? -adt : adt;
#pragma omp parallel for schedule(dynamic, 64)
    for (long long p = 0; p < n; ++p) {
        double x[3] = {0, 0, 0};
        for (int a = 0; a < dim; ++a) x[a] = x0[a * n + p];
        int cell = cells ? cells[p] : 0;
        unsigned char st = ORA_OK;
        double te = t0 + T;
        if (field_kind >= 2 && cell < 0) {
            st = ORA_OUTSIDE;
            te = t0;
        }
        double mg = rmax;
        for (long long s = 0; s < nsteps && st == ORA_OK; ++s) {
            double t = t0 + (double)s * h;
            double k1[3], k2[3], k3[3], k4[3], y[3];
            if (bi) mg = fmin(mg, boundary_dist(bi, x, rmax));
            int out = eval_u(&src, x, t, &cell, k1);
            if (!out) {
                for (int a = 0; a < dim; ++a) y[a] = x[a] + 0.5 * h * k1[a];
                if (bi) mg = fmin(mg, boundary_dist(bi, y, rmax));
                out = eval_u(&src, y, t + 0.5 * h, &cell, k2);
            }
            if (!out) {
                for (int a = 0; a < dim; ++a) y[a] = x[a] + 0.5 * h * k2[a];
                if (bi) mg = fmin(mg, boundary_dist(bi, y, rmax));
                out = eval_u(&src, y, t + 0.5 * h, &cell, k3);
            }
            if (!out) {
                for (int a = 0; a < dim; ++a) y[a] = x[a] + h * k3[a];
                if (bi) mg = fmin(mg, boundary_dist(bi, y, rmax));
                out = eval_u(&src, y, t + h, &cell, k4);
            }
            if (out) { /* a stage left the mesh: freeze at the start of the step */
                st = ORA_LEFT;
                te = t;
                break;
            }
            for (int a = 0; a < dim; ++a)
                x[a] = x[a] + h / 6.0 * (k1[a] + 2.0 * k2[a] + 2.0 * k3[a] + k4[a]);
            if (field_kind == 0 && rect_left((const ora_rect_field *)field, x)) {
                st = ORA_LEFT;
                te = t + h;
            }
        }
        for (int a = 0; a < dim; ++a) xT[a * n + p] = x[a];
        status[p] = st;
        t_exit[p] = te;
        if (margin) margin[p] = mg;
    }
    return nsteps;
}

long long ora_rk4(int field_kind, const void *field, int dim, long long n,
                  const double *x0, const int *cells, double t0, double T, double dt,
                  double *xT, unsigned char *status, double *t_exit)
{
    return rk4_impl(field_kind, field, dim, n, x0, cells, t0, T, dt, xT, status, t_exit, NULL, 0.0, NULL);
}

long long ora_rk4_margin(int field_kind, const void *field, int dim, long long n,
                         const double *x0, const int *cells, double t0, double T, double dt,
                         double *xT, unsigned char *status, double *t_exit,
                         const ora_bindex *bi, double rmax, double *margin)
{
    return rk4_impl(field_kind, field, dim, n, x0, cells, t0, T, dt, xT, status, t_exit, bi, rmax, margin);
}

/* ====================================================================
 * Distance to the boundary of a mesh: the faces of tets (edges of
 * triangles) with no neighbour across them.  The tests use it to tell the
 * tracers whose exit decision is close: a stage point within rounding of
 * the boundary can be inside in one precision and outside in another, as
 * Sec. 3.1's cell search decides by the sign of a barycentric coordinate.
 * ==================================================================== */

struct ora_bindex {
    int dim;
    long long nfaces;
    double *fv;          /* [nfaces][dim][dim]: the face's dim vertices            */
    double lo[3], cell;  /* grid over the faces' bounding box, grown by rmax      */
    long long g[3];
    long long *start;    /* [cells + 1] CSR of the faces whose box + rmax meets   */
    long long *items;    /*   the grid cell                                       */
};

static double dot_n(const double *a, const double *b, int dim)
{
    double s = 0.0;
    for (int i = 0; i < dim; ++i) s += a[i] * b[i];
    return s;
}

/* distance from p to the segment [a, b] */
static double seg_dist(const double *p, const double *a, const double *b, int dim)
{
    double e[3], w[3];
    for (int i = 0; i < dim; ++i) {
        e[i] = b[i] - a[i];
        w[i] = p[i] - a[i];
    }
    double ee = dot_n(e, e, dim), t = ee > 0.0 ? dot_n(w, e, dim) / ee : 0.0;
    t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
    double d2 = 0.0;
    for (int i = 0; i < dim; ++i) {
        double r = w[i] - t * e[i];
        d2 += r * r;
    }
    return sqrt(d2);
}

static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* distance from p to the triangle (a, b, c) in 3D: to its plane when p projects inside it (the
 * normal component drops out of each edge's side test), else to the nearest edge */
static double tri_dist(const double *p, const double *a, const double *b, const double *c)
{
    double e0[3], e1[3], n[3];
    for (int i = 0; i < 3; ++i) {
        e0[i] = b[i] - a[i];
        e1[i] = c[i] - a[i];
    }
    cross3(e0, e1, n);
    double nn = dot_n(n, n, 3);
    if (nn > 0.0) {
        const double *v[3] = {a, b, c};
        int inside = 1;
        for (int k = 0; k < 3; ++k) {
            const double *u = v[k], *w = v[(k + 1) % 3];
            double e[3], q[3], x[3];
            for (int i = 0; i < 3; ++i) {
                e[i] = w[i] - u[i];
                q[i] = p[i] - u[i];
            }
            cross3(e, q, x);
            if (dot_n(x, n, 3) < 0.0) inside = 0;
        }
        if (inside) {
            double w[3] = {p[0] - a[0], p[1] - a[1], p[2] - a[2]};
            return fabs(dot_n(w, n, 3)) / sqrt(nn);
        }
    }
    double d = seg_dist(p, a, b, 3);
    d = fmin(d, seg_dist(p, b, c, 3));
    return fmin(d, seg_dist(p, c, a, 3));
}

static double face_dist(const ora_bindex *bi, long long f, const double *p)
{
    const double *v = bi->fv + (size_t)f * bi->dim * bi->dim;
    if (bi->dim == 2) return seg_dist(p, v, v + 2, 2);
    return tri_dist(p, v, v + 3, v + 6);
}

double ora_boundary_distance_brute(const ora_bindex *bi, const double *p)
{
    double d = INFINITY;
    for (long long f = 0; f < bi->nfaces; ++f) d = fmin(d, face_dist(bi, f, p));
    return d;
}

static long long grid_index(const ora_bindex *bi, const double *p, int clampit)
{
    long long idx = 0, mul = 1;
    for (int d = 0; d < bi->dim; ++d) {
        long long c = (long long)floor((p[d] - bi->lo[d]) / bi->cell);
        if (c < 0 || c >= bi->g[d]) {
            if (!clampit) return -1;
            c = c < 0 ? 0 : bi->g[d] - 1;
        }
        idx += c * mul;
        mul *= bi->g[d];
    }
    return idx;
}

static double boundary_dist(const ora_bindex *bi, const double *x, double rmax)
{
    long long c = grid_index(bi, x, 0);
    if (c < 0) return rmax;   /* outside the grid: farther than rmax from every face */
    double d = rmax;
    for (long long q = bi->start[c]; q < bi->start[c + 1]; ++q) d = fmin(d, face_dist(bi, bi->items[q], x));
    return d;
}

double ora_boundary_distance(const ora_bindex *bi, const double *p, double rmax)
{
    return boundary_dist(bi, p, rmax);
}

/* index the boundary faces of a tet (kind 2) or triangle (kind 3) field for distances up to rmax */
ora_bindex *ora_boundary_build(int kind, const void *field, double rmax)
{
    const int dim = kind == 3 ? 2 : 3, nv = dim + 1;
    long long ncells;
    const int *cells, *nbrs;
    const float *pts;
    if (kind == 3) {
        const ora_tri_field *f = (const ora_tri_field *)field;
        ncells = f->ncells;
        cells = f->tris;
        nbrs = f->nbrs;
        pts = f->xy;
    } else {
        const ora_tet_field *f = (const ora_tet_field *)field;
        ncells = f->ncells;
        cells = f->tets;
        nbrs = f->nbrs;
        pts = f->xyz;
    }
    ora_bindex *bi = (ora_bindex *)calloc(1, sizeof(ora_bindex));
    bi->dim = dim;
    for (long long t = 0; t < ncells; ++t)
        for (int v = 0; v < nv; ++v) bi->nfaces += nbrs[t * nv + v] < 0;
    bi->fv = (double *)malloc(sizeof(double) * (size_t)(bi->nfaces ? bi->nfaces : 1) * dim * dim);
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    long long f = 0;
    for (long long t = 0; t < ncells; ++t)
        for (int v = 0; v < nv; ++v) {
            if (nbrs[t * nv + v] >= 0) continue;
            int k = 0;
            for (int w = 0; w < nv; ++w) {   /* the face opposite vertex v */
                if (w == v) continue;
                const float *q = pts + (size_t)cells[t * nv + w] * dim;
                for (int d = 0; d < dim; ++d) {
                    double x = (double)q[d];
                    bi->fv[((size_t)f * dim + k) * dim + d] = x;
                    lo[d] = fmin(lo[d], x);
                    hi[d] = fmax(hi[d], x);
                }
                ++k;
            }
            ++f;
        }
    /* about one face per grid cell, never finer than rmax */
    double vol = 1.0;
    for (int d = 0; d < dim; ++d) {
        lo[d] -= rmax;
        hi[d] += rmax;
        vol *= hi[d] - lo[d];
    }
    double cell = pow(vol / (double)(bi->nfaces ? bi->nfaces : 1), 1.0 / dim);
    bi->cell = fmax(cell, rmax);
    long long ncell = 1;
    for (int d = 0; d < 3; ++d) {
        bi->lo[d] = d < dim ? lo[d] : 0.0;
        bi->g[d] = d < dim ? (long long)ceil((hi[d] - lo[d]) / bi->cell) : 1;
        if (bi->g[d] < 1) bi->g[d] = 1;
        ncell *= bi->g[d];
    }
    bi->start = (long long *)calloc((size_t)ncell + 1, sizeof(long long));
    /* two passes: count, then fill, the cells each face's box grown by rmax meets */
    for (int pass = 0; pass < 2; ++pass) {
        long long *cur = NULL;
        if (pass == 1) {
            for (long long c = 0; c < ncell; ++c) bi->start[c + 1] += bi->start[c];
            bi->items = (long long *)malloc(sizeof(long long) * (size_t)(bi->start[ncell] ? bi->start[ncell] : 1));
            cur = (long long *)malloc(sizeof(long long) * (size_t)ncell);
            memcpy(cur, bi->start, sizeof(long long) * (size_t)ncell);
        }
        for (long long q = 0; q < bi->nfaces; ++q) {
            long long c0[3] = {0, 0, 0}, c1[3] = {0, 0, 0};
            for (int d = 0; d < dim; ++d) {
                double a = INFINITY, b = -INFINITY;
                for (int k = 0; k < dim; ++k) {
                    double x = bi->fv[((size_t)q * dim + k) * dim + d];
                    a = fmin(a, x);
                    b = fmax(b, x);
                }
                c0[d] = (long long)floor((a - rmax - bi->lo[d]) / bi->cell);
                c1[d] = (long long)floor((b + rmax - bi->lo[d]) / bi->cell);
                if (c0[d] < 0) c0[d] = 0;
                if (c1[d] >= bi->g[d]) c1[d] = bi->g[d] - 1;
            }
            for (long long k = c0[2]; k <= c1[2]; ++k)
                for (long long j = c0[1]; j <= c1[1]; ++j)
                    for (long long i = c0[0]; i <= c1[0]; ++i) {
                        long long c = i + bi->g[0] * (j + bi->g[1] * k);
                        if (pass == 0)
                            bi->start[c + 1] += 1;
                        else
                            bi->items[cur[c]++] = q;
                    }
        }
        free(cur);
    }
    return bi;
}

void ora_boundary_free(ora_bindex *bi)
{
    if (!bi) return;
    free(bi->fv);
    free(bi->start);
    free(bi->items);
    free(bi);
}

/* RK4 on Eq. 2 together with its variational equation dM/dt = J(x, t) M, M(t0) = I, on a
 * rectilinear field (Sec. 1: the linearised flow map, the alternative to finite differences of
 * the seed grid).  Same steps, stage times and leaving rule as ora_rk4; M [n][dim][dim] is the
 * derivative of the final position with respect to the seed, frozen with the tracer.          */
/* velocity and Jacobian of any field kind; 0 inside, 1 outside (meshes) */
static int eval_uJ(int kind, const void *field, const double *x, double t, int *cell, double *u, double *J)
{
    if (kind == 0) return ora_rect_velocity_grad((const ora_rect_field *)field, x, t, u, J);
    if (kind == 3) return ora_tri_velocity_grad((const ora_tri_field *)field, x, t, cell, u, J);
    return ora_tet_velocity_grad((const ora_tet_field *)field, x, t, cell, u, J);
}

long long ora_rk4_var_kind(int field_kind, const void *field, int dim, long long n, const double *x0, const int *cells,
                           double t0, double T, double dt, double *xT, double *Mout, unsigned char *status,
                           double *t_exit)
{
    double adt = fabs(dt);
    long long nsteps = (long long)floor(fabs(T) / adt + 0.5);
    double h = (T < 0.0) ? -adt : adt;
#pragma omp parallel for schedule(dynamic, 64)
    for (long long p = 0; p < n; ++p) {
        double x[3] = {0, 0, 0}, M[9] = {0}, y[3], Y[9], ku[4][3], kM[4][9], J[9];
        for (int a = 0; a < dim; ++a) {
            x[a] = x0[a * n + p];
            M[a * dim + a] = 1.0;
        }
        int cell = cells ? cells[p] : 0;
        unsigned char st = ORA_OK;
        double te = t0 + T;
        if (field_kind >= 2 && cell < 0) {
            st = ORA_OUTSIDE;
            te = t0;
        }
        for (long long s = 0; s < nsteps && st == ORA_OK; ++s) {
            double t = t0 + (double)s * h;
            const double ct[4] = {0.0, 0.5, 0.5, 1.0};
            int out = 0;
            for (int q = 0; q < 4 && !out; ++q) {
                for (int a = 0; a < dim; ++a) y[a] = q == 0 ? x[a] : x[a] + ct[q] * h * ku[q - 1][a];
                for (int e = 0; e < dim * dim; ++e) Y[e] = q == 0 ? M[e] : M[e] + ct[q] * h * kM[q - 1][e];
                out = eval_uJ(field_kind, field, y, t + ct[q] * h, &cell, ku[q], J);
                if (out) break;
                for (int a = 0; a < dim; ++a)
                    for (int b = 0; b < dim; ++b) {
                        double acc = 0.0;
                        for (int c = 0; c < dim; ++c) acc += J[a * dim + c] * Y[c * dim + b];
                        kM[q][a * dim + b] = acc;
                    }
            }
            if (out) { /* meshes: a stage left the mesh, freeze at the start of the step */
                st = ORA_LEFT;
                te = t;
                break;
            }
            for (int a = 0; a < dim; ++a) x[a] = x[a] + h / 6.0 * (ku[0][a] + 2.0 * ku[1][a] + 2.0 * ku[2][a] + ku[3][a]);
            for (int e = 0; e < dim * dim; ++e)
                M[e] = M[e] + h / 6.0 * (kM[0][e] + 2.0 * kM[1][e] + 2.0 * kM[2][e] + kM[3][e]);
            if (field_kind == 0 && rect_left((const ora_rect_field *)field, x)) {
                st = ORA_LEFT;
                te = t + h;
            }
        }
        for (int a = 0; a < dim; ++a) xT[a * n + p] = x[a];
        for (int e = 0; e < dim * dim; ++e) Mout[p * dim * dim + e] = M[e];
        status[p] = st;
        t_exit[p] = te;
    }
    return nsteps;
}

long long ora_rk4_var(const ora_rect_field *f, long long n, const double *x0, double t0, double T, double dt,
                      double *xT, double *Mout, unsigned char *status, double *t_exit)
{
    return ora_rk4_var_kind(0, f, f->dim, n, x0, NULL, t0, T, dt, xT, Mout, status, t_exit);
}

/* Dormand-Prince 5(4) tableau (Dormand & Prince 1980). */
static const double DP_C[7] = {0.0, 1.0 / 5.0, 3.0 / 10.0, 4.0 / 5.0, 8.0 / 9.0, 1.0, 1.0};
static const double DP_A[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5.0, 0, 0, 0, 0, 0},
    {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0, 0},
    {44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0, 0, 0, 0},
    {19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0, 0, 0},
    {9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0, 0},
    {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0}};
static const double DP_B[7] = {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0,
                               -2187.0 / 6784.0, 11.0 / 84.0, 0.0};
static const double DP_BS[7] = {5179.0 / 57600.0, 0.0, 7571.0 / 16695.0, 393.0 / 640.0,
                                -92097.0 / 339200.0, 187.0 / 2100.0, 1.0 / 40.0};

typedef struct {
    double x[3];
    double k1[3];   /* FSAL: derivative at (x, t) */
    int have_k1;
    int cell;
    unsigned char st;
    double te;
    long long attempts, accepted;
} dp_tracer;

/* One DP5(4) trial from (x, t) with step h.  Fills xn (5th order), err (the
 * scaled norm) and k7 (derivative at xn, t + h).  Returns 1 if a stage point
 * is outside the mesh.                                                      */
static int dp_trial(const vel_src *src, int dim, dp_tracer *tr, double t, double h,
                    double rtol, double atol, double *xn, double *k7, double *err)
{
    double k[7][3];
    double y[3];
    int cell = tr->cell;
    if (!tr->have_k1) {
        if (eval_u(src, tr->x, t, &cell, tr->k1)) return 1;
        tr->have_k1 = 1;
        tr->cell = cell;
    }
    for (int a = 0; a < dim; ++a) k[0][a] = tr->k1[a];
    for (int s = 1; s < 7; ++s) {
        for (int a = 0; a < dim; ++a) {
            double acc = 0.0;
            for (int j = 0; j < s; ++j) acc += DP_A[s][j] * k[j][a];
            y[a] = tr->x[a] + h * acc;
        }
        if (eval_u(src, y, t + DP_C[s] * h, &cell, k[s])) return 1;
    }
    double e = 0.0;
    for (int a = 0; a < dim; ++a) {
        /* 5th-order solution: same sum as the last stage point (b = a_7j) */
        double acc = 0.0, ea = 0.0;
        for (int j = 0; j < 6; ++j) acc += DP_B[j] * k[j][a];
        for (int s = 0; s < 7; ++s) ea += (DP_B[s] - DP_BS[s]) * k[s][a];
        ea = h * ea;
        double x5 = tr->x[a] + h * acc;
        xn[a] = x5;
        k7[a] = k[6][a];
        double sc = atol + rtol * fmax(fabs(tr->x[a]), fabs(x5));
        double r = fabs(ea) / sc;
        if (r > e) e = r;
    }
    *err = e;
    tr->cell = cell;
    return 0;
}

static double dp_factor(double err)
{
    if (err == 0.0) return 5.0;
    double f = 0.9 * pow(err, -0.2);
    if (f < 0.2) f = 0.2;
    if (f > 5.0) f = 5.0;
    return f;
}

long long ora_dp45(int field_kind, const void *field, int dim, long long n,
                   const double *x0, const int *cells, double t0, double T,
                   double h0, double rtol, double atol, long long max_steps,
                   int group, int adaptive,
                   double *xT, unsigned char *status, double *t_exit,
                   long long *nsteps_out)
{
    vel_src src = {field_kind, field, dim};
    if (group < 1) group = 1;
    double dir = (T < 0.0) ? -1.0 : 1.0;
    double tend = t0 + T;
    long long ngroups = (n + group - 1) / group;
    long long total_acc = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total_acc)
    for (long long g = 0; g < ngroups; ++g) {
        long long p0 = g * group;
        long long p1 = p0 + group < n ? p0 + group : n;
        int m = (int)(p1 - p0);
        dp_tracer *tr = (dp_tracer *)calloc((size_t)m, sizeof(dp_tracer));
        for (int q = 0; q < m; ++q) {
            long long p = p0 + q;
            for (int a = 0; a < dim; ++a) tr[q].x[a] = x0[a * n + p];
            tr[q].cell = cells ? cells[p] : 0;
            tr[q].st = ORA_OK;
            tr[q].te = tend;
            if (field_kind >= 2 && tr[q].cell < 0) {
                tr[q].st = ORA_OUTSIDE;
                tr[q].te = t0;
            }
        }
        double t = t0;
        double h = dir * fabs(h0);
        long long attempts = 0;
        double xn[32][3], k7[32][3], err[32];
        int outm[32];
        while (1) {
            int live = 0;
            for (int q = 0; q < m; ++q) live += (tr[q].st == ORA_OK);
            if (!live) break;
            if (dir * (tend - t) <= 0.0) break;
            if (attempts >= max_steps) {
                for (int q = 0; q < m; ++q)
                    if (tr[q].st == ORA_OK) {
                        tr[q].st = ORA_MAXSTEPS;
                        tr[q].te = t;
                    }
                break;
            }
            double hs = h;
            int last = dir * (t + hs - tend) >= 0.0;
            if (last) hs = tend - t; /* land on t0 + T */
            attempts++;
            int all_ok = 1;
            double hmin = 0.0;
            int have_h = 0;
            for (int q = 0; q < m; ++q) {
                if (tr[q].st != ORA_OK) continue;
                outm[q] = dp_trial(&src, dim, &tr[q], t, hs, rtol, atol, xn[q], k7[q], &err[q]);
                if (outm[q]) continue;
                if (adaptive && err[q] > 1.0) all_ok = 0;
                double hq = hs * dp_factor(err[q]);
                if (!have_h || fabs(hq) < fabs(hmin)) {
                    hmin = hq;
                    have_h = 1;
                }
            }
            /* a stage outside the mesh: that tracer leaves, frozen at the
             * start of the step, and takes no part in the vote             */
            for (int q = 0; q < m; ++q)
                if (tr[q].st == ORA_OK && outm[q]) {
                    tr[q].st = ORA_LEFT;
                    tr[q].te = t;
                }
            if (!adaptive || all_ok) {
                double tn = last ? tend : t + hs; /* the interval of Eq. 2 ends exactly at t0 + T */
                for (int q = 0; q < m; ++q) {
                    if (tr[q].st != ORA_OK) continue;
                    for (int a = 0; a < dim; ++a) {
                        tr[q].x[a] = xn[q][a];
                        tr[q].k1[a] = k7[q][a];
                    }
                    tr[q].accepted++;
                    /* same rule as the fixed-step path: a rectilinear tracer more than one
                     * cell outside a non-periodic axis has left the domain              */
                    if (field_kind == 0 && rect_left((const ora_rect_field *)field, tr[q].x)) {
                        tr[q].st = ORA_LEFT;
                        tr[q].te = tn;
                    }
                }
                t = tn;
            }
            if (adaptive && have_h) h = hmin;
        }
        for (int q = 0; q < m; ++q) {
            long long p = p0 + q;
            for (int a = 0; a < dim; ++a) xT[a * n + p] = tr[q].x[a];
            status[p] = tr[q].st;
            t_exit[p] = tr[q].te;
            if (nsteps_out) nsteps_out[p] = tr[q].accepted;
            total_acc += tr[q].accepted;
        }
        free(tr);
    }
    return total_acc;
}

/* ====================================================================
 * Flow-map gradient by finite differences on the seed lattice (Sec. 2
 * "Cauchy-Green"), C = grad F^T grad F (Eq. 1), eigenvalues, FTLE.
 * ==================================================================== */

/* lattice neighbour of seed (i,j,k) at offset off along axis b; returns the id
 * or -1 when it falls off a non-periodic edge; *wrap gets the number of
 * periods crossed (positive upward).                                        */
static long long lattice_nbr(int dim, const int n[3], const int periodic[3], const long long idx[3],
                             int b, int off, int *wrap)
{
    long long c[3] = {idx[0], idx[1], dim == 3 ? idx[2] : 0};
    long long v = c[b] + off;
    *wrap = 0;
    if (periodic[b]) {
        while (v < 0) {
            v += n[b];
            (*wrap)--;
        }
        while (v >= n[b]) {
            v -= n[b];
            (*wrap)++;
        }
    } else if (v < 0 || v >= n[b]) {
        return -1;
    }
    c[b] = v;
    return c[0] + (long long)n[0] * (c[1] + (long long)n[1] * c[2]);
}

void ora_flowmap_gradient(int dim, const int n[3], const double h[3],
                          const int periodic[3], const double period[3],
                          const double *xT, const unsigned char *status, double *grad)
{
    long long nz = (dim == 3) ? n[2] : 1;
    long long N = (long long)n[0] * n[1] * nz;
#pragma omp parallel for schedule(static)
    for (long long p = 0; p < N; ++p) {
        long long idx[3] = {p % n[0], (p / n[0]) % n[1], p / ((long long)n[0] * n[1])};
        double *G = grad + p * dim * dim;
        for (int e = 0; e < dim * dim; ++e) G[e] = NAN;
        if (status[p] != ORA_OK) continue;
        for (int b = 0; b < dim; ++b) {
            int wp1, wm1, wp2, wm2;
            long long qp1 = lattice_nbr(dim, n, periodic, idx, b, 1, &wp1);
            long long qm1 = lattice_nbr(dim, n, periodic, idx, b, -1, &wm1);
            long long qp2 = lattice_nbr(dim, n, periodic, idx, b, 2, &wp2);
            long long qm2 = lattice_nbr(dim, n, periodic, idx, b, -2, &wm2);
            int okp1 = qp1 >= 0 && status[qp1] == ORA_OK;
            int okm1 = qm1 >= 0 && status[qm1] == ORA_OK;
            int okp2 = qp2 >= 0 && status[qp2] == ORA_OK;
            int okm2 = qm2 >= 0 && status[qm2] == ORA_OK;
            for (int a = 0; a < dim; ++a) {
                /* neighbour position, shifted by the periods crossed on axis b */
                double F0 = xT[a * N + p];
                double Fp1 = 0, Fm1 = 0, Fp2 = 0, Fm2 = 0;
                double sh = (a == b) ? period[b] : 0.0;
                if (qp1 >= 0) Fp1 = xT[a * N + qp1] + (double)wp1 * sh;
                if (qm1 >= 0) Fm1 = xT[a * N + qm1] + (double)wm1 * sh;
                if (qp2 >= 0) Fp2 = xT[a * N + qp2] + (double)wp2 * sh;
                if (qm2 >= 0) Fm2 = xT[a * N + qm2] + (double)wm2 * sh;
                double d;
                if (okp1 && okm1)
                    d = (Fp1 - Fm1) / (2.0 * h[b]);
                else if (okp1 && okp2)
                    d = (-3.0 * F0 + 4.0 * Fp1 - Fp2) / (2.0 * h[b]);
                else if (okm1 && okm2)
                    d = (3.0 * F0 - 4.0 * Fm1 + Fm2) / (2.0 * h[b]);
                else
                    d = NAN;
                G[a * dim + b] = d;
            }
        }
    }
}

void ora_cauchy_green(int dim, long long n, const double *grad, double *C)
{
    int np = (dim == 2) ? 3 : 6;
#pragma omp parallel for schedule(static)
    for (long long p = 0; p < n; ++p) {
        const double *G = grad + p * dim * dim;
        double *Cp = C + p * np;
        int o = 0;
        for (int i = 0; i < dim; ++i)
            for (int j = i; j < dim; ++j) {
                double s = 0.0;
                for (int a = 0; a < dim; ++a) s += G[a * dim + i] * G[a * dim + j];
                Cp[o++] = s;
            }
    }
}

/* cyclic Jacobi eigenvalue iteration (Golub & Van Loan, Sec. 8.5); with vec != NULL the
 * rotations are also accumulated, V <- V J, so column i of V is the eigenvector of A[i][i]
 * (Sec. 2 "Cauchy-Green": eigenvalues and eigenvectors of C at each seed) */
int ora_eigvec_sym(int dim, const double *Cp, double *eig, double *vec)
{
    double A[3][3], V[3][3];
    int o = 0;
    for (int i = 0; i < dim; ++i)
        for (int j = i; j < dim; ++j) {
            A[i][j] = Cp[o];
            A[j][i] = Cp[o];
            o++;
        }
    for (int i = 0; i < dim; ++i)
        for (int j = 0; j < dim; ++j) V[i][j] = i == j ? 1.0 : 0.0;
    for (int i = 0; i < dim; ++i)
        if (isnan(A[i][i])) {
            for (int r = 0; r < dim; ++r) eig[r] = NAN;
            if (vec)
                for (int r = 0; r < dim * dim; ++r) vec[r] = NAN;
            return 0;
        }
    int sweep;
    for (sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int i = 0; i < dim; ++i) {
            diag += A[i][i] * A[i][i];
            for (int j = 0; j < dim; ++j)
                if (i != j) off += A[i][j] * A[i][j];
        }
        if (off == 0.0 || off <= 1e-36 * diag) break;
        for (int p = 0; p < dim - 1; ++p)
            for (int q = p + 1; q < dim; ++q) {
                if (A[p][q] == 0.0) continue;
                double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0);
                double s = t * c;
                /* A <- J^T A J with the rotation in the (p, q) plane */
                for (int k = 0; k < dim; ++k) {
                    double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < dim; ++k) {
                    double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < dim; ++k) {
                    double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
    }
    int idx[3] = {0, 1, 2};
    for (int i = 0; i < dim; ++i) eig[i] = A[i][i];
    for (int i = 0; i < dim; ++i) /* ascending insertion sort, carrying the columns */
        for (int j = i + 1; j < dim; ++j)
            if (eig[j] < eig[i]) {
                double tmp = eig[i];
                eig[i] = eig[j];
                eig[j] = tmp;
                int ti = idx[i];
                idx[i] = idx[j];
                idx[j] = ti;
            }
    if (vec)
        for (int k = 0; k < dim; ++k)
            for (int r = 0; r < dim; ++r) vec[k * dim + r] = V[r][idx[k]];
    return sweep;
}

int ora_eig_sym(int dim, const double *Cp, double *eig) { return ora_eigvec_sym(dim, Cp, eig, NULL); }

/* eigenvalues (ascending) and unit eigenvectors of n packed tensors */
void ora_cg_eigen(int dim, long long n, const double *C, double *eig, double *vec)
{
    int np = (dim == 2) ? 3 : 6;
#pragma omp parallel for schedule(static)
    for (long long p = 0; p < n; ++p) ora_eigvec_sym(dim, C + p * np, eig + p * dim, vec + p * dim * dim);
}

void ora_ftle(int dim, long long n, const double *C, double T, double *lambda_max, double *ftle)
{
    int np = (dim == 2) ? 3 : 6;
#pragma omp parallel for schedule(static)
    for (long long p = 0; p < n; ++p) {
        double eig[3];
        ora_eig_sym(dim, C + p * np, eig);
        double lm = eig[dim - 1];
        if (lambda_max) lambda_max[p] = lm;
        ftle[p] = log(sqrt(lm)) / fabs(T);
    }
}
