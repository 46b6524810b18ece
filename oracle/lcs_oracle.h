/*
 * lcs_oracle.h -- plain FP64 CPU oracle for the LCS flow-map / FTLE hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the slow, literal definition that the
 * CUDA library is checked against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant with the CUDA library, and it includes nothing from it.
 *
 * Paper: Ameli, Desai, Shadden, "Development of an efficient and flexible
 * pipeline for Lagrangian coherent structure computation" (arXiv 2209.13775).
 *   Eq. 1  Cauchy-Green tensor C = grad(F)^T grad(F) of the flow map F.
 *   Eq. 2  advection ODE dx/dt = u(x, t) integrated over (t0, tf) from a seed grid.
 *   Sec. 2 "Interpolator": velocity interpolated in space, and linearly in time
 *          between two frames.
 *   Sec. 2 "Seed": seeds on a structured grid; on unstructured data the cell
 *          holding each seed.
 *   Sec. 2 "Flow Map": single-step Runge-Kutta integration; trajectories that
 *          leave the data domain.
 *   Sec. 2 "Cauchy-Green": central differences of final positions, eigenvalues.
 *   Sec. 3.1: local cell search on tetrahedral grids (triangular grids in 2D),
 *          used for the 2D unstructured stenosis data of Sec. 4.
 *
 * Arrays are plain C arrays.  Positions are SoA: x[0..N), then y[0..N), then
 * z[0..N).  Seed index is x-fastest: id = i + nx*(j + ny*k).
 * Built with -ffp-contract=off so that no multiply-add is fused.
 */
#ifndef LCS_ORACLE_H
#define LCS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* tracer status values written by the integrators */
#define ORA_OK 0        /* inside the domain at the end of the interval      */
#define ORA_LEFT 1      /* left the domain; frozen at its last position      */
#define ORA_OUTSIDE 2   /* seed started outside the domain (tet meshes)      */
#define ORA_MAXSTEPS 3  /* adaptive integrator hit its step cap              */

/* ------------------------------------------------------------------ fields */

/* Velocity frames on a 2D/3D rectilinear grid (Sec. 2, "Interpolator").
 * node (i,j,k) sits at origin + (i,j,k)*spacing.  frames is
 * [nframes][nz][ny][nx][dim] FP32 (nz = 1 in 2D); it is read promoted to FP64.
 * A periodic axis has n cells (node n-1 connects back to node 0), so its
 * period is n*spacing; a non-periodic axis has n-1 cells.                   */
typedef struct {
    int dim;
    int n[3];
    double origin[3];
    double spacing[3];
    int periodic[3];
    int nframes;
    const double *times;   /* nframes increasing frame times               */
    int time_periodic;     /* wrap t into [times[0], times[0] + period)      */
    double period;
    const float *frames;
} ora_rect_field;

/* Velocity frames on a tetrahedral mesh (Sec. 3.1: velocity data given on
 * tetrahedra; P1 interpolation inside a tet).                               */
typedef struct {
    long long nnodes, ncells;
    const float *xyz;      /* [nnodes][3]                                   */
    const int *tets;       /* [ncells][4] node ids                          */
    const int *nbrs;       /* [ncells][4] tet across the face opposite vertex v, -1 = boundary */
    int nframes;
    const double *times;
    int time_periodic;
    double period;
    const float *frames;   /* [nframes][nnodes][3]                          */
    int walk_limit;        /* cap on walk steps before brute force          */
} ora_tet_field;

/* Velocity frames on a triangle mesh (2D unstructured data such as the
 * stenosis geometries of Sec. 4; P1 interpolation inside a triangle).       */
typedef struct {
    long long nnodes, ncells;
    const float *xy;       /* [nnodes][2]                                   */
    const int *tris;       /* [ncells][3] node ids                          */
    const int *nbrs;       /* [ncells][3] triangle across the edge opposite vertex v, -1 = boundary */
    int nframes;
    const double *times;
    int time_periodic;
    double period;
    const float *frames;   /* [nframes][nnodes][2]                          */
    int walk_limit;        /* cap on walk steps before brute force          */
} ora_tri_field;

/* Analytic velocity fields.  Used by the pins that need a smooth field
 * (order of convergence, conservation laws); they never feed the GPU.       */
#define ORA_AN_GYRE 0     /* double gyre: p[0]=A, p[1]=eps, p[2]=omega                  */
#define ORA_AN_ABC 1      /* ABC flow, A(t) = p[0] + p[3]*t*sin(pi t); B = p[1], C = p[2] */
#define ORA_AN_AFFINE 2   /* u = (A0 + t A1) x + (b0 + t b1); p = A0[9],A1[9],b0[3],b1[3] */
#define ORA_AN_PIPE 3     /* Poiseuille pipe + swirl; p[0]=R, p[1]=L, p[2]=s_amp, p[3..6]=phases */
typedef struct {
    int kind;
    int dim;
    double p[24];
} ora_analytic_field;

/* ------------------------------------------------------------ primitives */

/* Frame bracket for time t: largest k with times[k] <= t (after the periodic
 * wrap), clamped to [0, nframes-2]; alpha = (t - t_k)/(t_{k+1} - t_k), clamped
 * to [0,1] when time is not periodic.  Linear-in-time rule of Sec. 2.       */
void ora_time_locate(const double *times, int nframes, int time_periodic,
                     double period, double t, int *k, double *alpha);

/* u(x, t) on rectilinear frames.  Returns 0.  Queries on a non-periodic axis
 * are clamped to the grid box.                                              */
int ora_rect_velocity(const ora_rect_field *f, const double *x, double t, double *u);
/* u and its spatial Jacobian J[c * dim + d] = d u_c / d x_d (zero across a clamped axis). */
int ora_rect_velocity_grad(const ora_rect_field *f, const double *x, double t, double *u, double *J);

/* u(x, t) from an analytic field.  Returns 0.                               */
int ora_analytic_velocity(const ora_analytic_field *f, const double *x, double t, double *u);

/* u(x, t) on a tet mesh: FP64 walk from *cell (barycentric tolerance 1e-12),
 * every tet tested when the walk reaches a boundary face, P1 interpolation.
 * *cell is the walk's start (in) and the containing tet (out).
 * Returns 0 inside, 1 outside the mesh.                                     */
int ora_tet_velocity(const ora_tet_field *f, const double *x, double t, int *cell, double *u);

/* u(x, t) on a triangle mesh: FP64 walk from *cell (barycentric tolerance
 * 1e-12), every triangle tested when the walk reaches a boundary edge, P1
 * interpolation.  *cell is the walk's start (in) and the containing triangle (out).
 * Returns 0 inside, 1 outside the mesh.                                     */
int ora_tri_velocity(const ora_tri_field *f, const double *x, double t, int *cell, double *u);

/* ---------------------------------------------------------- seed grid (a2) */

/* Structured seed lattice (Sec. 2, "Seed"): along axis a,
 *   x_i = lo + i * step,  step = (hi - lo)/(n - 1)  (endpoint[a] != 0)
 *                         step = (hi - lo)/n        (endpoint[a] == 0, periodic)
 * in FP64, then rounded to FP32.  out is [dim][N] SoA, seed id x-fastest.   */
void ora_seed_grid(int dim, const int n[3], const double lo[3], const double hi[3],
                   const int endpoint[3], float *out);

/* --------------------------------------------------------- integrators */

/* Fixed-step classical RK4 on Eq. 2 (Sec. 2 "Flow Map"; Sec. 3.1).
 *   dt carries the sign of T; nsteps = round(|T|/|dt|); t_n = t0 + n*dt.
 * field_kind: 0 = rectilinear (ora_rect_field), 1 = analytic, 2 = tet,
 * 3 = triangle mesh (ora_tri_field).
 * x0 is [dim][n] FP64 SoA; xT the same layout.  status/t_exit per seed.
 * Rectilinear: a tracer more than one cell outside a non-periodic axis after
 * a step is LEFT, frozen there, t_exit = end time of that step.
 * Tet / triangle: a stage point outside the mesh makes the tracer LEFT, frozen at the
 * start of the step, t_exit = t_n.  cells (meshes only, may be NULL otherwise) is
 * the start cell per seed, -1 = seed outside (status OUTSIDE).
 * Returns the number of steps per tracer.                                   */
/* RK4 on Eq. 2 with the variational equation dM/dt = J M, M(t0) = I: final positions,
 * M [n][dim][dim], status and exit time as ora_rk4 (field_kind and cells as there;
 * ora_rk4_var is the rectilinear case).                                            */
long long ora_rk4_var_kind(int field_kind, const void *field, int dim, long long n, const double *x0, const int *cells,
                           double t0, double T, double dt, double *xT, double *M, unsigned char *status,
                           double *t_exit);
/* u and its spatial Jacobian J [dim][dim] on meshes (constant inside a cell); as ora_tet_velocity /
 * ora_tri_velocity otherwise.                                                                       */
int ora_tet_velocity_grad(const ora_tet_field *f, const double *x, double t, int *cell, double *u, double *J);
int ora_tri_velocity_grad(const ora_tri_field *f, const double *x, double t, int *cell, double *u, double *J);
long long ora_rk4_var(const ora_rect_field *f, long long n, const double *x0, double t0, double T, double dt,
                      double *xT, double *M, unsigned char *status, double *t_exit);

long long ora_rk4(int field_kind, const void *field, int dim, long long n,
                  const double *x0, const int *cells, double t0, double T, double dt,
                  double *xT, unsigned char *status, double *t_exit);

/* Distance to the boundary of a tet (field_kind 2) or triangle (3) mesh: the
 * faces (edges) with no neighbour across them.  ora_boundary_build indexes
 * them on a grid for queries up to rmax; ora_boundary_distance returns the
 * exact distance from p when it is below rmax, else rmax;
 * ora_boundary_distance_brute tests every face (no cap).  The distance to a
 * face is the distance to its plane (line) where p projects inside it, else
 * to its nearest edge (end point).                                          */
typedef struct ora_bindex ora_bindex;
ora_bindex *ora_boundary_build(int field_kind, const void *field, double rmax);
void ora_boundary_free(ora_bindex *bi);
double ora_boundary_distance(const ora_bindex *bi, const double *p, double rmax);
double ora_boundary_distance_brute(const ora_bindex *bi, const double *p);

/* ora_rk4 that also returns margin[n]: per tracer, the smallest distance to
 * the mesh boundary (capped at rmax) of any stage point it evaluated, the one
 * that left included.  Tracers whose margin exceeds the difference between
 * two computations of the same trajectory reach the same exit decisions.    */
long long ora_rk4_margin(int field_kind, const void *field, int dim, long long n,
                         const double *x0, const int *cells, double t0, double T, double dt,
                         double *xT, unsigned char *status, double *t_exit,
                         const ora_bindex *bi, double rmax, double *margin);

/* Dormand-Prince 5(4) with FSAL (the RK45 of the adaptive path).
 *   err = max_i |e_i| / (atol + rtol * max(|x_i|, |xnew_i|)), accept iff err <= 1,
 *   h_new = h * min(5, max(0.2, 0.9 * err^(-1/5)))   (factor 5 when err == 0).
 * group == 1: every seed steps on its own.  group == 32: seeds 32g..32g+31
 * share h; a step is accepted only if every live member accepts, and the
 * next h is the smallest member proposal.  adaptive == 0 takes fixed steps
 * of h0 with no error control (used by the order tests).  max_steps caps
 * attempted steps per seed (status MAXSTEPS).  nsteps_out (may be NULL)
 * receives the accepted steps per seed.                                     */
long long ora_dp45(int field_kind, const void *field, int dim, long long n,
                   const double *x0, const int *cells, double t0, double T,
                   double h0, double rtol, double atol, long long max_steps,
                   int group, int adaptive,
                   double *xT, unsigned char *status, double *t_exit,
                   long long *nsteps_out);

/* -------------------------------------------- flow-map gradient, C, FTLE */

/* grad F by finite differences on the seed lattice (Sec. 2 "Cauchy-Green"):
 * per axis b, in order of preference
 *   central      (F(p+e_b) - F(p-e_b)) / (2 h_b)
 *   forward 2nd  (-3F(p) + 4F(p+e_b) - F(p+2e_b)) / (2 h_b)
 *   backward 2nd ( 3F(p) - 4F(p-e_b) + F(p-2e_b)) / (2 h_b)
 * using only points that exist on the lattice and have status OK; none -> NaN.
 * A periodic axis wraps, and a neighbour across the wrap gets +-period[b] on
 * component b.  xT is [dim][N] FP64.  grad is [N][dim][dim], grad[a][b] =
 * dF_a/dx_b.                                                                */
void ora_flowmap_gradient(int dim, const int n[3], const double h[3],
                          const int periodic[3], const double period[3],
                          const double *xT, const unsigned char *status, double *grad);

/* Eq. 1: C = grad(F)^T grad(F), packed upper triangle, row by row:
 * 2D (C00, C01, C11); 3D (C00, C01, C02, C11, C12, C22).                    */
void ora_cauchy_green(int dim, long long n, const double *grad, double *C);

/* Eigenvalues of a packed symmetric dim x dim matrix by cyclic Jacobi
 * rotations to convergence; ascending order.  Returns sweeps used.          */
int ora_eig_sym(int dim, const double *Cpacked, double *eig);

/* The same with eigenvectors (Sec. 2 "Cauchy-Green"): vec[k * dim + r] is
 * component r of the unit eigenvector of eig[k] (vec may be NULL).          */
int ora_eigvec_sym(int dim, const double *Cpacked, double *eig, double *vec);

/* ora_eigvec_sym over n packed tensors: eig [n][dim], vec [n][dim][dim].     */
void ora_cg_eigen(int dim, long long n, const double *C, double *eig, double *vec);

/* FTLE from the largest eigenvalue of C: sigma = ln(sqrt(lambda_max)) / |T|.
 * lambda_max out (may be NULL); NaN in C gives NaN.                         */
void ora_ftle(int dim, long long n, const double *C, double T, double *lambda_max, double *ftle);

/* ------------------------------------------------------- tet geometry */

/* Sign of the orientation determinant of (a, b, c, d) evaluated exactly:
 * +1, 0 or -1; positive when d lies on the side of plane (a, b, c) where
 * (b-a) x (c-a) points.  Inputs are FP32 coordinates.                       */
int ora_orient3d_exact(const float *a, const float *b, const float *c, const float *d);

/* Exact containment of point p in the closed tet t: 1 if inside or on its
 * boundary.  *on_boundary set when some orientation is exactly zero.        */
int ora_tet_contains(const ora_tet_field *f, long long t, const float *p, int *on_boundary);

/* Lowest id among the closed tets containing p, by testing every tet;
 * -1 when none does.                                                        */
long long ora_tet_locate_brute(const ora_tet_field *f, const float *p);

/* Walk from start (Sec. 3.1 local search): cross a face whose plane separates
 * p from the tet until none does; then the tie-break of lowest id among the
 * closed tets holding p.  Falls back to brute force past walk_limit or when
 * the walk reaches a boundary face (the mesh need not be convex).
 * Returns the tet id or -1 if p is outside the mesh.                        */
long long ora_tet_locate_walk(const ora_tet_field *f, long long start, const float *p);

/* ------------------------------------------------- triangle geometry */

/* Sign of the orientation determinant (b - a) x (c - a) of three FP32 points,
 * evaluated exactly: +1 when c lies left of the directed line a -> b.       */
int ora_orient2d_exact(const float *a, const float *b, const float *c);

/* Exact containment of p in the closed triangle t (as ora_tet_contains).   */
int ora_tri_contains(const ora_tri_field *f, long long t, const float *p, int *on_boundary);

/* Lowest id among the closed triangles containing p; -1 when none does.    */
long long ora_tri_locate_brute(const ora_tri_field *f, const float *p);

/* Walk from start across edges whose line separates p from the triangle,
 * then the lowest-id tie-break among the closed triangles holding p (as
 * ora_tet_locate_walk).  A walk that reaches a boundary edge falls back to
 * brute force (the mesh need not be convex).  Returns the triangle id or -1
 * outside the mesh.                                                         */
long long ora_tri_locate_walk(const ora_tri_field *f, long long start, const float *p);

/* Set the OpenMP thread count (<= 0: leave the runtime default).  Returns
 * the count in effect.                                                      */
int ora_set_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
