/*
 * lcs.h -- C ABI of liblcs, a GB300 (sm_103a) library for the data-parallel hot
 * path of Lagrangian coherent structure computation: sampling the flow map of
 * an interpolated unsteady velocity field over a structured seed grid, then the
 * flow-map gradient, the Cauchy-Green tensor, its largest eigenvalue and the
 * FTLE field.
 *
 * Paper: S. Ameli, Y. Desai, S. C. Shadden, "Development of an efficient and
 * flexible pipeline for Lagrangian coherent structure computation"
 * (arXiv 2209.13775).  Each call below names the passage that defines it.
 *
 * Conventions (all calls):
 *  - Every call returns lcs_status and never aborts; the message of the last
 *    failure on a context is available from lcs_last_error().
 *  - Work is stream-ordered on the context's CUDA stream.  A call that writes a
 *    HOST buffer synchronises that stream before it returns; a call that writes
 *    a DEVICE buffer returns as soon as the work is queued.
 *  - The caller owns every array it passes; the library copies what it keeps.
 *    Handles (lcs_field, lcs_seeds, lcs_flowmap) own device memory allocated by
 *    the library until the matching lcs_free_*().
 *  - Positions are SoA: x[0..N), y[0..N), z[0..N).  Seed index is x-fastest:
 *    id = i + nx*(j + ny*k).  Batched outputs are job-major.
 *  - A context is not thread-safe; use one per host thread.
 *  - Handles may be used with any context on the same device.  The library
 *    orders work only on the calling context's stream: when two contexts touch
 *    one handle, the caller orders them (events, or a call that synchronises
 *    its stream, such as lcs_update_frames).
 */
#ifndef LCS_H
#define LCS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LCS_OK = 0,
    LCS_EINVAL = 1,       /* bad argument or descriptor                         */
    LCS_ENOMEM = 2,       /* device allocation failed                           */
    LCS_ECUDA = 3,        /* a CUDA runtime call failed                          */
    LCS_ETIMEOUT = 4,     /* a bounded device-side wait gave up                  */
    LCS_EWALK = 5,        /* a tet walk hit its step limit                       */
    LCS_EMAXSTEPS = 6,    /* an adaptive integration hit max_steps               */
    LCS_EUNSUPPORTED = 7  /* combination not implemented                         */
} lcs_status;

/* grid kinds, storage precisions, integrators */
enum { LCS_RECTILINEAR = 0, LCS_TET = 1, LCS_TRI = 2 };
enum { LCS_F32 = 0, LCS_F16 = 1, LCS_BF16 = 2 };
enum { LCS_RK4 = 0, LCS_RK45 = 1, LCS_SURROGATE = 2 };

/* per-tracer status written by lcs_advect */
enum {
    LCS_TRACER_OK = 0,        /* inside the domain at t0 + T                            */
    LCS_TRACER_LEFT = 1,      /* left the domain; frozen, exit time recorded            */
    LCS_TRACER_OUTSIDE = 2,   /* seed not inside the domain at t0                       */
    LCS_TRACER_MAXSTEPS = 3,  /* adaptive step cap reached                              */
    LCS_TRACER_WALKFAIL = 4   /* tet walk exceeded walk_limit                           */
};

typedef struct lcs_ctx lcs_ctx;
typedef struct lcs_field lcs_field;
typedef struct lcs_seeds lcs_seeds;
typedef struct lcs_flowmap lcs_flowmap;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device` that queues work on `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the
 * handle.  Errors: LCS_EINVAL (NULL out, bad device), LCS_ECUDA.            */
lcs_status lcs_create(lcs_ctx **out, int device, void *stream);

/* Destroy a context (NULL is a no-op).  Handles created on it must be freed
 * first.                                                                    */
void lcs_destroy(lcs_ctx *ctx);

/* Message of the last failure on ctx ("" when none).  Owned by ctx.        */
const char *lcs_last_error(const lcs_ctx *ctx);

/* Switch the stream later calls queue on.                                   */
lcs_status lcs_set_stream(lcs_ctx *ctx, void *stream);

/* The CUDA device index of ctx (-1 for NULL), so that a binding can check
 * that caller-owned device buffers sit on it.                              */
int lcs_context_device(const lcs_ctx *ctx);

/* Wait for the context's stream, then read and clear the device-side error
 * word: LCS_EWALK / LCS_ETIMEOUT / LCS_EMAXSTEPS when a kernel recorded one.  */
lcs_status lcs_synchronize(lcs_ctx *ctx);

/* --------------------------------------------------------- field (a1, a3) */

/* Velocity data (Sec. 2 "Reader"/"Cache"/"Interpolator"): nodal velocity
 * frames at increasing times, interpolated linearly in time and
 * bilinearly / trilinearly (rectilinear) or piecewise-linearly (tets in 3D,
 * triangles in 2D: Sec. 3.1, Sec. 3.2's 2D unstructured stenosis data) in
 * space.  Rectilinear node (i,j,k) sits at origin + (i,j,k)*spacing; a
 * periodic axis has n cells (node n-1 joins node 0) and period n*spacing;
 * queries on a non-periodic axis are clamped to the box.  Time outside
 * [t_first, t_last] uses the end frame unless time_periodic, which wraps t
 * into [t_first, t_first + period).                                         */
typedef struct {
    int dim;                    /* 2 or 3 (tets: 3, triangles: 2)                    */
    int kind;                   /* LCS_RECTILINEAR | LCS_TET | LCS_TRI                */
    int n[3];                   /* rectilinear nodes per axis (n[2] unused in 2D)     */
    double origin[3];
    double spacing[3];
    int periodic[3];            /* per-axis spatial periodicity (rectilinear)         */
    int nframes;                /* >= 1                                               */
    const double *frame_times;  /* HOST, nframes, strictly increasing                 */
    int time_periodic;
    double period;
    int storage;                /* LCS_F32 | LCS_F16 | LCS_BF16 (velocity storage)    */
    /* tetrahedral meshes (kind == LCS_TET) and triangle meshes (LCS_TRI), HOST:     */
    long long nnodes, ncells;
    const float *node_xyz;      /* [nnodes][3] (tets) or [nnodes][2] (triangles)      */
    const int *tets;            /* [ncells][4] node ids (tets), [ncells][3] (triangles,
                                   either orientation; the mesh need not be convex)   */
    const int *nbrs;            /* [ncells][4] tet across the face opposite vertex j
                                   ([ncells][3]: triangle across the edge opposite
                                   vertex j), -1 on the boundary; NULL: built by the
                                   library                                           */
} lcs_field_desc;

/* Copy velocity frames into device storage.  frames is FP32,
 * [nframes][nz][ny][nx][dim] (rectilinear) or [nframes][nnodes][dim] (meshes),
 * in host memory or, if frames_on_device, device memory.  The library
 * converts to desc->storage (FP16/BF16 round to nearest).  The call checks
 * every value for finiteness on the device and synchronises the stream.
 * Host frames pass through a staging buffer that the context keeps (grown
 * to the largest upload, freed with the context).
 * Errors: LCS_EINVAL (descriptor, a non-finite velocity or node coordinate,
 * a mesh cell of zero area or volume), LCS_ENOMEM, LCS_ECUDA.               */
lcs_status lcs_load_field(lcs_ctx *ctx, const lcs_field_desc *desc, const float *frames,
                          int frames_on_device, lcs_field **out);

/* Spatial dimension of a loaded field (2 or 3; 0 for NULL).                 */
int lcs_field_dim(const lcs_field *field);

/* Replace the frames of a loaded field with new data of the same shape
 * (same conventions and finiteness check as lcs_load_field).  Returns once
 * the new frames are in place (the stream is synchronised), so work queued
 * afterwards on any stream sees them.  No queued work may still read the
 * field: to upload while an advection runs, update the other field of a
 * double buffer, from a second context on its own stream.                  */
lcs_status lcs_update_frames(lcs_ctx *ctx, lcs_field *field, const float *frames,
                             int frames_on_device);

void lcs_free_field(lcs_field *field);

/* --------------------------------------------------------- seed grid (a2) */

/* Structured seed lattice (Sec. 2 "Seed"): along axis a,
 *   x_i = lo[a] + i * step,  step = (hi[a] - lo[a]) / (n[a] - 1)   (periodic[a] == 0)
 *                            step = (hi[a] - lo[a]) / n[a]         (periodic[a] != 0)
 * evaluated in FP64 with round-to-nearest and no fused operations, then
 * rounded to FP32 -- bit-identical to that definition.  A periodic axis makes
 * the finite differences of lcs_cauchy_green / lcs_ftle wrap with period
 * hi[a] - lo[a].                                                            */
typedef struct {
    int dim;
    int n[3];
    double lo[3], hi[3];
    int periodic[3];
} lcs_seed_desc;

/* Generate the lattice on the device.  If `field` is a tet or triangle mesh,
 * also locate the cell holding each seed with exact orientation predicates:
 * the lowest cell id among the closed cells containing the seed, -1 if none
 * (Sec. 2 "Seed": the cell of each seed on unstructured data).  field may be
 * NULL.
 * Errors: LCS_EINVAL, LCS_ENOMEM, LCS_ECUDA.                                */
lcs_status lcs_seed_grid(lcs_ctx *ctx, const lcs_seed_desc *desc, const lcs_field *field,
                         lcs_seeds **out);

/* Number of seeds of a lattice.                                             */
long long lcs_seeds_count(const lcs_seeds *seeds);

/* Copy seed positions ([dim][N] FP32) and/or cell ids ([N] int32, -1 outside,
 * only for seeds made on a mesh field) to host or device buffers (either may be
 * NULL).                                                                    */
lcs_status lcs_seeds_get(lcs_ctx *ctx, const lcs_seeds *seeds, float *xyz, int *cells,
                         int on_device);

void lcs_free_seeds(lcs_seeds *seeds);

/* Auxiliary points around each seed (Sec. 2 "Seed" and "Cauchy-Green": a
 * second way to difference the flow map, with points placed close around
 * each seed instead of its lattice neighbours).  From a lattice of N seeds
 * made by lcs_seed_grid on a rectilinear field, a point set of N * 2 * dim
 * points: point (p * dim + b) * 2 + s is seed p moved by +delta[b] (s = 0) or
 * -delta[b] (s = 1) along axis b, computed in FP64 and rounded to FP32.
 * lcs_advect advects it like any seeds (lcs_seeds_count gives the points);
 * lcs_cauchy_green, lcs_ftle and lcs_cg_eigen on its flow map then form, per
 * lattice seed (N outputs),
 *   grad F[a][b] = (F_a(p, b, 0) - F_a(p, b, 1)) / (x0_b(p, b, 0) - x0_b(p, b, 1))
 * in FP64 from the FP32 positions, x0 the FP32 starting points (so the divisor
 * is the spacing the points really have); NaN unless all 2 dim points are OK.
 * delta [dim] HOST, each > 0 and finite.  Not for lcs_ftle_early; for a
 * lattice made on a mesh field use lcs_seed_aux_field.
 * Errors: LCS_EINVAL, LCS_ENOMEM, LCS_ECUDA.                               */
lcs_status lcs_seed_aux(lcs_ctx *ctx, const lcs_seeds *lattice, const double *delta, lcs_seeds **out);

/* lcs_seed_aux for a lattice made by lcs_seed_grid on `field`: on a tet or
 * triangle field the auxiliary points also get their exact cells (as
 * lcs_seed_grid locates seeds), so lcs_advect takes them on that field; a
 * point outside the mesh is OUTSIDE and its seed's grad F NaN.  On a
 * rectilinear field (or NULL) it is lcs_seed_aux.
 * Errors: LCS_EINVAL (a lattice not made on this mesh field), LCS_ENOMEM,
 * LCS_ECUDA.                                                                */
lcs_status lcs_seed_aux_field(lcs_ctx *ctx, const lcs_seeds *lattice, const lcs_field *field, const double *delta,
                              lcs_seeds **out);

/* ------------------------------------------------- flow map (a3-a8, a12) */

/* Integration options (Sec. 2 "Flow Map": single-step Runge-Kutta; Eq. 2
 * integrated over (t0, t0 + T); T < 0 integrates backward).
 *  LCS_RK4   fixed step |dt|, |T|/|dt| must be an integer (within 1e-9).
 *            Steps at t_n = t0 + n*dt, stages at t_n, t_n + dt/2, t_n + dt.
 *  LCS_RK45  Dormand-Prince 5(4) with one step size per warp of 32 seeds
 *            (32 consecutive seed ids): a step is accepted only when every
 *            live lane accepts (err <= 1, err = max_i |e_i| / (atol + rtol *
 *            max(|x_i|, |x_new_i|))), and the next step is the smallest lane
 *            proposal h * min(5, max(0.2, 0.9 err^-1/5)).  On every
 *            field kind.
 *  LCS_SURROGATE  2D non-periodic rectilinear fields, one job, T = K tau > 0
 *            with tau the network's step and tau = S dt: per sub-interval k
 *            every tracer proposes x + displacement(x, t0 + k tau); in each
 *            group of 32 consecutive seeds one audited lane (lowbias32 hash of
 *            k and the group index, modulo the group size) integrates RK4 (step
 *            dt) over the sub-interval, and the whole group integrates RK4
 *            instead when |proposal - RK4| > gate_tol or any lane's
 *            rho > log10(gate_tol).  The RK4 arithmetic is that of LCS_RK4, so
 *            gate_tol = 0 reproduces it bit for bit.
 * Batches: njobs > 1 integrates the same seeds for each (job_t0[j], job_T[j])
 * pair in one persistent launch.
 * Snapshots (LCS_RK4, every field kind): nsnap > 0 also keeps the flow
 * map at intermediate horizons of every integration, so one run yields the
 * Cauchy-Green tensor at several times (Sec. 3.1 and Sec. 4: the flow map of
 * an interval from the steps of a longer integration).  Snapshot s of job j
 * lands in flow-map slot njobs + j * nsnap + s and holds the state after
 * min(|snap_T[s]|, |T_j|) / dt steps (position, status, exit time; a tracer
 * that left before keeps its frozen state), with |T| = min(|snap_T[s]|, |T_j|)
 * for lcs_ftle; it equals, bit for bit, a separate run with that horizon.
 * The flow map then needs njobs * (1 + nsnap) slots.                       */
#define LCS_MAX_SNAP 8
typedef struct {
    int method;                 /* LCS_RK4 | LCS_RK45 | LCS_SURROGATE                */
    double t0, T;               /* single job (njobs <= 1)                            */
    int njobs;                  /* 0 or 1: single job; > 1: batch                     */
    const double *job_t0;       /* HOST [njobs] when njobs > 1                        */
    const double *job_T;        /* HOST [njobs]                                       */
    double dt;                  /* RK4 step magnitude                                 */
    double rtol, atol, h0;      /* RK45                                               */
    long long max_steps;        /* RK45 attempted-step cap per warp (0 = 10^6)        */
    int walk_limit;             /* mesh walk steps per point location (0 = 512); on
                                   triangles the bin lists settle a walk that stops  */
    int block_threads;          /* 0 = library choice                                 */
    int variant;                /* 0 = library choice; 1 = cached gather;
                                   2 = shared-memory frame ring (2D rectilinear);
                                   3 = tracers re-bundled by cell between episodes (3D);
                                   4 = persistent shared-memory ring pulling (job, tile)
                                       items longest-job first (2D, batches);
                                   5 = the field blended once to every stage time of
                                       every job (2D time slices; up to 16 GiB; the
                                       default in 2D when they take at most 2 GiB)     */
    const void *surrogate;      /* LCS_SURROGATE: the lcs_mlp to step with            */
    int episode_steps;          /* variant 3: RK4 steps between re-bundlings (0 = 40) */
    int tracers_per_thread;     /* variants 2 and 4: 1 or 2 tracers per thread (0 = 1) */
    int use_graph;              /* capture the launches of this call in a CUDA graph,
                                   cached on the context and replayed while the same
                                   field, seeds, flow map and options come back      */
    double gate_tol;            /* LCS_SURROGATE: audit threshold (0 = every
                                   sub-interval by RK4, +inf = never)              */
    int nsnap;                  /* 0..LCS_MAX_SNAP snapshots per integration        */
    const double *snap_T;       /* HOST [nsnap]: horizon magnitudes, > 0, strictly
                                   increasing, each a whole number of steps dt    */
    int variational;            /* LCS_RK4, no snapshots: also integrate grad F by
                                   the variational equations (lcs_flowmap_grad,
                                   lcs_ftle_variational); every field kind         */
    double wait_limit;          /* seconds a block of the shared-memory frame ring
                                   (variants 2 and 4) waits for a frame copy before
                                   it stops integrating and the next lcs_synchronize
                                   reports LCS_ETIMEOUT (the flow map of that call is
                                   then incomplete); 0 = 1 s, at most 60 s; under
                                   1e-6 a copy not complete at its first test counts
                                   as late.  Copies already issued are always waited
                                   for (with the 1 s bound) before a block exits.  A
                                   short limit lets a caller fail fast             */
} lcs_advect_opts;

/* Flow-map storage for `njobs` integrations of one lattice.                 */
lcs_status lcs_flowmap_create(lcs_ctx *ctx, const lcs_seeds *seeds, int njobs, lcs_flowmap **out);

/* Advect every seed through the field and write x(t0 + T) per job into fm,
 * with per-tracer status and exit time (a tracer leaving the domain is
 * frozen: rectilinear when more than one cell outside a non-periodic axis
 * after a step, at that step's end time; tets and triangles when a stage
 * point falls outside the mesh, at the start of that step).
 * Errors: LCS_EINVAL (options, a flow map with too few slots),
 * LCS_EUNSUPPORTED (e.g. snapshots with RK45 or the surrogate), LCS_ECUDA.      */
lcs_status lcs_advect(lcs_ctx *ctx, const lcs_field *field, const lcs_seeds *seeds,
                      const lcs_advect_opts *opts, lcs_flowmap *fm);

/* Copy job `job` of a flow map: positions [dim][N] FP32 (unwrapped across
 * periodic axes), status [N] uint8, exit time [N] FP32.  Any may be NULL.   */
lcs_status lcs_flowmap_get(lcs_ctx *ctx, const lcs_flowmap *fm, int job, float *xyz,
                           unsigned char *status, float *t_exit, int on_device);

/* Overwrite job `job` of a flow map with caller-supplied tracer end states,
 * so that lcs_cauchy_green / lcs_ftle / lcs_cg_eigen evaluate Eq. 1 and the
 * FTLE on a flow map computed elsewhere (another integrator, a file).
 * xyz [dim][N] FP32 (unwrapped across periodic axes), status [N] uint8
 * (LCS_TRACER_* codes), t_exit [N] FP32 or NULL (left unchanged); T is the
 * job's integration time (its sign the direction; the FTLE divides by |T|).
 * Buffers are all host or all device (on_device); the library copies them.
 * The flow map's variational grad F (every job), if any, is invalidated.
 * Errors: LCS_EINVAL (null flow map or xyz/status, job out of range, T zero or
 * not finite, a host status value above LCS_TRACER_WALKFAIL), LCS_ECUDA.      */
lcs_status lcs_flowmap_set(lcs_ctx *ctx, lcs_flowmap *fm, int job, const float *xyz,
                           const unsigned char *status, const float *t_exit, double T, int on_device);

/* grad F of every tracer of job `job` from the variational equations (Sec. 1:
 * the linearised flow map, the alternative to differencing the seed grid):
 * lcs_advect with opts.variational integrates dM/dt = J(x, t) M, M(t0) = I,
 * next to Eq. 2 with the same RK4 stages, J the spatial Jacobian of the
 * interpolant (piecewise: per cell on meshes, zero across an axis where a
 * rectilinear query is clamped to the box); M is frozen with a tracer that
 * leaves.  grad [N][dim][dim] FP32,
 * grad[(p*dim + a)*dim + b] = d x_a(T) / d x0_b.
 * Errors: LCS_EINVAL when no variational integration wrote this flow map.   */
lcs_status lcs_flowmap_grad(lcs_ctx *ctx, const lcs_flowmap *fm, int job, float *grad, int on_device);

/* Per-tracer step counts of job `job` ([N] int32).  After LCS_RK45: accepted
 * steps (32 consecutive seeds step together, so the tracers of a group that
 * stay live to the end report the same count, and a tracer that stopped early
 * the count it had reached).  After LCS_SURROGATE: the sub-intervals the
 * tracer integrated with RK4 because its group failed the audit.
 * Errors: LCS_EINVAL when neither integration wrote this flow map.          */
lcs_status lcs_flowmap_steps(lcs_ctx *ctx, const lcs_flowmap *fm, int job, int *steps, int on_device);

void lcs_free_flowmap(lcs_flowmap *fm);

/* Choose the launch options of an lcs_advect call (variant, block_threads,
 * tracers_per_thread, episode_steps) by timing candidates with CUDA events on
 * these very inputs, and write the fastest back into *opts (other fields are
 * read, not changed).  The choice is remembered in the text file cache_path
 * (NULL: no cache), keyed by device, field shape, seed count and jobs; a later
 * call with the same key returns without timing.  Tuning runs lcs_advect into
 * a temporary flow map (allocated and freed here).
 * Errors: LCS_EINVAL, LCS_EUNSUPPORTED (not RK4 on a rectilinear field), and
 * those of lcs_advect.                                                      */
lcs_status lcs_autotune(lcs_ctx *ctx, const lcs_field *field, const lcs_seeds *seeds, lcs_advect_opts *opts,
                        const char *cache_path);

/* ------------------------------------------ learned surrogate (a13, a14) */

/* A multilayer perceptron 7 -> 128 -> 128 -> 128 -> 128 -> 3 with SiLU after each
 * hidden layer maps features of a point (x, y) at time t of a 2D field,
 *   phi = (x - cx, y - cy, sin(omega t), cos(omega t), sin(kx x), cos(kx x), sin(ky y)),
 * to outputs o: the displacement over one step tau is out_scale * (o0, o1), and
 * o2 = rho predicts log10 of that displacement's error.  It stands in for the
 * integrator over a sub-interval (the paper has no such network; the local
 * flow-map approximations it mentions among related work, Sec. 4, are the
 * nearest idea).  Parameters: LCS_MLP_NPARAMS FP32 values packed as
 *   W0[128][7] b0[128] W1[128][128] b1 W2 b2 W3 b3 W4[3][128] b4[3]
 * (row-major W[out][in]); the library keeps them in FP32 and computes with BF16
 * copies of the weights and BF16 activations, FP32 accumulation and FP32 biases,
 * on the tensor cores.                                                      */
#define LCS_MLP_NPARAMS 50947

typedef struct lcs_mlp lcs_mlp;

typedef struct {
    double center[2];           /* (cx, cy)                                         */
    double kx, ky, omega;       /* spatial and temporal frequencies of phi         */
    double tau;                 /* step of the surrogate (> 0)                     */
    double out_scale;           /* displacement = out_scale * (o0, o1) (> 0)       */
} lcs_mlp_desc;

/* Network with the given parameters (host or device, copied).
 * Errors: LCS_EINVAL (descriptor), LCS_ENOMEM, LCS_ECUDA.                    */
lcs_status lcs_mlp_create(lcs_ctx *ctx, const lcs_mlp_desc *desc, const float *params, int on_device,
                          lcs_mlp **out);
/* Replace / read the FP32 parameters; setting them also resets Adam's state. */
lcs_status lcs_mlp_set_params(lcs_ctx *ctx, lcs_mlp *mlp, const float *params, int on_device);
lcs_status lcs_mlp_get_params(lcs_ctx *ctx, const lcs_mlp *mlp, float *params, int on_device);
void lcs_mlp_free(lcs_mlp *mlp);

/* Outputs o [3][n] (o0, o1, o2 rows) at points xyt [3][n] (x, y, t rows).    */
lcs_status lcs_mlp_forward(lcs_ctx *ctx, const lcs_mlp *mlp, long long n, const float *xyt, float *out,
                           int on_device);

/* Mean loss over n samples (n a positive multiple of 128) and its gradient
 * [LCS_MLP_NPARAMS] (grads may be NULL; loss: host pointer or NULL):
 *   loss = mean of (o0 - dx/s)^2 + (o1 - dy/s)^2
 *          + rho_weight (o2 - log10(|s (o0, o1) - d| + 1e-7))^2,
 * s = out_scale, d = disp [2][n] the integrator's displacement over tau from
 * the points xyt [3][n]; the log10 target is a constant of the gradient.
 * The gradient also stays in the network for lcs_mlp_adam.                 */
lcs_status lcs_mlp_loss_grad(lcs_ctx *ctx, lcs_mlp *mlp, long long n, const float *xyt, const float *disp,
                             double rho_weight, float *grads, double *loss, int on_device);

/* One Adam step (Kingma & Ba) on the FP32 parameters with gradient grads
 * (NULL: the last lcs_mlp_loss_grad), learning rate lr, moments beta1, beta2,
 * and eps; bias corrections use the network's own step count.              */
lcs_status lcs_mlp_adam(lcs_ctx *ctx, lcs_mlp *mlp, const float *grads, int on_device, double lr, double beta1,
                        double beta2, double eps);

typedef struct {
    long long batch;            /* samples per step, a positive multiple of 128     */
    int epochs;                 /* passes over the samples                         */
    double lr, lr_min;          /* cosine decay from lr to lr_min over all steps   */
    double beta1, beta2, eps;   /* Adam                                            */
    double rho_weight;          /* weight of the error head's loss term            */
    double dt;                  /* RK4 step of the targets (tau a multiple of it)  */
} lcs_train_desc;

/* Train on the field: targets are the RK4 (step dt) displacements over tau from
 * every sample (x0, y0, t0) of samples [3][ns], then epochs of Adam steps over
 * consecutive batches (ns / batch of them; the samples are taken in the given
 * order, so pass them shuffled).  loss_per_epoch (host, [epochs], or NULL):
 * mean training loss of each epoch.  2D rectilinear fields.
 * Errors: LCS_EINVAL, LCS_EUNSUPPORTED, LCS_ECUDA.                          */
lcs_status lcs_surrogate_train(lcs_ctx *ctx, const lcs_field *field, lcs_mlp *mlp, const lcs_train_desc *desc,
                               long long ns, const float *samples, int on_device, double *loss_per_epoch);

/* ------------------------------------------------ tensor-core GEMM (BF16) */

/* C[M x N] = A[M x K] * B[N x K]^T (accumulate = 1: C += ...) on the tcgen05
 * tensor cores, FP32 accumulation; the trainer of the surrogate is built on it.
 * Device pointers: A, B BF16 with K contiguous (row strides lda, ldb in elements,
 * multiples of 8), C FP32 (row stride ldc).  K must be a multiple of 16 and N
 * be 16 or a multiple of 128; splits > 1 cuts K into that many ranges summed
 * with atomics.  No counterpart in the paper.
 * Errors: LCS_EINVAL (shapes), LCS_ECUDA.                                   */
lcs_status lcs_gemm_bf16(lcs_ctx *ctx, long long M, int N, long long K, const void *A, long long lda, const void *B,
                         long long ldb, float *C, long long ldc, int splits, int accumulate);

/* ---------------------------------------- grad F, C, lambda_max, FTLE (a9-a11) */

/* Cauchy-Green tensor C = grad(F)^T grad(F) (Eq. 1) with grad F from finite
 * differences of the final positions on the seed lattice (Sec. 2
 * "Cauchy-Green"), in FP64 from the FP32 positions.  Per axis b the stencil
 * is, in order of preference, central (F(p+e_b) - F(p-e_b)) / 2h_b, forward
 * (-3F(p) + 4F(p+e_b) - F(p+2e_b)) / 2h_b or backward (3F(p) - 4F(p-e_b) +
 * F(p-2e_b)) / 2h_b, using only lattice points with status OK; none -> NaN.
 * Output packed per seed: 2D (C00, C01, C11), 3D (C00, C01, C02, C11, C12,
 * C22), FP64.  job = -1 writes every job, job-major.
 * Errors: LCS_EINVAL (a lattice with fewer than 3 seeds along an axis, where
 * no difference rule applies; auxiliary-point and variational flow maps are
 * exempt), LCS_ECUDA.                                                       */
lcs_status lcs_cauchy_green(lcs_ctx *ctx, const lcs_flowmap *fm, int job, double *C,
                            int on_device);

/* FTLE sigma = ln(sqrt(lambda_max(C))) / |T| (Sec. 1: the FTLE is derived from
 * the largest eigenvalue of C) as FP32 [N], NaN where C is undefined;
 * optionally lambda_max [N] FP64 and C (as lcs_cauchy_green) from the same
 * pass.  lambda_max and C may be NULL.  job = -1 writes every job.
 * Errors: as lcs_cauchy_green.                                              */
lcs_status lcs_ftle(lcs_ctx *ctx, const lcs_flowmap *fm, int job, float *ftle, double *lambda_max,
                    double *C, int on_device);

/* FTLE (and optionally lambda_max and C, as lcs_ftle) from the variational
 * grad F of lcs_flowmap_grad instead of finite differences: C = M^T M in FP64
 * from the FP32 M, per tracer, NaN for a tracer that is not OK.            */
lcs_status lcs_ftle_variational(lcs_ctx *ctx, const lcs_flowmap *fm, int job, float *ftle, double *lambda_max,
                                double *C, int on_device);

/* Early Cauchy-Green evaluation (Sec. 2 "Flow Map": for trajectories that exit
 * the data, the CG tensor is formed ahead of the horizon wherever such a
 * trajectory is used).  fm holds job `job` of an lcs_advect call made with field, seeds and
 * opts (LCS_RK4, any field kind).  Each seed's finite differences use the
 * lattice neighbours the differences choose from the seeds valid at the start
 * (as lcs_cauchy_green: central, or one-sided at a non-periodic lattice edge
 * or beside seeds outside a mesh); m = the fewest steps the seed or one of
 * them stayed in the domain (all steps if still OK at the end; otherwise one
 * less than the step it left in on rectilinear fields, the steps before the
 * one it failed in on meshes).  m = all steps: the FTLE of lcs_ftle; 0 < m:
 * grad F from those tracers re-integrated over m steps (the same arithmetic,
 * so the positions they had after step m), C, lambda_max and
 * sigma = ln(sqrt(lambda_max)) / (m |dt|); m = 0: NaN.  ftle [N] FP32,
 * t_eval [N] FP32 (optional): the horizon each value belongs to.
 * Synchronises the context's stream (the number of early seeds sizes the
 * second pass).  Errors: LCS_EINVAL, LCS_EUNSUPPORTED, LCS_ENOMEM, LCS_ECUDA. */
lcs_status lcs_ftle_early(lcs_ctx *ctx, const lcs_field *field, const lcs_seeds *seeds, const lcs_advect_opts *opts,
                          const lcs_flowmap *fm, int job, float *ftle, float *t_eval, int on_device);

/* Eigenvalues and eigenvectors of C at every seed (Sec. 2 "Cauchy-Green" lists
 * both among the filter's per-seed outputs), C as lcs_cauchy_green.  eigval [N][dim] FP64 in
 * ascending order; eigvec [N][dim][dim] FP64, eigvec[(p*dim + k)*dim + r]
 * = component r of the unit eigenvector of eigval[p][k], its largest-magnitude
 * component positive.  Cyclic Jacobi rotations in FP64 to a relative
 * off-diagonal threshold (16 sweeps at most).  NaN where C is undefined.
 * Either output may be NULL; job = -1 writes every job.
 * Errors: LCS_EINVAL, LCS_ECUDA.                                            */
lcs_status lcs_cg_eigen(lcs_ctx *ctx, const lcs_flowmap *fm, int job, double *eigval, double *eigvec,
                        int on_device);

/* ------------------------------------------------------------ kernel timing */

/* Time the library's kernels by phase with CUDA events recorded on the
 * context's stream around each launch (off by default; costs two event
 * records per launch).  Phases: */
enum {
    LCS_PHASE_ADVECT = 0,     /* advection kernels (RK4 step loops)                  */
    LCS_PHASE_REBUNDLE = 1,   /* re-bundling by cell (scan, permutation, gather)      */
    LCS_PHASE_SLICES = 2,     /* time slices of the field for an episode              */
    LCS_PHASE_CG = 3          /* finite differences, Cauchy-Green, eigenvalue, FTLE   */
};
lcs_status lcs_timing_enable(lcs_ctx *ctx, int on);

/* Wait for the recorded launches of `phase`, return their summed duration in
 * milliseconds and their count (either pointer may be NULL), and start a new
 * tally.                                                                    */
lcs_status lcs_timing_read(lcs_ctx *ctx, int phase, double *ms, long long *launches);

/* ------------------------------------- advection without device allocation */

/* No counterpart in the paper: an interface for callers that cannot allocate
 * device memory.  lcs_advect grows a context-owned scratch buffer with
 * cudaMalloc when a call needs more room; some callers must not let that
 * happen -- a plugin running inside another runtime's execution phase, where
 * that runtime owns the device memory and forbids allocation; a process that
 * handed nearly all device memory to a pool up front; a latency-bound loop
 * that cannot afford an allocation that may synchronise the device.
 *
 * lcs_advect_rk4_noalloc integrates one job with fixed-step RK4 (the same
 * schedule and kernels, so the same results as lcs_advect with method
 * LCS_RK4) on a field already loaded by lcs_load_field, and allocates
 * nothing: its working memory (the per-stage frame schedule) is a 1 MiB array
 * compiled into the library, which every GPU that loads the library holds
 * until the process exits.  The caller passes every input and output as
 * DEVICE pointers on ctx's device:
 *   seeds   [3 or 2][n] FP32 SoA start positions (e.g. from lcs_seeds_get)
 *   xyz     [dim][n] FP32 final positions (unwrapped on periodic axes)
 *   status  [n] uint8, t_exit [n] FP32 (as lcs_flowmap_get)
 * Limits: |T|/|dt| must be an integer <= LCS_NOALLOC_MAX_STEPS, else
 * LCS_EINVAL with nothing queued.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress), so make that first call
 * before any stream capture.  All calls share the one array: two calls whose
 * work overlaps on the GPU (different streams, or different contexts on one
 * device) race on it; calls queued on one stream are ordered and safe.
 * Nothing in the array needs to start at zero: each call writes every entry
 * it reads before reading it.                                               */
#define LCS_NOALLOC_MAX_STEPS 43680
lcs_status lcs_advect_rk4_noalloc(lcs_ctx *ctx, const lcs_field *field, const float *seeds, long long n,
                                  double t0, double T, double dt, float *xyz, unsigned char *status,
                                  float *t_exit);

#ifdef __cplusplus
}
#endif
#endif
