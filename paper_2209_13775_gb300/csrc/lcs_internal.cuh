// lcs_internal.cuh -- shared declarations of liblcs's translation units.
//
// Library-private: handle layouts, kernel parameter blocks, launchers and the
// small device helpers (storage loads, bounded mbarrier waits) that more than
// one kernel file uses.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "lcs.h"

// device error word bits (OR-ed by kernels, read by lcs_synchronize)
#define LCS_ERRBIT_TIMEOUT 1u
#define LCS_ERRBIT_WALK 2u
#define LCS_ERRBIT_MAXSTEPS 4u

// bound on any device-side wait: a copy that has not landed after this long is
// treated as failed (error bit set, the waiting block stops its work)
#define LCS_WAIT_LIMIT_NS 1000000000ull

// kernel phases timed with CUDA events when a context's timing is on
#define LCS_NPHASES 4

struct lcs_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    unsigned int *d_errword = nullptr;   // device error flags
    int num_sms = 0;
    size_t smem_optin = 0;               // max dynamic shared memory per block
    // scratch: device memory the library reuses across calls (queue counters)
    void *d_scratch = nullptr;
    size_t scratch_bytes = 0;
    // staging of frames uploaded from host memory (grown as needed) and the finiteness flag
    float *d_stage = nullptr;
    size_t stage_bytes = 0;
    int *d_flag = nullptr;
    // CUDA graphs of lcs_advect calls (opts.use_graph), keyed by handles and options
    struct GraphEntry {
        std::string key;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        unsigned long long last_use = 0;
    };
    std::vector<GraphEntry> graphs;
    unsigned long long graph_clock = 0;
    cudaStream_t cap_stream = nullptr;   // capture stream (graphs launch on `stream`)
    // per-phase event timing (lcs_timing_enable / lcs_timing_read)
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    cudaEvent_t ev_open[LCS_NPHASES] = {};
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_done[LCS_NPHASES];
};

// next unique handle id
unsigned long long lcs_next_uid();

// bracket the launches of one phase with events on stream s (no-ops unless timing is on)
void lcs_tm_begin(lcs_ctx *ctx, int phase, cudaStream_t s);
void lcs_tm_end(lcs_ctx *ctx, int phase, cudaStream_t s);

struct lcs_field {
    unsigned long long uid = 0;          // unique for the process lifetime (graph cache keys)
    lcs_ctx *ctx = nullptr;
    int dim = 0, kind = 0, storage = 0;
    int n[3] = {1, 1, 1};
    double origin[3] = {0, 0, 0}, spacing[3] = {1, 1, 1};
    int periodic[3] = {0, 0, 0};
    int nframes = 0;
    std::vector<double> times;
    int time_periodic = 0;
    double period = 0.0;
    double *d_times = nullptr;
    // velocity slabs: [nslabs][frame_stride bytes]; node v occupies vec stored components.
    // 2D: one slab per frame, (u, v) per node.  3D: one slab per frame interval k holding
    // (u_k, 0, u_{k+1}, 0) per node, so one load brings both frames of a corner.
    void *d_frames = nullptr;
    int nslabs = 0;
    int vec = 0;                       // stored components per node (2 in 2D, 8 in 3D)
    size_t elem_bytes = 4;             // bytes per stored component
    size_t frame_bytes = 0;            // unpadded bytes per slab
    size_t frame_stride = 0;           // padded bytes per slab (multiple of 256)
    long long nodes = 0;
    // tetrahedral mesh
    long long ncells = 0;
    float4 *d_xyz = nullptr;           // [nodes]
    int4 *d_tets = nullptr;            // [ncells]
    int4 *d_nbrs = nullptr;            // [ncells]
    float4 *d_tetmap = nullptr;        // [ncells][4]: rows of the inverse affine map + v0, then nbrs
    int bin_n[3] = {0, 0, 0};          // bin grid over the nodes' bounding box (meshes)
    float bin_lo[3] = {0, 0, 0}, bin_inv[3] = {0, 0, 0};
    // triangle mesh (d_tets, d_nbrs hold (a, b, c, 0) and (n0, n1, n2, -1))
    float2 *d_xy = nullptr;            // [nodes]
    float4 *d_trimap = nullptr;        // [ncells] (M00, M01, M10, M11) of the inverse affine map
    float2 *d_triv0 = nullptr;         // [ncells] vertex 0
    int *d_bstart = nullptr;           // [nbins + 1] CSR (meshes): cells whose bounding box meets a bin
    int *d_blist = nullptr;
    long long nbins = 0;
    int convex = 0;                    // mesh proven convex: a walk that meets the boundary is outside
};

static inline bool lcs_is_mesh(const lcs_field *f) { return f->kind == LCS_TET || f->kind == LCS_TRI; }

// true when the cells form one component across their nv neighbours per cell (-1: none)
bool mesh_connected(const int *nbrs, long long nc, int nv);

// tetrahedral store (tet_store.cu): positions, tets, neighbours (built when null), inverse
// affine maps and the bin lists; exact seed location
cudaError_t tet_build_store(lcs_field *f, const float *xyz_host, const int *tets_host, const int *nbrs_host,
                            cudaStream_t s);
cudaError_t tet_locate_seeds(const lcs_field *f, const float *seeds, long long N, int *cells, cudaStream_t s);

// triangle store (tri_store.cu): positions, triangles, neighbours (built when null), inverse
// affine maps and the bin lists; exact seed location
cudaError_t tri_build_store(lcs_field *f, const float *xy_host, const int *tris_host, const int *nbrs_host,
                            cudaStream_t s);
cudaError_t tri_locate_seeds(const lcs_field *f, const float *seeds, long long N, int *cells, cudaStream_t s);

struct lcs_seeds {
    unsigned long long uid = 0;          // unique for the process lifetime (graph cache keys)
    int dim = 0;
    int n[3] = {1, 1, 1};
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    int periodic[3] = {0, 0, 0};
    long long N = 0;
    float *d_xyz = nullptr;            // [dim][N]
    int *d_cells = nullptr;            // [N] when made on a tet field
    unsigned long long field_uid = 0;  // the tet field the cells refer to
    double h[3] = {1, 1, 1};           // lattice step per axis
    double period[3] = {0, 0, 0};      // hi - lo on periodic axes
    long long aux_base_N = 0;          // > 0: auxiliary points of a lattice of that many seeds (lcs_seed_aux)
    double aux_delta[3] = {0, 0, 0};
};

struct lcs_flowmap {
    unsigned long long uid = 0;          // unique for the process lifetime (graph cache keys)
    lcs_ctx *ctx = nullptr;
    const lcs_seeds *seeds = nullptr;
    int dim = 0, njobs = 0;
    long long N = 0;
    float *d_xyz = nullptr;            // [njobs][dim][N]
    unsigned char *d_status = nullptr; // [njobs][N]
    float *d_texit = nullptr;          // [njobs][N]
    int *d_steps = nullptr;            // [njobs][N] accepted adaptive steps (after an RK45 advect)
    float *d_grad = nullptr;           // [njobs][N][dim][dim] variational grad F (opts.variational)
    bool grad_valid = false;
    std::vector<double> T;             // per job
    double *d_absT = nullptr;          // [njobs] |T|, written by the schedule kernel
};

// ------------------------------------------------------------ rectilinear

struct RectParams {
    int n[3];
    int periodic[3];
    float origin[3];
    float inv_h[3];
    float hi_node[3];     // origin + (n-1) h  (clamp limit, non-periodic axes)
    float left_lo[3];     // origin - h        (LEFT below)
    float left_hi[3];     // origin + n h      (LEFT above)
    float L[3];           // n h               (period, periodic axes)
    long long sy, sz;     // node strides
    long long fstride;    // nodes per padded frame (in stored vectors)
};

// stage schedule entry: frame k and the FP32 weight alpha of frame k+1
struct SchedEntry {
    int k;
    float a;
};

// Batch of integrations passed by value to the schedule kernel (no host copy).
#define LCS_MAX_JOBS 512
struct JobTable {
    int njobs;
    int nsteps_max;
    double t0[LCS_MAX_JOBS];
    double h[LCS_MAX_JOBS];     // signed step
    double T[LCS_MAX_JOBS];     // requested horizon
    int nsteps[LCS_MAX_JOBS];
    int order[LCS_MAX_JOBS];    // jobs by decreasing step count (work-queue order)
    int nsnap = 0;              // snapshots per job (lcs_advect_opts.nsnap)
    int snap_n[LCS_MAX_SNAP];   // their step counts |snap_T| / dt (capped per job at nsteps)
    double snap_T[LCS_MAX_SNAP];// their horizon magnitudes
};

// per-job values the schedule kernel leaves in device scratch for the advection kernels
struct JobDev {
    int *nsteps;     // [njobs]
    float *h;        // [njobs]
    float *t0;       // [njobs]
    float *tend;     // [njobs]
    double *absT;    // [njobs] (the flow map's copy, for the FTLE)
    int *order;      // [njobs] JobTable::order on the device, or null
    double *t0d;     // [njobs] FP64 start times, or null
    double *Td;      // [njobs] FP64 horizons, or null
    int *snap_n = nullptr;  // [LCS_MAX_SNAP] snapshot step counts, or null
    float *snap_te = nullptr;  // [njobs][nsnap] end time t0 + T of each snapshot (a tracer still OK there)
};

struct Rk4Launch {
    lcs_ctx *ctx;
    const lcs_field *field;
    const float *seeds;       // [dim][N]
    long long N;
    int njobs;
    int nsteps_max;
    const SchedEntry *sched;  // [njobs][nsteps_max][3]
    const int *job_nsteps;    // [njobs]
    const float *job_h;       // [njobs] signed step
    const float *job_t0;      // [njobs]
    const float *job_tend;    // [njobs]
    float *out_xyz;           // [njobs][dim][N]
    unsigned char *out_status;
    float *out_texit;
    int block_threads;
    int variant;              // 1 gather, 2 shared-memory ring (2D), 3 re-bundled episodes (3D),
                              // 4 persistent shared-memory ring over a job/tile work queue (2D),
                              // 5 per-stage time slices (2D)
    int episode_steps;        // variant 3: steps between re-bundling (0 = default)
    const int *host_nsteps;   // [njobs] host copy of the step counts
    void *work;               // variant 3 working memory (rk4_sorted_scratch_bytes), or null
    int tracers_per_thread;   // ring kernels: 1 or 2
    unsigned *queue;          // variant 4: work-queue counter in device scratch, or null
    const int *job_order;     // variant 4: [njobs] jobs by decreasing step count (device), or null
    float *out_grad = nullptr;  // variational grad F [njobs][N][dim][dim], or null
    int nsnap = 0;            // snapshots per job: slot njobs + job * nsnap + s after min(snap_n[s], nsteps)
    const int *snap_n = nullptr;  // [nsnap] on the device (written by the schedule kernel)
    const int *host_snap_n = nullptr;  // [nsnap] the same on the host
    const float *snap_te = nullptr;    // [njobs][nsnap] snapshot end times (device)
    unsigned long long wait_ns = LCS_WAIT_LIMIT_NS;  // ring kernels: bound on a wait for a frame copy
};

// smallest seed count for which lcs_advect picks the re-bundled kernel by default
#define LCS_SORTED_MIN_SEEDS 262144
// default RK4 steps per re-bundled episode
#define LCS_EPISODE_STEPS 40

size_t rk4_sorted_scratch_bytes(long long N, const lcs_field *f, int episode_steps, bool variational);
// variant 5 (2D time slices): their bytes for these jobs, and the most lcs_advect reserves for them
size_t rk4_slice2d_bytes(const lcs_field *f, int njobs, const int *host_nsteps);
#define LCS_SLICE2D_MAX_BYTES (16ULL << 30)
#define LCS_SLICE2D_DEFAULT_BYTES (2ULL << 30)

RectParams make_rect_params(const lcs_field *f);

cudaError_t launch_rk4_schedule(const double *d_times, int nframes, int time_periodic, double period,
                                const JobTable &J, JobDev D, SchedEntry *d_sched, cudaStream_t s);

// returns the variant actually used (1 or 2), or -1 on a launch error
int launch_rk4_rect(lcs_ctx *ctx, const Rk4Launch &L, cudaStream_t s);

// ------------------------------------------------- tets and adaptive stepping

cudaError_t launch_rk4_tet(lcs_ctx *ctx, const Rk4Launch &L, const int *cells0, int walk_limit, cudaStream_t s);

// ------------------------------------------------------ grad F / C / FTLE

struct CgLaunch {
    int dim;
    int n[3];
    int periodic[3];
    double h[3];
    double period[3];
    double h2[3], rh2[3];        // 2 h and RN(1 / (2 h)), filled by launch_cg_ftle
    long long N;
    int job0, njobs;
    const float *xyz;            // flow map base [njobs_total][dim][N]
    const unsigned char *status; // [njobs_total][N]
    const float *texit = nullptr; // [njobs_total][N] (early evaluation only)
    const float *x0aux = nullptr; // auxiliary points: their FP32 starting points [dim][npts]; null: lattice
    const float *grad = nullptr;  // variational grad F [njobs_total][N][dim][dim]; null: differences
    long long npts = 0;          // auxiliary points per job (N * 2 dim)
    const double *absT;          // [njobs_total] |T|
    double *C;                   // [njobs][N][np] or null
    double *lam;                 // [njobs][N] or null
    float *ftle;                 // [njobs][N] or null
    double *eigval;              // [njobs][N][dim] or null (lcs_cg_eigen)
    double *eigvec;              // [njobs][N][dim][dim] or null
};

cudaError_t launch_cg_ftle(const CgLaunch &L, cudaStream_t s);

// early Cauchy-Green evaluation (early_cg.cu): phase 0 scans the seeds of slot `job` (writes
// t_eval and lists the early ones), phase 1 re-integrates the listed stencils and writes their FTLE
struct EarlyLaunch {
    CgLaunch cg;                 // lattice, flow map (positions, status, exit times), outputs unused
    int phase;
    int job, ns;                 // slot and its RK4 step count
    double t0, adt;              // the job's start time and |dt|
    float absT;                  // |T| (the regular seeds' horizon)
    unsigned *count;             // listed seeds (device)
    int2 *list;                  // [N] (seed, steps m) of the listed seeds
    long long nlisted;           // phase 1: the count, read back
    float *pos;                  // phase 1: [nlisted][2 dim + 1][dim] re-integrated stencil positions
    float *t_eval, *ftle;        // [N] outputs (device)
    const lcs_field *field;
    const float *seeds;          // [dim][N]
    int nsteps_max;
    const SchedEntry *sched;     // [njobs][nsteps_max][3]
    const float *job_h;          // [njobs]
    const int *cells0 = nullptr; // mesh fields: [N] start cells of the seeds (-1 outside)
    int walk_limit = 0;          // mesh fields: walk steps per location
};

cudaError_t launch_early_cg(const EarlyLaunch &E, cudaStream_t s);

// grow the context's reusable device scratch (dropping captured graphs that point into it)
lcs_status lcs_scratch_reserve(lcs_ctx *ctx, size_t bytes);

// set the context's last error (printf-style) and return st (lcs_api.cu)
lcs_status lcs_fail(lcs_ctx *ctx, lcs_status st, const char *fmt, ...);

#define LCS_CUDA_TRY(ctx, call)                                                                        \
    do {                                                                                               \
        cudaError_t e__ = (call);                                                                      \
        if (e__ != cudaSuccess)                                                                        \
            return lcs_fail((ctx), e__ == cudaErrorMemoryAllocation ? LCS_ENOMEM : LCS_ECUDA, "%s: %s", \
                            #call, cudaGetErrorString(e__));                                           \
    } while (0)

// ------------------------------------------------------------------ misc

cudaError_t launch_seed_aux(int dim, const float *lattice, long long N, const double *delta, float *out,
                            cudaStream_t s);
cudaError_t launch_seed_grid(int dim, const int n[3], const double lo[3], const double hi[3],
                             const int periodic[3], long long N, float *out, cudaStream_t s);

cudaError_t launch_convert_rect(const float *src, int nframes, int nslabs, long long nodes, int dim, int vec,
                                int storage, size_t slab_stride, void *dst, int *nonfinite, cudaStream_t s);

// ---------------------------------------------------------- device helpers

#ifdef __CUDACC__

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// 1D bulk copy global -> shared, completion counted on bar (16-byte aligned, size % 16 == 0)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// One RK4 position update with its rounding error carried (compensated summation, Kahan 1965):
// x + c is the tracer's coordinate, c the part below the last bit of x.  The increment
// h/6 (k1 + 2 k2 + 2 k3 + k4), plus c, is added to x, and c becomes what that sum lost: d - (s - x)
// is the exact rounding error of s = x + d whenever |x| >= |d| (Dekker's Fast2Sum), which holds
// except for a coordinate within one step of zero, where the error left is below ulp(d).  So the
// rounding of each step's sum no longer accumulates in the position: on the double gyre at
// 2048 x 1024 seeds it was the largest error of the FP32 FTLE (median 1.7e-5 over |T| = 2, 2.0e-6
// with the rounding carried).  Stage points use x alone, an error of |c| |du/dx| h per step, far
// below what the carried rounding removes.
__device__ __forceinline__ void rk4_advance(float &x, float &c, float h6, float k1, float k2, float k3, float k4)
{
    const float d = fmaf(h6, (k1 + k4) + 2.0f * (k2 + k3), c);
    const float s = x + d;
    c = d - (s - x);
    x = s;
}

// x + c += d with the error of x + d recovered by Knuth's TwoSum (exact for any operands): the
// periodic shifts of a wrapped coordinate, where |d| = L may exceed |x|
__device__ __forceinline__ void add_carried(float &x, float &c, float d)
{
    const float s = x + d;
    const float bp = s - x;
    c += (x - (s - bp)) + (d - bp);
    x = s;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// non-blocking test of the phase with the given parity
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, unsigned parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait for the phase with the given parity; false when limit_ns ran out.  try_wait may
// itself suspend the thread for a system-dependent time (microseconds) before it answers, so a
// limit shorter than the default polls with the non-blocking test_wait instead, and a limit under
// a microsecond (below what %globaltimer resolves) is a single test.
__device__ __forceinline__ bool mbar_wait_limit(uint64_t *bar, unsigned parity, uint64_t limit_ns)
{
    if (limit_ns < 1000) return mbar_test_wait(bar, parity);
    if (limit_ns < LCS_WAIT_LIMIT_NS) {
        if (mbar_test_wait(bar, parity)) return true;
        const uint64_t t0 = global_ns();
        while (!mbar_test_wait(bar, parity))
            if (global_ns() - t0 > limit_ns) return false;
        return true;
    }
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity)
{
    return mbar_wait_limit(bar, parity, LCS_WAIT_LIMIT_NS);
}

#endif  // __CUDACC__
