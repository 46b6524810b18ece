// noalloc.cu -- lcs_advect_rk4_noalloc: fixed-step RK4 advection that allocates
// no device memory.
//
// lcs_advect keeps its per-job values and its stage schedule (frame bracket of
// every RK4 stage) in scratch memory that the context allocates and grows on
// demand.  This entry point runs the same schedule and advection kernels with
// that working memory taken from a fixed array in the library image instead, so
// that callers which must not allocate device memory can still integrate.
#include "lcs_internal.cuh"

#include <math.h>

#include <mutex>

// Working memory of lcs_advect_rk4_noalloc.  Every GPU that loads the library
// holds this 1 MiB array until the process exits.
#define LCS_NOALLOC_SCRATCH_BYTES (1u << 20)
#define LCS_NOALLOC_HEADER 256u                // per-job values: offsets 0, 16, 32, 48 (4 bytes), 64 (8 bytes)
#define LCS_NOALLOC_MAX_DEVICES 64
static __device__ __align__(256) unsigned char g_noalloc_scratch[LCS_NOALLOC_SCRATCH_BYTES];
// the step limit published in lcs.h is exactly what the array holds after the header: three
// schedule entries (one per distinct RK4 stage time) per step
static_assert(LCS_NOALLOC_MAX_STEPS ==
                  (LCS_NOALLOC_SCRATCH_BYTES - LCS_NOALLOC_HEADER) / (3 * sizeof(SchedEntry)),
              "LCS_NOALLOC_MAX_STEPS must be the step count the scratch array holds");
static_assert(64 + sizeof(double) <= LCS_NOALLOC_HEADER, "the per-job values must fit the header");
static_assert(LCS_NOALLOC_HEADER % 16 == 0, "schedule entries must start 16-byte aligned");

#define NA_STR2(x) #x
#define NA_STR(x) NA_STR2(x)

// device address of g_noalloc_scratch per device, looked up once per device
static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[LCS_NOALLOC_MAX_DEVICES];

static lcs_status na_fail(lcs_ctx *ctx, lcs_status st, const char *msg)
{
    if (ctx) ctx->err = msg;
    return st;
}

extern "C" lcs_status lcs_advect_rk4_noalloc(lcs_ctx *ctx, const lcs_field *f, const float *seeds, long long n,
                                             double t0, double T, double dt, float *xyz, unsigned char *status,
                                             float *t_exit)
{
    if (!ctx) return LCS_EINVAL;
    if (!f || !seeds || !xyz || !status || !t_exit)
        return na_fail(ctx, LCS_EINVAL, "lcs_advect_rk4_noalloc: null argument");
    if (f->kind != LCS_RECTILINEAR)
        return na_fail(ctx, LCS_EUNSUPPORTED, "lcs_advect_rk4_noalloc: rectilinear fields only");
    if (n < 0) return na_fail(ctx, LCS_EINVAL, "lcs_advect_rk4_noalloc: negative seed count");
    double adt = fabs(dt);
    if (!(adt > 0.0) || !isfinite(adt) || !isfinite(t0) || !isfinite(T))
        return na_fail(ctx, LCS_EINVAL, "lcs_advect_rk4_noalloc: t0, T and dt must be finite, dt != 0");
    double r = fabs(T) / adt;
    long long ns = (long long)floor(r + 0.5);
    if (fabs(r - (double)ns) > 1e-9 * (r > 1.0 ? r : 1.0))
        return na_fail(ctx, LCS_EINVAL, "lcs_advect_rk4_noalloc: |T|/|dt| is not an integer");
    if (ns > LCS_NOALLOC_MAX_STEPS)
        return na_fail(ctx, LCS_EINVAL,
                       "lcs_advect_rk4_noalloc: |T|/|dt| exceeds LCS_NOALLOC_MAX_STEPS (" NA_STR(LCS_NOALLOC_MAX_STEPS)
                       "), the most RK4 steps its fixed " NA_STR(LCS_NOALLOC_SCRATCH_BYTES) "-byte scratch holds; "
                       "use lcs_advect");
    if (ctx->device < 0 || ctx->device >= LCS_NOALLOC_MAX_DEVICES)
        return na_fail(ctx, LCS_EINVAL, "lcs_advect_rk4_noalloc: device index too large");
    if (cudaSetDevice(ctx->device) != cudaSuccess)
        return na_fail(ctx, LCS_ECUDA, "lcs_advect_rk4_noalloc: cudaSetDevice failed");
    if (f->dim != 2 && f->dim != 3) return na_fail(ctx, LCS_EINVAL, "lcs_advect_rk4_noalloc: field dim must be 2 or 3");
    // the kernels dereference these pointers: refuse host memory and other devices' memory before any
    // launch (the sizes behind them cannot be checked here; the caller guarantees them)
    const void *bufs[4] = {seeds, xyz, status, t_exit};
    for (const void *b : bufs) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, b) != cudaSuccess) {
            cudaGetLastError();
            return na_fail(ctx, LCS_EINVAL, "lcs_advect_rk4_noalloc: a buffer is not CUDA memory");
        }
        if ((a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) || a.device != ctx->device)
            return na_fail(ctx, LCS_EINVAL, "lcs_advect_rk4_noalloc: every buffer must be device memory on the "
                                            "context's device");
    }
    void *base;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_addr[ctx->device]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                ctx->err = std::string("lcs_advect_rk4_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
                return LCS_ECUDA;
            }
            g_noalloc_addr[ctx->device] = p;
        }
        base = g_noalloc_addr[ctx->device];
    }
    // one job; the table travels as a kernel parameter (no host or device buffer)
    JobTable J;
    J.njobs = 1;
    J.nsteps_max = (int)ns;
    J.t0[0] = t0;
    J.T[0] = T;
    J.h[0] = T < 0.0 ? -adt : adt;
    J.nsteps[0] = (int)ns;
    J.order[0] = 0;
    char *p = (char *)base;
    JobDev D;
    D.nsteps = (int *)(p + 0);
    D.h = (float *)(p + 16);
    D.t0 = (float *)(p + 32);
    D.tend = (float *)(p + 48);
    D.absT = (double *)(p + 64);
    D.order = nullptr;
    D.t0d = nullptr;
    D.Td = nullptr;
    SchedEntry *sched = (SchedEntry *)(p + LCS_NOALLOC_HEADER);
    // every schedule entry and per-job value the advection reads is written by the schedule kernel
    // first, so nothing in the array needs clearing between calls
    cudaError_t e = launch_rk4_schedule(f->d_times, f->nframes, f->time_periodic, f->period, J, D, sched, ctx->stream);
    if (e != cudaSuccess) return na_fail(ctx, LCS_ECUDA, "lcs_advect_rk4_noalloc: schedule launch failed");
    if (n == 0) return LCS_OK;
    Rk4Launch L;
    L.ctx = ctx;
    L.field = f;
    L.seeds = seeds;
    L.N = n;
    L.njobs = 1;
    L.nsteps_max = (int)ns;
    L.sched = sched;
    L.job_nsteps = D.nsteps;
    L.job_h = D.h;
    L.job_t0 = D.t0;
    L.job_tend = D.tend;
    L.out_xyz = xyz;
    L.out_status = status;
    L.out_texit = t_exit;
    L.block_threads = 0;
    L.variant = f->dim == 3 ? 1 : 0;   // the re-bundled 3D kernel needs allocated working memory
    L.episode_steps = 0;
    L.host_nsteps = J.nsteps;
    L.work = nullptr;
    L.tracers_per_thread = 1;
    L.queue = nullptr;
    L.job_order = nullptr;
    if (launch_rk4_rect(ctx, L, ctx->stream) < 0)
        return na_fail(ctx, LCS_ECUDA, "lcs_advect_rk4_noalloc: advection launch failed");
    return LCS_OK;
}
