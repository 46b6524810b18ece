// lcs_api.cu -- the C ABI of liblcs (declared in include/lcs.h): handles,
// argument checks, device memory, and the order of launches for each call.
//
// Paper passages per call are given in lcs.h.  This file holds only host logic
// plus the two bulk conversion kernels (frame storage, seed lattice).
#include "lcs_internal.cuh"
#include "dp45_args.cuh"
#include "mlp_internal.cuh"

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>

// ------------------------------------------------------------------- errors

lcs_status lcs_fail(lcs_ctx *ctx, lcs_status st, const char *fmt, ...)
{
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return st;
}

#define CUDA_TRY(ctx, call)                                                                        \
    do {                                                                                           \
        cudaError_t e__ = (call);                                                                  \
        if (e__ != cudaSuccess)                                                                    \
            return lcs_fail((ctx), e__ == cudaErrorMemoryAllocation ? LCS_ENOMEM : LCS_ECUDA, "%s: %s", \
                        #call, cudaGetErrorString(e__));                                           \
    } while (0)

// ------------------------------------------------------------------ context

unsigned long long lcs_next_uid()
{
    static std::atomic<unsigned long long> next{1};
    return next.fetch_add(1);
}

static void graph_cache_clear(lcs_ctx *ctx)
{
    for (auto &g : ctx->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
    }
    ctx->graphs.clear();
}

extern "C" lcs_status lcs_create(lcs_ctx **out, int device, void *stream)
{
    if (!out) return LCS_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return LCS_EINVAL;
    lcs_ctx *c = new (std::nothrow) lcs_ctx();
    if (!c) return LCS_ENOMEM;
    c->device = device;
    c->stream = (cudaStream_t)stream;
    int sms = 0, optin = 0;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess ||
        cudaMalloc(&c->d_errword, sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(c->d_errword, 0, sizeof(unsigned)) != cudaSuccess) {
        if (c->d_errword) cudaFree(c->d_errword);
        delete c;
        return LCS_ECUDA;
    }
    c->num_sms = sms;
    c->smem_optin = (size_t)optin - 1024;  // room for the kernels' static shared state
    *out = c;
    return LCS_OK;
}

static void tm_release_all(lcs_ctx *ctx)
{
    for (int p = 0; p < LCS_NPHASES; ++p) {
        for (auto &pr : ctx->ev_done[p]) {
            ctx->ev_pool.push_back(pr.first);
            ctx->ev_pool.push_back(pr.second);
        }
        ctx->ev_done[p].clear();
        if (ctx->ev_open[p]) ctx->ev_pool.push_back(ctx->ev_open[p]);
        ctx->ev_open[p] = nullptr;
    }
}

extern "C" void lcs_destroy(lcs_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->d_errword) cudaFree(ctx->d_errword);
    if (ctx->d_scratch) cudaFree(ctx->d_scratch);
    if (ctx->d_stage) cudaFree(ctx->d_stage);
    if (ctx->d_flag) cudaFree(ctx->d_flag);
    tm_release_all(ctx);
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    graph_cache_clear(ctx);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    delete ctx;
}

static cudaEvent_t tm_event(lcs_ctx *ctx)
{
    if (!ctx->ev_pool.empty()) {
        cudaEvent_t e = ctx->ev_pool.back();
        ctx->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

void lcs_tm_begin(lcs_ctx *ctx, int phase, cudaStream_t s)
{
    if (!ctx || !ctx->timing || phase < 0 || phase >= LCS_NPHASES || ctx->ev_open[phase]) return;
    cudaEvent_t e = tm_event(ctx);
    if (e && cudaEventRecord(e, s) == cudaSuccess) ctx->ev_open[phase] = e;
}

void lcs_tm_end(lcs_ctx *ctx, int phase, cudaStream_t s)
{
    if (!ctx || !ctx->timing || phase < 0 || phase >= LCS_NPHASES || !ctx->ev_open[phase]) return;
    cudaEvent_t e = tm_event(ctx);
    if (e && cudaEventRecord(e, s) == cudaSuccess) ctx->ev_done[phase].push_back({ctx->ev_open[phase], e});
    ctx->ev_open[phase] = nullptr;
}

extern "C" lcs_status lcs_timing_enable(lcs_ctx *ctx, int on)
{
    if (!ctx) return LCS_EINVAL;
    ctx->timing = on != 0;
    if (!ctx->timing) tm_release_all(ctx);
    return LCS_OK;
}

extern "C" lcs_status lcs_timing_read(lcs_ctx *ctx, int phase, double *ms, long long *launches)
{
    if (!ctx) return LCS_EINVAL;
    if (phase < 0 || phase >= LCS_NPHASES) return lcs_fail(ctx, LCS_EINVAL, "lcs_timing_read: phase %d", phase);
    CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    double tot = 0.0;
    long long n = 0;
    for (auto &pr : ctx->ev_done[phase]) {
        CUDA_TRY(ctx, cudaEventSynchronize(pr.second));
        float t = 0.0f;
        CUDA_TRY(ctx, cudaEventElapsedTime(&t, pr.first, pr.second));
        tot += t;
        ++n;
        ctx->ev_pool.push_back(pr.first);
        ctx->ev_pool.push_back(pr.second);
    }
    ctx->ev_done[phase].clear();
    if (ms) *ms = tot;
    if (launches) *launches = n;
    return LCS_OK;
}

extern "C" const char *lcs_last_error(const lcs_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : "null context";
}

extern "C" int lcs_context_device(const lcs_ctx *ctx) { return ctx ? ctx->device : -1; }

extern "C" int lcs_field_dim(const lcs_field *f) { return f ? f->dim : 0; }

extern "C" lcs_status lcs_set_stream(lcs_ctx *ctx, void *stream)
{
    if (!ctx) return LCS_EINVAL;
    ctx->stream = (cudaStream_t)stream;
    return LCS_OK;
}

extern "C" lcs_status lcs_synchronize(lcs_ctx *ctx)
{
    if (!ctx) return LCS_EINVAL;
    CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    unsigned w = 0;
    CUDA_TRY(ctx, cudaMemcpy(&w, ctx->d_errword, sizeof w, cudaMemcpyDeviceToHost));
    if (w) {
        CUDA_TRY(ctx, cudaMemset(ctx->d_errword, 0, sizeof w));
        if (w & LCS_ERRBIT_TIMEOUT) return lcs_fail(ctx, LCS_ETIMEOUT, "a device-side wait gave up");
        if (w & LCS_ERRBIT_WALK) return lcs_fail(ctx, LCS_EWALK, "a tet walk exceeded walk_limit");
        if (w & LCS_ERRBIT_MAXSTEPS) return lcs_fail(ctx, LCS_EMAXSTEPS, "an adaptive integration hit max_steps");
    }
    return LCS_OK;
}

// grow the context's reusable device scratch to at least `bytes`
lcs_status lcs_scratch_reserve(lcs_ctx *ctx, size_t bytes)
{
    if (bytes <= ctx->scratch_bytes) return LCS_OK;
    if (ctx->d_scratch) {
        CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        graph_cache_clear(ctx);  // captured graphs point into the old scratch
        cudaFree(ctx->d_scratch);
        ctx->d_scratch = nullptr;
        ctx->scratch_bytes = 0;
    }
    size_t b = std::max(bytes, (size_t)1 << 20);
    CUDA_TRY(ctx, cudaMalloc(&ctx->d_scratch, b));
    ctx->scratch_bytes = b;
    return LCS_OK;
}

// ----------------------------------------------------------- frame storage

// FP32 [nframes][nodes][dim] -> [nframes][frame_stride bytes] of `vec` stored components
template <typename T>
__device__ __forceinline__ T to_store(float v);
template <>
__device__ __forceinline__ float to_store<float>(float v) { return v; }
template <>
__device__ __forceinline__ __half to_store<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// 2D rectilinear: slab f = frame f, node v = (u, v).  Triangles: slab k = interval pair
// (k, k+1), node v = (u_k, v_k, u_{k+1}, v_{k+1}).  3D: slab k = interval pair, node v =
// (u_k, 0, u_{k+1}, 0) so that one load brings both frames of a node (a single frame is
// paired with itself).
// Every frame value is read by at least one slab (frame f by slab f, the last one also as the
// k + 1 side of the last slab), so the pass also flags any non-finite value in *nonfinite.
template <typename T>
__global__ void convert_rect_kernel(const float *__restrict__ src, int nframes, int nslabs, long long nodes, int dim,
                                    int vec, size_t slab_stride, char *__restrict__ dst, int *__restrict__ nonfinite)
{
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)nslabs * nodes) return;
    long long f = idx / nodes, v = idx % nodes;
    T *o = reinterpret_cast<T *>(dst + (size_t)f * slab_stride) + v * vec;
    bool ok = true;
    if (dim == 2 && vec == 2) {
        const float *s = src + idx * 2;
        ok = isfinite(s[0]) && isfinite(s[1]);
        o[0] = to_store<T>(s[0]);
        o[1] = to_store<T>(s[1]);
    } else if (dim == 2) {  // triangle meshes: (u_k, v_k, u_{k+1}, v_{k+1}) per node
        long long f1 = f + 1 < nframes ? f + 1 : f;
        const float *a = src + (f * nodes + v) * 2, *b = src + (f1 * nodes + v) * 2;
        ok = isfinite(a[0]) && isfinite(a[1]) && isfinite(b[0]) && isfinite(b[1]);
        o[0] = to_store<T>(a[0]);
        o[1] = to_store<T>(a[1]);
        o[2] = to_store<T>(b[0]);
        o[3] = to_store<T>(b[1]);
    } else {
        long long f1 = f + 1 < nframes ? f + 1 : f;
        const float *a = src + (f * nodes + v) * 3, *b = src + (f1 * nodes + v) * 3;
        for (int c = 0; c < 3; ++c) {
            ok = ok && isfinite(a[c]) && isfinite(b[c]);
            o[c] = to_store<T>(a[c]);
            o[4 + c] = to_store<T>(b[c]);
        }
        o[3] = to_store<T>(0.0f);
        o[7] = to_store<T>(0.0f);
    }
    if (!ok) atomicOr(nonfinite, 1);
}

cudaError_t launch_convert_rect(const float *src, int nframes, int nslabs, long long nodes, int dim, int vec,
                                int storage, size_t slab_stride, void *dst, int *nonfinite, cudaStream_t s)
{
    long long total = (long long)nslabs * nodes;
    if (total == 0) return cudaSuccess;
    int bt = 256;
    unsigned grid = (unsigned)((total + bt - 1) / bt);
    if (storage == LCS_F32)
        convert_rect_kernel<float>
            <<<grid, bt, 0, s>>>(src, nframes, nslabs, nodes, dim, vec, slab_stride, (char *)dst, nonfinite);
    else if (storage == LCS_F16)
        convert_rect_kernel<__half>
            <<<grid, bt, 0, s>>>(src, nframes, nslabs, nodes, dim, vec, slab_stride, (char *)dst, nonfinite);
    else
        convert_rect_kernel<__nv_bfloat16>
            <<<grid, bt, 0, s>>>(src, nframes, nslabs, nodes, dim, vec, slab_stride, (char *)dst, nonfinite);
    return cudaGetLastError();
}

static lcs_status upload_frames(lcs_ctx *ctx, lcs_field *f, const float *frames, int on_device)
{
    const size_t n_in = (size_t)f->nframes * f->nodes * f->dim;
    const float *src = frames;
    if (!ctx->d_flag) CUDA_TRY(ctx, cudaMalloc((void **)&ctx->d_flag, sizeof(int)));
    if (!on_device) {
        // host frames go through the context's staging buffer, grown when a larger upload comes
        // (every upload ends with the stream synchronised, so the buffer is free between calls)
        const size_t bytes = n_in * sizeof(float);
        if (bytes > ctx->stage_bytes) {
            if (ctx->d_stage) cudaFree(ctx->d_stage);
            ctx->d_stage = nullptr;
            ctx->stage_bytes = 0;
            cudaError_t e = cudaMalloc((void **)&ctx->d_stage, bytes);
            if (e != cudaSuccess)
                return lcs_fail(ctx, e == cudaErrorMemoryAllocation ? LCS_ENOMEM : LCS_ECUDA, "frame staging: %s",
                                cudaGetErrorString(e));
            ctx->stage_bytes = bytes;
        }
        cudaError_t e = cudaMemcpyAsync(ctx->d_stage, frames, bytes, cudaMemcpyHostToDevice, ctx->stream);
        if (e != cudaSuccess) return lcs_fail(ctx, LCS_ECUDA, "frame upload: %s", cudaGetErrorString(e));
        src = ctx->d_stage;
    }
    // velocity data must be finite (a NaN would spread through every tracer that touches it): the
    // conversion flags any non-finite value it reads
    int hflag = 0;
    cudaError_t e = cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream);
    if (e == cudaSuccess)
        e = launch_convert_rect(src, f->nframes, f->nslabs, f->nodes, f->dim, f->vec, f->storage, f->frame_stride,
                                f->d_frames, ctx->d_flag, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return lcs_fail(ctx, LCS_ECUDA, "frame conversion: %s", cudaGetErrorString(e));
    if (hflag) return lcs_fail(ctx, LCS_EINVAL, "frames hold a non-finite velocity value");
    return LCS_OK;
}

// Tetrahedral (Sec. 3.1) or triangle (2D) mesh: frames as interval pairs per node, plus the
// mesh store.
static lcs_status load_tet_field(lcs_ctx *ctx, const lcs_field_desc *d, const float *frames, int frames_on_device,
                                 lcs_field **out)
{
    const bool tri = d->kind == LCS_TRI;
    const int dim = tri ? 2 : 3, nv = dim + 1;
    if (d->dim != dim)
        return lcs_fail(ctx, LCS_EINVAL, tri ? "lcs_load_field: triangle meshes are 2D" : "lcs_load_field: tet meshes are 3D");
    if (d->storage < LCS_F32 || d->storage > LCS_BF16) return lcs_fail(ctx, LCS_EINVAL, "lcs_load_field: storage");
    if (d->nnodes < nv || d->ncells < 1 || !d->node_xyz || !d->tets)
        return lcs_fail(ctx, LCS_EINVAL, "lcs_load_field: a mesh needs nnodes >= %d, ncells >= 1, node_xyz, cells", nv);
    if (d->nnodes >= (1LL << 31) || d->ncells >= (1LL << 31))
        return lcs_fail(ctx, LCS_EINVAL, "lcs_load_field: more than 2^31 nodes or tets");
    if (d->nframes < 1 || !d->frame_times) return lcs_fail(ctx, LCS_EINVAL, "lcs_load_field: need >= 1 frame");
    for (int k = 1; k < d->nframes; ++k)
        if (!(d->frame_times[k] > d->frame_times[k - 1]))
            return lcs_fail(ctx, LCS_EINVAL, "lcs_load_field: frame_times must increase");
    if (d->time_periodic && !(d->period > 0.0)) return lcs_fail(ctx, LCS_EINVAL, "lcs_load_field: period must be > 0");
    for (long long q = 0; q < nv * d->ncells; ++q) {
        if (d->tets[q] < 0 || d->tets[q] >= d->nnodes)
            return lcs_fail(ctx, LCS_EINVAL, "lcs_load_field: cell %lld names node %d", q / nv, d->tets[q]);
        if (d->nbrs && (d->nbrs[q] < -1 || d->nbrs[q] >= d->ncells))
            return lcs_fail(ctx, LCS_EINVAL, "lcs_load_field: cell %lld has neighbour %d", q / nv, d->nbrs[q]);
    }
    for (long long q = 0; q < (long long)dim * d->nnodes; ++q)
        if (!isfinite(d->node_xyz[q])) return lcs_fail(ctx, LCS_EINVAL, "lcs_load_field: non-finite node coordinate");
    // a cell of zero area or volume has no inverse map (its barycentric coordinates would not exist)
    for (long long c = 0; c < d->ncells; ++c) {
        const int *v = d->tets + (long long)nv * c;
        const float *a = d->node_xyz + (long long)dim * v[0];
        double e[3][3];
        for (int r = 0; r < dim; ++r)
            for (int k = 0; k < dim; ++k) e[r][k] = (double)d->node_xyz[(long long)dim * v[r + 1] + k] - a[k];
        const double det = tri ? e[0][0] * e[1][1] - e[0][1] * e[1][0]
                               : e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
                                     e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                                     e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
        if (!(det != 0.0)) return lcs_fail(ctx, LCS_EINVAL, "lcs_load_field: cell %lld is degenerate", c);
    }
    CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    lcs_field *f = new (std::nothrow) lcs_field();
    if (!f) return lcs_fail(ctx, LCS_ENOMEM, "host allocation");
    f->ctx = ctx;
    f->uid = lcs_next_uid();
    f->dim = dim;
    f->kind = d->kind;
    f->storage = d->storage;
    f->nframes = d->nframes;
    f->times.assign(d->frame_times, d->frame_times + d->nframes);
    f->time_periodic = d->time_periodic != 0;
    f->period = d->period;
    f->nodes = d->nnodes;
    f->ncells = d->ncells;
    f->vec = tri ? 4 : 8;
    f->nslabs = f->nframes > 1 ? f->nframes - 1 : 1;
    f->elem_bytes = d->storage == LCS_F32 ? 4 : 2;
    f->frame_bytes = (size_t)f->nodes * f->vec * f->elem_bytes;
    f->frame_stride = (f->frame_bytes + 255) & ~(size_t)255;
    lcs_status st = LCS_OK;
    cudaError_t e = cudaMalloc(&f->d_frames, f->frame_stride * f->nslabs);
    if (e == cudaSuccess) e = cudaMalloc(&f->d_times, sizeof(double) * f->nframes);
    if (e == cudaSuccess)
        e = cudaMemcpy(f->d_times, f->times.data(), sizeof(double) * f->nframes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = tri ? tri_build_store(f, d->node_xyz, d->tets, d->nbrs, ctx->stream)
                : tet_build_store(f, d->node_xyz, d->tets, d->nbrs, ctx->stream);
    if (e != cudaSuccess)
        st = lcs_fail(ctx, e == cudaErrorMemoryAllocation ? LCS_ENOMEM : LCS_ECUDA, "lcs_load_field: %s",
                  cudaGetErrorString(e));
    else
        st = upload_frames(ctx, f, frames, frames_on_device);
    if (st != LCS_OK) {
        lcs_free_field(f);
        return st;
    }
    *out = f;
    return LCS_OK;
}

extern "C" lcs_status lcs_load_field(lcs_ctx *ctx, const lcs_field_desc *d, const float *frames,
                                     int frames_on_device, lcs_field **out)
{
    if (!ctx) return LCS_EINVAL;
    if (!d || !frames || !out) return lcs_fail(ctx, LCS_EINVAL, "lcs_load_field: null argument");
    *out = nullptr;
    if (d->kind == LCS_TET || d->kind == LCS_TRI) return load_tet_field(ctx, d, frames, frames_on_device, out);
    if (d->kind != LCS_RECTILINEAR) return lcs_fail(ctx, LCS_EINVAL, "lcs_load_field: unknown kind %d", d->kind);
    if (d->dim != 2 && d->dim != 3) return lcs_fail(ctx, LCS_EINVAL, "lcs_load_field: dim must be 2 or 3");
    if (d->storage < LCS_F32 || d->storage > LCS_BF16) return lcs_fail(ctx, LCS_EINVAL, "lcs_load_field: storage");
    if (d->nframes < 1 || !d->frame_times) return lcs_fail(ctx, LCS_EINVAL, "lcs_load_field: need >= 1 frame");
    for (int k = 1; k < d->nframes; ++k)
        if (!(d->frame_times[k] > d->frame_times[k - 1]))
            return lcs_fail(ctx, LCS_EINVAL, "lcs_load_field: frame_times must increase");
    if (d->time_periodic && !(d->period > 0.0)) return lcs_fail(ctx, LCS_EINVAL, "lcs_load_field: period must be > 0");
    long long nodes = 1;
    for (int a = 0; a < d->dim; ++a) {
        int minn = d->periodic[a] ? 3 : 2;
        if (d->n[a] < minn) return lcs_fail(ctx, LCS_EINVAL, "lcs_load_field: axis %d needs >= %d nodes", a, minn);
        if (!(d->spacing[a] > 0.0)) return lcs_fail(ctx, LCS_EINVAL, "lcs_load_field: spacing must be > 0");
        nodes *= d->n[a];
    }
    if (nodes >= (1LL << 31)) return lcs_fail(ctx, LCS_EINVAL, "lcs_load_field: more than 2^31 nodes per frame");
    CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    lcs_field *f = new (std::nothrow) lcs_field();
    if (!f) return lcs_fail(ctx, LCS_ENOMEM, "host allocation");
    f->ctx = ctx;
    f->uid = lcs_next_uid();
    f->dim = d->dim;
    f->kind = d->kind;
    f->storage = d->storage;
    for (int a = 0; a < 3; ++a) {
        f->n[a] = a < d->dim ? d->n[a] : 1;
        f->origin[a] = a < d->dim ? d->origin[a] : 0.0;
        f->spacing[a] = a < d->dim ? d->spacing[a] : 1.0;
        f->periodic[a] = a < d->dim ? (d->periodic[a] != 0) : 0;
    }
    f->nframes = d->nframes;
    f->times.assign(d->frame_times, d->frame_times + d->nframes);
    f->time_periodic = d->time_periodic != 0;
    f->period = d->period;
    f->nodes = nodes;
    f->vec = d->dim == 2 ? 2 : 8;
    f->nslabs = d->dim == 2 ? f->nframes : (f->nframes > 1 ? f->nframes - 1 : 1);
    f->elem_bytes = d->storage == LCS_F32 ? 4 : 2;
    f->frame_bytes = (size_t)nodes * f->vec * f->elem_bytes;
    f->frame_stride = (f->frame_bytes + 255) & ~(size_t)255;
    lcs_status st = LCS_OK;
    cudaError_t e = cudaMalloc(&f->d_frames, f->frame_stride * f->nslabs);
    if (e == cudaSuccess) e = cudaMemsetAsync(f->d_frames, 0, f->frame_stride * f->nslabs, ctx->stream);
    if (e == cudaSuccess) e = cudaMalloc(&f->d_times, sizeof(double) * f->nframes);
    if (e == cudaSuccess)
        e = cudaMemcpy(f->d_times, f->times.data(), sizeof(double) * f->nframes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        st = lcs_fail(ctx, e == cudaErrorMemoryAllocation ? LCS_ENOMEM : LCS_ECUDA, "lcs_load_field: %s",
                  cudaGetErrorString(e));
    } else {
        st = upload_frames(ctx, f, frames, frames_on_device);
    }
    if (st != LCS_OK) {
        lcs_free_field(f);
        return st;
    }
    *out = f;
    return LCS_OK;
}

extern "C" lcs_status lcs_update_frames(lcs_ctx *ctx, lcs_field *f, const float *frames, int frames_on_device)
{
    if (!ctx) return LCS_EINVAL;
    if (!f || !frames) return lcs_fail(ctx, LCS_EINVAL, "lcs_update_frames: null argument");
    CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    return upload_frames(ctx, f, frames, frames_on_device);
}

extern "C" void lcs_free_field(lcs_field *f)
{
    if (!f) return;
    if (f->ctx) cudaSetDevice(f->ctx->device);
    cudaFree(f->d_frames);
    cudaFree(f->d_times);
    cudaFree(f->d_xyz);
    cudaFree(f->d_tets);
    cudaFree(f->d_nbrs);
    cudaFree(f->d_tetmap);
    cudaFree(f->d_xy);
    cudaFree(f->d_trimap);
    cudaFree(f->d_triv0);
    cudaFree(f->d_bstart);
    cudaFree(f->d_blist);
    delete f;
}

// -------------------------------------------------------------- seed grid

// x_i = lo + i * step with step = (hi - lo) / (n - 1) (or / n on periodic axes);
// FP64 round-to-nearest, no fused operations, then rounded to FP32
__global__ void seed_grid_kernel(int dim, int nx, int ny, double lo0, double lo1, double lo2, double hi0,
                                 double hi1, double hi2, int n0, int n1, int n2, int p0, int p1, int p2,
                                 long long N, float *__restrict__ out)
{
    long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= N) return;
    long long i = id % nx, j = (id / nx) % ny, k = id / ((long long)nx * ny);
    const double lo[3] = {lo0, lo1, lo2}, hi[3] = {hi0, hi1, hi2};
    const int n[3] = {n0, n1, n2}, per[3] = {p0, p1, p2};
    const long long ix[3] = {i, j, k};
    for (int a = 0; a < dim; ++a) {
        double step;
        if (per[a])
            step = __ddiv_rn(__dsub_rn(hi[a], lo[a]), (double)n[a]);
        else
            step = n[a] > 1 ? __ddiv_rn(__dsub_rn(hi[a], lo[a]), (double)(n[a] - 1)) : 0.0;
        double x = __dadd_rn(lo[a], __dmul_rn((double)ix[a], step));
        out[a * N + id] = __double2float_rn(x);
    }
}

cudaError_t launch_seed_grid(int dim, const int n[3], const double lo[3], const double hi[3], const int periodic[3],
                             long long N, float *out, cudaStream_t s)
{
    if (N == 0) return cudaSuccess;
    int bt = 256;
    unsigned grid = (unsigned)((N + bt - 1) / bt);
    seed_grid_kernel<<<grid, bt, 0, s>>>(dim, n[0], n[1], lo[0], lo[1], lo[2], hi[0], hi[1], hi[2], n[0], n[1],
                                         n[2], periodic[0], periodic[1], periodic[2], N, out);
    return cudaGetLastError();
}

// auxiliary point (p * dim + b) * 2 + s = seed p moved by (1 - 2s) delta[b] along axis b
__global__ void seed_aux_kernel(int dim, const float *__restrict__ lat, long long N, double d0, double d1,
                                double d2, float *__restrict__ out)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long M = N * 2 * dim;
    if (t >= M) return;
    const long long p = t / (2 * dim);
    const int b = (int)((t / 2) % dim), sgn = (int)(t & 1);
    const double d = b == 0 ? d0 : (b == 1 ? d1 : d2);
    for (int a = 0; a < dim; ++a) {
        const float x = lat[a * N + p];
        out[a * M + t] = a == b ? __double2float_rn(__dadd_rn((double)x, sgn ? -d : d)) : x;
    }
}

cudaError_t launch_seed_aux(int dim, const float *lattice, long long N, const double *delta, float *out,
                            cudaStream_t s)
{
    const long long M = N * 2 * dim;
    if (M == 0) return cudaSuccess;
    seed_aux_kernel<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(dim, lattice, N, delta[0], delta[1],
                                                                  dim > 2 ? delta[2] : 0.0, out);
    return cudaGetLastError();
}

// auxiliary points of a lattice; on a mesh field (the lattice made on it) also their exact cells
static lcs_status seed_aux(lcs_ctx *ctx, const lcs_seeds *lat, const lcs_field *field, const double *delta,
                           lcs_seeds **out, const char *who)
{
    if (!ctx) return LCS_EINVAL;
    if (!lat || !delta || !out) return lcs_fail(ctx, LCS_EINVAL, "%s: null argument", who);
    *out = nullptr;
    const bool mesh = field && lcs_is_mesh(field);
    if (lat->aux_base_N > 0) return lcs_fail(ctx, LCS_EINVAL, "%s: auxiliary points of auxiliary points", who);
    if (mesh && (!lat->d_cells || lat->field_uid != field->uid))
        return lcs_fail(ctx, LCS_EINVAL, "%s: the lattice must come from lcs_seed_grid on this mesh field", who);
    if (!mesh && lat->d_cells)
        return lcs_fail(ctx, LCS_EINVAL, "%s: a lattice made on a mesh field needs that field", who);
    for (int a = 0; a < lat->dim; ++a)
        if (!(delta[a] > 0.0) || !isfinite(delta[a]))
            return lcs_fail(ctx, LCS_EINVAL, "%s: delta[%d] = %g must be finite and > 0", who, a, delta[a]);
    if (lat->N > ((1LL << 31) - 1) / (2 * lat->dim)) return lcs_fail(ctx, LCS_EINVAL, "%s: too many seeds", who);
    lcs_seeds *s = new (std::nothrow) lcs_seeds(*lat);
    if (!s) return lcs_fail(ctx, LCS_ENOMEM, "host allocation");
    s->uid = lcs_next_uid();
    s->aux_base_N = lat->N;
    s->N = lat->N * 2 * lat->dim;
    for (int a = 0; a < 3; ++a) s->aux_delta[a] = a < lat->dim ? delta[a] : 0.0;
    s->d_xyz = nullptr;
    s->d_cells = nullptr;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_xyz, sizeof(float) * s->dim * (size_t)s->N);
    if (e == cudaSuccess) e = launch_seed_aux(s->dim, lat->d_xyz, lat->N, s->aux_delta, s->d_xyz, ctx->stream);
    if (e == cudaSuccess && mesh) {
        s->field_uid = field->uid;
        e = cudaMalloc(&s->d_cells, sizeof(int) * (size_t)s->N);
        if (e == cudaSuccess)
            e = field->kind == LCS_TRI ? tri_locate_seeds(field, s->d_xyz, s->N, s->d_cells, ctx->stream)
                                       : tet_locate_seeds(field, s->d_xyz, s->N, s->d_cells, ctx->stream);
    }
    if (e != cudaSuccess) {
        lcs_free_seeds(s);
        return lcs_fail(ctx, e == cudaErrorMemoryAllocation ? LCS_ENOMEM : LCS_ECUDA, "%s: %s", who,
                        cudaGetErrorString(e));
    }
    *out = s;
    return LCS_OK;
}

extern "C" lcs_status lcs_seed_aux(lcs_ctx *ctx, const lcs_seeds *lat, const double *delta, lcs_seeds **out)
{
    return seed_aux(ctx, lat, nullptr, delta, out, "lcs_seed_aux");
}

extern "C" lcs_status lcs_seed_aux_field(lcs_ctx *ctx, const lcs_seeds *lat, const lcs_field *field,
                                         const double *delta, lcs_seeds **out)
{
    return seed_aux(ctx, lat, field, delta, out, "lcs_seed_aux_field");
}

extern "C" lcs_status lcs_seed_grid(lcs_ctx *ctx, const lcs_seed_desc *d, const lcs_field *field, lcs_seeds **out)
{
    if (!ctx) return LCS_EINVAL;
    if (!d || !out) return lcs_fail(ctx, LCS_EINVAL, "lcs_seed_grid: null argument");
    *out = nullptr;
    if (d->dim != 2 && d->dim != 3) return lcs_fail(ctx, LCS_EINVAL, "lcs_seed_grid: dim must be 2 or 3");
    if (field && field->dim != d->dim) return lcs_fail(ctx, LCS_EINVAL, "lcs_seed_grid: dim differs from the field's");

    long long N = 1;
    for (int a = 0; a < d->dim; ++a) {
        if (d->n[a] < 1) return lcs_fail(ctx, LCS_EINVAL, "lcs_seed_grid: n[%d] < 1", a);
        if (!(d->hi[a] >= d->lo[a])) return lcs_fail(ctx, LCS_EINVAL, "lcs_seed_grid: hi < lo on axis %d", a);
        N *= d->n[a];
    }
    CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    lcs_seeds *s = new (std::nothrow) lcs_seeds();
    if (!s) return lcs_fail(ctx, LCS_ENOMEM, "host allocation");
    s->uid = lcs_next_uid();
    s->dim = d->dim;
    s->N = N;
    for (int a = 0; a < 3; ++a) {
        s->n[a] = a < d->dim ? d->n[a] : 1;
        s->lo[a] = a < d->dim ? d->lo[a] : 0.0;
        s->hi[a] = a < d->dim ? d->hi[a] : 0.0;
        s->periodic[a] = a < d->dim ? (d->periodic[a] != 0) : 0;
        if (s->periodic[a]) {
            s->h[a] = (s->hi[a] - s->lo[a]) / s->n[a];
            s->period[a] = s->hi[a] - s->lo[a];
        } else {
            s->h[a] = s->n[a] > 1 ? (s->hi[a] - s->lo[a]) / (s->n[a] - 1) : 1.0;
            s->period[a] = 0.0;
        }
    }
    cudaError_t e = cudaMalloc(&s->d_xyz, sizeof(float) * s->dim * (size_t)N);
    if (e == cudaSuccess) e = launch_seed_grid(s->dim, s->n, s->lo, s->hi, s->periodic, N, s->d_xyz, ctx->stream);
    if (e == cudaSuccess && field && lcs_is_mesh(field)) {
        s->field_uid = field->uid;
        e = cudaMalloc(&s->d_cells, sizeof(int) * (size_t)N);
        if (e == cudaSuccess)
            e = field->kind == LCS_TRI ? tri_locate_seeds(field, s->d_xyz, N, s->d_cells, ctx->stream)
                                       : tet_locate_seeds(field, s->d_xyz, N, s->d_cells, ctx->stream);
    }
    if (e != cudaSuccess) {
        lcs_free_seeds(s);
        return lcs_fail(ctx, e == cudaErrorMemoryAllocation ? LCS_ENOMEM : LCS_ECUDA, "lcs_seed_grid: %s",
                    cudaGetErrorString(e));
    }
    *out = s;
    return LCS_OK;
}

extern "C" long long lcs_seeds_count(const lcs_seeds *s)
{
    return s ? s->N : 0;
}

extern "C" lcs_status lcs_seeds_get(lcs_ctx *ctx, const lcs_seeds *s, float *xyz, int *cells, int on_device)
{
    if (!ctx) return LCS_EINVAL;
    if (!s) return lcs_fail(ctx, LCS_EINVAL, "lcs_seeds_get: null seeds");
    if (cells && !s->d_cells) return lcs_fail(ctx, LCS_EINVAL, "lcs_seeds_get: seeds carry no cell ids");
    CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (xyz) CUDA_TRY(ctx, cudaMemcpyAsync(xyz, s->d_xyz, sizeof(float) * s->dim * s->N, k, ctx->stream));
    if (cells) CUDA_TRY(ctx, cudaMemcpyAsync(cells, s->d_cells, sizeof(int) * s->N, k, ctx->stream));
    if (!on_device) CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return LCS_OK;
}

extern "C" void lcs_free_seeds(lcs_seeds *s)
{
    if (!s) return;
    cudaFree(s->d_xyz);
    cudaFree(s->d_cells);
    delete s;
}

// --------------------------------------------------------------- flow map

extern "C" lcs_status lcs_flowmap_create(lcs_ctx *ctx, const lcs_seeds *s, int njobs, lcs_flowmap **out)
{
    if (!ctx) return LCS_EINVAL;
    if (!s || !out) return lcs_fail(ctx, LCS_EINVAL, "lcs_flowmap_create: null argument");
    *out = nullptr;
    if (njobs < 1 || njobs > LCS_MAX_JOBS) return lcs_fail(ctx, LCS_EINVAL, "lcs_flowmap_create: njobs in [1, %d]", LCS_MAX_JOBS);
    CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    lcs_flowmap *fm = new (std::nothrow) lcs_flowmap();
    if (!fm) return lcs_fail(ctx, LCS_ENOMEM, "host allocation");
    fm->ctx = ctx;
    fm->uid = lcs_next_uid();
    fm->seeds = s;
    fm->dim = s->dim;
    fm->njobs = njobs;
    fm->N = s->N;
    fm->T.assign(njobs, 0.0);
    size_t N = (size_t)s->N;
    cudaError_t e = cudaMalloc(&fm->d_xyz, sizeof(float) * fm->dim * N * njobs);
    if (e == cudaSuccess) e = cudaMalloc(&fm->d_status, N * njobs);
    if (e == cudaSuccess) e = cudaMalloc(&fm->d_texit, sizeof(float) * N * njobs);
    if (e == cudaSuccess) e = cudaMalloc(&fm->d_absT, sizeof(double) * njobs);
    if (e == cudaSuccess) e = cudaMemsetAsync(fm->d_status, LCS_TRACER_OUTSIDE, N * njobs, ctx->stream);
    if (e != cudaSuccess) {
        lcs_free_flowmap(fm);
        return lcs_fail(ctx, e == cudaErrorMemoryAllocation ? LCS_ENOMEM : LCS_ECUDA, "lcs_flowmap_create: %s",
                    cudaGetErrorString(e));
    }
    *out = fm;
    return LCS_OK;
}

extern "C" void lcs_free_flowmap(lcs_flowmap *fm)
{
    if (!fm) return;
    cudaFree(fm->d_xyz);
    cudaFree(fm->d_status);
    cudaFree(fm->d_texit);
    cudaFree(fm->d_absT);
    cudaFree(fm->d_steps);
    cudaFree(fm->d_grad);
    delete fm;
}

// scratch layout for one lcs_advect call
struct AdvectScratch {
    JobDev jd;
    SchedEntry *sched;
};

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

struct AdvectLayout {
    size_t jb, sb, wb;
    bool want_work;
    int E;
};

static AdvectLayout advect_layout(const lcs_field *f, const lcs_seeds *s, const lcs_advect_opts *o, const JobTable &J)
{
    AdvectLayout Ly;
    Ly.jb = 2 * align256(sizeof(int) * J.njobs) + 3 * align256(sizeof(float) * J.njobs) + 256 +
            align256(sizeof(int) * LCS_MAX_SNAP) + align256(sizeof(float) * J.njobs * LCS_MAX_SNAP);
    Ly.sb = align256(sizeof(SchedEntry) * 3 * (size_t)J.njobs * std::max(J.nsteps_max, 1));
    Ly.want_work = f->dim == 3 && (o->variant == 3 || (o->variant == 0 && s->N >= LCS_SORTED_MIN_SEEDS));
    Ly.E = o->episode_steps > 0 ? std::min(o->episode_steps, 1024) : LCS_EPISODE_STEPS;
    Ly.wb = Ly.want_work ? rk4_sorted_scratch_bytes(s->N, f, Ly.E, o->variational != 0) : 0;
    if (f->dim == 2 && f->kind == LCS_RECTILINEAR && (o->variant == 5 || o->variant == 0)) {
        // 2D time slices: asked for (up to 16 GiB), or by default when they take at most 2 GiB
        const size_t b = rk4_slice2d_bytes(f, J.njobs, J.nsteps);
        Ly.want_work = b <= (o->variant == 5 ? LCS_SLICE2D_MAX_BYTES : LCS_SLICE2D_DEFAULT_BYTES);
        Ly.wb = Ly.want_work ? b : 0;
    }
    return Ly;
}

static lcs_status advect_rk4_rect(lcs_ctx *ctx, const lcs_field *f, const lcs_seeds *s, const lcs_advect_opts *o,
                                  lcs_flowmap *fm, JobTable &J)
{
    const AdvectLayout Ly = advect_layout(f, s, o, J);
    const size_t jb = Ly.jb, sb = Ly.sb;
    const bool want_work = Ly.want_work;
    const int E = Ly.E;
    lcs_status st = lcs_scratch_reserve(ctx, jb + sb + Ly.wb);
    if (st != LCS_OK) return st;
    char *p = (char *)ctx->d_scratch;
    JobDev D;
    D.nsteps = (int *)p;
    p += align256(sizeof(int) * J.njobs);
    D.h = (float *)p;
    p += align256(sizeof(float) * J.njobs);
    D.t0 = (float *)p;
    p += align256(sizeof(float) * J.njobs);
    D.tend = (float *)p;
    p += align256(sizeof(float) * J.njobs);
    D.absT = fm->d_absT;
    D.t0d = nullptr;
    D.Td = nullptr;
    D.order = (int *)p;
    p += align256(sizeof(int) * J.njobs);
    unsigned *queue = (unsigned *)p;
    p += 256;
    D.snap_n = (int *)p;
    p += align256(sizeof(int) * LCS_MAX_SNAP);
    D.snap_te = (float *)p;
    p += align256(sizeof(float) * J.njobs * LCS_MAX_SNAP);
    SchedEntry *sched = (SchedEntry *)p;
    CUDA_TRY(ctx, launch_rk4_schedule(f->d_times, f->nframes, f->time_periodic, f->period, J, D, sched, ctx->stream));
    Rk4Launch L;
    L.ctx = ctx;
    L.field = f;
    L.seeds = s->d_xyz;
    L.N = s->N;
    L.njobs = J.njobs;
    L.nsteps_max = J.nsteps_max;
    L.sched = sched;
    L.job_nsteps = D.nsteps;
    L.job_h = D.h;
    L.job_t0 = D.t0;
    L.job_tend = D.tend;
    L.out_xyz = fm->d_xyz;
    L.out_status = fm->d_status;
    L.out_texit = fm->d_texit;
    L.block_threads = o->block_threads;
    L.variant = o->variant;
    L.episode_steps = E;
    L.host_nsteps = J.nsteps;
    L.tracers_per_thread = o->tracers_per_thread >= 2 ? 2 : 1;
    L.queue = queue;
    L.job_order = D.order;
    L.out_grad = o->variational ? fm->d_grad : nullptr;
    L.nsnap = J.nsnap;
    L.snap_n = D.snap_n;
    L.host_snap_n = J.snap_n;
    L.snap_te = D.snap_te;
    L.work = want_work ? (char *)ctx->d_scratch + jb + sb : nullptr;
    if (o->wait_limit > 0.0) L.wait_ns = (unsigned long long)(o->wait_limit * 1e9);
    if (lcs_is_mesh(f)) {
        cudaError_t e = launch_rk4_tet(ctx, L, s->d_cells, o->walk_limit, ctx->stream);
        if (e != cudaSuccess) return lcs_fail(ctx, LCS_ECUDA, "lcs_advect: launch failed: %s", cudaGetErrorString(e));
        return LCS_OK;
    }
    if (launch_rk4_rect(ctx, L, ctx->stream) < 0)
        return lcs_fail(ctx, LCS_ECUDA, "lcs_advect: launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    return LCS_OK;
}

// Adaptive DP5(4) with one step per warp (every field kind)
static lcs_status advect_rk45(lcs_ctx *ctx, const lcs_field *f, const lcs_seeds *s, const lcs_advect_opts *o,
                              lcs_flowmap *fm)
{
    const int njobs = o->njobs > 1 ? o->njobs : 1;
    const double rtol = o->rtol > 0 ? o->rtol : 1e-6, atol = o->atol > 0 ? o->atol : 1e-6;
    const double h0 = o->h0 != 0 ? fabs(o->h0) : 0.01;
    if (!isfinite(rtol) || !isfinite(atol) || !isfinite(h0))
        return lcs_fail(ctx, LCS_EINVAL, "lcs_advect: rtol, atol and h0 must be finite");
    JobTable *J = new (std::nothrow) JobTable();
    if (!J) return lcs_fail(ctx, LCS_ENOMEM, "host allocation");
    J->njobs = njobs;
    J->nsteps_max = 0;
    for (int j = 0; j < njobs; ++j) {
        double t0 = o->njobs > 1 ? o->job_t0[j] : o->t0;
        double T = o->njobs > 1 ? o->job_T[j] : o->T;
        if (!isfinite(t0) || !isfinite(T)) {
            delete J;
            return lcs_fail(ctx, LCS_EINVAL, "lcs_advect: job %d has a non-finite t0 or T", j);
        }
        J->t0[j] = t0;
        J->T[j] = T;
        J->h[j] = 0.0;
        J->nsteps[j] = 0;
        J->order[j] = j;
        fm->T[j] = T;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    size_t need = 2 * align256(sizeof(int) * njobs) + 3 * align256(sizeof(float) * njobs) + 2 * align256(8 * njobs);
    lcs_status st = e == cudaSuccess ? lcs_scratch_reserve(ctx, need) : lcs_fail(ctx, LCS_ECUDA, "cudaSetDevice failed");
    if (st == LCS_OK && !fm->d_steps && cudaMalloc(&fm->d_steps, sizeof(int) * (size_t)fm->N * fm->njobs) != cudaSuccess)
        st = lcs_fail(ctx, LCS_ENOMEM, "lcs_advect: step counts");
    if (st != LCS_OK) {
        delete J;
        return st;
    }
    char *p = (char *)ctx->d_scratch;
    JobDev D;
    D.nsteps = (int *)p;
    p += align256(sizeof(int) * njobs);
    D.h = (float *)p;
    p += align256(sizeof(float) * njobs);
    D.t0 = (float *)p;
    p += align256(sizeof(float) * njobs);
    D.tend = (float *)p;
    p += align256(sizeof(float) * njobs);
    D.order = (int *)p;
    p += align256(sizeof(int) * njobs);
    D.t0d = (double *)p;
    p += align256(8 * njobs);
    D.Td = (double *)p;
    D.absT = fm->d_absT;
    e = launch_rk4_schedule(f->d_times, f->nframes, f->time_periodic, f->period, *J, D, nullptr,
                            ctx->stream);  // per-job values only (no RK4 steps)
    delete J;
    if (e != cudaSuccess) return lcs_fail(ctx, LCS_ECUDA, "lcs_advect: %s", cudaGetErrorString(e));
    Dp45Args A;
    memset(&A, 0, sizeof A);
    A.seeds = s->d_xyz;
    A.cells0 = lcs_is_mesh(f) ? s->d_cells : nullptr;
    A.N = s->N;
    A.job_t0 = D.t0d;
    A.job_T = D.Td;
    A.h0 = (float)h0;
    A.rtol = (float)rtol;
    A.atol = (float)atol;
    A.max_steps = o->max_steps > 0 ? o->max_steps : 1000000;
    A.out_xyz = fm->d_xyz;
    A.out_status = fm->d_status;
    A.out_texit = fm->d_texit;
    A.out_steps = fm->d_steps;
    e = launch_dp45(ctx, f, A, njobs, o->block_threads, o->walk_limit, ctx->stream);
    if (e != cudaSuccess) return lcs_fail(ctx, LCS_ECUDA, "lcs_advect: RK45 launch failed: %s", cudaGetErrorString(e));
    return LCS_OK;
}

extern "C" lcs_status lcs_flowmap_steps(lcs_ctx *ctx, const lcs_flowmap *fm, int job, int *steps, int on_device)
{
    if (!ctx) return LCS_EINVAL;
    if (!fm || !steps) return lcs_fail(ctx, LCS_EINVAL, "lcs_flowmap_steps: null argument");
    if (job < 0 || job >= fm->njobs) return lcs_fail(ctx, LCS_EINVAL, "lcs_flowmap_steps: job %d out of range", job);
    if (!fm->d_steps) return lcs_fail(ctx, LCS_EINVAL, "lcs_flowmap_steps: no adaptive integration wrote this flow map");
    CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    CUDA_TRY(ctx, cudaMemcpyAsync(steps, fm->d_steps + (size_t)job * fm->N, sizeof(int) * (size_t)fm->N,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    if (!on_device) CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return LCS_OK;
}

// graph cache key: the handles' unique ids, the options that shape the launches, the jobs
static std::string graph_key(const lcs_ctx *ctx, const lcs_field *f, const lcs_seeds *s, const lcs_advect_opts *o,
                             const lcs_flowmap *fm, const JobTable &J)
{
    std::string k;
    char buf[256];
    snprintf(buf, sizeof buf, "%llu/%llu/%llu/%p/%zu/%d/%d/%d/%d/%d/%d/%a/v%d/w%d/l%a|", f->uid, s->uid, fm->uid,
             ctx->d_scratch, ctx->scratch_bytes, o->method, o->variant, o->block_threads, o->episode_steps,
             o->tracers_per_thread, J.njobs, o->dt, o->variational, o->walk_limit, o->wait_limit);
    k += buf;
    for (int j = 0; j < J.njobs; ++j) {
        snprintf(buf, sizeof buf, "%a,%a;", J.t0[j], J.T[j]);
        k += buf;
    }
    for (int q = 0; q < J.nsnap; ++q) {
        snprintf(buf, sizeof buf, "s%d,%a;", J.snap_n[q], J.snap_T[q]);
        k += buf;
    }
    return k;
}

// Capture the launches of one lcs_advect call into a CUDA graph (once per key), then replay it
// on the context stream.  The scratch is reserved before capture, since capture forbids allocation.
static lcs_status advect_graph(lcs_ctx *ctx, const lcs_field *f, const lcs_seeds *s, const lcs_advect_opts *o,
                               lcs_flowmap *fm, JobTable &J)
{
    const AdvectLayout Ly = advect_layout(f, s, o, J);
    lcs_status st = lcs_scratch_reserve(ctx, Ly.jb + Ly.sb + Ly.wb);
    if (st != LCS_OK) return st;
    const std::string key = graph_key(ctx, f, s, o, fm, J);
    ctx->graph_clock++;
    for (auto &g : ctx->graphs)
        if (g.key == key) {
            g.last_use = ctx->graph_clock;
            CUDA_TRY(ctx, cudaGraphLaunch(g.exec, ctx->stream));
            return LCS_OK;
        }
    if (!ctx->cap_stream) CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    cudaStream_t user = ctx->stream;
    const bool timing = ctx->timing;
    ctx->stream = ctx->cap_stream;
    ctx->timing = false;
    cudaError_t e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) st = advect_rk4_rect(ctx, f, s, o, fm, J);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(ctx->cap_stream, &graph) : e;
    ctx->stream = user;
    ctx->timing = timing;
    if (e != cudaSuccess || e2 != cudaSuccess || st != LCS_OK) {
        if (graph) cudaGraphDestroy(graph);
        if (st != LCS_OK) return st;
        return lcs_fail(ctx, LCS_ECUDA, "lcs_advect: graph capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return lcs_fail(ctx, LCS_ECUDA, "lcs_advect: graph instantiate: %s", cudaGetErrorString(e));
    }
    if (ctx->graphs.size() >= 8) {  // evict the least recently used
        auto it = std::min_element(ctx->graphs.begin(), ctx->graphs.end(),
                                   [](const lcs_ctx::GraphEntry &a, const lcs_ctx::GraphEntry &b) {
                                       return a.last_use < b.last_use;
                                   });
        cudaGraphExecDestroy(it->exec);
        cudaGraphDestroy(it->graph);
        ctx->graphs.erase(it);
    }
    lcs_ctx::GraphEntry g;
    g.key = key;
    g.graph = graph;
    g.exec = exec;
    g.last_use = ctx->graph_clock;
    ctx->graphs.push_back(g);
    CUDA_TRY(ctx, cudaGraphLaunch(exec, ctx->stream));
    return LCS_OK;
}

// The fixed-step jobs of an RK4 call (and its snapshot steps) from the options: |T| / |dt|
// must be a whole number of steps for every job and snapshot.
static lcs_status rk4_jobs(lcs_ctx *ctx, const lcs_advect_opts *o, int njobs, JobTable *J, const char *who)
{
    const double adt = fabs(o->dt);
    if (!(adt > 0.0) || !isfinite(adt)) return lcs_fail(ctx, LCS_EINVAL, "%s: dt must be finite and > 0", who);
    J->njobs = njobs;
    J->nsteps_max = 0;
    for (int j = 0; j < njobs; ++j) {
        double t0 = o->njobs > 1 ? o->job_t0[j] : o->t0;
        double T = o->njobs > 1 ? o->job_T[j] : o->T;
        if (!isfinite(t0) || !isfinite(T)) return lcs_fail(ctx, LCS_EINVAL, "%s: job %d has a non-finite t0 or T", who, j);
        double r = fabs(T) / adt;
        long long ns = (long long)floor(r + 0.5);
        if (fabs(r - (double)ns) > 1e-9 * std::max(1.0, r) || ns > (1LL << 30))
            return lcs_fail(ctx, LCS_EINVAL, "%s: |T|/|dt| = %.17g is not an integer (job %d)", who, r, j);
        J->t0[j] = t0;
        J->T[j] = T;
        J->h[j] = T < 0.0 ? -adt : adt;
        J->nsteps[j] = (int)ns;
        J->nsteps_max = std::max(J->nsteps_max, (int)ns);
        J->order[j] = j;
    }
    J->nsnap = o->nsnap;
    for (int q = 0; q < o->nsnap; ++q) {
        const double a = o->snap_T[q], r = a / adt;
        const long long n = (long long)floor(r + 0.5);
        if (!(a > 0.0) || !isfinite(a) || fabs(r - (double)n) > 1e-9 * std::max(1.0, r) || n > (1LL << 30) ||
            (q > 0 && !(a > o->snap_T[q - 1])))
            return lcs_fail(ctx, LCS_EINVAL, "%s: snap_T[%d] = %.17g must be > 0, increasing and a whole number of steps",
                            who, q, a);
        J->snap_n[q] = (int)n;
        J->snap_T[q] = a;
    }
    return LCS_OK;
}

extern "C" lcs_status lcs_advect(lcs_ctx *ctx, const lcs_field *f, const lcs_seeds *s, const lcs_advect_opts *o,
                                 lcs_flowmap *fm)
{
    if (!ctx) return LCS_EINVAL;
    if (!f || !s || !o || !fm) return lcs_fail(ctx, LCS_EINVAL, "lcs_advect: null argument");
    if (f->dim != s->dim) return lcs_fail(ctx, LCS_EINVAL, "lcs_advect: field and seeds differ in dim");
    if (fm->seeds != s) return lcs_fail(ctx, LCS_EINVAL, "lcs_advect: flow map was made for other seeds");
    int njobs = o->njobs > 1 ? o->njobs : 1;
    if (njobs > fm->njobs) return lcs_fail(ctx, LCS_EINVAL, "lcs_advect: %d jobs > flow map's %d", njobs, fm->njobs);
    if (o->nsnap < 0 || o->nsnap > LCS_MAX_SNAP || (o->nsnap > 0 && !o->snap_T))
        return lcs_fail(ctx, LCS_EINVAL, "lcs_advect: nsnap must be 0..%d with snap_T given", LCS_MAX_SNAP);
    if (o->variational && (o->method != LCS_RK4 || o->nsnap > 0 || s->aux_base_N > 0))
        return lcs_fail(ctx, LCS_EUNSUPPORTED,
                        "lcs_advect: the variational equations need LCS_RK4, a lattice and no snapshots");
    if (o->nsnap > 0) {
        if (o->method != LCS_RK4)
            return lcs_fail(ctx, LCS_EUNSUPPORTED, "lcs_advect: snapshots need LCS_RK4");
        if ((long long)njobs * (1 + o->nsnap) > fm->njobs)
            return lcs_fail(ctx, LCS_EINVAL, "lcs_advect: %d jobs with %d snapshots need %lld flow-map slots, not %d",
                            njobs, o->nsnap, (long long)njobs * (1 + o->nsnap), fm->njobs);
    }
    if (o->njobs > 1 && (!o->job_t0 || !o->job_T)) return lcs_fail(ctx, LCS_EINVAL, "lcs_advect: job arrays missing");
    if (!(o->wait_limit >= 0.0 && o->wait_limit <= 60.0))
        return lcs_fail(ctx, LCS_EINVAL, "lcs_advect: wait_limit must be 0..60 s");
    if (o->method != LCS_RK4 && o->method != LCS_RK45 && o->method != LCS_SURROGATE)
        return lcs_fail(ctx, LCS_EUNSUPPORTED, "lcs_advect: method %d not built in", o->method);
    if (o->method == LCS_SURROGATE) return advect_surrogate(ctx, f, s, o, fm);
    if (lcs_is_mesh(f) && (!s->d_cells || s->field_uid != f->uid))
        return lcs_fail(ctx, LCS_EINVAL, "lcs_advect: on a mesh field the seeds must come from lcs_seed_grid on that field");
    if (o->method == LCS_RK45) return advect_rk45(ctx, f, s, o, fm);
    JobTable *J = new (std::nothrow) JobTable();
    if (!J) return lcs_fail(ctx, LCS_ENOMEM, "host allocation");
    lcs_status bs = rk4_jobs(ctx, o, njobs, J, "lcs_advect");
    if (bs != LCS_OK) {
        delete J;
        return bs;
    }
    for (int j = 0; j < njobs; ++j) {
        fm->T[j] = J->T[j];
        for (int q = 0; q < J->nsnap; ++q) {
            const double a = J->snap_T[q], Tj = J->T[j];
            fm->T[njobs + j * J->nsnap + q] = Tj < 0.0 ? -std::min(a, -Tj) : std::min(a, Tj);
        }
    }
    // work-queue order of the persistent kernel: longest integrations first
    std::stable_sort(J->order, J->order + njobs, [&](int a, int b) { return J->nsteps[a] > J->nsteps[b]; });
    lcs_status st;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess && o->variational && !fm->d_grad)
        e = cudaMalloc(&fm->d_grad, sizeof(float) * fm->dim * fm->dim * (size_t)fm->N * fm->njobs);
    fm->grad_valid = o->variational != 0;
    if (e != cudaSuccess)
        st = lcs_fail(ctx, LCS_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    else if (o->use_graph)
        st = advect_graph(ctx, f, s, o, fm, *J);
    else
        st = advect_rk4_rect(ctx, f, s, o, fm, *J);
    delete J;
    return st;
}

extern "C" lcs_status lcs_flowmap_get(lcs_ctx *ctx, const lcs_flowmap *fm, int job, float *xyz,
                                      unsigned char *status, float *t_exit, int on_device)
{
    if (!ctx) return LCS_EINVAL;
    if (!fm) return lcs_fail(ctx, LCS_EINVAL, "lcs_flowmap_get: null flow map");
    if (job < 0 || job >= fm->njobs) return lcs_fail(ctx, LCS_EINVAL, "lcs_flowmap_get: job %d out of range", job);
    CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    size_t N = (size_t)fm->N;
    if (xyz)
        CUDA_TRY(ctx, cudaMemcpyAsync(xyz, fm->d_xyz + (size_t)job * fm->dim * N, sizeof(float) * fm->dim * N, k,
                                      ctx->stream));
    if (status) CUDA_TRY(ctx, cudaMemcpyAsync(status, fm->d_status + (size_t)job * N, N, k, ctx->stream));
    if (t_exit)
        CUDA_TRY(ctx, cudaMemcpyAsync(t_exit, fm->d_texit + (size_t)job * N, sizeof(float) * N, k, ctx->stream));
    if (!on_device) CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return LCS_OK;
}

extern "C" lcs_status lcs_flowmap_set(lcs_ctx *ctx, lcs_flowmap *fm, int job, const float *xyz,
                                      const unsigned char *status, const float *t_exit, double T, int on_device)
{
    if (!ctx) return LCS_EINVAL;
    const char *who = "lcs_flowmap_set";
    if (!fm || !xyz || !status) return lcs_fail(ctx, LCS_EINVAL, "%s: null argument", who);
    if (job < 0 || job >= fm->njobs) return lcs_fail(ctx, LCS_EINVAL, "%s: job %d out of range", who, job);
    if (!(T != 0.0 && std::isfinite(T))) return lcs_fail(ctx, LCS_EINVAL, "%s: T must be finite and nonzero", who);
    size_t N = (size_t)fm->N;
    if (!on_device)
        for (size_t i = 0; i < N; ++i)
            if (status[i] > LCS_TRACER_WALKFAIL)
                return lcs_fail(ctx, LCS_EINVAL, "%s: status[%zu] = %d is not a tracer status", who, i, (int)status[i]);
    CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CUDA_TRY(ctx, cudaMemcpyAsync(fm->d_xyz + (size_t)job * fm->dim * N, xyz, sizeof(float) * fm->dim * N, k,
                                  ctx->stream));
    CUDA_TRY(ctx, cudaMemcpyAsync(fm->d_status + (size_t)job * N, status, N, k, ctx->stream));
    if (t_exit)
        CUDA_TRY(ctx, cudaMemcpyAsync(fm->d_texit + (size_t)job * N, t_exit, sizeof(float) * N, k, ctx->stream));
    const double absT = fabs(T);
    CUDA_TRY(ctx, cudaMemcpyAsync(fm->d_absT + job, &absT, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));   // absT lives on this frame
    fm->T[job] = T;
    fm->grad_valid = false;
    return LCS_OK;
}

// ------------------------------------------------------ grad F, C, FTLE

static lcs_status cg_call(lcs_ctx *ctx, const lcs_flowmap *fm, int job, float *ftle, double *lam, double *C,
                          int on_device, const char *who, double *eigval = nullptr, double *eigvec = nullptr,
                          bool variational = false)
{
    if (!ctx) return LCS_EINVAL;
    if (!fm) return lcs_fail(ctx, LCS_EINVAL, "%s: null flow map", who);
    if (job < -1 || job >= fm->njobs) return lcs_fail(ctx, LCS_EINVAL, "%s: job %d out of range", who, job);
    const lcs_seeds *s = fm->seeds;
    const bool aux = s->aux_base_N > 0;
    if (variational && !(fm->d_grad && fm->grad_valid))
        return lcs_fail(ctx, LCS_EINVAL, "%s: no variational integration wrote this flow map", who);
    if (!aux && !variational)
        for (int a = 0; a < s->dim; ++a)
            if (s->n[a] < 3) return lcs_fail(ctx, LCS_EINVAL, "%s: the lattice needs >= 3 seeds per axis", who);
    CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    int j0 = job < 0 ? 0 : job, nj = job < 0 ? fm->njobs : 1;
    size_t N = (size_t)(aux ? s->aux_base_N : fm->N);   // outputs per job: one per lattice seed
    int np = fm->dim == 2 ? 3 : 6;
    CgLaunch L;
    L.dim = fm->dim;
    for (int a = 0; a < 3; ++a) {
        L.n[a] = s->n[a];
        L.periodic[a] = s->periodic[a];
        L.h[a] = s->h[a];
        L.period[a] = s->period[a];
    }
    L.N = (long long)N;
    L.job0 = j0;
    L.njobs = nj;
    L.xyz = fm->d_xyz;
    L.status = fm->d_status;
    L.absT = fm->d_absT;
    L.x0aux = aux ? s->d_xyz : nullptr;
    L.npts = fm->N;
    L.grad = variational ? fm->d_grad : nullptr;
    const size_t dim = (size_t)fm->dim;
    size_t bC = C ? sizeof(double) * np * N * nj : 0, bL = lam ? sizeof(double) * N * nj : 0,
           bF = ftle ? sizeof(float) * N * nj : 0, bE = eigval ? sizeof(double) * dim * N * nj : 0,
           bV = eigvec ? sizeof(double) * dim * dim * N * nj : 0;
    char *tmp = nullptr;
    if (!on_device && (bC + bL + bF + bE + bV) > 0)
        CUDA_TRY(ctx, cudaMallocAsync((void **)&tmp,
                                      align256(bC) + align256(bL) + align256(bF) + align256(bE) + align256(bV),
                                      ctx->stream));
    char *q = tmp;
    L.C = C ? (on_device ? C : (double *)q) : nullptr;
    if (C && !on_device) q += align256(bC);
    L.lam = lam ? (on_device ? lam : (double *)q) : nullptr;
    if (lam && !on_device) q += align256(bL);
    L.ftle = ftle ? (on_device ? ftle : (float *)q) : nullptr;
    if (ftle && !on_device) q += align256(bF);
    L.eigval = eigval ? (on_device ? eigval : (double *)q) : nullptr;
    if (eigval && !on_device) q += align256(bE);
    L.eigvec = eigvec ? (on_device ? eigvec : (double *)q) : nullptr;
    lcs_tm_begin(ctx, 3, ctx->stream);
    cudaError_t e = launch_cg_ftle(L, ctx->stream);
    lcs_tm_end(ctx, 3, ctx->stream);
    if (e == cudaSuccess && !on_device) {
        if (C) e = cudaMemcpyAsync(C, L.C, bC, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess && lam) e = cudaMemcpyAsync(lam, L.lam, bL, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess && ftle) e = cudaMemcpyAsync(ftle, L.ftle, bF, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess && eigval)
            e = cudaMemcpyAsync(eigval, L.eigval, bE, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess && eigvec)
            e = cudaMemcpyAsync(eigvec, L.eigvec, bV, cudaMemcpyDeviceToHost, ctx->stream);
    }
    if (tmp) cudaFreeAsync(tmp, ctx->stream);
    if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return lcs_fail(ctx, LCS_ECUDA, "%s: %s", who, cudaGetErrorString(e));
    return LCS_OK;
}

extern "C" lcs_status lcs_cauchy_green(lcs_ctx *ctx, const lcs_flowmap *fm, int job, double *C, int on_device)
{
    if (ctx && !C) return lcs_fail(ctx, LCS_EINVAL, "lcs_cauchy_green: null output");
    return cg_call(ctx, fm, job, nullptr, nullptr, C, on_device, "lcs_cauchy_green");
}

extern "C" lcs_status lcs_ftle(lcs_ctx *ctx, const lcs_flowmap *fm, int job, float *ftle, double *lambda_max,
                               double *C, int on_device)
{
    if (ctx && !ftle) return lcs_fail(ctx, LCS_EINVAL, "lcs_ftle: null output");
    return cg_call(ctx, fm, job, ftle, lambda_max, C, on_device, "lcs_ftle");
}

extern "C" lcs_status lcs_ftle_early(lcs_ctx *ctx, const lcs_field *f, const lcs_seeds *s, const lcs_advect_opts *o,
                                     const lcs_flowmap *fm, int job, float *ftle, float *t_eval, int on_device)
{
    if (!ctx) return LCS_EINVAL;
    const char *who = "lcs_ftle_early";
    if (!f || !s || !o || !fm || !ftle) return lcs_fail(ctx, LCS_EINVAL, "%s: null argument", who);
    if (o->method != LCS_RK4) return lcs_fail(ctx, LCS_EUNSUPPORTED, "%s: fixed-step RK4 only", who);
    if (f->dim != s->dim || fm->seeds != s) return lcs_fail(ctx, LCS_EINVAL, "%s: field, seeds and flow map differ", who);
    if (lcs_is_mesh(f) && (!s->d_cells || s->field_uid != f->uid))
        return lcs_fail(ctx, LCS_EINVAL, "%s: on a mesh field the seeds must come from lcs_seed_grid on it", who);
    if (s->aux_base_N > 0) return lcs_fail(ctx, LCS_EUNSUPPORTED, "%s: not for auxiliary points", who);
    const int njobs = o->njobs > 1 ? o->njobs : 1;
    if (job < 0 || job >= njobs || njobs > fm->njobs)
        return lcs_fail(ctx, LCS_EINVAL, "%s: job %d out of range of the options' %d jobs", who, job, njobs);
    for (int a = 0; a < s->dim; ++a)
        if (s->n[a] < 3) return lcs_fail(ctx, LCS_EINVAL, "%s: the lattice needs >= 3 seeds per axis", who);
    if ((long long)fm->N > (1LL << 31) - 1) return lcs_fail(ctx, LCS_EINVAL, "%s: too many seeds", who);
    JobTable *J = new (std::nothrow) JobTable();
    if (!J) return lcs_fail(ctx, LCS_ENOMEM, "host allocation");
    lcs_status st = rk4_jobs(ctx, o, njobs, J, who);
    if (st != LCS_OK) {
        delete J;
        return st;
    }
    J->nsnap = 0;
    const double t0 = J->t0[job], adt = fabs(J->h[job]), absT = fabs(J->T[job]);
    const int ns = J->nsteps[job];
    CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const size_t N = (size_t)fm->N;
    // one block of temporaries: per-job values, schedule, count, list, host-output staging
    const size_t bj = align256(sizeof(int) * njobs), bf = align256(sizeof(float) * njobs),
                 bd = align256(sizeof(double) * njobs),
                 bs = align256(sizeof(SchedEntry) * 3 * (size_t)njobs * std::max(J->nsteps_max, 1)),
                 bl = align256(sizeof(int2) * N), bo = on_device ? 0 : align256(sizeof(float) * N);
    char *tmp = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&tmp, 2 * bj + 3 * bf + bd + bs + 256 + bl + 2 * bo, ctx->stream);
    if (e != cudaSuccess) {
        delete J;
        return lcs_fail(ctx, LCS_ENOMEM, "%s: %s", who, cudaGetErrorString(e));
    }
    char *p = tmp;
    JobDev D;
    D.nsteps = (int *)p;
    p += bj;
    D.order = (int *)p;
    p += bj;
    D.h = (float *)p;
    p += bf;
    D.t0 = (float *)p;
    p += bf;
    D.tend = (float *)p;
    p += bf;
    D.absT = (double *)p;
    p += bd;
    D.t0d = nullptr;
    D.Td = nullptr;
    SchedEntry *sched = (SchedEntry *)p;
    p += bs;
    unsigned *count = (unsigned *)p;
    p += 256;
    int2 *list = (int2 *)p;
    p += bl;
    float *out_f = on_device ? ftle : (float *)p;
    p += bo;
    float *out_t = on_device ? t_eval : (t_eval ? (float *)p : nullptr);
    float *pos = nullptr;
    EarlyLaunch E;
    e = launch_rk4_schedule(f->d_times, f->nframes, f->time_periodic, f->period, *J, D, sched, ctx->stream);
    const int nsteps_max = J->nsteps_max;
    delete J;
    // the regular FTLE of every seed, then the early seeds overwrite theirs
    CgLaunch L;
    L.dim = fm->dim;
    for (int a = 0; a < 3; ++a) {
        L.n[a] = s->n[a];
        L.periodic[a] = s->periodic[a];
        L.h[a] = s->h[a];
        L.period[a] = s->period[a];
    }
    L.N = fm->N;
    L.job0 = job;
    L.njobs = 1;
    L.xyz = fm->d_xyz;
    L.status = fm->d_status;
    L.texit = fm->d_texit;
    L.absT = fm->d_absT;
    L.C = nullptr;
    L.lam = nullptr;
    L.ftle = out_f;
    L.eigval = nullptr;
    L.eigvec = nullptr;
    lcs_tm_begin(ctx, 3, ctx->stream);
    if (e == cudaSuccess) e = launch_cg_ftle(L, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, sizeof(unsigned), ctx->stream);
    E.cg = L;
    E.phase = 0;
    E.job = job;
    E.ns = ns;
    E.t0 = t0;
    E.adt = adt;
    E.absT = (float)absT;
    E.count = count;
    E.list = list;
    E.nlisted = 0;
    E.pos = nullptr;
    E.t_eval = out_t;
    E.ftle = out_f;
    E.field = f;
    E.seeds = s->d_xyz;
    E.nsteps_max = nsteps_max;
    E.sched = sched;
    E.job_h = D.h;
    E.cells0 = lcs_is_mesh(f) ? s->d_cells : nullptr;
    E.walk_limit = o->walk_limit;
    unsigned nl = 0;
    if (e == cudaSuccess) e = launch_early_cg(E, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nl, count, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess && nl > 0) {
        e = cudaMallocAsync((void **)&pos, sizeof(float) * (size_t)nl * (2 * fm->dim + 1) * fm->dim, ctx->stream);
        if (e == cudaSuccess) {
            E.phase = 1;
            E.nlisted = nl;
            E.pos = pos;
            e = launch_early_cg(E, ctx->stream);
        }
    }
    lcs_tm_end(ctx, 3, ctx->stream);
    if (e == cudaSuccess && !on_device) {
        e = cudaMemcpyAsync(ftle, out_f, sizeof(float) * N, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess && t_eval)
            e = cudaMemcpyAsync(t_eval, out_t, sizeof(float) * N, cudaMemcpyDeviceToHost, ctx->stream);
    }
    if (pos) cudaFreeAsync(pos, ctx->stream);
    cudaFreeAsync(tmp, ctx->stream);
    if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return lcs_fail(ctx, LCS_ECUDA, "%s: %s", who, cudaGetErrorString(e));
    return LCS_OK;
}

extern "C" lcs_status lcs_ftle_variational(lcs_ctx *ctx, const lcs_flowmap *fm, int job, float *ftle,
                                           double *lambda_max, double *C, int on_device)
{
    if (ctx && !ftle) return lcs_fail(ctx, LCS_EINVAL, "lcs_ftle_variational: null output");
    return cg_call(ctx, fm, job, ftle, lambda_max, C, on_device, "lcs_ftle_variational", nullptr, nullptr, true);
}

extern "C" lcs_status lcs_flowmap_grad(lcs_ctx *ctx, const lcs_flowmap *fm, int job, float *grad, int on_device)
{
    if (!ctx) return LCS_EINVAL;
    if (!fm || !grad) return lcs_fail(ctx, LCS_EINVAL, "lcs_flowmap_grad: null argument");
    if (job < 0 || job >= fm->njobs) return lcs_fail(ctx, LCS_EINVAL, "lcs_flowmap_grad: job %d out of range", job);
    if (!fm->d_grad || !fm->grad_valid)
        return lcs_fail(ctx, LCS_EINVAL, "lcs_flowmap_grad: no variational integration wrote this flow map");
    CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const size_t b = sizeof(float) * fm->dim * fm->dim * (size_t)fm->N;
    CUDA_TRY(ctx, cudaMemcpyAsync(grad, (const char *)fm->d_grad + b * job, b,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    if (!on_device) CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return LCS_OK;
}

extern "C" lcs_status lcs_cg_eigen(lcs_ctx *ctx, const lcs_flowmap *fm, int job, double *eigval, double *eigvec,
                                   int on_device)
{
    if (ctx && !eigval && !eigvec) return lcs_fail(ctx, LCS_EINVAL, "lcs_cg_eigen: null outputs");
    return cg_call(ctx, fm, job, nullptr, nullptr, nullptr, on_device, "lcs_cg_eigen", eigval, eigvec);
}
