// mlp_api.cu -- C ABI of the learned surrogate and of the tensor-core GEMM under it.
#include "mlp_internal.cuh"
#include "tc_common.cuh"

#include <math.h>

#include <new>

extern "C" lcs_status lcs_gemm_bf16(lcs_ctx *ctx, long long M, int N, long long K, const void *A, long long lda,
                                    const void *B, long long ldb, float *C, long long ldc, int splits, int accumulate)
{
    if (!ctx) return LCS_EINVAL;
    if (!A || !B || !C) return lcs_fail(ctx, LCS_EINVAL, "lcs_gemm_bf16: null pointer");
    if (M < 0 || N < 0 || K < 0 || K % 16 || lda % 8 || ldb % 8 || (N != 16 && N % 128) || lda < K || ldb < K ||
        ldc < N)
        return lcs_fail(ctx, LCS_EINVAL, "lcs_gemm_bf16: unsupported shape M=%lld N=%d K=%lld lda=%lld ldb=%lld", M, N,
                        K, lda, ldb);
    if ((uintptr_t)A % 16 || (uintptr_t)B % 16)
        return lcs_fail(ctx, LCS_EINVAL, "lcs_gemm_bf16: A and B must be 16-byte aligned");
    LCS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    LCS_CUDA_TRY(ctx, launch_gemm_bf16((const __nv_bfloat16 *)A, lda, (const __nv_bfloat16 *)B, ldb, C, ldc, M, N, K,
                                       splits, accumulate, ctx->d_errword, ctx->stream));
    return LCS_OK;
}

// ------------------------------------------------------------------ network state

namespace {

// FP32 master parameters -> the inference block (canonical operand tiles + biases) and the
// trainer's K-major BF16 operands and their transposes; one thread per destination element
__global__ void mlp_refresh_kernel(const float *__restrict__ p, unsigned char *__restrict__ tiles,
                                   __nv_bfloat16 *__restrict__ wk, __nv_bfloat16 *__restrict__ wt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    // inference tiles: W0 (128 x 16), W1..W3 (128 x 128), W4 (16 x 128) as BF16 elements
    const int n_w0 = 128 * 16, n_w = 128 * 128, n_w4 = 16 * 128;
    const int n_tiles = n_w0 + 3 * n_w + n_w4;
    const int n_k = n_tiles;                // trainer operands, same element counts
    const int n_t = 3 * n_w + 128 * 16;     // transposes of W1..W3 and W4
    if (i < n_tiles) {
        int r, k, R, l;
        uint32_t base;
        float v;
        if (i < n_w0) {
            l = 0, R = 128, r = i / 16, k = i % 16, base = 0;
            v = k < 7 ? p[MLP_OFF_W0 + r * 7 + k] : 0.0f;
        } else if (i < n_w0 + 3 * n_w) {
            const int j = i - n_w0;
            l = 1 + j / n_w, R = 128, r = (j % n_w) / 128, k = j % 128, base = 4096 + 32768u * (l - 1);
            v = p[MLP_OFF_W1 + (l - 1) * MLP_LAYER_STRIDE + r * 128 + k];
        } else {
            const int j = i - n_w0 - 3 * n_w;
            l = 4, R = 16, r = j / 128, k = j % 128, base = 102400;
            v = r < 3 ? p[MLP_OFF_W4 + r * 128 + k] : 0.0f;
        }
        const __nv_bfloat16 b = __float2bfloat16_rn(v);
        *reinterpret_cast<__nv_bfloat16 *>(tiles + base + ckm_offset(R, r, k)) = b;
        // trainer operand, row-major [out][in] with the same padding
        wk[i] = b;
        (void)l;
    } else if (i < n_tiles + n_t) {
        const int j = i - n_tiles;
        if (j < 3 * n_w) {  // W_l^T [in][out]
            const int l = 1 + j / n_w, in = (j % n_w) / 128, out = j % 128;
            wt[j] = __float2bfloat16_rn(p[MLP_OFF_W1 + (l - 1) * MLP_LAYER_STRIDE + out * 128 + in]);
        } else {            // W4^T [128 in][16 out]
            const int q = j - 3 * n_w, in = q / 16, out = q % 16;
            wt[j] = __float2bfloat16_rn(out < 3 ? p[MLP_OFF_W4 + out * 128 + in] : 0.0f);
        }
    } else if (i < n_tiles + n_t + 528) {
        const int j = i - n_tiles - n_t;     // biases b0..b3, then b4 padded to 16
        float v;
        if (j < 512)
            v = p[MLP_OFF_B0 + (j / 128) * MLP_LAYER_STRIDE + (j % 128)];
        else
            v = j - 512 < 3 ? p[MLP_OFF_B4 + (j - 512)] : 0.0f;
        reinterpret_cast<float *>(tiles + 106496)[j] = v;
    }
    (void)n_k;
}

}  // namespace

cudaError_t launch_mlp_refresh(lcs_mlp *m, cudaStream_t s)
{
    const int total = (128 * 16 + 3 * 128 * 128 + 16 * 128) + (3 * 128 * 128 + 128 * 16) + 528;
    mlp_refresh_kernel<<<(total + 255) / 256, 256, 0, s>>>(m->d_params, m->d_tiles, m->d_wk, m->d_wt);
    return cudaGetLastError();
}

static bool desc_ok(const lcs_mlp_desc *d)
{
    return d && isfinite(d->center[0]) && isfinite(d->center[1]) && isfinite(d->kx) && isfinite(d->ky) &&
           isfinite(d->omega) && d->tau > 0.0 && isfinite(d->tau) && d->out_scale > 0.0 && isfinite(d->out_scale);
}

extern "C" lcs_status lcs_mlp_create(lcs_ctx *ctx, const lcs_mlp_desc *d, const float *params, int on_device,
                                     lcs_mlp **out)
{
    if (!ctx) return LCS_EINVAL;
    if (!out || !params) return lcs_fail(ctx, LCS_EINVAL, "lcs_mlp_create: null argument");
    *out = nullptr;
    if (!desc_ok(d)) return lcs_fail(ctx, LCS_EINVAL, "lcs_mlp_create: descriptor (tau, out_scale > 0, finite)");
    LCS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    lcs_mlp *m = new (std::nothrow) lcs_mlp();
    if (!m) return lcs_fail(ctx, LCS_ENOMEM, "host allocation");
    m->uid = lcs_next_uid();
    m->ctx = ctx;
    m->d = *d;
    const size_t pb = sizeof(float) * MLP_NPARAMS;
    cudaError_t e = cudaMalloc(&m->d_params, pb);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_m, pb);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_v, pb);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_grad, pb);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_tiles, MLP_TILE_BYTES);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_wk, sizeof(__nv_bfloat16) * (128 * 16 + 3 * 128 * 128 + 16 * 128));
    if (e == cudaSuccess) e = cudaMalloc(&m->d_wt, sizeof(__nv_bfloat16) * (3 * 128 * 128 + 128 * 16));
    if (e == cudaSuccess) e = cudaMemsetAsync(m->d_m, 0, pb, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->d_v, 0, pb, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->d_params, params, pb, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            ctx->stream);
    if (e == cudaSuccess) e = launch_mlp_refresh(m, ctx->stream);
    if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        lcs_mlp_free(m);
        return lcs_fail(ctx, e == cudaErrorMemoryAllocation ? LCS_ENOMEM : LCS_ECUDA, "lcs_mlp_create: %s",
                        cudaGetErrorString(e));
    }
    *out = m;
    return LCS_OK;
}

extern "C" lcs_status lcs_mlp_set_params(lcs_ctx *ctx, lcs_mlp *m, const float *params, int on_device)
{
    if (!ctx) return LCS_EINVAL;
    if (!m || !params) return lcs_fail(ctx, LCS_EINVAL, "lcs_mlp_set_params: null argument");
    LCS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    LCS_CUDA_TRY(ctx, cudaMemcpyAsync(m->d_params, params, sizeof(float) * MLP_NPARAMS,
                                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
    LCS_CUDA_TRY(ctx, cudaMemsetAsync(m->d_m, 0, sizeof(float) * MLP_NPARAMS, ctx->stream));
    LCS_CUDA_TRY(ctx, cudaMemsetAsync(m->d_v, 0, sizeof(float) * MLP_NPARAMS, ctx->stream));
    m->adam_steps = 0;
    LCS_CUDA_TRY(ctx, launch_mlp_refresh(m, ctx->stream));
    if (!on_device) LCS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return LCS_OK;
}

extern "C" lcs_status lcs_mlp_get_params(lcs_ctx *ctx, const lcs_mlp *m, float *params, int on_device)
{
    if (!ctx) return LCS_EINVAL;
    if (!m || !params) return lcs_fail(ctx, LCS_EINVAL, "lcs_mlp_get_params: null argument");
    LCS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    LCS_CUDA_TRY(ctx, cudaMemcpyAsync(params, m->d_params, sizeof(float) * MLP_NPARAMS,
                                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    if (!on_device) LCS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return LCS_OK;
}

extern "C" void lcs_mlp_free(lcs_mlp *m)
{
    if (!m) return;
    if (m->ctx) cudaSetDevice(m->ctx->device);
    cudaFree(m->d_params);
    cudaFree(m->d_m);
    cudaFree(m->d_v);
    cudaFree(m->d_grad);
    cudaFree(m->d_tiles);
    cudaFree(m->d_wk);
    cudaFree(m->d_wt);
    cudaFree(m->d_work);
    delete m;
}

extern "C" lcs_status lcs_mlp_forward(lcs_ctx *ctx, const lcs_mlp *m, long long n, const float *xyt, float *out,
                                      int on_device)
{
    if (!ctx) return LCS_EINVAL;
    if (!m || (n > 0 && (!xyt || !out))) return lcs_fail(ctx, LCS_EINVAL, "lcs_mlp_forward: null argument");
    if (n < 0) return lcs_fail(ctx, LCS_EINVAL, "lcs_mlp_forward: n < 0");
    if (n == 0) return LCS_OK;
    LCS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    float *din = nullptr, *dout = nullptr;
    const float *src = xyt;
    float *dst = out;
    if (!on_device) {
        LCS_CUDA_TRY(ctx, cudaMallocAsync((void **)&din, sizeof(float) * 3 * n, ctx->stream));
        LCS_CUDA_TRY(ctx, cudaMallocAsync((void **)&dout, sizeof(float) * 3 * n, ctx->stream));
        LCS_CUDA_TRY(ctx, cudaMemcpyAsync(din, xyt, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, ctx->stream));
        src = din;
        dst = dout;
    }
    MlpStepArgs A;
    A.tiles = m->d_tiles;
    A.x = src;
    A.stride = n;
    A.n = n;
    A.t = src + 2 * n;
    A.t_uniform = 0.0f;
    A.cx = (float)m->d.center[0];
    A.cy = (float)m->d.center[1];
    A.kx = (float)m->d.kx;
    A.ky = (float)m->d.ky;
    A.omega = (float)m->d.omega;
    A.out_scale = (float)m->d.out_scale;
    A.mode = 0;
    A.out0 = dst;
    A.out1 = dst + n;
    A.out2 = dst + 2 * n;
    A.errword = ctx->d_errword;
    cudaError_t e = launch_mlp_step(A, ctx->num_sms, ctx->stream);
    if (e == cudaSuccess && !on_device)
        e = cudaMemcpyAsync(out, dout, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, ctx->stream);
    if (din) cudaFreeAsync(din, ctx->stream);
    if (dout) cudaFreeAsync(dout, ctx->stream);
    if (e != cudaSuccess) return lcs_fail(ctx, LCS_ECUDA, "lcs_mlp_forward: %s", cudaGetErrorString(e));
    if (!on_device) return lcs_synchronize(ctx);
    return LCS_OK;
}

// ------------------------------------------------------------------ gated advection

lcs_status advect_surrogate(lcs_ctx *ctx, const lcs_field *f, const lcs_seeds *s, const lcs_advect_opts *o,
                            lcs_flowmap *fm)
{
    const lcs_mlp *m = (const lcs_mlp *)o->surrogate;
    if (!m) return lcs_fail(ctx, LCS_EINVAL, "lcs_advect: LCS_SURROGATE needs opts->surrogate (an lcs_mlp)");
    if (f->kind != LCS_RECTILINEAR || f->dim != 2 || f->periodic[0] || f->periodic[1])
        return lcs_fail(ctx, LCS_EUNSUPPORTED, "lcs_advect: the surrogate runs on 2D non-periodic rectilinear fields");
    if (o->njobs > 1) return lcs_fail(ctx, LCS_EUNSUPPORTED, "lcs_advect: the surrogate integrates one job per call");
    const double tau = m->d.tau, adt = fabs(o->dt), T = o->T;
    const double rk = T / tau, rs = tau / adt;
    const long long K = (long long)floor(rk + 0.5), S = (long long)floor(rs + 0.5);
    if (!(T > 0.0) || !(adt > 0.0) || K < 1 || fabs(rk - K) > 1e-9 * rk || S < 1 || fabs(rs - S) > 1e-9 * rs ||
        K * S > (1LL << 30))
        return lcs_fail(ctx, LCS_EINVAL, "lcs_advect: the surrogate needs T = K tau (K >= 1) and tau = S dt, T > 0");
    if (!isfinite(o->t0)) return lcs_fail(ctx, LCS_EINVAL, "lcs_advect: t0 must be finite");
    const long long N = s->N;
    const long long ngrp = (N + 31) / 32;
    JobTable *J = new (std::nothrow) JobTable();
    if (!J) return lcs_fail(ctx, LCS_ENOMEM, "host allocation");
    J->njobs = 1;
    J->nsteps_max = (int)(K * S);
    J->t0[0] = o->t0;
    J->T[0] = T;
    J->h[0] = adt;
    J->nsteps[0] = (int)(K * S);
    J->order[0] = 0;
    fm->T[0] = T;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t sched_b = al(sizeof(SchedEntry) * 3 * (size_t)K * S);
    const size_t need = sched_b + al(sizeof(float) * 3 * N) + al(sizeof(float) * 2 * N) + al(ngrp) + 8 * al(64);
    LCS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    lcs_status st = lcs_scratch_reserve(ctx, need);
    if (st != LCS_OK) {
        delete J;
        return st;
    }
    if (!fm->d_steps) LCS_CUDA_TRY(ctx, cudaMalloc(&fm->d_steps, sizeof(int) * (size_t)fm->N * fm->njobs));
    char *p = (char *)ctx->d_scratch;
    SchedEntry *sched = (SchedEntry *)p;
    p += sched_b;
    float *xp = (float *)p;
    p += al(sizeof(float) * 3 * N);
    float *cxy = (float *)p;   // the tracer state's carried rounding (rk4_advance)
    p += al(sizeof(float) * 2 * N);
    unsigned char *flag = (unsigned char *)p;
    p += al(ngrp);
    JobDev D;
    D.nsteps = (int *)p;
    p += al(64);
    D.h = (float *)p;
    p += al(64);
    D.t0 = (float *)p;
    p += al(64);
    D.tend = (float *)p;
    p += al(64);
    D.order = nullptr;
    D.t0d = nullptr;
    D.Td = nullptr;
    D.absT = fm->d_absT;
    cudaError_t e = launch_rk4_schedule(f->d_times, f->nframes, f->time_periodic, f->period, *J, D, sched, ctx->stream);
    delete J;
    // tracer state: the flow map starts at the seeds, OK, exit time t0 + T, no fallbacks
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(fm->d_xyz, s->d_xyz, sizeof(float) * 2 * N, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(cxy, 0, sizeof(float) * 2 * N, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(fm->d_status, LCS_TRACER_OK, N, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(fm->d_steps, 0, sizeof(int) * N, ctx->stream);
    if (e == cudaSuccess) e = launch_fill_f32(fm->d_texit, N, (float)(o->t0 + T), ctx->stream);
    const float h32 = (float)adt, t032 = (float)o->t0;
    for (long long k = 0; k < K && e == cudaSuccess; ++k) {
        MlpStepArgs A;
        A.tiles = m->d_tiles;
        A.x = fm->d_xyz;
        A.stride = N;
        A.n = N;
        A.t = nullptr;
        A.t_uniform = (float)(o->t0 + (double)k * tau);
        A.cx = (float)m->d.center[0];
        A.cy = (float)m->d.center[1];
        A.kx = (float)m->d.kx;
        A.ky = (float)m->d.ky;
        A.omega = (float)m->d.omega;
        A.out_scale = (float)m->d.out_scale;
        A.mode = 1;
        A.out0 = xp;
        A.out1 = xp + N;
        A.out2 = xp + 2 * N;
        A.errword = ctx->d_errword;
        lcs_tm_begin(ctx, 0, ctx->stream);
        e = launch_mlp_step(A, ctx->num_sms, ctx->stream);
        lcs_tm_end(ctx, 0, ctx->stream);
        if (e != cudaSuccess) break;
        SurGateArgs G;
        G.n = N;
        G.step = (int)k;
        G.S = (int)S;
        G.h = h32;
        G.t0 = t032;
        G.tol = (float)o->gate_tol;
        G.log_tol = o->gate_tol > 0 ? (float)log10(o->gate_tol) : -INFINITY;
        G.rho = xp + 2 * N;
        G.xp = xp;
        G.xyz = fm->d_xyz;
        G.cxy = cxy;
        G.status = fm->d_status;
        G.texit = fm->d_texit;
        G.counts = fm->d_steps;
        G.flag = flag;
        G.sched = sched;
        G.errword = ctx->d_errword;
        lcs_tm_begin(ctx, 1, ctx->stream);
        e = launch_sur_gate(G, f, ctx->stream);
        lcs_tm_end(ctx, 1, ctx->stream);
    }
    if (e == cudaSuccess) e = launch_settle_f32(fm->d_xyz, cxy, 2 * N, ctx->stream);
    if (e != cudaSuccess) return lcs_fail(ctx, LCS_ECUDA, "lcs_advect (surrogate): %s", cudaGetErrorString(e));
    return LCS_OK;
}

// ------------------------------------------------------------------ training

extern "C" lcs_status lcs_mlp_loss_grad(lcs_ctx *ctx, lcs_mlp *m, long long n, const float *xyt, const float *disp,
                                        double rho_weight, float *grads, double *loss, int on_device)
{
    if (!ctx) return LCS_EINVAL;
    if (!m || !xyt || !disp) return lcs_fail(ctx, LCS_EINVAL, "lcs_mlp_loss_grad: null argument");
    if (n <= 0 || n % 128) return lcs_fail(ctx, LCS_EINVAL, "lcs_mlp_loss_grad: n must be a positive multiple of 128");
    if (!(rho_weight >= 0.0) || !isfinite(rho_weight))
        return lcs_fail(ctx, LCS_EINVAL, "lcs_mlp_loss_grad: rho_weight must be finite and >= 0");
    LCS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const float *dx = xyt, *dd = disp;
    float *tmp = nullptr;
    double *dl = nullptr;
    if (!on_device) {
        LCS_CUDA_TRY(ctx, cudaMallocAsync((void **)&tmp, sizeof(float) * 5 * n, ctx->stream));
        LCS_CUDA_TRY(ctx, cudaMemcpyAsync(tmp, xyt, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, ctx->stream));
        LCS_CUDA_TRY(ctx, cudaMemcpyAsync(tmp + 3 * n, disp, sizeof(float) * 2 * n, cudaMemcpyHostToDevice, ctx->stream));
        dx = tmp;
        dd = tmp + 3 * n;
    }
    LCS_CUDA_TRY(ctx, cudaMallocAsync((void **)&dl, sizeof(double), ctx->stream));
    cudaError_t e = mlp_loss_grad(m, dx, n, dd, n, n, (float)rho_weight, ctx->num_sms, ctx->d_errword, dl, ctx->stream);
    double lsum = 0.0;
    if (e == cudaSuccess && grads)
        e = cudaMemcpyAsync(grads, m->d_grad, sizeof(float) * MLP_NPARAMS,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && loss) e = cudaMemcpyAsync(&lsum, dl, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && loss) e = cudaStreamSynchronize(ctx->stream);
    if (tmp) cudaFreeAsync(tmp, ctx->stream);
    cudaFreeAsync(dl, ctx->stream);
    if (e != cudaSuccess) return lcs_fail(ctx, LCS_ECUDA, "lcs_mlp_loss_grad: %s", cudaGetErrorString(e));
    if (loss) *loss = lsum / (double)n;
    if (!on_device) return lcs_synchronize(ctx);
    return LCS_OK;
}

extern "C" lcs_status lcs_mlp_adam(lcs_ctx *ctx, lcs_mlp *m, const float *grads, int on_device, double lr, double beta1,
                                   double beta2, double eps)
{
    if (!ctx) return LCS_EINVAL;
    if (!m) return lcs_fail(ctx, LCS_EINVAL, "lcs_mlp_adam: null network");
    if (!(lr >= 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0))
        return lcs_fail(ctx, LCS_EINVAL, "lcs_mlp_adam: lr >= 0, 0 <= beta < 1, eps > 0");
    LCS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const float *g = m->d_grad;
    float *tmp = nullptr;
    if (grads && !on_device) {
        LCS_CUDA_TRY(ctx, cudaMallocAsync((void **)&tmp, sizeof(float) * MLP_NPARAMS, ctx->stream));
        LCS_CUDA_TRY(ctx, cudaMemcpyAsync(tmp, grads, sizeof(float) * MLP_NPARAMS, cudaMemcpyHostToDevice, ctx->stream));
        g = tmp;
    } else if (grads) {
        g = grads;
    }
    cudaError_t e = mlp_adam(m, g, lr, beta1, beta2, eps, ctx->stream);
    if (tmp) cudaFreeAsync(tmp, ctx->stream);
    if (e != cudaSuccess) return lcs_fail(ctx, LCS_ECUDA, "lcs_mlp_adam: %s", cudaGetErrorString(e));
    if (grads && !on_device) return lcs_synchronize(ctx);
    return LCS_OK;
}

extern "C" lcs_status lcs_surrogate_train(lcs_ctx *ctx, const lcs_field *f, lcs_mlp *m, const lcs_train_desc *d,
                                          long long ns, const float *samples, int on_device, double *loss_per_epoch)
{
    if (!ctx) return LCS_EINVAL;
    if (!f || !m || !d || !samples) return lcs_fail(ctx, LCS_EINVAL, "lcs_surrogate_train: null argument");
    if (f->kind != LCS_RECTILINEAR || f->dim != 2)
        return lcs_fail(ctx, LCS_EUNSUPPORTED, "lcs_surrogate_train: 2D rectilinear fields");
    const long long B = d->batch;
    if (B <= 0 || B % 128 || ns < B || d->epochs < 1)
        return lcs_fail(ctx, LCS_EINVAL, "lcs_surrogate_train: batch a positive multiple of 128, ns >= batch, epochs >= 1");
    const double rs = m->d.tau / d->dt;
    const long long S = (long long)floor(rs + 0.5);
    if (!(d->dt > 0.0) || S < 1 || fabs(rs - S) > 1e-9 * rs || S > (1 << 20))
        return lcs_fail(ctx, LCS_EINVAL, "lcs_surrogate_train: tau must be a multiple of dt > 0");
    if (!(d->lr >= 0.0) || !(d->lr_min >= 0.0) || !(d->beta1 >= 0.0 && d->beta1 < 1.0) ||
        !(d->beta2 >= 0.0 && d->beta2 < 1.0) || !(d->eps > 0.0) || !(d->rho_weight >= 0.0))
        return lcs_fail(ctx, LCS_EINVAL, "lcs_surrogate_train: optimiser settings");
    LCS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const long long nb = ns / B, total = nb * d->epochs;
    float *xs = nullptr, *disp = nullptr;
    double *losses = nullptr;
    LCS_CUDA_TRY(ctx, cudaMallocAsync((void **)&disp, sizeof(float) * 2 * ns, ctx->stream));
    LCS_CUDA_TRY(ctx, cudaMallocAsync((void **)&losses, sizeof(double) * total, ctx->stream));
    const float *xyt = samples;
    if (!on_device) {
        LCS_CUDA_TRY(ctx, cudaMallocAsync((void **)&xs, sizeof(float) * 3 * ns, ctx->stream));
        LCS_CUDA_TRY(ctx, cudaMemcpyAsync(xs, samples, sizeof(float) * 3 * ns, cudaMemcpyHostToDevice, ctx->stream));
        xyt = xs;
    }
    // integrator targets: RK4 displacement over tau from every sample
    cudaError_t e = mlp_targets(f, xyt, ns, (int)S, d->dt, disp, ctx->stream);
    if (e == cudaSuccess) e = mlp_reserve(m, B, ctx->stream);
    for (long long it = 0; it < total && e == cudaSuccess; ++it) {
        const long long b = it % nb;
        e = mlp_loss_grad(m, xyt + b * B, ns, disp + b * B, ns, B, (float)d->rho_weight, ctx->num_sms, ctx->d_errword,
                          losses + it, ctx->stream);
        if (e != cudaSuccess) break;
        const double lr = d->lr_min + 0.5 * (d->lr - d->lr_min) * (1.0 + cos(M_PI * (double)it / (double)total));
        e = mlp_adam(m, m->d_grad, lr, d->beta1, d->beta2, d->eps, ctx->stream);
    }
    std::vector<double> h;
    if (e == cudaSuccess && loss_per_epoch) {
        h.resize((size_t)total);
        e = cudaMemcpyAsync(h.data(), losses, sizeof(double) * total, cudaMemcpyDeviceToHost, ctx->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFreeAsync(disp, ctx->stream);
    cudaFreeAsync(losses, ctx->stream);
    if (xs) cudaFreeAsync(xs, ctx->stream);
    if (e != cudaSuccess) return lcs_fail(ctx, LCS_ECUDA, "lcs_surrogate_train: %s", cudaGetErrorString(e));
    if (loss_per_epoch)
        for (int ep = 0; ep < d->epochs; ++ep) {
            double s = 0.0;
            for (long long b = 0; b < nb; ++b) s += h[(size_t)(ep * nb + b)];
            loss_per_epoch[ep] = s / (double)(nb * B);
        }
    return lcs_synchronize(ctx);
}
