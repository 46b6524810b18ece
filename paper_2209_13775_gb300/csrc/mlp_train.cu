// mlp_train.cu -- training of the surrogate network: integrator targets, loss and
// gradients (reverse mode, layer by layer), Adam.
//
// A batch of B samples (B a multiple of 128) runs forward as four GEMMs into FP32
// pre-activations Z_l, each followed by a bias + SiLU kernel that writes the BF16
// activations H_{l+1} and their transposes, then the output GEMM and the loss kernel.
// Backward: the output layer's weight gradient by a SIMT reduction (3 rows), then per
// hidden layer dZ = dH * SiLU'(Z) (BF16, plus its transpose and the bias gradient),
// dW_l = dZ^T H_l as a split-K GEMM over the batch, and dH = dZ W_l.  Every GEMM runs
// on the tcgen05 tensor cores (mlp_gemm.cu) with BF16 operands and FP32 accumulation.
#include "mlp_internal.cuh"
#include "rect_device.cuh"

#include <math.h>

#include <new>

namespace {

__device__ __forceinline__ float tanh_a(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// SiLU of a pair of pre-activations exactly as the inference kernel computes it: h = z/2 rounded to
// BF16, then h + h tanh(h) in packed BF16 arithmetic
__device__ __forceinline__ __nv_bfloat162 silu_pair(float z0, float z1)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(0.5f * z0, 0.5f * z1);
    uint32_t hu = *reinterpret_cast<uint32_t *>(&h), t, d;
    asm("tanh.approx.bf16x2 %0, %1;" : "=r"(t) : "r"(hu));
    asm("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(hu), "r"(t), "r"(hu));
    return *reinterpret_cast<__nv_bfloat162 *>(&d);
}

__device__ __forceinline__ float silu_grad_f(float z)
{
    const float s = fmaf(0.5f, tanh_a(0.5f * z), 0.5f);
    return s * fmaf(z, 1.0f - s, 1.0f);
}

struct FeatParams {
    float cx, cy, kx, ky, omega;
};

// phi [B][16] and phi^T [16][B] (BF16) of the samples (x, y, t) [3][stride] from offset 0
__global__ void tr_features_kernel(const float *__restrict__ xyt, long long stride, long long B, FeatParams F,
                                   __nv_bfloat16 *__restrict__ phi, __nv_bfloat16 *__restrict__ phiT)
{
    const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (b >= B) return;
    const float x = xyt[b], y = xyt[stride + b], t = xyt[2 * stride + b];
    float sw, cw, sx, cx, sy, cy;
    sincosf(F.omega * t, &sw, &cw);
    sincosf(F.kx * x, &sx, &cx);
    sincosf(F.ky * y, &sy, &cy);
    const float f[7] = {x - F.cx, y - F.cy, sw, cw, sx, cx, sy};
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const __nv_bfloat16 v = __float2bfloat16_rn(k < 7 ? f[k] : 0.0f);
        phi[b * 16 + k] = v;
        phiT[(long long)k * B + b] = v;
    }
}

// Z += bias (in place, FP32); H = BF16(SiLU(Z)) [B][128] and H^T [128][B].  Block: 32 rows.
__global__ void __launch_bounds__(256) tr_silu_kernel(float *__restrict__ Z, const float *__restrict__ bias, long long B,
                                                      __nv_bfloat16 *__restrict__ H, __nv_bfloat16 *__restrict__ HT)
{
    __shared__ __nv_bfloat16 tile[128][34];
    const long long r0 = (long long)blockIdx.x * 32;
    for (int e = threadIdx.x; e < 32 * 64; e += 256) {
        const int rr = e >> 6, c = (e & 63) * 2;
        const long long row = r0 + rr;
        if (row >= B) continue;
        const float z0 = Z[row * 128 + c] + bias[c], z1 = Z[row * 128 + c + 1] + bias[c + 1];
        Z[row * 128 + c] = z0;
        Z[row * 128 + c + 1] = z1;
        const __nv_bfloat162 h = silu_pair(z0, z1);
        *reinterpret_cast<__nv_bfloat162 *>(H + row * 128 + c) = h;
        tile[c][rr] = h.x;
        tile[c + 1][rr] = h.y;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * 128; e += 256) {
        const int c = e >> 5, rr = e & 31;
        if (r0 + rr < B) HT[(long long)c * B + r0 + rr] = tile[c][rr];
    }
}

// loss and dL/do per sample; dO (BF16 [B][16], zero beyond column 2) and dOf (FP32 [B][3])
__global__ void __launch_bounds__(256) tr_loss_kernel(const float *__restrict__ O, const float *__restrict__ b4,
                                                      const float *__restrict__ disp, long long dstride, long long B,
                                                      float s, float wr, __nv_bfloat16 *__restrict__ dO,
                                                      float *__restrict__ dOf, double *__restrict__ loss)
{
    const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double l = 0.0;
    if (b < B) {
        const float o0 = O[b * 16] + b4[0], o1 = O[b * 16 + 1] + b4[1], o2 = O[b * 16 + 2] + b4[2];
        const float dx = disp[b], dy = disp[dstride + b];
        const float e0 = o0 - dx / s, e1 = o1 - dy / s;
        const float px = fmaf(s, o0, -dx), py = fmaf(s, o1, -dy);
        const float rt = log10f(sqrtf(px * px + py * py) + 1e-7f);
        const float er = o2 - rt;
        l = (double)e0 * e0 + (double)e1 * e1 + (double)wr * er * er;
        const float inv = 1.0f / (float)B;
        const float g0 = 2.0f * e0 * inv, g1 = 2.0f * e1 * inv, g2 = 2.0f * wr * er * inv;
        dOf[b * 3] = g0;
        dOf[b * 3 + 1] = g1;
        dOf[b * 3 + 2] = g2;
#pragma unroll
        for (int k = 0; k < 16; ++k) dO[b * 16 + k] = __float2bfloat16_rn(k == 0 ? g0 : k == 1 ? g1 : k == 2 ? g2 : 0.0f);
    }
    // block sum of the per-sample losses
    for (int off = 16; off > 0; off >>= 1) l += __shfl_down_sync(0xffffffffu, l, off);
    __shared__ double part[8];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        atomicAdd(loss, t);
    }
}

// output layer: dW4[j][k] = sum_b dO[b][j] H4[b][k], db4[j] = sum_b dO[b][j]; thread k, block = row chunk
__global__ void __launch_bounds__(128) tr_out_grad_kernel(const float *__restrict__ dOf,
                                                          const __nv_bfloat16 *__restrict__ H4, long long B,
                                                          long long rows_per_block, float *__restrict__ grad)
{
    const int k = threadIdx.x;
    const long long b0 = blockIdx.x * rows_per_block;
    const long long b1 = b0 + rows_per_block < B ? b0 + rows_per_block : B;
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, s0 = 0.0f, s1 = 0.0f, s2 = 0.0f;
    for (long long b = b0; b < b1; ++b) {
        const float h = __bfloat162float(H4[b * 128 + k]);
        const float g0 = dOf[b * 3], g1 = dOf[b * 3 + 1], g2 = dOf[b * 3 + 2];
        a0 = fmaf(g0, h, a0);
        a1 = fmaf(g1, h, a1);
        a2 = fmaf(g2, h, a2);
        s0 += g0;
        s1 += g1;
        s2 += g2;
    }
    atomicAdd(grad + MLP_OFF_W4 + k, a0);
    atomicAdd(grad + MLP_OFF_W4 + 128 + k, a1);
    atomicAdd(grad + MLP_OFF_W4 + 256 + k, a2);
    if (k == 0) {
        atomicAdd(grad + MLP_OFF_B4, s0);
        atomicAdd(grad + MLP_OFF_B4 + 1, s1);
        atomicAdd(grad + MLP_OFF_B4 + 2, s2);
    }
}

// dZ = dH * SiLU'(Z): BF16 [B][128] and its transpose; bias gradient (column sums) into db
__global__ void __launch_bounds__(256) tr_silu_grad_kernel(const float *__restrict__ dH, const float *__restrict__ Z,
                                                           long long B, __nv_bfloat16 *__restrict__ dZ,
                                                           __nv_bfloat16 *__restrict__ dZT, float *__restrict__ db)
{
    __shared__ __nv_bfloat16 tile[128][34];
    __shared__ float csum[2][128];
    const long long r0 = (long long)blockIdx.x * 32;
    float acc = 0.0f;  // this thread's column is (threadIdx.x & 127), rows of parity (threadIdx.x >> 7)
    for (int e = threadIdx.x; e < 32 * 128; e += 256) {
        const int rr = e >> 7, c = e & 127;
        const long long row = r0 + rr;
        float g = 0.0f;
        if (row < B) g = dH[row * 128 + c] * silu_grad_f(Z[row * 128 + c]);
        acc += g;
        const __nv_bfloat16 v = __float2bfloat16_rn(g);
        if (row < B) dZ[row * 128 + c] = v;
        tile[c][rr] = v;
    }
    csum[threadIdx.x >> 7][threadIdx.x & 127] = acc;
    __syncthreads();
    if (threadIdx.x < 128) atomicAdd(db + threadIdx.x, csum[0][threadIdx.x] + csum[1][threadIdx.x]);
    for (int e = threadIdx.x; e < 32 * 128; e += 256) {
        const int c = e >> 5, rr = e & 31;
        if (r0 + rr < B) dZT[(long long)c * B + r0 + rr] = tile[c][rr];
    }
}

// dW0 from the padded [128][16] GEMM result into the packed [128][7] gradient
__global__ void tr_dw0_kernel(const float *__restrict__ tmp, float *__restrict__ grad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 128 * 7) grad[MLP_OFF_W0 + i] = tmp[(i / 7) * 16 + (i % 7)];
}

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int n, float lr, float b1, float b2, float eps, float bc1, float bc2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
    const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

// RK4 displacement over tau of each sample (x0, y0, t0), steps of dt; frame times FP32 in smem
template <int ST>
__global__ void __launch_bounds__(256) tr_targets_kernel(RectParams P, const char *__restrict__ frames, size_t fstride,
                                                         const double *__restrict__ times, int nf, int tp, float period,
                                                         const float *__restrict__ xyt, long long n, int S, float h,
                                                         float *__restrict__ disp)
{
    extern __shared__ float s_t[];
    for (int q = threadIdx.x; q < nf; q += blockDim.x) s_t[q] = (float)times[q];
    __syncthreads();
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float x[2] = {xyt[i], xyt[n + i]}, cx[2] = {0.0f, 0.0f};
    const float t0 = xyt[2 * n + i];
    auto bracket = [&](float t, int &k, float &a) {
        if (nf <= 1) {
            k = 0;
            a = 0.0f;
            return;
        }
        float tt = t;
        if (tp) tt = t - period * floorf((t - s_t[0]) / period);
        int lo = 0, hi = nf - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_t[mid] <= tt)
                lo = mid;
            else
                hi = mid - 1;
        }
        k = lo < nf - 2 ? lo : nf - 2;
        a = (tt - s_t[k]) / (s_t[k + 1] - s_t[k]);
        if (!tp) a = fminf(fmaxf(a, 0.0f), 1.0f);
    };
    for (int s = 0; s < S; ++s) {
        const float ts = fmaf((float)s, h, t0);
        int k0, k1, k2;
        float a0, a1, a2;
        bracket(ts, k0, a0);
        bracket(ts + 0.5f * h, k1, a1);
        bracket(ts + h, k2, a2);
        rk4_step<2, ST, SRC_GLOBAL>(P, x, cx, h, frames + (size_t)k0 * fstride, frames + (size_t)(k0 + 1) * fstride,
                                    a0, frames + (size_t)k1 * fstride, frames + (size_t)(k1 + 1) * fstride, a1,
                                    frames + (size_t)k2 * fstride, frames + (size_t)(k2 + 1) * fstride, a2);
    }
    disp[i] = (x[0] - xyt[i]) + cx[0];
    disp[n + i] = (x[1] - xyt[n + i]) + cx[1];
}

size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// work space carve-up for a batch capacity of B samples
struct Work {
    __nv_bfloat16 *phi, *phiT, *H[5], *HT[5], *dO, *dZ, *dZT;
    float *Z[4], *O, *dOf, *dH, *dw0;
    double *loss;
};

size_t work_bytes(long long B)
{
    size_t b = 0;
    b += 2 * al256(sizeof(__nv_bfloat16) * 16 * B);        // phi, phiT
    b += 8 * al256(sizeof(__nv_bfloat16) * 128 * B);       // H1..H4, HT1..HT4
    b += al256(sizeof(__nv_bfloat16) * 16 * B);            // dO
    b += 2 * al256(sizeof(__nv_bfloat16) * 128 * B);       // dZ, dZT
    b += 4 * al256(sizeof(float) * 128 * B);               // Z0..Z3
    b += al256(sizeof(float) * 16 * B) + al256(sizeof(float) * 3 * B) + al256(sizeof(float) * 128 * B);
    b += al256(sizeof(float) * 128 * 16) + al256(sizeof(double));
    return b;
}

Work carve(void *base, long long B)
{
    Work w;
    char *p = (char *)base;
    auto take = [&](size_t bytes) {
        char *q = p;
        p += al256(bytes);
        return q;
    };
    w.phi = (__nv_bfloat16 *)take(sizeof(__nv_bfloat16) * 16 * B);
    w.phiT = (__nv_bfloat16 *)take(sizeof(__nv_bfloat16) * 16 * B);
    w.H[0] = w.phi;
    w.HT[0] = w.phiT;
    for (int l = 1; l <= 4; ++l) {
        w.H[l] = (__nv_bfloat16 *)take(sizeof(__nv_bfloat16) * 128 * B);
        w.HT[l] = (__nv_bfloat16 *)take(sizeof(__nv_bfloat16) * 128 * B);
    }
    w.dO = (__nv_bfloat16 *)take(sizeof(__nv_bfloat16) * 16 * B);
    w.dZ = (__nv_bfloat16 *)take(sizeof(__nv_bfloat16) * 128 * B);
    w.dZT = (__nv_bfloat16 *)take(sizeof(__nv_bfloat16) * 128 * B);
    for (int l = 0; l < 4; ++l) w.Z[l] = (float *)take(sizeof(float) * 128 * B);
    w.O = (float *)take(sizeof(float) * 16 * B);
    w.dOf = (float *)take(sizeof(float) * 3 * B);
    w.dH = (float *)take(sizeof(float) * 128 * B);
    w.dw0 = (float *)take(sizeof(float) * 128 * 16);
    w.loss = (double *)take(sizeof(double));
    return w;
}

}  // namespace

// offsets of the trainer's BF16 operands inside lcs_mlp::d_wk / d_wt
static const __nv_bfloat16 *wk_layer(const lcs_mlp *m, int l)
{
    return l == 0 ? m->d_wk : l < 4 ? m->d_wk + 128 * 16 + (size_t)(l - 1) * 128 * 128 : m->d_wk + 128 * 16 + 3 * 128 * 128;
}

static const __nv_bfloat16 *wt_layer(const lcs_mlp *m, int l)  // l = 1..4
{
    return m->d_wt + (size_t)(l - 1) * 128 * 128;
}

cudaError_t mlp_reserve(lcs_mlp *m, long long B, cudaStream_t s)
{
    if (B <= m->cap) return cudaSuccess;
    if (m->d_work) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
        cudaFree(m->d_work);
        m->d_work = nullptr;
        m->cap = 0;
    }
    cudaError_t e = cudaMalloc(&m->d_work, work_bytes(B));
    if (e == cudaSuccess) m->cap = B;
    return e;
}

// gradient of the mean loss over B samples (B a multiple of 128) into m->d_grad; loss into *d_loss
cudaError_t mlp_loss_grad(lcs_mlp *m, const float *xyt, long long xstride, const float *disp, long long dstride,
                          long long B, float rho_weight, int num_sms, unsigned *errword, double *d_loss, cudaStream_t s)
{
    cudaError_t e = mlp_reserve(m, B, s);
    if (e != cudaSuccess) return e;
    Work w = carve(m->d_work, B);
    const float *bias = m->d_params;  // biases read from the FP32 master copy
    FeatParams F{(float)m->d.center[0], (float)m->d.center[1], (float)m->d.kx, (float)m->d.ky, (float)m->d.omega};
    const unsigned g256 = (unsigned)((B + 255) / 256), g32 = (unsigned)((B + 31) / 32);
    e = cudaMemsetAsync(m->d_grad, 0, sizeof(float) * MLP_NPARAMS, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.dw0, 0, sizeof(float) * 128 * 16, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.loss, 0, sizeof(double), s);
    if (e != cudaSuccess) return e;
    tr_features_kernel<<<g256, 256, 0, s>>>(xyt, xstride, B, F, w.phi, w.phiT);
    // forward
    for (int l = 0; l < 4; ++l) {
        const int K = l == 0 ? 16 : 128;
        e = launch_gemm_bf16(w.H[l], K, wk_layer(m, l), K, w.Z[l], 128, B, 128, K, 1, 0, errword, s);
        if (e != cudaSuccess) return e;
        const float *b = bias + (l == 0 ? MLP_OFF_B0 : MLP_OFF_B0 + l * MLP_LAYER_STRIDE);
        tr_silu_kernel<<<g32, 256, 0, s>>>(w.Z[l], b, B, w.H[l + 1], w.HT[l + 1]);
    }
    e = launch_gemm_bf16(w.H[4], 128, wk_layer(m, 4), 128, w.O, 16, B, 16, 128, 1, 0, errword, s);
    if (e != cudaSuccess) return e;
    tr_loss_kernel<<<g256, 256, 0, s>>>(w.O, bias + MLP_OFF_B4, disp, dstride, B, (float)m->d.out_scale, rho_weight,
                                        w.dO, w.dOf, w.loss);
    // backward: output layer
    const long long rpb = 512;
    tr_out_grad_kernel<<<(unsigned)((B + rpb - 1) / rpb), 128, 0, s>>>(w.dOf, w.H[4], B, rpb, m->d_grad);
    e = launch_gemm_bf16(w.dO, 16, wt_layer(m, 4), 16, w.dH, 128, B, 128, 16, 1, 0, errword, s);
    if (e != cudaSuccess) return e;
    const int splits = (int)(B / 512 < num_sms ? (B / 512 > 0 ? B / 512 : 1) : num_sms);
    for (int l = 3; l >= 0; --l) {
        float *db = m->d_grad + (l == 0 ? MLP_OFF_B0 : MLP_OFF_B0 + l * MLP_LAYER_STRIDE);
        tr_silu_grad_kernel<<<g32, 256, 0, s>>>(w.dH, w.Z[l], B, w.dZ, w.dZT, db);
        if (l > 0) {
            e = launch_gemm_bf16(w.dZT, B, w.HT[l], B, m->d_grad + MLP_OFF_W1 + (l - 1) * MLP_LAYER_STRIDE, 128, 128,
                                 128, B, splits, 1, errword, s);
            if (e != cudaSuccess) return e;
            e = launch_gemm_bf16(w.dZ, 128, wt_layer(m, l), 128, w.dH, 128, B, 128, 128, 1, 0, errword, s);
        } else {
            e = launch_gemm_bf16(w.dZT, B, w.HT[0], B, w.dw0, 16, 128, 16, B, splits, 1, errword, s);
        }
        if (e != cudaSuccess) return e;
    }
    tr_dw0_kernel<<<4, 256, 0, s>>>(w.dw0, m->d_grad);
    if (d_loss) e = cudaMemcpyAsync(d_loss, w.loss, sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}

cudaError_t mlp_adam(lcs_mlp *m, const float *grad, double lr, double b1, double b2, double eps, cudaStream_t s)
{
    m->adam_steps += 1;
    const double bc1 = 1.0 - pow(b1, (double)m->adam_steps), bc2 = 1.0 - pow(b2, (double)m->adam_steps);
    adam_kernel<<<(MLP_NPARAMS + 255) / 256, 256, 0, s>>>(m->d_params, grad, m->d_m, m->d_v, MLP_NPARAMS, (float)lr,
                                                         (float)b1, (float)b2, (float)eps, (float)bc1, (float)bc2);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_mlp_refresh(m, s);
    return e;
}

cudaError_t mlp_targets(const lcs_field *f, const float *xyt, long long n, int S, double dt, float *disp, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const RectParams P = make_rect_params(f);
    const size_t smem = sizeof(float) * (size_t)(f->nframes > 0 ? f->nframes : 1);
    const unsigned grid = (unsigned)((n + 255) / 256);
    const float h = (float)dt, per = (float)f->period;
    const char *fr = (const char *)f->d_frames;
    if (f->storage == LCS_F32)
        tr_targets_kernel<LCS_F32><<<grid, 256, smem, s>>>(P, fr, f->frame_stride, f->d_times, f->nframes,
                                                          f->time_periodic, per, xyt, n, S, h, disp);
    else if (f->storage == LCS_F16)
        tr_targets_kernel<LCS_F16><<<grid, 256, smem, s>>>(P, fr, f->frame_stride, f->d_times, f->nframes,
                                                          f->time_periodic, per, xyt, n, S, h, disp);
    else
        tr_targets_kernel<LCS_BF16><<<grid, 256, smem, s>>>(P, fr, f->frame_stride, f->d_times, f->nframes,
                                                           f->time_periodic, per, xyt, n, S, h, disp);
    return cudaGetLastError();
}
