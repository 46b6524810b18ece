// mlp_infer.cu -- the surrogate network on the tcgen05 tensor cores, and the gated
// surrogate advection built on it.
//
// Network (7 -> 128 -> 128 -> 128 -> 128 -> 3, SiLU): per tile of 128 tracers, features
// phi(x, y, t) are rounded to BF16 into a shared-memory operand tile; each layer is one
// 128 x N x K MMA chain into a TMEM accumulator (FP32), and its epilogue adds the FP32
// bias, applies SiLU (h + h tanh(h) with h = z/2, in packed BF16 arithmetic) and writes the
// BF16 activations back as the next layer's operand.  The weights (104 KB of BF16 operand tiles) and biases stay in
// shared memory for the whole persistent launch.  Three warpgroups work on three tiles at a
// time, so each tile's epilogue overlaps the others' MMAs on the tensor core.
//
// Gated advection over one surrogate step tau (the audit of each 32-tracer group against
// the integrator of Eq. 2, and the integrator where the audit fails) runs in two SIMT
// kernels after the network: an audit kernel with one thread per group, and an apply
// kernel with one thread per tracer that either takes the proposal or integrates the
// sub-interval with the same RK4 arithmetic as the fixed-step path.
#include "mlp_internal.cuh"
#include "rect_device.cuh"
#include "tc_common.cuh"

#include <math.h>

namespace {

constexpr uint32_t OFF_W0 = 0, OFF_W1 = 4096, OFF_W2 = 36864, OFF_W3 = 69632, OFF_W4 = 102400, OFF_BIAS = 106496;
constexpr uint32_t OFF_WG = MLP_TILE_BYTES;  // per-warpgroup region: phi tile (4 KB) + activations (32 KB)
constexpr uint32_t WG_BYTES = 4096 + 32768;
constexpr int NWG = 3;  // warpgroups (tiles in flight) per CTA
constexpr uint32_t INFER_SMEM = MLP_TILE_BYTES + NWG * WG_BYTES;

__device__ __forceinline__ void wg_sync(int g) { asm volatile("bar.sync %0, 128;" ::"r"(1 + g) : "memory"); }

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

__device__ __forceinline__ uint32_t tanh_bf16x2(uint32_t h)
{
    uint32_t t;
    asm("tanh.approx.bf16x2 %0, %1;" : "=r"(t) : "r"(h));
    return t;
}

__device__ __forceinline__ uint32_t fma_bf16x2(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// one hidden layer's epilogue for tile row r: the 128 FP32 accumulator columns (all loads in
// flight before one wait), h = z/2 = acc/2 + b/2 (hb holds b/2) rounded to BF16 pairs, and
// SiLU(z) = h + h tanh(h) in packed BF16 arithmetic, stored as row r of the next operand tile
__device__ __forceinline__ void hidden_epilogue(uint32_t ta, const float *hb, unsigned char *tile, int r)
{
#pragma unroll
    for (int half = 0; half < 128; half += 64) {
        uint32_t acc[64];
        tmem_ld32_async(ta + half, acc);
        tmem_ld32_async(ta + half + 32, acc + 32);
        tmem_wait_ld32(acc);
        tmem_wait_ld32(acc + 32);
#pragma unroll
        for (int c = 0; c < 64; c += 8) {
            uint32_t w[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float h0 = fmaf(__uint_as_float(acc[c + 2 * j]), 0.5f, hb[half + c + 2 * j]);
                const float h1 = fmaf(__uint_as_float(acc[c + 2 * j + 1]), 0.5f, hb[half + c + 2 * j + 1]);
                const uint32_t h2 = pack_bf16(h0, h1);
                w[j] = fma_bf16x2(h2, tanh_bf16x2(h2), h2);
            }
            *reinterpret_cast<uint4 *>(tile + ckm_offset(128, r, half + c)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

__global__ void __launch_bounds__(NWG * 128, 1) mlp_step_kernel(MlpStepArgs A)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t bar_w, bar_g[NWG];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag[NWG];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int g = warp >> 2;           // warpgroup
    const int r = tid & 127;           // tile row = TMEM lane
    const int wq = warp & 3;
    if (tid == 0) {
        mbar_init(&bar_w, 1);
        for (int q = 0; q < NWG; ++q) {
            mbar_init(&bar_g[q], 1);
            abort_flag[q] = 0;
        }
        mbar_fence_init();
    }
    if (warp == 0) tmem_alloc(&tmem_base, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
        mbar_arrive_expect_tx(&bar_w, MLP_TILE_BYTES);
        bulk_g2s(smem, A.tiles, MLP_TILE_BYTES, &bar_w);
    }
    const bool have_w = !__syncthreads_or(!tc_wait(&bar_w, 0, A.errword));
    if (have_w) {  // hidden-layer biases are used halved (the epilogue works with z / 2)
        float *b = reinterpret_cast<float *>(smem + OFF_BIAS);
        for (int q = tid; q < 512; q += blockDim.x) b[q] *= 0.5f;
        __syncthreads();
    }
    const uint32_t tmem = tmem_base + (uint32_t)(g * 128);
    unsigned char *sPhi = smem + OFF_WG + g * WG_BYTES;
    unsigned char *sAct = sPhi + 4096;
    const float *bias = reinterpret_cast<const float *>(smem + OFF_BIAS);
    const uint32_t uPhi = smem_u32(sPhi), uAct = smem_u32(sAct), uW = smem_u32(smem);
    const uint32_t id128 = tc_idesc_bf16(128, 128), id16 = tc_idesc_bf16(128, 16);
    const long long ntiles = (A.n + 127) / 128;
    unsigned phase = 0;
    for (long long tile = (long long)blockIdx.x * NWG + g; have_w && tile < ntiles; tile += (long long)NWG * gridDim.x) {
        const long long i = tile * 128 + r;
        const bool live = i < A.n;
        float x = 0.0f, y = 0.0f, t = A.t_uniform;
        if (live) {
            x = A.x[i];
            y = A.x[A.stride + i];
            if (A.t) t = A.t[i];
        }
        {   // features -> BF16 row r of the phi tile (K = 16, columns 7..15 zero)
            float sw, cw, sx, cx, sy, cy;
            sincosf(A.omega * t, &sw, &cw);
            sincosf(A.kx * x, &sx, &cx);
            sincosf(A.ky * y, &sy, &cy);
            const uint4 lo = make_uint4(pack_bf16(x - A.cx, y - A.cy), pack_bf16(sw, cw), pack_bf16(sx, cx),
                                        pack_bf16(sy, 0.0f));
            *reinterpret_cast<uint4 *>(sPhi + ckm_offset(128, r, 0)) = lo;
            *reinterpret_cast<uint4 *>(sPhi + ckm_offset(128, r, 8)) = make_uint4(0, 0, 0, 0);
        }
        float o[3] = {0.0f, 0.0f, 0.0f};
        for (int l = 0; l < 5; ++l) {
            fence_async_smem();
            tc_fence_before();
            wg_sync(g);
            if (r == 0) {
                tc_fence_after();
                if (l == 0) {
                    tc_mma(tmem, tc_desc(uPhi, 2048, 128), tc_desc(uW + OFF_W0, 2048, 128), id128, false);
                } else {
                    const uint32_t wofs = l == 1 ? OFF_W1 : l == 2 ? OFF_W2 : l == 3 ? OFF_W3 : OFF_W4;
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk) {
                        const uint64_t ad = tc_desc(uAct + kk * 4096, 2048, 128);
                        const uint64_t bd = l < 4 ? tc_desc(uW + wofs + kk * 4096, 2048, 128)
                                                  : tc_desc(uW + wofs + kk * 512, 256, 128);
                        tc_mma(tmem, ad, bd, l < 4 ? id128 : id16, kk > 0);
                    }
                }
                tc_commit(&bar_g[g]);
            }
            if (!tc_wait(&bar_g[g], phase, A.errword)) abort_flag[g] = 1;
            phase ^= 1;
            wg_sync(g);  // every thread of the warpgroup sees the same abort flag
            if (abort_flag[g]) break;
            tc_fence_after();
            const uint32_t ta = tmem + ((uint32_t)(wq * 32) << 16);
            if (l < 4) {
                hidden_epilogue(ta, bias + l * 128, sAct, r);
            } else {
                float v[16];
                tmem_ld16(ta, v);
                o[0] = v[0] + bias[512];
                o[1] = v[1] + bias[513];
                o[2] = v[2] + bias[514];
            }
        }
        if (abort_flag[g]) break;
        if (live) {
            if (A.mode == 0) {
                A.out0[i] = o[0];
                A.out1[i] = o[1];
                A.out2[i] = o[2];
            } else {
                A.out0[i] = fmaf(A.out_scale, o[0], x);
                A.out1[i] = fmaf(A.out_scale, o[1], y);
                A.out2[i] = o[2];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_free(tmem_base, 512);
}

// one thread per 32-tracer group: audit lane's RK4 over the sub-interval vs its proposal,
// and the group's largest predicted error; flag = 1 sends the group to the integrator
template <int ST>
__global__ void __launch_bounds__(256) sur_audit_kernel(SurGateArgs G, RectParams P, const char *__restrict__ frames,
                                                        size_t fstride)
{
    const long long grp = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long ngrp = (G.n + 31) / 32;
    if (grp >= ngrp) return;
    const long long i0 = grp * 32;
    const int m = (int)(G.n - i0 < 32 ? G.n - i0 : 32);
    bool fall = false;
    for (int q = 0; q < m; ++q)
        if (G.rho[i0 + q] > G.log_tol || !(G.rho[i0 + q] == G.rho[i0 + q])) fall = true;
    const long long a = i0 + (long long)(lowbias32(lowbias32((unsigned)G.step) ^ (unsigned)grp) % (unsigned)m);
    if (!fall && G.status[a] == LCS_TRACER_OK && G.tol < INFINITY) {
        float x[2] = {G.xyz[a], G.xyz[G.n + a]}, c[2] = {G.cxy[a], G.cxy[G.n + a]};
        const SchedEntry *sc = G.sched + (size_t)G.step * G.S * 3;
        for (int n = 0; n < G.S; ++n) {
            SchedEntry e0 = load_sched(sc + 3 * n), e1 = load_sched(sc + 3 * n + 1), e2 = load_sched(sc + 3 * n + 2);
            rk4_step<2, ST, SRC_GLOBAL>(P, x, c, G.h, frames + (size_t)e0.k * fstride,
                                        frames + (size_t)(e0.k + 1) * fstride, e0.a, frames + (size_t)e1.k * fstride,
                                        frames + (size_t)(e1.k + 1) * fstride, e1.a, frames + (size_t)e2.k * fstride,
                                        frames + (size_t)(e2.k + 1) * fstride, e2.a);
        }
        const float dx = G.xp[a] - (x[0] + c[0]), dy = G.xp[G.n + a] - (x[1] + c[1]);
        const float res = sqrtf(dx * dx + dy * dy);
        fall = !(res <= G.tol);
    }
    G.flag[grp] = fall ? 1 : 0;
}

// one thread per tracer: take the proposal, or integrate the sub-interval where the group failed
template <int ST>
__global__ void __launch_bounds__(256) sur_apply_kernel(SurGateArgs G, RectParams P, const char *__restrict__ frames,
                                                        size_t fstride)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= G.n || G.status[i] != LCS_TRACER_OK) return;
    float x[2], c[2] = {0.0f, 0.0f};
    const int step = G.step;
    if (G.flag[i >> 5]) {
        x[0] = G.xyz[i];
        x[1] = G.xyz[G.n + i];
        c[0] = G.cxy[i];
        c[1] = G.cxy[G.n + i];
        const SchedEntry *sc = G.sched + (size_t)step * G.S * 3;
        for (int n = 0; n < G.S; ++n) {
            SchedEntry e0 = load_sched(sc + 3 * n), e1 = load_sched(sc + 3 * n + 1), e2 = load_sched(sc + 3 * n + 2);
            rk4_step<2, ST, SRC_GLOBAL>(P, x, c, G.h, frames + (size_t)e0.k * fstride,
                                        frames + (size_t)(e0.k + 1) * fstride, e0.a, frames + (size_t)e1.k * fstride,
                                        frames + (size_t)(e1.k + 1) * fstride, e1.a, frames + (size_t)e2.k * fstride,
                                        frames + (size_t)(e2.k + 1) * fstride, e2.a);
            if (rect_left<2>(P, x)) {
                G.status[i] = LCS_TRACER_LEFT;
                G.texit[i] = fmaf((float)(step * G.S + n + 1), G.h, G.t0);
                break;
            }
        }
        G.counts[i] += 1;
    } else {
        x[0] = G.xp[i];
        x[1] = G.xp[G.n + i];
        if (rect_left<2>(P, x)) {
            G.status[i] = LCS_TRACER_LEFT;
            G.texit[i] = fmaf((float)((step + 1) * G.S), G.h, G.t0);
        }
    }
    G.xyz[i] = x[0];
    G.xyz[G.n + i] = x[1];
    G.cxy[i] = c[0];   // a proposal starts without a carried rounding
    G.cxy[G.n + i] = c[1];
}

__global__ void fill_f32_kernel(float *p, long long n, float v)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// x + c rounded once: the flow map of the surrogate path, as the fixed-step kernels store it
__global__ void settle_f32_kernel(float *x, const float *c, long long n)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) x[i] = x[i] + c[i];
}

}  // namespace

cudaError_t launch_fill_f32(float *p, long long n, float v, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    fill_f32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, n, v);
    return cudaGetLastError();
}

cudaError_t launch_settle_f32(float *x, const float *c, long long n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    settle_f32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, c, n);
    return cudaGetLastError();
}

cudaError_t launch_mlp_step(const MlpStepArgs &A, int num_sms, cudaStream_t s)
{
    if (A.n <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(mlp_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)INFER_SMEM);
    if (e != cudaSuccess) return e;
    const long long pairs = ((A.n + 127) / 128 + NWG - 1) / NWG;
    const int grid = (int)(pairs < num_sms ? pairs : num_sms);
    mlp_step_kernel<<<grid, NWG * 128, INFER_SMEM, s>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_sur_gate(const SurGateArgs &G, const lcs_field *f, cudaStream_t s)
{
    if (G.n <= 0) return cudaSuccess;
    const RectParams P = make_rect_params(f);
    const char *fr = (const char *)f->d_frames;
    const long long ngrp = (G.n + 31) / 32;
    const unsigned ga = (unsigned)((ngrp + 255) / 256), gt = (unsigned)((G.n + 255) / 256);
    if (f->storage == LCS_F32) {
        sur_audit_kernel<LCS_F32><<<ga, 256, 0, s>>>(G, P, fr, f->frame_stride);
        sur_apply_kernel<LCS_F32><<<gt, 256, 0, s>>>(G, P, fr, f->frame_stride);
    } else if (f->storage == LCS_F16) {
        sur_audit_kernel<LCS_F16><<<ga, 256, 0, s>>>(G, P, fr, f->frame_stride);
        sur_apply_kernel<LCS_F16><<<gt, 256, 0, s>>>(G, P, fr, f->frame_stride);
    } else {
        sur_audit_kernel<LCS_BF16><<<ga, 256, 0, s>>>(G, P, fr, f->frame_stride);
        sur_apply_kernel<LCS_BF16><<<gt, 256, 0, s>>>(G, P, fr, f->frame_stride);
    }
    return cudaGetLastError();
}
