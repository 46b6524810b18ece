// mlp_internal.cuh -- the surrogate network's device state and the kernels around it.
#pragma once

#include "lcs_internal.cuh"

#include <cuda_bf16.h>

// C[M x N] (+)= A[M x K] * B[N x K]^T on the tensor cores (mlp_gemm.cu).  A, B BF16 with K
// contiguous (lda, ldb multiples of 8), K a multiple of 16, N = 16 or a multiple of 128;
// split-K partial sums and accumulate = 1 add into C with atomics.
cudaError_t launch_gemm_bf16(const __nv_bfloat16 *A, long long lda, const __nv_bfloat16 *B, long long ldb, float *C,
                             long long ldc, long long M, int N, long long K, int splits, int accumulate,
                             unsigned *errword, cudaStream_t s);

// ------------------------------------------------------------ the network

#define MLP_IN 7
#define MLP_HID 128
#define MLP_NPARAMS 50947
// offsets of the packed FP32 parameters W0[128][7] b0[128] W1 b1 W2 b2 W3 b3 W4[3][128] b4[3]
#define MLP_OFF_W0 0
#define MLP_OFF_B0 896
#define MLP_OFF_W1 1024
#define MLP_LAYER_STRIDE 16512  // 128 * 128 + 128
#define MLP_OFF_W4 50560
#define MLP_OFF_B4 50944
// inference block: BF16 operand tiles in the canonical K-major layout, then FP32 biases:
// W0 [128][16] at 0, W1..W3 [128][128] at 4096 + 32768 (l - 1), W4 [16][128] at 102400,
// biases b0..b3 [4][128] and b4 [16] at 106496
#define MLP_TILE_BYTES 108608

struct lcs_mlp {
    unsigned long long uid = 0;
    lcs_ctx *ctx = nullptr;
    lcs_mlp_desc d{};
    float *d_params = nullptr;        // FP32 master copy [MLP_NPARAMS]
    float *d_m = nullptr, *d_v = nullptr;  // Adam moments
    long long adam_steps = 0;
    unsigned char *d_tiles = nullptr; // inference block (MLP_TILE_BYTES)
    __nv_bfloat16 *d_wk = nullptr;    // trainer operands: W0 [128][16], W1..W3 [128][128], W4 [16][128]
    __nv_bfloat16 *d_wt = nullptr;    // transposes: W1^T..W3^T [128][128], W4^T [128][16]
    float *d_grad = nullptr;          // gradient [MLP_NPARAMS]
    // trainer work space for batches of up to `cap` samples
    long long cap = 0;
    void *d_work = nullptr;
};

struct MlpStepArgs {
    const void *tiles;        // inference block in device memory
    const float *x;           // x at x[i], y at x[stride + i]
    long long stride, n;
    const float *t;           // per-tracer time, or null: t_uniform
    float t_uniform;
    float cx, cy, kx, ky, omega, out_scale;
    int mode;                 // 0: out = (o0, o1, o2); 1: out = (x + s o0, y + s o1, o2)
    float *out0, *out1, *out2;
    unsigned *errword;
};

struct SurGateArgs {
    long long n;
    int step, S;              // surrogate step index, RK4 steps per surrogate step
    float h, t0;              // RK4 step and start time (FP32, as the fixed-step path)
    float tol, log_tol;
    const float *rho;         // [n] predicted log10 error
    const float *xp;          // [2][n] proposals
    float *xyz;               // [2][n] tracer state
    float *cxy;               // [2][n] its carried rounding (rk4_advance)
    unsigned char *status;
    float *texit;
    int *counts;              // [n] sub-intervals integrated by RK4
    unsigned char *flag;      // [ceil(n / 32)]
    const SchedEntry *sched;  // [K * S * 3] stage schedule of the whole interval
    unsigned *errword;
};

// 32-bit integer hash (Wellons' lowbias32): picks the audited lane of each group
__host__ __device__ __forceinline__ unsigned lowbias32(unsigned x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

cudaError_t launch_mlp_step(const MlpStepArgs &A, int num_sms, cudaStream_t s);
cudaError_t launch_fill_f32(float *p, long long n, float v, cudaStream_t s);
cudaError_t launch_settle_f32(float *x, const float *c, long long n, cudaStream_t s);
cudaError_t launch_sur_gate(const SurGateArgs &G, const lcs_field *f, cudaStream_t s);
cudaError_t launch_mlp_refresh(lcs_mlp *m, cudaStream_t s);
lcs_status advect_surrogate(lcs_ctx *ctx, const lcs_field *f, const lcs_seeds *s, const lcs_advect_opts *o,
                            lcs_flowmap *fm);

// trainer (mlp_train.cu)
cudaError_t mlp_reserve(lcs_mlp *m, long long B, cudaStream_t s);
cudaError_t mlp_loss_grad(lcs_mlp *m, const float *xyt, long long xstride, const float *disp, long long dstride,
                          long long B, float rho_weight, int num_sms, unsigned *errword, double *d_loss, cudaStream_t s);
cudaError_t mlp_adam(lcs_mlp *m, const float *grad, double lr, double b1, double b2, double eps, cudaStream_t s);
cudaError_t mlp_targets(const lcs_field *f, const float *xyt, long long n, int S, double dt, float *disp,
                        cudaStream_t s);
