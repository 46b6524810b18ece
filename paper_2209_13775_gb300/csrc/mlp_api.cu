// mlp_api.cu -- C ABI of the learned surrogate and of the tensor-core GEMM under it.
#include "mlp_internal.cuh"

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
