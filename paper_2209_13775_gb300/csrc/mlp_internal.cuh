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
