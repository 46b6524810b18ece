// mlp_gemm.cu -- BF16 GEMM on the tcgen05 tensor cores, used by the surrogate trainer.
//
//   C[M x N] (+)= A[M x K] * B[N x K]^T      A, B: BF16, K contiguous; C: FP32
//
// One CTA of 128 threads computes a 128 x BN tile (BN = 16 or 128) over a K range (split-K
// partial sums are added with atomics).  Per 64-wide K chunk the four warps copy A and B
// into the canonical K-major shared-memory layout, one thread issues four
// 128 x BN x 16 MMAs into the TMEM accumulator and commits them to an mbarrier, and the
// chunk buffer is reused once the MMAs have completed.  The epilogue reads the
// accumulator lane by lane (warp w holds rows 32w .. 32w+31) and writes C.
#include "mlp_internal.cuh"
#include "tc_common.cuh"

namespace {

constexpr int GB_M = 128, GB_K = 64;

template <int BN>
__global__ void __launch_bounds__(128) gemm_bf16_kernel(const __nv_bfloat16 *__restrict__ A, long long lda,
                                                        const __nv_bfloat16 *__restrict__ B, long long ldb,
                                                        float *__restrict__ C, long long ldc, long long M, int N,
                                                        long long K, long long kchunk, int atomic,
                                                        unsigned *errword)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    // A chunk at 0 (16 KB), B chunk at 48 KB (up to 16 KB); the 96 KB allocation covers every
    // core matrix a descriptor of either chunk can address
    unsigned char *sA = smem;
    unsigned char *sB = smem + 49152;
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    constexpr uint32_t TCOLS = BN < 32 ? 32 : BN;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long m0 = (long long)blockIdx.x * GB_M;
    const int n0 = blockIdx.y * BN;
    const long long k0 = (long long)blockIdx.z * kchunk;
    const long long k1 = k0 + kchunk < K ? k0 + kchunk : K;
    if (tid == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        mbar_fence_init();
    }
    if (warp == 0) tmem_alloc(&tmem_base, TCOLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = tc_idesc_bf16(GB_M, BN);
    unsigned phase = 0;
    bool first = true;
    for (long long kc = k0; kc < k1; kc += GB_K) {
        const int kn = (int)(k1 - kc < GB_K ? k1 - kc : GB_K);  // multiple of 16
        // A: 128 rows x kn columns as 16-byte segments (8 BF16); zero beyond M
        for (int c = tid; c < GB_M * (GB_K / 8); c += 128) {
            const int r = c >> 3, kg = c & 7;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (kg * 8 < kn && m0 + r < M) v = *reinterpret_cast<const uint4 *>(A + (m0 + r) * lda + kc + kg * 8);
            *reinterpret_cast<uint4 *>(sA + ckm_offset(GB_M, r, kg * 8)) = v;
        }
        for (int c = tid; c < BN * (GB_K / 8); c += 128) {
            const int r = c >> 3, kg = c & 7;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (kg * 8 < kn && n0 + r < N) v = *reinterpret_cast<const uint4 *>(B + (long long)(n0 + r) * ldb + kc + kg * 8);
            *reinterpret_cast<uint4 *>(sB + ckm_offset(BN, r, kg * 8)) = v;
        }
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
            for (int kk = 0; kk < kn / 16; ++kk) {
                const uint64_t ad = tc_desc(a0 + kk * 2 * (GB_M / 8) * 128, (GB_M / 8) * 128, 128);
                const uint64_t bd = tc_desc(b0 + kk * 2 * (BN / 8) * 128, (BN / 8) * 128, 128);
                tc_mma(tmem, ad, bd, idesc, !first || kk > 0);
            }
            tc_commit(&bar);
        }
        first = false;
        if (!tc_wait(&bar, phase, errword)) abort_flag = 1;
        phase ^= 1;
        __syncthreads();
        if (abort_flag) break;
    }
    tc_fence_after();
    if (!abort_flag && !first) {
        const long long row = m0 + warp * 32 + lane;
#pragma unroll
        for (int c = 0; c < BN; c += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c, v);
            if (row < M) {
                float *out = C + row * ldc + n0 + c;
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (n0 + c + j < N) {
                        if (atomic)
                            atomicAdd(out + j, v[j]);
                        else
                            out[j] = v[j];
                    }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_free(tmem, TCOLS);
}

}  // namespace

cudaError_t launch_gemm_bf16(const __nv_bfloat16 *A, long long lda, const __nv_bfloat16 *B, long long ldb, float *C,
                             long long ldc, long long M, int N, long long K, int splits, int accumulate,
                             unsigned *errword, cudaStream_t s)
{
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    if (K % 16 || lda % 8 || ldb % 8 || (N != 16 && N % 128)) return cudaErrorInvalidValue;
    if (splits < 1) splits = 1;
    long long kchunk = (K + splits - 1) / splits;
    kchunk = (kchunk + GB_K - 1) / GB_K * GB_K;
    splits = (int)((K + kchunk - 1) / kchunk);
    const int atomic = accumulate || splits > 1;
    const size_t smem = 98304;
    dim3 grid((unsigned)((M + GB_M - 1) / GB_M), (unsigned)(N == 16 ? 1 : N / 128), (unsigned)splits);
    if (N == 16) {
        cudaError_t e = cudaFuncSetAttribute(gemm_bf16_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        gemm_bf16_kernel<16><<<grid, 128, smem, s>>>(A, lda, B, ldb, C, ldc, M, N, K, kchunk, atomic, errword);
    } else {
        cudaError_t e = cudaFuncSetAttribute(gemm_bf16_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        gemm_bf16_kernel<128><<<grid, 128, smem, s>>>(A, lda, B, ldb, C, ldc, M, N, K, kchunk, atomic, errword);
    }
    return cudaGetLastError();
}
