// bench_peaks.cu -- measurement probes of bench.py (not part of the library): the roofline
// denominators this GPU reaches with simple loops (FP32 and FP64 fused multiply-add throughput,
// L2-resident and HBM read bandwidth), and the cost of one warp-wide 16-byte gather from L1 for
// lane address patterns that separate the two limits of the L1 data stage.
//
// Each loop is the plainest form of its resource: independent FMA chains per thread (enough
// of them to cover the pipe latency), or grid-stride 16-byte loads folded into a sum that is
// stored so the compiler keeps them.  Grids are sized in multiples of the SM count.  Every
// gather index is masked into its buffer.
#include <cuda_runtime.h>

namespace {

constexpr int CHAINS = 8;

template <typename T>
__global__ void __launch_bounds__(256) fma_loop_kernel(T a, T b, int iters, T *__restrict__ out)
{
    T v[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) v[c] = (T)(threadIdx.x + c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) v[c] = fma(v[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += v[c];
    if (s == (T)-1.2345) out[0] = s;   // never true for these inputs; keeps the chains alive
}

__global__ void __launch_bounds__(256) read_loop_kernel(const float4 *__restrict__ buf, long long n, int reps,
                                                        float *__restrict__ out)
{
    float acc = 0.0f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r)
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
            const float4 q = __ldg(buf + i);
            acc += q.x + q.y + q.z + q.w;
        }
    if (acc == -1.2345f) out[0] = acc;
}


// 16-byte gathers from an L1-resident buffer: lane l of a warp reads lane_offset(pattern, l) float4s
// past a per-iteration base (1024-aligned, masked into the buffer).  The patterns place the 8 lanes
// of each quarter warp (which one 128-bit load request serves per L1 data-stage wavefront at best)
// in 1, 2, 4 or 8 distinct 128-byte lines, with distinct or colliding 16-byte bank groups.
__device__ __forceinline__ unsigned lane_offset(int pattern, unsigned l)
{
    const unsigned q = l & 7, w = l >> 3;
    switch (pattern) {
    case 0: return l;                                  // 1 line per quarter
    case 1: return q + 8 * ((q >> 2) & 1) + 256 * w;   // 2 lines, distinct bank groups
    case 2: return q + 8 * ((q >> 1) & 3) + 256 * w;   // 4 lines, distinct bank groups
    case 3: return 9 * q + 256 * w;                    // 8 lines, distinct bank groups
    case 4: return 8 * q + 256 * w;                    // 8 lines, one bank group
    case 5: return 8 * (q & 1) + 256 * w;              // 2 lines, one bank group, 2 addresses
    default: return 0;
    }
}

__global__ void __launch_bounds__(256) gather_pattern_kernel(const float4 *__restrict__ buf, unsigned mask,
                                                             int pattern, int iters, float *__restrict__ out)
{
    const unsigned lane = threadIdx.x & 31, w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned off = lane_offset(pattern, lane);
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    unsigned s = w * 2654435761u + 12345u;
    for (int it = 0; it < iters; ++it) {
        s = s * 1664525u + 1013904223u;
        const unsigned base = (s >> 4) & mask & ~1023u;
        const float4 a = __ldg(buf + ((base + off) & mask));
        acc.x += a.x;
        acc.y += a.y;
        acc.z += a.z;
        acc.w += a.w;
    }
    if (acc.x + acc.y + acc.z + acc.w == -1.2345f) out[0] = acc.x;
}

}  // namespace

#define BENCH_L1_PATTERNS 6

// peaks[4]: FP32 FMA TFLOP/s, FP64 FMA TFLOP/s, read GB/s of a 32 MB (L2-resident) buffer, read
// GB/s of a 4 GiB buffer.  Returns 0, or the CUDA error code.
extern "C" int bench_probe_peaks(int device, double *peaks)
{
    if (!peaks) return (int)cudaErrorInvalidValue;
    int sms = 0;
    cudaStream_t s = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const size_t l2_bytes = (size_t)32 << 20, hbm_bytes = (size_t)4 << 30;
    char *buf = nullptr;
    double *sink = nullptr;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMalloc(&buf, hbm_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&sink, 64);
    if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, hbm_bytes, s);
    auto timed = [&](auto launch, float *ms) {
        launch();   // warm-up
        cudaEventRecord(e0, s);
        launch();
        cudaEventRecord(e1, s);
        cudaError_t r = cudaEventSynchronize(e1);
        if (r == cudaSuccess) r = cudaEventElapsedTime(ms, e0, e1);
        return r == cudaSuccess ? cudaGetLastError() : r;
    };
    const unsigned fgrid = (unsigned)sms * 16;   // 16 blocks of 256 per SM: full occupancy
    float ms = 0.0f;
    if (e == cudaSuccess) {   // FP32 FMA: 2 flops each
        const int iters = 1 << 14;
        e = timed([&] { fma_loop_kernel<float><<<fgrid, 256, 0, s>>>(1.0000001f, 1e-7f, iters, (float *)sink); }, &ms);
        peaks[0] = 2.0 * CHAINS * iters * (double)fgrid * 256 / (ms * 1e-3) / 1e12;
    }
    if (e == cudaSuccess) {   // FP64 FMA
        const int iters = 1 << 10;
        e = timed([&] { fma_loop_kernel<double><<<fgrid, 256, 0, s>>>(1.0000000001, 1e-12, iters, sink); }, &ms);
        peaks[1] = 2.0 * CHAINS * iters * (double)fgrid * 256 / (ms * 1e-3) / 1e12;
    }
    if (e == cudaSuccess) {   // a 32 MB buffer read 256 times: L2-resident after the first pass
        const int reps = 256;
        const long long n = (long long)(l2_bytes / 16);
        e = timed([&] { read_loop_kernel<<<(unsigned)sms * 8, 256, 0, s>>>((const float4 *)buf, n, reps, (float *)sink); },
                  &ms);
        peaks[2] = (double)l2_bytes * reps / (ms * 1e-3) / 1e9;
    }
    if (e == cudaSuccess) {   // 4 GiB read once from HBM
        const long long n = (long long)(hbm_bytes / 16);
        e = timed([&] { read_loop_kernel<<<(unsigned)sms * 8, 256, 0, s>>>((const float4 *)buf, n, 1, (float *)sink); },
                  &ms);
        peaks[3] = (double)hbm_bytes / (ms * 1e-3) / 1e9;
    }
    cudaFree(buf);
    cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return (int)e;
}

// clk[BENCH_L1_PATTERNS]: SM clock cycles per warp-wide 16-byte gather request (per SM, all SMs
// busy) for each lane pattern of lane_offset; 4 cycles is one wavefront per quarter warp.  Returns
// 0, or the CUDA error code.
extern "C" int bench_probe_l1(int device, double *clk)
{
    if (!clk) return (int)cudaErrorInvalidValue;
    int sms = 0, khz = 0;
    const unsigned R = 1u << 13;   // 128 KB of float4: L1-resident
    float4 *buf = nullptr;
    float *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, device);
    if (e == cudaSuccess) e = cudaMalloc(&buf, R * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&sink, 64);
    if (e == cudaSuccess) e = cudaMemset(buf, 0, R * sizeof(float4));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const unsigned blocks = (unsigned)sms * 8;
    const int iters = 4000;
    for (int p = 0; p < BENCH_L1_PATTERNS && e == cudaSuccess; ++p) {
        float best = 1e30f;
        for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
            cudaEventRecord(e0);
            gather_pattern_kernel<<<blocks, 256>>>(buf, R - 1, p, iters, sink);
            cudaEventRecord(e1);
            e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (ms < best) best = ms;
        }
        const double requests = (double)blocks * 8 * iters;
        clk[p] = best * 1e-3 * khz * 1e3 * sms / requests;
    }
    cudaFree(buf);
    cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return (int)e;
}
