// advect_episodes.cu -- 3D RK4 advection with tracers re-bundled by cell between
// episodes of a few steps.
//
// Paper: Eq. 2 integrated with RK4 (Sec. 2 "Flow Map", Sec. 3.1); Sec. 3.2 notes that
// tracers with nearby indices stop needing nearby velocity data as the seed grid
// evolves, and cites re-organising particles into spatially coherent bundles as
// the remedy.  That is what this file does on the GPU.
//
// Tracers of one warp drift apart in a mixing flow, and then the 32 lanes of a warp
// read unrelated cells: every load splits into many L1 wavefronts.  So the
// integration runs in episodes of E steps; before each one the tracer records are
// re-bundled by a counting sort on the x-fastest index of the cell they sit in, and
// consecutive threads sit in the same rows of cells again.  A tracer's arithmetic
// does not depend on which thread runs it, so the flow map is bit-identical to the
// one-pass kernel.
//
// Per episode (FP32 storage): the field is blended once to every distinct stage
// time of the episode (a "time slice", stored as three component planes of
// x-neighbour pairs); the advection then reads 8-byte entries of three planes per
// stencil row.  FP16/BF16 storage reads the 16-byte interval pairs directly.
#include "rect_device.cuh"

// Resident 256-thread blocks per SM the advection kernel is compiled for, with time
// slices (FP32) and with interval pairs (FP16/BF16): 4 caps both at 64 registers
// (32 warps per SM).  Their stencil gathers are latency-bound, and the occupancy
// pays more than the few bytes spilled cost (the full-size ABC workload: 217 -> 145 ms
// per 400 steps with slices; 199 -> 173 ms with FP16 pairs).  5 (48 registers) is
// slower again.
#ifndef LCS_EP_MINB
#define LCS_EP_MINB 4
#endif
#ifndef LCS_EP_MINB_PAIRS
#define LCS_EP_MINB_PAIRS 4
#endif

// 32-byte tracer record: one sector per tracer for the re-bundling scatter
struct __align__(16) Tracer {
    float x, y, z;          // wrapped into [origin, origin + L) on periodic axes
    int id;                 // seed index
    short ix, iy, iz;       // periods crossed per axis
    unsigned char st, pad;  // status
    float te;               // exit time
    float unused;
};
static_assert(sizeof(Tracer) == 32, "tracer record must be one 32-byte sector");

// x-fastest index of the cell holding x (coarsened by `shift` bits)
__device__ __forceinline__ unsigned cell_key(const RectParams &P, const float *x, int shift)
{
    int c[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float sd = (x[d] - P.origin[d]) * P.inv_h[d];
        int v = isfinite(sd) ? (int)floorf(fminf(fmaxf(sd, 0.0f), (float)P.n[d])) : 0;
        int hi = P.periodic[d] ? P.n[d] - 1 : P.n[d] - 2;
        c[d] = min(max(v, 0), hi);
    }
    return (unsigned)((c[0] + P.sy * (long long)c[1] + P.sz * (long long)c[2]) >> shift);
}

__global__ void ep_init_kernel(RectParams P, const float *__restrict__ seeds, long long N, Tracer *__restrict__ S,
                               const float *__restrict__ job_tend, int job, int shift, unsigned *__restrict__ keys,
                               unsigned *__restrict__ hist)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    float x[3] = {seeds[i], seeds[N + i], seeds[2 * N + i]};
    int img[3] = {0, 0, 0};
    wrap_periodic<3>(P, x, img);
    Tracer t;
    t.x = x[0];
    t.y = x[1];
    t.z = x[2];
    t.id = (int)i;
    t.ix = (short)img[0];
    t.iy = (short)img[1];
    t.iz = (short)img[2];
    t.st = LCS_TRACER_OK;
    t.pad = 0;
    t.te = job_tend[job];
    t.unused = 0.0f;
    S[i] = t;
    unsigned k = cell_key(P, x, shift);
    keys[i] = k;
    atomicAdd(hist + k, 1u);
}

// ------------------------------------------------------------ counting sort

// exclusive scan of a 1024-thread block (one value per thread)
__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned *total)
{
    __shared__ unsigned wsum[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned t = lane < nw ? wsum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        wsum[lane] = t;
    }
    __syncthreads();
    unsigned pre = (w > 0 ? wsum[w - 1] : 0u) + x - v;
    *total = wsum[nw - 1];
    __syncthreads();
    return pre;
}

#define SCAN_ITEMS 4
#define SCAN_TILE (1024 * SCAN_ITEMS)

__global__ void __launch_bounds__(1024) scan_reduce_kernel(const unsigned *__restrict__ in, long long n,
                                                           unsigned *__restrict__ bsum)
{
    long long base = (long long)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    unsigned t = 0;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q)
        if (base + q < n) t += in[base + q];
    unsigned tot;
    block_excl_scan(t, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// one block: exclusive scan of up to 1024 * SCAN_ITEMS block sums, in place
__global__ void __launch_bounds__(1024) scan_top_kernel(unsigned *__restrict__ bsum, int nb)
{
    int base = threadIdx.x * SCAN_ITEMS;
    unsigned v[SCAN_ITEMS], t = 0;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        v[q] = base + q < nb ? bsum[base + q] : 0u;
        t += v[q];
    }
    unsigned tot;
    unsigned pre = block_excl_scan(t, &tot);
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        if (base + q < nb) bsum[base + q] = pre;
        pre += v[q];
    }
}

__global__ void __launch_bounds__(1024) scan_down_kernel(const unsigned *__restrict__ in, long long n,
                                                         const unsigned *__restrict__ bsum,
                                                         unsigned *__restrict__ out)
{
    long long base = (long long)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    unsigned v[SCAN_ITEMS], t = 0;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        v[q] = base + q < n ? in[base + q] : 0u;
        t += v[q];
    }
    unsigned tot;
    unsigned pre = block_excl_scan(t, &tot) + bsum[blockIdx.x];
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        if (base + q < n) out[base + q] = pre;
        pre += v[q];
    }
}

__global__ void ep_scatter_kernel(const Tracer *__restrict__ A, Tracer *__restrict__ B, long long N,
                                  const unsigned *__restrict__ keys, unsigned *__restrict__ cursor)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    unsigned p = atomicAdd(cursor + keys[i], 1u);
    B[p] = A[i];
}

// ------------------------------------------------------------- time slices

// Every distinct stage time of steps [s0, s1) gets one slice (the end of step n and
// the start of step n + 1 usually share it).  One thread builds the table:
// smap[3 (n - s0) + stage] = slice, stab[slice] = (k, alpha), slice count in *nsl.
__global__ void ep_slice_table_kernel(const SchedEntry *__restrict__ sched, int nsteps_max, int job, int s0,
                                      int s1, int *__restrict__ smap, SchedEntry *__restrict__ stab,
                                      int *__restrict__ nsl)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const SchedEntry *sc = sched + (size_t)job * nsteps_max * 3;
    int m = 0;
    SchedEntry last = {-1, 0.0f};
    for (int n = s0; n < s1; ++n)
        for (int st = 0; st < 3; ++st) {
            SchedEntry e = sc[3 * n + st];
            bool same = m > 0 && e.k == last.k && __float_as_int(e.a) == __float_as_int(last.a);
            if (!same) {
                stab[m++] = e;
                last = e;
            }
            smap[3 * (n - s0) + st] = m - 1;
        }
    *nsl = m;
}

__device__ __forceinline__ void blend_node(const char *pair, int v, float a, float *u)
{
    float va[3], vb[3];
    Pair3<LCS_F32>::ld(pair, v, va, vb);
    const float g = 1.0f - a;
#pragma unroll
    for (int c = 0; c < 3; ++c) u[c] = a == 0.0f ? va[c] : tblend(va[c], vb[c], a, g);
}

// slice j = the field blended to stab[j] (interp3p's arithmetic), as three planes:
// plane c, node v -> (u_c(v), u_c(v + x)), x wrapped on a periodic axis
__global__ void ep_slice_fill_kernel(RectParams P, const char *__restrict__ pairs, size_t fstride, long long nodes,
                                     const SchedEntry *__restrict__ stab, const int *__restrict__ nsl,
                                     float2 *__restrict__ slices, size_t plane_stride)
{
    const int j = blockIdx.y;
    if (j >= *nsl) return;
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= nodes) return;
    const SchedEntry e = stab[j];
    const char *pair = pairs + (size_t)e.k * fstride;
    const int nx = P.n[0];
    const int i = (int)(v % nx);
    const int i1 = P.periodic[0] ? (i + 1 == nx ? 0 : i + 1) : min(i + 1, nx - 1);
    float u0[3], u1[3];
    blend_node(pair, (int)v, e.a, u0);
    blend_node(pair, (int)(v - i + i1), e.a, u1);
    float2 *base = slices + (size_t)j * 3 * plane_stride;
#pragma unroll
    for (int c = 0; c < 3; ++c) base[c * plane_stride + v] = make_float2(u0[c], u1[c]);
}

// ---------------------------------------------------------------- advection

// Steps [s0, min(s1, nsteps)) of every tracer record, then the cell key of its new
// position for the next re-bundling.  SLICES: FP32 time slices; else interval pairs.
template <int ST, bool SLICES, int PM>
__global__ void __launch_bounds__(256, SLICES ? LCS_EP_MINB : LCS_EP_MINB_PAIRS) ep_advect3_kernel(RectParams P, const char *__restrict__ pairs,
                                                         size_t fstride, const float2 *__restrict__ slices,
                                                         size_t plane_stride, const int *__restrict__ smap, Rk4Args A,
                                                         Tracer *__restrict__ S, int job, int s0, int s1, int shift,
                                                         unsigned *__restrict__ keys, unsigned *__restrict__ hist)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= A.N) return;
    Tracer t = S[i];
    float x[3] = {t.x, t.y, t.z};
    if (t.st == LCS_TRACER_OK) {
        int img[3] = {t.ix, t.iy, t.iz};
        const int ns = A.job_nsteps[job];
        const float h = A.job_h[job];
        const int e = min(s1, ns);
        const SchedEntry *sc = A.sched + (size_t)job * A.nsteps_max * 3;
        CornerCache cc;       // SLICES
        cc.v0 = -1;
        cc.slice = -1;
        PairCache pc;         // interval pairs
        pc.v0 = -1;
        pc.k = -1;
        pc.a = 0.0f;
        for (int n = s0; n < e; ++n) {
            if constexpr (SLICES) {
                const int *m = smap + 3 * (n - s0);
                rk4_step3c<PM>(P, x, h, slices, __ldg(m), __ldg(m + 1), __ldg(m + 2), plane_stride, cc);
            } else {
                SchedEntry e0 = load_sched(sc + 3 * n), e1 = load_sched(sc + 3 * n + 1),
                           e2 = load_sched(sc + 3 * n + 2);
                rk4_step3pc<ST, PM>(P, x, h, pairs, fstride, e0, e1, e2, pc);
            }
            wrap_periodic<3, PM>(P, x, img);
            if (rect_left<3, PM>(P, x)) {
                t.st = LCS_TRACER_LEFT;
                t.te = fmaf((float)(n + 1), h, A.job_t0[job]);
                break;
            }
        }
        t.x = x[0];
        t.y = x[1];
        t.z = x[2];
        t.ix = (short)img[0];
        t.iy = (short)img[1];
        t.iz = (short)img[2];
        S[i] = t;
    }
    if (keys) {
        unsigned k = cell_key(P, x, shift);
        keys[i] = k;
        atomicAdd(hist + k, 1u);
    }
}

__global__ void ep_finalize_kernel(RectParams P, const Tracer *__restrict__ S, long long N, float *__restrict__ out_xyz,
                                   unsigned char *__restrict__ out_st, float *__restrict__ out_te)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const Tracer t = S[i];
    const long long id = t.id;
    const float x[3] = {t.x, t.y, t.z};
    const int img[3] = {t.ix, t.iy, t.iz};
#pragma unroll
    for (int d = 0; d < 3; ++d) out_xyz[d * N + id] = P.periodic[d] ? fmaf((float)img[d], P.L[d], x[d]) : x[d];
    out_st[id] = t.st;
    out_te[id] = t.te;
}

// ------------------------------------------------------------------- driver

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// coarsen cell keys so that at most 2^24 bins exist (the scan handles 4096 tiles of 4096)
static int sort_shift(long long nodes)
{
    int shift = 0;
    while (((nodes - 1) >> shift) + 1 > (1LL << 24)) ++shift;
    return shift;
}

static size_t slice_bytes(long long nodes, int E)
{
    return al256(8 * (size_t)nodes) * 9 * E + al256(sizeof(int) * 3 * E) + al256(sizeof(SchedEntry) * 3 * E) + 256;
}

size_t rk4_sorted_scratch_bytes(long long N, long long nodes, int storage, int E)
{
    long long nbins = ((nodes - 1) >> sort_shift(nodes)) + 1;
    long long nb = (nbins + SCAN_TILE - 1) / SCAN_TILE;
    size_t b = 2 * al256(sizeof(Tracer) * N) + al256(4 * N) + 2 * al256(4 * nbins) + al256(4 * nb);
    if (storage == LCS_F32) b += slice_bytes(nodes, E);
    return b;
}

template <int ST>
static cudaError_t episodes(const RectParams &P, const lcs_field *f, const Rk4Args &A, const Rk4Launch &L,
                            cudaStream_t s)
{
    const long long N = A.N;
    const int shift = sort_shift(f->nodes);
    const long long nbins = ((f->nodes - 1) >> shift) + 1;
    const long long nb = (nbins + SCAN_TILE - 1) / SCAN_TILE;
    if (nb > 1024 * SCAN_ITEMS) return cudaErrorInvalidValue;
    const int E = L.episode_steps > 0 ? L.episode_steps : LCS_EPISODE_STEPS;
    char *p = (char *)L.work;
    Tracer *SA = (Tracer *)p;
    p += al256(sizeof(Tracer) * N);
    Tracer *SB = (Tracer *)p;
    p += al256(sizeof(Tracer) * N);
    unsigned *keys = (unsigned *)p;
    p += al256(4 * N);
    unsigned *hist = (unsigned *)p;
    p += al256(4 * nbins);
    unsigned *cursor = (unsigned *)p;
    p += al256(4 * nbins);
    unsigned *bsum = (unsigned *)p;
    p += al256(4 * nb);
    constexpr bool SL = ST == LCS_F32;
    const size_t plane_stride = al256(8 * (size_t)f->nodes) / 8;
    float2 *slices = nullptr;
    int *smap = nullptr, *nsl = nullptr;
    SchedEntry *stab = nullptr;
    if (SL) {
        slices = (float2 *)p;
        p += al256(8 * (size_t)f->nodes) * 9 * E;
        smap = (int *)p;
        p += al256(sizeof(int) * 3 * E);
        stab = (SchedEntry *)p;
        p += al256(sizeof(SchedEntry) * 3 * E);
        nsl = (int *)p;
    }
    const int bt = 256;
    const unsigned grid = (unsigned)((N + bt - 1) / bt);
    const int abt = L.block_threads > 0 && L.block_threads <= 256 ? L.block_threads : 256;
    const unsigned agrid = (unsigned)((N + abt - 1) / abt);
    for (int job = 0; job < L.njobs; ++job) {
        const int ns = L.host_nsteps[job];
        cudaMemsetAsync(hist, 0, 4 * nbins, s);
        ep_init_kernel<<<grid, bt, 0, s>>>(P, A.seeds, N, SA, A.job_tend, job, shift, keys, hist);
        for (int s0 = 0; s0 < ns; s0 += E) {
            const int s1 = s0 + E < ns ? s0 + E : ns;
            const bool last = s1 >= ns;
            lcs_tm_begin(L.ctx, 1, s);
            scan_reduce_kernel<<<(unsigned)nb, 1024, 0, s>>>(hist, nbins, bsum);
            scan_top_kernel<<<1, 1024, 0, s>>>(bsum, (int)nb);
            scan_down_kernel<<<(unsigned)nb, 1024, 0, s>>>(hist, nbins, bsum, cursor);
            ep_scatter_kernel<<<grid, bt, 0, s>>>(SA, SB, N, keys, cursor);
            if (!last) cudaMemsetAsync(hist, 0, 4 * nbins, s);
            lcs_tm_end(L.ctx, 1, s);
            lcs_tm_begin(L.ctx, 2, s);
            if (SL) {
                ep_slice_table_kernel<<<1, 32, 0, s>>>(A.sched, A.nsteps_max, job, s0, s1, smap, stab, nsl);
                dim3 fg((unsigned)((f->nodes + 255) / 256), (unsigned)(3 * (s1 - s0)));
                ep_slice_fill_kernel<<<fg, 256, 0, s>>>(P, (const char *)f->d_frames, f->frame_stride, f->nodes, stab,
                                                         nsl, slices, plane_stride);
            }
            lcs_tm_end(L.ctx, 2, s);
            lcs_tm_begin(L.ctx, 0, s);
            // compile-time periodicity for the common all-periodic and non-periodic boxes
            const int pm = P.periodic[0] | (P.periodic[1] << 1) | (P.periodic[2] << 2);
            unsigned *kk = last ? nullptr : keys;
            const char *pr = (const char *)f->d_frames;
            if (pm == 7)
                ep_advect3_kernel<ST, SL, 7><<<agrid, abt, 0, s>>>(P, pr, f->frame_stride, slices, plane_stride, smap,
                                                                   A, SB, job, s0, s1, shift, kk, hist);
            else if (pm == 0)
                ep_advect3_kernel<ST, SL, 0><<<agrid, abt, 0, s>>>(P, pr, f->frame_stride, slices, plane_stride, smap,
                                                                   A, SB, job, s0, s1, shift, kk, hist);
            else
                ep_advect3_kernel<ST, SL, -1><<<agrid, abt, 0, s>>>(P, pr, f->frame_stride, slices, plane_stride,
                                                                    smap, A, SB, job, s0, s1, shift, kk, hist);
            lcs_tm_end(L.ctx, 0, s);
            Tracer *tmp = SA;
            SA = SB;
            SB = tmp;
        }
        ep_finalize_kernel<<<grid, bt, 0, s>>>(P, SA, N, A.out_xyz + (size_t)job * 3 * N, A.out_status + (size_t)job * N,
                                               A.out_texit + (size_t)job * N);
    }
    return cudaGetLastError();
}

cudaError_t launch_rk4_episodes(const RectParams &P, const lcs_field *f, const Rk4Args &A, const Rk4Launch &L,
                                cudaStream_t s)
{
    if (f->storage == LCS_F32) return episodes<LCS_F32>(P, f, A, L, s);
    if (f->storage == LCS_F16) return episodes<LCS_F16>(P, f, A, L, s);
    return episodes<LCS_BF16>(P, f, A, L, s);
}
