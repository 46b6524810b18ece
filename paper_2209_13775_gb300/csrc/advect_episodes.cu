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
// re-bundled by a counting sort on the key of the cell they sit in (cells grouped in
// bricks), the records moved by a gather through the resulting permutation, and
// consecutive threads sit in the same few cells again.  A tracer's arithmetic
// does not depend on which thread runs it, so the flow map is bit-identical to the
// one-pass kernel.
//
// Per episode the field is blended once, in FP32, to every distinct stage time of the
// episode (a "time slice", stored as xy-quads of the three components interleaved per node, on a
// lattice with a halo on periodic axes); the advection then reads two 16-byte quads per component and
// stencil, and keeps the last stencil's corners in registers for the next stage that
// reads the same slice from the same cell.  FP16/BF16 storage is widened in the fill.
#include "rect_device.cuh"

// Resident 256-thread blocks per SM the advection kernel is compiled for: 4 caps it at
// 64 registers (32 warps per SM).  Its stencil gathers are latency-bound, and the
// occupancy pays more than the few bytes spilled cost (the full-size ABC workload:
// 217 -> 145 ms per 400 steps when introduced); 5 (48 registers, more spills) and a
// 56-register cap with 128-thread blocks (36 warps) are slower.
#ifndef LCS_EP_MINB
#define LCS_EP_MINB 4
#endif

// 48-byte tracer record (three 16-byte loads) moved by the re-bundling gather
struct __align__(16) Tracer {
    float x, y, z;          // wrapped into [origin, origin + L) on periodic axes
    int id;                 // seed index
    float cx, cy, cz;       // the coordinates' carried rounding (rk4_advance)
    float te;               // exit time
    short ix, iy, iz;       // periods crossed per axis
    unsigned char st, pad;  // status
    float unused[2];
};
static_assert(sizeof(Tracer) == 48, "tracer record must be three 16-byte words");

// Re-bundling order: cells grouped in bricks of 2^EP_BRICK cells per axis, bricks in
// x-fastest order and cells x-fastest inside a brick.  A wave of resident blocks then holds
// tracers of a compact block of cells rather than a thin slab, and the slices it reads in
// an episode stay in L2 for longer: 8^3 bricks took the ABC episode kernel from 121.9 to
// 113.9 ms per 400 steps (4^3: 115.2 ms; plain x-fastest cells: EP_BRICK 0).
#ifndef EP_BRICK
#define EP_BRICK 3
#endif

__host__ __device__ __forceinline__ long long brick_count(int n) { return (n + (1 << EP_BRICK) - 1) >> EP_BRICK; }

// number of distinct cell keys before coarsening
static long long key_space(const lcs_field *f)
{
    return brick_count(f->n[0]) * brick_count(f->n[1]) * brick_count(f->n[2]) << (3 * EP_BRICK);
}

// key of the cell holding x (coarsened by `shift` bits)
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
    constexpr int B = EP_BRICK, M = (1 << EP_BRICK) - 1;
    const long long bx = brick_count(P.n[0]), by = brick_count(P.n[1]);
    const long long brick = (c[0] >> B) + bx * ((c[1] >> B) + by * (long long)(c[2] >> B));
    const long long k = (brick << (3 * B)) | (c[0] & M) | ((c[1] & M) << B) | ((c[2] & M) << (2 * B));
    return (unsigned)(k >> shift);
}

// ctr[key] += 1 for every calling lane, one atomic per distinct key among the lanes that arrive
// together (consecutive records of a re-bundled order mostly share a cell); returns each lane's
// slot: the counter's old value plus the lane's rank among the lanes with its key
__device__ __forceinline__ unsigned warp_add_one(unsigned *ctr, unsigned key)
{
    const unsigned act = __activemask();
    const unsigned m = __match_any_sync(act, key);
    const unsigned lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    unsigned base = 0;
    if ((int)lane == leader) base = atomicAdd(ctr + key, (unsigned)__popc(m));
    base = __shfl_sync(act, base, leader);
    return base + (unsigned)__popc(m & ((1u << lane) - 1u));
}

__global__ void ep_init_kernel(RectParams P, const float *__restrict__ seeds, long long N, Tracer *__restrict__ S,
                               const float *__restrict__ job_tend, int job, int shift, unsigned *__restrict__ keys,
                               unsigned *__restrict__ hist)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    float x[3] = {seeds[i], seeds[N + i], seeds[2 * N + i]}, c[3] = {0.0f, 0.0f, 0.0f};
    int img[3] = {0, 0, 0};
    wrap_periodic<3>(P, x, c, img);
    Tracer t;
    t.x = x[0];
    t.y = x[1];
    t.z = x[2];
    t.cx = c[0];
    t.cy = c[1];
    t.cz = c[2];
    t.id = (int)i;
    t.ix = (short)img[0];
    t.iy = (short)img[1];
    t.iz = (short)img[2];
    t.st = LCS_TRACER_OK;
    t.pad = 0;
    t.te = job_tend[job];
    t.unused[0] = t.unused[1] = 0.0f;
    S[i] = t;
    unsigned k = cell_key(P, x, shift);
    keys[i] = k;
    warp_add_one(hist, k);
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

// the re-bundled order as a permutation: slot p of the new order takes record perm[p] of the old
__global__ void ep_perm_kernel(long long N, const unsigned *__restrict__ keys, unsigned *__restrict__ cursor,
                               unsigned *__restrict__ perm)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    perm[warp_add_one(cursor, keys[i])] = (unsigned)i;
}

// slot p of the new order from record perm[p] of the old: gathered reads, coalesced writes (a
// scatter writes 48-byte records to scattered slots, which costs more); the variational grad F
// ([9][N] planes) moves with the records
__global__ void ep_gather_kernel(const Tracer *__restrict__ A, Tracer *__restrict__ B, long long N,
                                 const unsigned *__restrict__ perm, const float *__restrict__ MA,
                                 float *__restrict__ MB)
{
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= N) return;
    const long long i = __ldg(perm + p);
    B[p] = A[i];
    if (MA) {
#pragma unroll
        for (int e = 0; e < 9; ++e) MB[e * N + p] = MA[e * N + i];
    }
}

// grad F = I in seed order ([9][N] planes)
__global__ void ep_var_init_kernel(float *__restrict__ M, long long N)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
#pragma unroll
    for (int e = 0; e < 9; ++e) M[e * N + i] = e % 4 == 0 ? 1.0f : 0.0f;
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

// Time slices.  Slice j is the field blended to stage time stab[j] in FP32 (interp3p's
// arithmetic on the stored frames, widened from FP16/BF16 storage), as xy-quads on a lattice extended by
// a halo of SLICE_HALO nodes on each side of every periodic axis: extended node (I, J, K) holds,
// for c = 0, 1, 2 in turn, the float4 (u_c(i, j, k), u_c(i1, j, k), u_c(i, j1, k), u_c(i1, j1, k))
// with (i, j, k) the field node the extended node wraps to and i1, j1 the next node along
// x and y (wrapped, or clamped on a closed axis).  A trilinear stencil is then two 16-byte
// loads per component (its two z-rows), the three of a row in one 48-byte run (interleaving
// the components rather than keeping three planes cut the episode kernel from 113.2 to
// 111.2 ms per 400 steps at C2), and stencil points a few cells outside the periodic box need
// no index wrapping: the halo holds the wrapped values.
//
// Rows and planes of a slice are padded (pitches R and Q nodes, R = 4 and Q = 2 mod 8) so that
// the 8 nodes of any 2 x 2 x 2 block of cells start in 8 different 16-byte bank groups of a
// 128-byte line: the L1 data stage serves the 8 lanes of a quarter warp in one wavefront only
// when no two of them read different addresses in the same bank group, and the stencil loads of
// nearby tracers then rarely collide.  Unpadded, z-neighbours (Q = 132^2 = 0 mod 8 on the ABC
// grid) always collided; a count of the collisions along RK4 trajectories of the ABC flow gave
// 1.78 wavefronts per quarter warp unpadded, 1.01 padded.
#define SLICE_HALO 2

struct SliceGeom {
    int H[3];        // halo nodes on each side of an axis (periodic axes only)
    int N[3];        // extended node counts n + 2H
    int R;           // row pitch in nodes (>= N[0], = 4 mod 8)
    long long nxy;   // plane pitch in nodes (>= R * N[1], = 2 mod 8)
    long long nodes; // nodes of one slice plane, padding included (nxy * N[2])
};

static SliceGeom slice_geom(const lcs_field *f)
{
    SliceGeom G;
    for (int d = 0; d < 3; ++d) {
        G.H[d] = f->periodic[d] ? SLICE_HALO : 0;
        G.N[d] = f->n[d] + 2 * G.H[d];
    }
    G.R = G.N[0] + ((4 - G.N[0]) & 7);
    const long long q = (long long)G.R * G.N[1];
    G.nxy = q + ((2 - q) & 7);
    G.nodes = G.nxy * G.N[2];
    return G;
}

// field node of extended index I along an axis (any n >= 1: the halo may span several periods)
__device__ __forceinline__ int slice_src(int I, int H, int n, bool per)
{
    if (!per) return I;
    int i = (I - H) % n;
    return i < 0 ? i + n : i;
}

// One thread per extended node writes that node's quads in every slice of the episode:
// the four interval-pair records of its quad are read once per frame interval k and
// blended to each slice time in registers, u = (1 - a) u_k + a u_{k+1} as interp3p blends
// (u_k itself when a = 0), so the slices cost little more than their writes.
template <int ST>
__global__ void ep_slice_fill_kernel(RectParams P, SliceGeom G, const char *__restrict__ pairs, size_t fstride,
                                     const SchedEntry *__restrict__ stab, const int *__restrict__ nsl,
                                     float4 *__restrict__ slices, size_t plane_stride)
{
    // a block's 256 nodes are consecutive, so their interleaved quads (3 per node) form one run
    // of 768 float4 per slice: staged in shared memory and stored coalesced (padding nodes get 0)
    __shared__ float4 stage[256 * 3];
    const long long vb = (long long)blockIdx.x * 256;
    const long long v = vb + threadIdx.x;
    const int nb = (int)min(256LL, G.nodes - vb);
    bool live = v < G.nodes;
    int corner[4] = {0, 0, 0, 0};
    if (live) {
        const int K = (int)(v / G.nxy);
        const long long rem = v - (long long)K * G.nxy;
        const int J = (int)(rem / G.R);
        const int I = (int)(rem - (long long)J * G.R);
        live = J < G.N[1] && I < G.N[0];
        const bool px = P.periodic[0], py = P.periodic[1];
        const int i = slice_src(I, G.H[0], P.n[0], px);
        const int jj = slice_src(J, G.H[1], P.n[1], py);
        const int k = slice_src(K, G.H[2], P.n[2], P.periodic[2]);
        const int i1 = px ? (i + 1 == P.n[0] ? 0 : i + 1) : min(i + 1, P.n[0] - 1);
        const int j1 = py ? (jj + 1 == P.n[1] ? 0 : jj + 1) : min(jj + 1, P.n[1] - 1);
        const long long zk = k * P.sz;
        if (live) {
            corner[0] = (int)(i + jj * P.sy + zk);
            corner[1] = (int)(i1 + jj * P.sy + zk);
            corner[2] = (int)(i + j1 * P.sy + zk);
            corner[3] = (int)(i1 + j1 * P.sy + zk);
        }
    }
    const int m = __ldg(nsl);
    float ua[4][3], ub[4][3];
    int kc = -1;
    for (int j = 0; j < m; ++j) {
        const SchedEntry e = load_sched(stab + j);
        if (live) {
            if (e.k != kc) {
                const char *pair = pairs + (size_t)e.k * fstride;
#pragma unroll
                for (int q = 0; q < 4; ++q) Pair3<ST>::ld(pair, corner[q], ua[q], ub[q]);
                kc = e.k;
            }
            const float g = 1.0f - e.a;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float u[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) u[q] = e.a == 0.0f ? ua[q][c] : tblend(ua[q][c], ub[q][c], e.a, g);
                stage[3 * threadIdx.x + c] = make_float4(u[0], u[1], u[2], u[3]);
            }
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) stage[3 * threadIdx.x + c] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
        __syncthreads();
        float4 *base = slices + (size_t)j * 3 * plane_stride + 3 * vb;
        for (int q = threadIdx.x; q < 3 * nb; q += 256) base[q] = stage[q];
        __syncthreads();
    }
}

// Cell of x along axis d on the extended lattice, with the fraction f: the same s, floor and
// f as axis_cell, so the weights are the same.  A periodic index beyond the halo (a stencil
// point more than SLICE_HALO - 1 cells outside the box) is flagged in `out` and wrapped by
// the caller.
template <int PM>
__device__ __forceinline__ int axis_cell_ext(const RectParams &P, const SliceGeom &G, int d, float x, float &f,
                                             int &raw, bool &out)
{
    if (per_axis<PM>(P, d)) {
        float s = (x - P.origin[d]) * P.inv_h[d];
        float fl = floorf(s);
        raw = (int)fl;
        f = s - fl;
        const int e = raw + G.H[d];
        out = out || (unsigned)e > (unsigned)(G.N[d] - 2);
        return e;
    } else {
        float xc = fminf(fmaxf(x, P.origin[d]), P.hi_node[d]);
        float s = (xc - P.origin[d]) * P.inv_h[d];
        int i = min((int)s, P.n[d] - 2);
        f = s - (float)i;
        raw = i;
        return i;
    }
}

// Trilinear weights of x (make_stencil's products) and the extended base node of its cell.
template <int PM>
__device__ __forceinline__ int stencil_ext(const RectParams &P, const SliceGeom &G, const float *x, float *w)
{
    float fx, fy, fz;
    int rx, ry, rz;
    bool out = false;
    int ix = axis_cell_ext<PM>(P, G, 0, x[0], fx, rx, out);
    int iy = axis_cell_ext<PM>(P, G, 1, x[1], fy, ry, out);
    int iz = axis_cell_ext<PM>(P, G, 2, x[2], fz, rz, out);
    if (out) {   // rare: wrap every periodic axis into the box (the others are already in range)
        if (per_axis<PM>(P, 0)) ix = wrap_index_slow(rx, P.n[0]) + G.H[0];
        if (per_axis<PM>(P, 1)) iy = wrap_index_slow(ry, P.n[1]) + G.H[1];
        if (per_axis<PM>(P, 2)) iz = wrap_index_slow(rz, P.n[2]) + G.H[2];
    }
    const float gx = 1.0f - fx, gy = 1.0f - fy, gz = 1.0f - fz;
    const float a = gy * gz, b = fy * gz, c = gy * fz, d = fy * fz;
    w[0] = gx * a;
    w[1] = fx * a;
    w[2] = gx * b;
    w[3] = fx * b;
    w[4] = gx * c;
    w[5] = fx * c;
    w[6] = gx * d;
    w[7] = fx * d;
    return ix + iy * G.R + iz * (int)G.nxy;
}

// Corner cache: the two z-row quads of the 3 components of the cell a tracer's last stage
// evaluation read, with the cell's extended base node and the slice they came from.
// Stage 3 of an RK4 step reads the same slice as stage 2 (t_n + h/2), and stage 1 of step
// n + 1 the same slice as stage 4 of step n (t_n + h) whenever the schedule gives both the
// same (k, alpha); in a smooth flow the second point of each pair is almost always in the
// same cell as the first, so its corners are already in registers.  The base node fixes
// all eight corners, so a reuse reads exactly what a reload would: bit-identical results.
struct QuadCache {
    float4 q[2][3];
    int v0;
    int slice;
};

// u(x) from slice `slice` (3 planes of plane_stride quads at pl); the products and their
// order are interp3p's: corners (i0,j0,k0), (i1,j0,k0), (i0,j1,k0), (i1,j1,k0), then k1.
__device__ __forceinline__ void interp3q(int v0, const float *w, const float4 *__restrict__ pl, int slice,
                                         size_t plane_stride, int nxy, QuadCache &cc, float *u)
{
    if (v0 != cc.v0 || slice != cc.slice) {
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) cc.q[r][c] = __ldg(pl + 3 * (v0 + r * nxy) + c);
        cc.v0 = v0;
        cc.slice = slice;
    }
    float acc[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int r = 0; r < 2; ++r) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            acc[c] = fmaf(w[4 * r], cc.q[r][c].x, acc[c]);
            acc[c] = fmaf(w[4 * r + 1], cc.q[r][c].y, acc[c]);
            acc[c] = fmaf(w[4 * r + 2], cc.q[r][c].z, acc[c]);
            acc[c] = fmaf(w[4 * r + 3], cc.q[r][c].w, acc[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) u[c] = acc[c];
}

// One RK4 step in 3D from slices m0, m1, m2 (stage times t_n, t_n + h/2, t_n + h).
template <int PM>
__device__ __forceinline__ void rk4_step3q(const RectParams &P, const SliceGeom &G, float *x, float *cx, float h,
                                           const float4 *__restrict__ slices, int m0, int m1, int m2, size_t ps,
                                           QuadCache &cc)
{
    float k1[3], k2[3], k3[3], k4[3], y[3], w[8];
    const float hh = 0.5f * h;
    const size_t ss = 3 * ps;
    const int nxy = (int)G.nxy;
    int v = stencil_ext<PM>(P, G, x, w);
    interp3q(v, w, slices + (size_t)m0 * ss, m0, ps, nxy, cc, k1);
#pragma unroll
    for (int c = 0; c < 3; ++c) y[c] = fmaf(hh, k1[c], x[c]);
    v = stencil_ext<PM>(P, G, y, w);
    interp3q(v, w, slices + (size_t)m1 * ss, m1, ps, nxy, cc, k2);
#pragma unroll
    for (int c = 0; c < 3; ++c) y[c] = fmaf(hh, k2[c], x[c]);
    v = stencil_ext<PM>(P, G, y, w);
    interp3q(v, w, slices + (size_t)m1 * ss, m1, ps, nxy, cc, k3);
#pragma unroll
    for (int c = 0; c < 3; ++c) y[c] = fmaf(h, k3[c], x[c]);
    v = stencil_ext<PM>(P, G, y, w);
    interp3q(v, w, slices + (size_t)m2 * ss, m2, ps, nxy, cc, k4);
    const float h6 = h * (1.0f / 6.0f);
#pragma unroll
    for (int c = 0; c < 3; ++c) rk4_advance(x[c], cx[c], h6, k1[c], k2[c], k3[c], k4[c]);
}

// ------------------------------------------------- variational equations

// stencil_ext plus, for the Jacobian, the fractions and the per-axis factor d s / d x: 1 / h
// where the query moves with x, 0 on a non-periodic axis where x lies outside the box (the
// clamped query does not move)
template <int PM>
__device__ __forceinline__ int stencil_ext_grad(const RectParams &P, const SliceGeom &G, const float *x, float *w,
                                                float *f, float *on)
{
    int r[3];
    bool out = false;
    int ix = axis_cell_ext<PM>(P, G, 0, x[0], f[0], r[0], out);
    int iy = axis_cell_ext<PM>(P, G, 1, x[1], f[1], r[1], out);
    int iz = axis_cell_ext<PM>(P, G, 2, x[2], f[2], r[2], out);
    if (out) {
        if (per_axis<PM>(P, 0)) ix = wrap_index_slow(r[0], P.n[0]) + G.H[0];
        if (per_axis<PM>(P, 1)) iy = wrap_index_slow(r[1], P.n[1]) + G.H[1];
        if (per_axis<PM>(P, 2)) iz = wrap_index_slow(r[2], P.n[2]) + G.H[2];
    }
    const float gx = 1.0f - f[0], gy = 1.0f - f[1], gz = 1.0f - f[2];
    const float a = gy * gz, b = f[1] * gz, c = gy * f[2], d = f[1] * f[2];
    w[0] = gx * a;
    w[1] = f[0] * a;
    w[2] = gx * b;
    w[3] = f[0] * b;
    w[4] = gx * c;
    w[5] = f[0] * c;
    w[6] = gx * d;
    w[7] = f[0] * d;
#pragma unroll
    for (int k = 0; k < 3; ++k)
        on[k] = (per_axis<PM>(P, k) || (x[k] >= P.origin[k] && x[k] <= P.hi_node[k])) ? P.inv_h[k] : 0.0f;
    return ix + iy * G.R + iz * (int)G.nxy;
}

// u(x) as interp3q and its Jacobian J[c][d] = sum_q (d w_q / d x_d) u_q[c], corner q with offsets
// (q & 1, (q >> 1) & 1, q >> 2), the one-pass variational kernel's products in its order
__device__ __forceinline__ void interp3q_grad(int v0, const float *w, const float *f, const float *on,
                                              const float4 *__restrict__ pl, int slice, size_t plane_stride, int nxy,
                                              QuadCache &cc, float *u, float (*J)[3])
{
    interp3q(v0, w, pl, slice, plane_stride, nxy, cc, u);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            float acc = 0.0f;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                float wq = ((q >> d) & 1) ? 1.0f : -1.0f;
#pragma unroll
                for (int e = 0; e < 3; ++e)
                    if (e != d) wq *= ((q >> e) & 1) ? f[e] : 1.0f - f[e];
                const float4 qv = cc.q[q >> 2][c];
                const float uq = (q & 3) == 0 ? qv.x : (q & 3) == 1 ? qv.y : (q & 3) == 2 ? qv.z : qv.w;
                acc = fmaf(wq, uq, acc);
            }
            J[c][d] = acc * on[d];
        }
}

// Steps [s0, min(s1, nsteps)) of every tracer record with the variational equations dM/dt = J M
// next to Eq. 2: x follows rk4_step3q's arithmetic, M ([9][N] planes, slot-ordered like S) the
// one-pass variational kernel's, so both match the other paths bit for bit.
template <int PM>
__global__ void __launch_bounds__(256, 2) ep_var3_kernel(RectParams P, SliceGeom G, const float4 *__restrict__ slices,
                                                        size_t plane_stride, const int *__restrict__ smap, Rk4Args A,
                                                        Tracer *__restrict__ S, float *__restrict__ M9, int job,
                                                        int s0, int s1, int shift, unsigned *__restrict__ keys,
                                                        unsigned *__restrict__ hist)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= A.N) return;
    const long long N = A.N;
    Tracer t = S[i];
    float x[3] = {t.x, t.y, t.z}, cx[3] = {t.cx, t.cy, t.cz};
    if (t.st == LCS_TRACER_OK) {
        int img[3] = {t.ix, t.iy, t.iz};
        float M[3][3];
#pragma unroll
        for (int e = 0; e < 9; ++e) M[e / 3][e % 3] = M9[e * N + i];
        const int ns = A.job_nsteps[job];
        const float h = A.job_h[job], hh = 0.5f * h, h6 = h * (1.0f / 6.0f);
        const size_t ss = 3 * plane_stride;
        const int nxy = (int)G.nxy;
        const int e1 = min(s1, ns);
        QuadCache cc;
        cc.v0 = -1;
        cc.slice = -1;
        for (int n = s0; n < e1; ++n) {
            const int *m = smap + 3 * (n - s0);
            const int ms[3] = {__ldg(m), __ldg(m + 1), __ldg(m + 2)};
            float k[4][3], S03[3][3], S12[3][3], Kp[3][3];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int sl = ms[q == 0 ? 0 : (q == 3 ? 2 : 1)];
                const float c = q == 0 ? 0.0f : (q == 3 ? h : hh);
                float y[3], Y[3][3], w[8], f[3], on[3], J[3][3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    y[a] = q == 0 ? x[a] : fmaf(c, k[q - 1][a], x[a]);
#pragma unroll
                    for (int b = 0; b < 3; ++b) Y[a][b] = q == 0 ? M[a][b] : fmaf(c, Kp[a][b], M[a][b]);
                }
                const int v = stencil_ext_grad<PM>(P, G, y, w, f, on);
                interp3q_grad(v, w, f, on, slices + (size_t)sl * ss, sl, plane_stride, nxy, cc, k[q], J);
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        float acc = 0.0f;
#pragma unroll
                        for (int cc2 = 0; cc2 < 3; ++cc2) acc = fmaf(J[a][cc2], Y[cc2][b], acc);
                        Kp[a][b] = acc;
                        if (q == 0) S03[a][b] = acc;
                        else if (q == 1) S12[a][b] = acc;
                        else if (q == 2) S12[a][b] = S12[a][b] + acc;
                        else S03[a][b] = S03[a][b] + acc;
                    }
            }
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                rk4_advance(x[a], cx[a], h6, k[0][a], k[1][a], k[2][a], k[3][a]);
#pragma unroll
                for (int b = 0; b < 3; ++b) M[a][b] = fmaf(h6, S03[a][b] + 2.0f * S12[a][b], M[a][b]);
            }
            wrap_periodic<3, PM>(P, x, cx, img);
            if (rect_left<3, PM>(P, x)) {
                t.st = LCS_TRACER_LEFT;
                t.te = fmaf((float)(n + 1), h, A.job_t0[job]);
                break;
            }
        }
        t.x = x[0];
        t.y = x[1];
        t.z = x[2];
        t.cx = cx[0];
        t.cy = cx[1];
        t.cz = cx[2];
        t.ix = (short)img[0];
        t.iy = (short)img[1];
        t.iz = (short)img[2];
        S[i] = t;
#pragma unroll
        for (int e = 0; e < 9; ++e) M9[e * N + i] = M[e / 3][e % 3];
    }
    if (keys) {
        unsigned k = cell_key(P, x, shift);
        keys[i] = k;
        warp_add_one(hist, k);
    }
}

// ---------------------------------------------------------------- advection

// tracer record t into output slot `slot`; snap >= 0: the slot is snapshot entry snap
// (job * nsnap + s) of the call, whose end time a tracer still OK records as its exit time
__device__ __forceinline__ void ep_store(const RectParams &P, const Rk4Args &A, int slot, const Tracer &t, int snap)
{
    const long long N = A.N, id = t.id;
    const float x[3] = {t.x, t.y, t.z}, c[3] = {t.cx, t.cy, t.cz};
    const int img[3] = {t.ix, t.iy, t.iz};
    float *o = A.out_xyz + (size_t)slot * 3 * N;
#pragma unroll
    for (int d = 0; d < 3; ++d) o[d * N + id] = out_coord(P, d, x[d], c[d], img[d]);
    A.out_status[(size_t)slot * N + id] = t.st;
    A.out_texit[(size_t)slot * N + id] = snap >= 0 && t.st == LCS_TRACER_OK ? __ldg(A.snap_te + snap) : t.te;
}

// Steps [s0, min(s1, nsteps)) of every tracer record through the episode's time slices,
// then the cell key of its new position for the next re-bundling.
template <int PM>
__global__ void __launch_bounds__(256, LCS_EP_MINB) ep_advect3_kernel(RectParams P, SliceGeom G,
                                                                      const float4 *__restrict__ slices,
                                                                      size_t plane_stride, const int *__restrict__ smap,
                                                                      Rk4Args A, Tracer *__restrict__ S, int job,
                                                                      int s0, int s1, int shift,
                                                                      unsigned *__restrict__ keys,
                                                                      unsigned *__restrict__ hist)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= A.N) return;
    Tracer t = S[i];
    float x[3] = {t.x, t.y, t.z}, cx[3] = {t.cx, t.cy, t.cz};
    if (t.st == LCS_TRACER_OK) {
        int img[3] = {t.ix, t.iy, t.iz};
        const int ns = A.job_nsteps[job];
        const float h = A.job_h[job];
        const int e = min(s1, ns);
        QuadCache cc;
        cc.v0 = -1;
        cc.slice = -1;
        for (int n = s0; n < e; ++n) {
            const int *m = smap + 3 * (n - s0);
            rk4_step3q<PM>(P, G, x, cx, h, slices, __ldg(m), __ldg(m + 1), __ldg(m + 2), plane_stride, cc);
            wrap_periodic<3, PM>(P, x, cx, img);
            if (rect_left<3, PM>(P, x)) {
                t.st = LCS_TRACER_LEFT;
                t.te = fmaf((float)(n + 1), h, A.job_t0[job]);
                break;
            }
        }
        t.x = x[0];
        t.y = x[1];
        t.z = x[2];
        t.cx = cx[0];
        t.cy = cx[1];
        t.cz = cx[2];
        t.ix = (short)img[0];
        t.iy = (short)img[1];
        t.iz = (short)img[2];
        S[i] = t;
    }
    if (keys) {
        unsigned k = cell_key(P, x, shift);
        keys[i] = k;
        warp_add_one(hist, k);
    }
}

// every tracer record into flow-map slot `slot` (snapshot entry snap, see ep_store): an episode
// ends at each snapshot step before the end of the integration
__global__ void ep_snapshot_kernel(RectParams P, const Tracer *__restrict__ S, Rk4Args A, int slot, int snap)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= A.N) return;
    ep_store(P, A, slot, S[i], snap);
}

// final state of every tracer record into slot `job`, and into the job's snapshot slots whose
// horizon is the whole integration; with M9, the variational grad F of the job
__global__ void ep_finalize_kernel(RectParams P, const Tracer *__restrict__ S, Rk4Args A, int job,
                                   const float *__restrict__ M9)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= A.N) return;
    const Tracer t = S[i];
    ep_store(P, A, job, t, -1);
    if (M9) {
        float *o = A.out_grad + ((size_t)job * A.N + t.id) * 9;
#pragma unroll
        for (int e = 0; e < 9; ++e) o[e] = M9[e * A.N + i];
    }
    const int ns = A.job_nsteps[job];
    for (int q = 0; q < A.nsnap; ++q)
        if (snap_step(A, q, ns) == ns) ep_store(P, A, snap_slot(A, job, q), t, job * A.nsnap + q);
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

// up to 3 distinct stage times per step, 3 component planes per slice
static size_t slice_bytes(const SliceGeom &G, int E)
{
    return al256(16 * (size_t)G.nodes) * 9 * E + al256(sizeof(int) * 3 * E) + al256(sizeof(SchedEntry) * 3 * E) +
           256;
}

size_t rk4_sorted_scratch_bytes(long long N, const lcs_field *f, int E, bool variational)
{
    const long long keys = key_space(f);
    long long nbins = ((keys - 1) >> sort_shift(keys)) + 1;
    long long nb = (nbins + SCAN_TILE - 1) / SCAN_TILE;
    size_t b = 2 * al256(sizeof(Tracer) * N) + 2 * al256(4 * N) + 2 * al256(4 * nbins) + al256(4 * nb);
    b += slice_bytes(slice_geom(f), E);
    if (variational) b += 2 * al256(sizeof(float) * 9 * N);   // grad F planes, ping-pong with the records
    return b;
}

template <int ST>
static cudaError_t episodes(const RectParams &P, const lcs_field *f, const Rk4Args &A, const Rk4Launch &L,
                            cudaStream_t s)
{
    const long long N = A.N;
    const long long nkeys = key_space(f);
    const int shift = sort_shift(nkeys);
    const long long nbins = ((nkeys - 1) >> shift) + 1;
    const long long nb = (nbins + SCAN_TILE - 1) / SCAN_TILE;
    if (nb > 1024 * SCAN_ITEMS || N > 0xffffffffLL) return cudaErrorInvalidValue;
    const int E = L.episode_steps > 0 ? L.episode_steps : LCS_EPISODE_STEPS;
    char *p = (char *)L.work;
    Tracer *SA = (Tracer *)p;
    p += al256(sizeof(Tracer) * N);
    Tracer *SB = (Tracer *)p;
    p += al256(sizeof(Tracer) * N);
    unsigned *keys = (unsigned *)p;
    p += al256(4 * N);
    unsigned *perm = (unsigned *)p;
    p += al256(4 * N);
    unsigned *hist = (unsigned *)p;
    p += al256(4 * nbins);
    unsigned *cursor = (unsigned *)p;
    p += al256(4 * nbins);
    unsigned *bsum = (unsigned *)p;
    p += al256(4 * nb);
    const SliceGeom G = slice_geom(f);
    if (G.nodes > (1LL << 30)) return cudaErrorInvalidValue;
    const size_t plane_stride = al256(16 * (size_t)G.nodes) / 16;
    float4 *slices = nullptr;
    int *smap = nullptr, *nsl = nullptr;
    SchedEntry *stab = nullptr;
    {
        slices = (float4 *)p;
        p += al256(16 * (size_t)G.nodes) * 9 * E;
        smap = (int *)p;
        p += al256(sizeof(int) * 3 * E);
        stab = (SchedEntry *)p;
        p += al256(sizeof(SchedEntry) * 3 * E);
        nsl = (int *)p;
    }
    // variational grad F: [9][N] planes after the rest of the working memory, moved with the records
    const bool var = A.out_grad != nullptr;
    float *MA = nullptr, *MB = nullptr;
    if (var) {
        MA = (float *)((char *)L.work + rk4_sorted_scratch_bytes(N, f, E, false));
        MB = (float *)((char *)MA + al256(sizeof(float) * 9 * N));
    }
    const int bt = 256;
    const unsigned grid = (unsigned)((N + bt - 1) / bt);
    const int abt = L.block_threads > 0 && L.block_threads <= 256 ? L.block_threads : 256;
    const unsigned agrid = (unsigned)((N + abt - 1) / abt);
    for (int job = 0; job < L.njobs; ++job) {
        const int ns = L.host_nsteps[job];
        cudaMemsetAsync(hist, 0, 4 * nbins, s);
        ep_init_kernel<<<grid, bt, 0, s>>>(P, A.seeds, N, SA, A.job_tend, job, shift, keys, hist);
        if (var) ep_var_init_kernel<<<grid, bt, 0, s>>>(MA, N);
        int snext = 0;   // next snapshot before the end of the job: episodes end there
        while (snext < L.nsnap && L.host_snap_n[snext] <= 0) ++snext;
        for (int s0 = 0, s1; s0 < ns; s0 = s1) {
            s1 = s0 + E < ns ? s0 + E : ns;
            int snap_out = -1;
            if (snext < L.nsnap && L.host_snap_n[snext] < ns && L.host_snap_n[snext] <= s1) {
                s1 = L.host_snap_n[snext];
                snap_out = L.njobs + job * L.nsnap + snext;
                ++snext;
            }
            const bool last = s1 >= ns;
            lcs_tm_begin(L.ctx, 1, s);
            scan_reduce_kernel<<<(unsigned)nb, 1024, 0, s>>>(hist, nbins, bsum);
            scan_top_kernel<<<1, 1024, 0, s>>>(bsum, (int)nb);
            scan_down_kernel<<<(unsigned)nb, 1024, 0, s>>>(hist, nbins, bsum, cursor);
            ep_perm_kernel<<<grid, bt, 0, s>>>(N, keys, cursor, perm);
            ep_gather_kernel<<<grid, bt, 0, s>>>(SA, SB, N, perm, MA, MB);
            if (!last) cudaMemsetAsync(hist, 0, 4 * nbins, s);
            lcs_tm_end(L.ctx, 1, s);
            lcs_tm_begin(L.ctx, 2, s);
            ep_slice_table_kernel<<<1, 32, 0, s>>>(A.sched, A.nsteps_max, job, s0, s1, smap, stab, nsl);
            ep_slice_fill_kernel<ST><<<(unsigned)((G.nodes + 255) / 256), 256, 0, s>>>(
                P, G, (const char *)f->d_frames, f->frame_stride, stab, nsl, slices, plane_stride);
            lcs_tm_end(L.ctx, 2, s);
            lcs_tm_begin(L.ctx, 0, s);
            // compile-time periodicity for the common all-periodic and non-periodic boxes
            const int pm = P.periodic[0] | (P.periodic[1] << 1) | (P.periodic[2] << 2);
            unsigned *kk = last ? nullptr : keys;
            if (var) {
                if (pm == 7)
                    ep_var3_kernel<7><<<agrid, abt, 0, s>>>(P, G, slices, plane_stride, smap, A, SB, MB, job, s0, s1,
                                                           shift, kk, hist);
                else if (pm == 0)
                    ep_var3_kernel<0><<<agrid, abt, 0, s>>>(P, G, slices, plane_stride, smap, A, SB, MB, job, s0, s1,
                                                           shift, kk, hist);
                else
                    ep_var3_kernel<-1><<<agrid, abt, 0, s>>>(P, G, slices, plane_stride, smap, A, SB, MB, job, s0,
                                                            s1, shift, kk, hist);
            } else if (pm == 7)
                ep_advect3_kernel<7><<<agrid, abt, 0, s>>>(P, G, slices, plane_stride, smap, A, SB, job, s0, s1, shift,
                                                          kk, hist);
            else if (pm == 0)
                ep_advect3_kernel<0><<<agrid, abt, 0, s>>>(P, G, slices, plane_stride, smap, A, SB, job, s0, s1, shift,
                                                          kk, hist);
            else
                ep_advect3_kernel<-1><<<agrid, abt, 0, s>>>(P, G, slices, plane_stride, smap, A, SB, job, s0, s1,
                                                           shift, kk, hist);
            lcs_tm_end(L.ctx, 0, s);
            if (snap_out >= 0)
                ep_snapshot_kernel<<<grid, bt, 0, s>>>(P, SB, A, snap_out, snap_out - L.njobs);
            Tracer *tmp = SA;
            SA = SB;
            SB = tmp;
            float *mt = MA;
            MA = MB;
            MB = mt;
        }
        ep_finalize_kernel<<<grid, bt, 0, s>>>(P, SA, A, job, MA);
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
