// tet_store.cu -- tetrahedral velocity fields: device store, inverse affine maps, a
// bin grid of walk starts, and the exact location of seeds (Sec. 2 "Seed": on
// unstructured data the Seed filter finds the cell holding each seed; Sec. 3.1: the
// local cell search on tetrahedra).
#include "tet_device.cuh"

#include <math.h>

#include <algorithm>
#include <vector>

#define BIN_EMPTY 0x7f7f7f7f  // what a 0x7f byte fill leaves in an int

// 32-bit integer hash (Wellons' lowbias32): face order of the stochastic walk
__device__ __forceinline__ unsigned lowbias32_t(unsigned x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// ------------------------------------------------------------ device kernels

__global__ void tet_xyz_kernel(const float *__restrict__ xyz, long long n, float4 *__restrict__ out)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = make_float4(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], 0.0f);
}

// inverse of E = [v1 - v0, v2 - v0, v3 - v0] (columns) in FP64, rounded to FP32 rows
__global__ void tet_map_kernel(const float4 *__restrict__ xyz, const int4 *__restrict__ tets, long long nc,
                               float4 *__restrict__ tmap)
{
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= nc) return;
    const int4 q = tets[t];
    const float4 p0 = xyz[q.x], p1 = xyz[q.y], p2 = xyz[q.z], p3 = xyz[q.w];
    const double e[3][3] = {{(double)p1.x - p0.x, (double)p2.x - p0.x, (double)p3.x - p0.x},
                            {(double)p1.y - p0.y, (double)p2.y - p0.y, (double)p3.y - p0.y},
                            {(double)p1.z - p0.z, (double)p2.z - p0.z, (double)p3.z - p0.z}};
    const double c00 = e[1][1] * e[2][2] - e[1][2] * e[2][1], c01 = e[1][2] * e[2][0] - e[1][0] * e[2][2],
                 c02 = e[1][0] * e[2][1] - e[1][1] * e[2][0];
    const double det = e[0][0] * c00 + e[0][1] * c01 + e[0][2] * c02;
    const double id = 1.0 / det;
    double m[3][3];
    m[0][0] = c00 * id;
    m[0][1] = (e[0][2] * e[2][1] - e[0][1] * e[2][2]) * id;
    m[0][2] = (e[0][1] * e[1][2] - e[0][2] * e[1][1]) * id;
    m[1][0] = c01 * id;
    m[1][1] = (e[0][0] * e[2][2] - e[0][2] * e[2][0]) * id;
    m[1][2] = (e[0][2] * e[1][0] - e[0][0] * e[1][2]) * id;
    m[2][0] = c02 * id;
    m[2][1] = (e[0][1] * e[2][0] - e[0][0] * e[2][1]) * id;
    m[2][2] = (e[0][0] * e[1][1] - e[0][1] * e[1][0]) * id;
    const float v0[3] = {p0.x, p0.y, p0.z};
    for (int r = 0; r < 3; ++r)
        tmap[3 * t + r] = make_float4((float)m[r][0], (float)m[r][1], (float)m[r][2], v0[r]);
}

struct BinGrid {
    float lo[3], inv[3];
    int n[3];
};

__device__ __forceinline__ long long bin_of(const BinGrid &B, float x, float y, float z)
{
    const float p[3] = {x, y, z};
    int c[3];
    for (int d = 0; d < 3; ++d) {
        float s = (p[d] - B.lo[d]) * B.inv[d];
        int v = isfinite(s) ? (int)floorf(s) : 0;
        c[d] = min(max(v, 0), B.n[d] - 1);
    }
    return c[0] + (long long)B.n[0] * (c[1] + (long long)B.n[1] * c[2]);
}

// each bin remembers the lowest-id tet whose centroid falls in it
__global__ void tet_bin_kernel(const float4 *__restrict__ xyz, const int4 *__restrict__ tets, long long nc, BinGrid B,
                               int *__restrict__ bins)
{
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= nc) return;
    const int4 q = tets[t];
    const float4 a = xyz[q.x], b = xyz[q.y], c = xyz[q.z], d = xyz[q.w];
    atomicMin(bins + bin_of(B, 0.25f * (a.x + b.x + c.x + d.x), 0.25f * (a.y + b.y + c.y + d.y),
                            0.25f * (a.z + b.z + c.z + d.z)),
              (int)t);
}

// empty bins borrow the tet of the nearest filled bin within two rings, else tet 0
__global__ void tet_bin_fill_kernel(BinGrid B, const int *__restrict__ in, int *__restrict__ out)
{
    long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long nb = (long long)B.n[0] * B.n[1] * B.n[2];
    if (b >= nb) return;
    int v = in[b];
    if (v != BIN_EMPTY) {
        out[b] = v;
        return;
    }
    const int x = (int)(b % B.n[0]), y = (int)((b / B.n[0]) % B.n[1]), z = (int)(b / ((long long)B.n[0] * B.n[1]));
    int best = BIN_EMPTY, bestd = 1 << 30;
    for (int dz = -2; dz <= 2; ++dz)
        for (int dy = -2; dy <= 2; ++dy)
            for (int dx = -2; dx <= 2; ++dx) {
                int X = x + dx, Y = y + dy, Z = z + dz;
                if (X < 0 || Y < 0 || Z < 0 || X >= B.n[0] || Y >= B.n[1] || Z >= B.n[2]) continue;
                int w = in[X + (long long)B.n[0] * (Y + (long long)B.n[1] * Z)];
                int dd = dx * dx + dy * dy + dz * dz;
                if (w != BIN_EMPTY && (dd < bestd || (dd == bestd && w < best))) {
                    best = w;
                    bestd = dd;
                }
            }
    out[b] = best == BIN_EMPTY ? 0 : best;
}

__device__ __forceinline__ void vtx(const TetDev &T, int node, float *p)
{
    const float4 v = T.xyz[node];
    p[0] = v.x;
    p[1] = v.y;
    p[2] = v.z;
}

// signs of the barycentric coordinates of p in tet c, exactly
__device__ void exact_signs(const TetDev &T, int c, const float *p, int *sg)
{
    const int4 q = T.tets[c];
    float v[4][3];
    vtx(T, q.x, v[0]);
    vtx(T, q.y, v[1]);
    vtx(T, q.z, v[2]);
    vtx(T, q.w, v[3]);
    const int D = orient3d_sign(v[0], v[1], v[2], v[3]);
    sg[0] = D * orient3d_sign(p, v[1], v[2], v[3]);
    sg[1] = D * orient3d_sign(v[0], p, v[2], v[3]);
    sg[2] = D * orient3d_sign(v[0], v[1], p, v[3]);
    sg[3] = D * orient3d_sign(v[0], v[1], v[2], p);
}

__device__ bool exact_contains(const TetDev &T, int c, const float *p)
{
    int sg[4];
    exact_signs(T, c, p, sg);
    return sg[0] >= 0 && sg[1] >= 0 && sg[2] >= 0 && sg[3] >= 0;
}

__device__ int exact_brute(const TetDev &T, const float *p)
{
    for (long long c = 0; c < T.ncells; ++c)
        if (exact_contains(T, (int)c, p)) return (int)c;
    return -1;
}

// Lowest id among the closed tets holding p, -1 outside the mesh.
//  1. An FP32 walk (as in the integrator) from the bin's tet gets next to p cheaply.
//  2. An exact walk from there: exact orientation signs decide containment, and among the faces
//     whose exact sign is negative the walk crosses the first one in an order rotated by a
//     hash of (seed, step) -- a remembering stochastic walk, which cannot cycle on degenerate
//     (cospherical) configurations the way a deterministic choice can.  The result does not
//     depend on the path: it is the unique lowest-id closed tet holding p.
//  3. Where p lies on a face, edge or vertex, a breadth-first search over the closed tets across
//     faces holding p collects every holder and keeps the lowest id.
__global__ void tet_seed_locate_kernel(TetDev T, const float *__restrict__ seeds, long long N, BinGrid B,
                                       const int *__restrict__ bins, int walk_limit, int *__restrict__ cells)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float p[3] = {seeds[i], seeds[N + i], seeds[2 * N + i]};
    int c = bins[bin_of(B, p[0], p[1], p[2])];
    {   // 1. FP32 walk, bounded
        float lam[4];
        for (int it = 0; it < 1024; ++it) {
            tet_bary(T, c, p, lam);
            int jm = 0;
            float lm = lam[0];
            for (int j = 1; j < 4; ++j)
                if (lam[j] < lm) {
                    lm = lam[j];
                    jm = j;
                }
            if (!(lm < -1e-6f)) break;
            const int4 nb = T.nbrs[c];
            const int n = jm == 0 ? nb.x : jm == 1 ? nb.y : jm == 2 ? nb.z : nb.w;
            if (n < 0) break;
            c = n;
        }
    }
    int res = -2;
    int sg[4];
    for (int it = 0; it < walk_limit; ++it) {  // 2. exact walk
        exact_signs(T, c, p, sg);
        if (sg[0] >= 0 && sg[1] >= 0 && sg[2] >= 0 && sg[3] >= 0) {
            res = c;
            break;
        }
        const int rot = (int)(lowbias32_t((unsigned)i * 0x9E3779B9u ^ (unsigned)it) & 3u);
        int jm = 0;
        for (int q = 0; q < 4; ++q) {
            const int j = (q + rot) & 3;
            if (sg[j] < 0) {
                jm = j;
                break;
            }
        }
        const int4 nb = T.nbrs[c];
        const int n = jm == 0 ? nb.x : jm == 1 ? nb.y : jm == 2 ? nb.z : nb.w;
        if (n < 0) {
            res = -1;
            break;
        }
        c = n;
    }
    if (res == -2) {  // walk limit: fall back to testing every tet
        cells[i] = exact_brute(T, p);
        return;
    }
    if (res < 0 || (sg[0] > 0 && sg[1] > 0 && sg[2] > 0 && sg[3] > 0)) {
        cells[i] = res;
        return;
    }
    // 3. p on a face, edge or vertex of res: breadth-first over the closed tets across faces holding p
    constexpr int CAP = 128;
    int stack[CAP], seen[CAP];
    int ns = 0, nseen = 0, best = res;
    stack[ns++] = res;
    seen[nseen++] = res;
    while (ns > 0) {
        const int cc = stack[--ns];
        best = min(best, cc);
        int s2[4];
        exact_signs(T, cc, p, s2);
        const int4 nb = T.nbrs[cc];
        const int nn[4] = {nb.x, nb.y, nb.z, nb.w};
        for (int j = 0; j < 4; ++j) {
            if (s2[j] != 0 || nn[j] < 0) continue;
            bool dup = false;
            for (int q = 0; q < nseen; ++q) dup |= seen[q] == nn[j];
            if (dup || !exact_contains(T, nn[j], p)) continue;
            if (nseen >= CAP || ns >= CAP) {
                cells[i] = exact_brute(T, p);
                return;
            }
            seen[nseen++] = nn[j];
            stack[ns++] = nn[j];
        }
    }
    cells[i] = best;
}

// ------------------------------------------------------------------ host side

// tet across the face opposite vertex j, by matching sorted vertex triples
static void build_neighbours(const int *tets, long long nc, std::vector<int> &nbrs)
{
    struct Face {
        int a, b, c;
        long long tf;  // tet * 4 + j
    };
    std::vector<Face> f((size_t)nc * 4);
    for (long long t = 0; t < nc; ++t)
        for (int j = 0; j < 4; ++j) {
            int v[3], m = 0;
            for (int k = 0; k < 4; ++k)
                if (k != j) v[m++] = tets[4 * t + k];
            std::sort(v, v + 3);
            f[(size_t)(4 * t + j)] = {v[0], v[1], v[2], 4 * t + j};
        }
    std::sort(f.begin(), f.end(), [](const Face &x, const Face &y) {
        if (x.a != y.a) return x.a < y.a;
        if (x.b != y.b) return x.b < y.b;
        if (x.c != y.c) return x.c < y.c;
        return x.tf < y.tf;
    });
    nbrs.assign((size_t)nc * 4, -1);
    for (size_t i = 0; i + 1 < f.size(); ++i)
        if (f[i].a == f[i + 1].a && f[i].b == f[i + 1].b && f[i].c == f[i + 1].c) {
            nbrs[(size_t)f[i].tf] = (int)(f[i + 1].tf / 4);
            nbrs[(size_t)f[i + 1].tf] = (int)(f[i].tf / 4);
            ++i;
        }
}

cudaError_t tet_build_store(lcs_field *f, const float *xyz_host, const int *tets_host, const int *nbrs_host,
                            cudaStream_t s)
{
    const long long nn = f->nodes, nc = f->ncells;
    std::vector<int> nb_built;
    if (!nbrs_host) {
        build_neighbours(tets_host, nc, nb_built);
        nbrs_host = nb_built.data();
    }
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (long long i = 0; i < nn; ++i)
        for (int d = 0; d < 3; ++d) {
            lo[d] = std::min(lo[d], xyz_host[3 * i + d]);
            hi[d] = std::max(hi[d], xyz_host[3 * i + d]);
        }
    BinGrid B;
    const double vol = std::max(1e-30, (double)(hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]));
    const double cell = cbrt(vol / std::max(1.0, (double)nc / 2.0));  // about two tets per bin
    for (int d = 0; d < 3; ++d) {
        double ext = std::max((double)(hi[d] - lo[d]), 1e-30);
        B.n[d] = (int)std::min(1024.0, std::max(1.0, ceil(ext / cell)));
        B.lo[d] = lo[d];
        B.inv[d] = (float)(B.n[d] / ext);
    }
    const long long nbins = (long long)B.n[0] * B.n[1] * B.n[2];
    f->bin_n[0] = B.n[0];
    f->bin_n[1] = B.n[1];
    f->bin_n[2] = B.n[2];
    for (int d = 0; d < 3; ++d) {
        f->bin_lo[d] = B.lo[d];
        f->bin_inv[d] = B.inv[d];
    }
    float *dxyz = nullptr;
    int *tmpbins = nullptr;
    cudaError_t e = cudaMalloc(&f->d_xyz, sizeof(float4) * nn);
    if (e == cudaSuccess) e = cudaMalloc(&f->d_tets, sizeof(int4) * nc);
    if (e == cudaSuccess) e = cudaMalloc(&f->d_nbrs, sizeof(int4) * nc);
    if (e == cudaSuccess) e = cudaMalloc(&f->d_tetmap, sizeof(float4) * 3 * nc);
    if (e == cudaSuccess) e = cudaMalloc(&f->d_bins, sizeof(int) * nbins);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&dxyz, sizeof(float) * 3 * nn, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&tmpbins, sizeof(int) * nbins, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dxyz, xyz_host, sizeof(float) * 3 * nn, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f->d_tets, tets_host, sizeof(int4) * nc, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f->d_nbrs, nbrs_host, sizeof(int4) * nc, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(tmpbins, 0x7f, sizeof(int) * nbins, s);  // BIN_EMPTY
    if (e != cudaSuccess) {
        if (dxyz) cudaFreeAsync(dxyz, s);
        if (tmpbins) cudaFreeAsync(tmpbins, s);
        return e;
    }
    const int bt = 256;
    tet_xyz_kernel<<<(unsigned)((nn + bt - 1) / bt), bt, 0, s>>>(dxyz, nn, f->d_xyz);
    tet_map_kernel<<<(unsigned)((nc + bt - 1) / bt), bt, 0, s>>>(f->d_xyz, f->d_tets, nc, f->d_tetmap);
    tet_bin_kernel<<<(unsigned)((nc + bt - 1) / bt), bt, 0, s>>>(f->d_xyz, f->d_tets, nc, B, tmpbins);
    tet_bin_fill_kernel<<<(unsigned)((nbins + bt - 1) / bt), bt, 0, s>>>(B, tmpbins, f->d_bins);
    e = cudaGetLastError();
    cudaFreeAsync(dxyz, s);
    cudaFreeAsync(tmpbins, s);
    return e;
}

cudaError_t tet_locate_seeds(const lcs_field *f, const float *seeds, long long N, int walk_limit, int *cells,
                             cudaStream_t s)
{
    if (N == 0) return cudaSuccess;
    TetDev T;
    T.xyz = f->d_xyz;
    T.tets = f->d_tets;
    T.nbrs = f->d_nbrs;
    T.tmap = f->d_tetmap;
    T.pairs = (const char *)f->d_frames;
    T.fstride = f->frame_stride;
    T.ncells = f->ncells;
    T.walk_limit = walk_limit;
    T.tol = 0.0f;
    BinGrid B;
    for (int d = 0; d < 3; ++d) {
        B.n[d] = f->bin_n[d];
        B.lo[d] = f->bin_lo[d];
        B.inv[d] = f->bin_inv[d];
    }
    const int bt = 128;
    tet_seed_locate_kernel<<<(unsigned)((N + bt - 1) / bt), bt, 0, s>>>(T, seeds, N, B, f->d_bins, walk_limit,
                                                                        cells);
    return cudaGetLastError();
}
