// tet_store.cu -- tetrahedral velocity fields: device store, inverse affine maps, the
// bin lists, and the exact location of seeds (Sec. 2 "Seed": on unstructured data the
// Seed filter finds the cell holding each seed; Sec. 3.1: the local cell search on
// tetrahedra).
//
// Bins: a uniform grid over the nodes' bounding box with about two tets per bin; each bin
// lists, in increasing id, every tet whose bounding box meets it.  A point's bin therefore
// lists every tet that holds it: the seed location's walks and the integrator's walk fall back
// to that list when they meet a boundary face, so the mesh need not be convex.
#include "tet_device.cuh"

#include <math.h>

#include <algorithm>
#include <vector>

// ------------------------------------------------------------ device kernels

__global__ void tet_xyz_kernel(const float *__restrict__ xyz, long long n, float4 *__restrict__ out)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = make_float4(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], 0.0f);
}

// inverse of E = [v1 - v0, v2 - v0, v3 - v0] (columns) in FP64, rounded to FP32 rows, and the
// cell's neighbours as the record's fourth row
__global__ void tet_map_kernel(const float4 *__restrict__ xyz, const int4 *__restrict__ tets,
                               const int4 *__restrict__ nbrs, long long nc, float4 *__restrict__ tmap)
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
        tmap[4 * t + r] = make_float4((float)m[r][0], (float)m[r][1], (float)m[r][2], v0[r]);
    const int4 nb = nbrs[t];
    tmap[4 * t + 3] = make_float4(__int_as_float(nb.x), __int_as_float(nb.y), __int_as_float(nb.z), __int_as_float(nb.w));
}

struct BinGrid {
    float lo[3], inv[3];
    int n[3];
};

__device__ __forceinline__ void tet_bbox_bins(const BinGrid &B, const float4 *xyz, int4 q, int *b0, int *b1)
{
    const float4 a = xyz[q.x], b = xyz[q.y], c = xyz[q.z], d = xyz[q.w];
    const float lo[3] = {fminf(fminf(a.x, b.x), fminf(c.x, d.x)), fminf(fminf(a.y, b.y), fminf(c.y, d.y)),
                         fminf(fminf(a.z, b.z), fminf(c.z, d.z))};
    const float hi[3] = {fmaxf(fmaxf(a.x, b.x), fmaxf(c.x, d.x)), fmaxf(fmaxf(a.y, b.y), fmaxf(c.y, d.y)),
                         fmaxf(fmaxf(a.z, b.z), fmaxf(c.z, d.z))};
    for (int k = 0; k < 3; ++k) {
        b0[k] = mesh_bin_axis(lo[k], B.lo[k], B.inv[k], B.n[k]);
        b1[k] = mesh_bin_axis(hi[k], B.lo[k], B.inv[k], B.n[k]);
    }
}

__global__ void tet_bin_count_kernel(const float4 *__restrict__ xyz, const int4 *__restrict__ tets, long long nc,
                                     BinGrid B, int *__restrict__ count)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= nc) return;
    int b0[3], b1[3];
    tet_bbox_bins(B, xyz, tets[t], b0, b1);
    for (int z = b0[2]; z <= b1[2]; ++z)
        for (int y = b0[1]; y <= b1[1]; ++y)
            for (int x = b0[0]; x <= b1[0]; ++x) atomicAdd(count + x + B.n[0] * (y + (long long)B.n[1] * z), 1);
}

__global__ void tet_bin_fill_kernel(const float4 *__restrict__ xyz, const int4 *__restrict__ tets, long long nc,
                                    BinGrid B, const int *__restrict__ start, int *__restrict__ cursor,
                                    int *__restrict__ list)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= nc) return;
    int b0[3], b1[3];
    tet_bbox_bins(B, xyz, tets[t], b0, b1);
    for (int z = b0[2]; z <= b1[2]; ++z)
        for (int y = b0[1]; y <= b1[1]; ++y)
            for (int x = b0[0]; x <= b1[0]; ++x) {
                const long long b = x + B.n[0] * (y + (long long)B.n[1] * z);
                list[start[b] + atomicAdd(cursor + b, 1)] = (int)t;
            }
}

// each bin's list in increasing id (insertion sort: lists are short)
__global__ void tet_bin_sort_kernel(const int *__restrict__ start, long long nbins, int *__restrict__ list)
{
    const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (b >= nbins) return;
    const int s = start[b], e = start[b + 1];
    for (int i = s + 1; i < e; ++i) {
        const int v = list[i];
        int j = i - 1;
        while (j >= s && list[j] > v) {
            list[j + 1] = list[j];
            --j;
        }
        list[j + 1] = v;
    }
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

// lowest id among the closed tets of bin b holding p (the bin lists every holder of its points,
// in increasing id), -1 if none; a tet whose bounding box misses p is skipped without the exact test
__device__ int exact_bin_scan(const TetDev &T, int b, const float *p)
{
    for (int q = T.bstart[b]; q < T.bstart[b + 1]; ++q) {
        const int c = T.blist[q];
        const int4 v = T.tets[c];
        const float4 A = T.xyz[v.x], B = T.xyz[v.y], C = T.xyz[v.z], D = T.xyz[v.w];
        if (p[0] < fminf(fminf(A.x, B.x), fminf(C.x, D.x)) || p[0] > fmaxf(fmaxf(A.x, B.x), fmaxf(C.x, D.x)) ||
            p[1] < fminf(fminf(A.y, B.y), fminf(C.y, D.y)) || p[1] > fmaxf(fmaxf(A.y, B.y), fmaxf(C.y, D.y)) ||
            p[2] < fminf(fminf(A.z, B.z), fminf(C.z, D.z)) || p[2] > fmaxf(fmaxf(A.z, B.z), fmaxf(C.z, D.z)))
            continue;
        if (exact_contains(T, c, p)) return c;
    }
    return -1;
}

// Lowest id among the closed tets holding p, -1 outside the mesh.
//  1. An FP32 walk (as in the integrator) from the first tet listed for p's bin gets next to p.
//  2. An exact walk from there: exact orientation signs decide containment, and among the faces
//     whose exact sign is negative the walk crosses the first one in an order rotated by a
//     hash of (seed, step) -- a remembering stochastic walk, which cannot cycle on degenerate
//     (cospherical) configurations the way a deterministic choice can.  A walk that meets a
//     boundary face (the mesh need not be convex) or its step limit is settled by the bin list.
//  3. Where p lies on a face, edge or vertex, a breadth-first search over the closed tets across
//     faces holding p collects every holder and keeps the lowest id.
__global__ void tet_seed_locate_kernel(TetDev T, const float *__restrict__ seeds, long long N, int walk_limit,
                                       int *__restrict__ cells)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float p[3] = {seeds[i], seeds[N + i], seeds[2 * N + i]};
    if (!(isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2]))) {
        cells[i] = -1;
        return;
    }
    const int b = tet_bin(T, p);
    if (T.bstart[b] == T.bstart[b + 1]) {  // no tet's bounding box meets the bin
        cells[i] = -1;
        return;
    }
    int c = T.blist[T.bstart[b]];
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
    bool it_boundary = false;
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
            it_boundary = true;
            break;
        }
        c = n;
    }
    if (res < 0) {  // a boundary face (outside, if the mesh is convex) or the walk limit: the bin list decides
        cells[i] = T.convex && it_boundary ? -1 : exact_bin_scan(T, b, p);
        return;
    }
    if (sg[0] > 0 && sg[1] > 0 && sg[2] > 0 && sg[3] > 0) {
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
                cells[i] = exact_bin_scan(T, b, p);
                return;
            }
            seen[nseen++] = nn[j];
            stack[ns++] = nn[j];
        }
    }
    cells[i] = best;
}

// a boundary face (a, b, c) with the tet's fourth vertex `in` on its interior side: the mesh is
// concave at an edge of the face when the neighbouring boundary face's far vertex w lies strictly
// on the other side (exact signs)
__global__ void tet_convex_kernel(const float4 *__restrict__ xyz, const int *__restrict__ chk, long long n,
                                  int *__restrict__ convex)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int *q = chk + 5 * i;
    float v[5][3];
    for (int k = 0; k < 5; ++k) {
        const float4 p = xyz[q[k]];
        v[k][0] = p.x;
        v[k][1] = p.y;
        v[k][2] = p.z;
    }
    const int s_in = orient3d_sign(v[0], v[1], v[2], v[3]), s_w = orient3d_sign(v[0], v[1], v[2], v[4]);
    if (s_in * s_w < 0) atomicExch(convex, 0);
}

// ------------------------------------------------------------------ host side

bool mesh_connected(const int *nbrs, long long nc, int nv)
{
    if (nc == 0) return true;
    std::vector<char> seen((size_t)nc, 0);
    std::vector<int> stack(1, 0);
    seen[0] = 1;
    long long count = 1;
    while (!stack.empty()) {
        const int c = stack.back();
        stack.pop_back();
        for (int j = 0; j < nv; ++j) {
            const int n = nbrs[(size_t)nv * c + j];
            if (n >= 0 && !seen[(size_t)n]) {
                seen[(size_t)n] = 1;
                ++count;
                stack.push_back(n);
            }
        }
    }
    return count == nc;
}

// For every boundary edge shared by exactly two boundary faces, two checks (face, interior vertex,
// far vertex of the other face) as 5 node ids each.  Returns false when some boundary edge is not
// shared by exactly two boundary faces (then the mesh is not treated as convex).
static bool tet_convexity_checks(const int *tets, const int *nbrs, long long nc, std::vector<int> &chk)
{
    struct E {
        int u, v;
        long long tj;  // boundary face: tet * 4 + j
        int w;         // the face's vertex off the edge
    };
    std::vector<E> e;
    for (long long t = 0; t < nc; ++t)
        for (int j = 0; j < 4; ++j) {
            if (nbrs[4 * t + j] >= 0) continue;
            int f[3], m = 0;
            for (int k = 0; k < 4; ++k)
                if (k != j) f[m++] = tets[4 * t + k];
            for (int k = 0; k < 3; ++k) {
                int u = f[k], v = f[(k + 1) % 3];
                if (u > v) std::swap(u, v);
                e.push_back({u, v, 4 * t + j, f[(k + 2) % 3]});
            }
        }
    std::sort(e.begin(), e.end(), [](const E &x, const E &y) {
        if (x.u != y.u) return x.u < y.u;
        if (x.v != y.v) return x.v < y.v;
        return x.tj < y.tj;
    });
    auto face = [&](long long tj, int *q) {
        const long long t = tj / 4;
        const int j = (int)(tj % 4);
        int m = 0;
        for (int k = 0; k < 4; ++k)
            if (k != j) q[m++] = tets[4 * t + k];
        q[3] = tets[4 * t + j];
    };
    for (size_t i = 0; i < e.size();) {
        size_t k = i;
        while (k < e.size() && e[k].u == e[i].u && e[k].v == e[i].v) ++k;
        if (k - i != 2) return false;
        int q[4];
        for (int s = 0; s < 2; ++s) {
            face(e[i + s].tj, q);
            chk.insert(chk.end(), {q[0], q[1], q[2], q[3], e[i + 1 - s].w});
        }
        i = k;
    }
    return true;
}

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
    for (int d = 0; d < 3; ++d) {
        f->bin_n[d] = B.n[d];
        f->bin_lo[d] = B.lo[d];
        f->bin_inv[d] = B.inv[d];
    }
    f->nbins = nbins;
    float *dxyz = nullptr;
    int *count = nullptr, *cursor = nullptr;
    cudaError_t e = cudaMalloc(&f->d_xyz, sizeof(float4) * nn);
    if (e == cudaSuccess) e = cudaMalloc(&f->d_tets, sizeof(int4) * nc);
    if (e == cudaSuccess) e = cudaMalloc(&f->d_nbrs, sizeof(int4) * nc);
    if (e == cudaSuccess) e = cudaMalloc(&f->d_tetmap, sizeof(float4) * 4 * nc);
    if (e == cudaSuccess) e = cudaMalloc(&f->d_bstart, sizeof(int) * (nbins + 1));
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&dxyz, sizeof(float) * 3 * nn, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&count, sizeof(int) * nbins, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&cursor, sizeof(int) * nbins, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dxyz, xyz_host, sizeof(float) * 3 * nn, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f->d_tets, tets_host, sizeof(int4) * nc, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f->d_nbrs, nbrs_host, sizeof(int4) * nc, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, sizeof(int) * nbins, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cursor, 0, sizeof(int) * nbins, s);
    const int bt = 256;
    const unsigned gc = (unsigned)((nc + bt - 1) / bt);
    if (e == cudaSuccess) {
        tet_xyz_kernel<<<(unsigned)((nn + bt - 1) / bt), bt, 0, s>>>(dxyz, nn, f->d_xyz);
        tet_map_kernel<<<gc, bt, 0, s>>>(f->d_xyz, f->d_tets, f->d_nbrs, nc, f->d_tetmap);
        tet_bin_count_kernel<<<gc, bt, 0, s>>>(f->d_xyz, f->d_tets, nc, B, count);
        e = cudaGetLastError();
    }
    // the CSR offsets on the host (load time only)
    std::vector<int> h((size_t)nbins), st((size_t)nbins + 1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), count, sizeof(int) * nbins, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    long long total = 0;
    if (e == cudaSuccess) {
        for (long long b = 0; b < nbins; ++b) {
            st[(size_t)b] = (int)total;
            total += h[(size_t)b];
        }
        st[(size_t)nbins] = (int)total;
        if (total >= (1LL << 31)) e = cudaErrorInvalidValue;
    }
    if (e == cudaSuccess) e = cudaMalloc(&f->d_blist, sizeof(int) * std::max(total, 1LL));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(f->d_bstart, st.data(), sizeof(int) * (nbins + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        tet_bin_fill_kernel<<<gc, bt, 0, s>>>(f->d_xyz, f->d_tets, nc, B, f->d_bstart, cursor, f->d_blist);
        tet_bin_sort_kernel<<<(unsigned)((nbins + bt - 1) / bt), bt, 0, s>>>(f->d_bstart, nbins, f->d_blist);
        e = cudaGetLastError();
    }
    // convex (connected, every boundary edge convex): then a walk that meets the boundary is outside
    std::vector<int> chk;
    int convex = mesh_connected(nbrs_host, nc, 4) && tet_convexity_checks(tets_host, nbrs_host, nc, chk) ? 1 : 0;
    int *dchk = nullptr, *dflag = nullptr;
    const long long nchk = (long long)chk.size() / 5;
    if (e == cudaSuccess && convex && nchk > 0) {
        e = cudaMallocAsync((void **)&dchk, sizeof(int) * chk.size(), s);
        if (e == cudaSuccess) e = cudaMallocAsync((void **)&dflag, sizeof(int), s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dchk, chk.data(), sizeof(int) * chk.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dflag, &convex, sizeof(int), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) {
            tet_convex_kernel<<<(unsigned)((nchk + bt - 1) / bt), bt, 0, s>>>(f->d_xyz, dchk, nchk, dflag);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(&convex, dflag, sizeof(int), cudaMemcpyDeviceToHost, s);
    }
    if (dxyz) cudaFreeAsync(dxyz, s);
    if (count) cudaFreeAsync(count, s);
    if (cursor) cudaFreeAsync(cursor, s);
    if (dchk) cudaFreeAsync(dchk, s);
    if (dflag) cudaFreeAsync(dflag, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host values above go out of scope
    f->convex = e == cudaSuccess ? convex : 0;
    return e;
}

TetDev tet_dev(const lcs_field *f, int walk_limit)
{
    TetDev T;
    T.xyz = f->d_xyz;
    T.tets = f->d_tets;
    T.nbrs = f->d_nbrs;
    T.tmap = f->d_tetmap;
    T.bstart = f->d_bstart;
    T.blist = f->d_blist;
    for (int d = 0; d < 3; ++d) {
        T.blo[d] = f->bin_lo[d];
        T.binv[d] = f->bin_inv[d];
        T.bn[d] = f->bin_n[d];
    }
    T.pairs = (const char *)f->d_frames;
    T.fstride = f->frame_stride;
    T.ncells = f->ncells;
    T.walk_limit = walk_limit > 0 ? walk_limit : 512;
    T.tol = 1e-6f;
    T.convex = f->convex;
    return T;
}

cudaError_t tet_locate_seeds(const lcs_field *f, const float *seeds, long long N, int *cells, cudaStream_t s)
{
    if (N == 0) return cudaSuccess;
    const TetDev T = tet_dev(f, 0);
    const int bt = 128;
    tet_seed_locate_kernel<<<(unsigned)((N + bt - 1) / bt), bt, 0, s>>>(T, seeds, N, 1 << 16, cells);
    return cudaGetLastError();
}
