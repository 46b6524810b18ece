// tri_store.cu -- triangle-mesh velocity fields: device store, inverse affine maps, the
// bin lists, and the exact location of seeds (Sec. 2 "Seed": on unstructured data the
// Seed filter finds the cell holding each seed; Sec. 3.1: the cell search on triangles).
//
// Bins: a uniform grid over the nodes' bounding box with about two triangles per bin; each
// bin lists, in increasing id, every triangle whose bounding box meets it.  A point's bin
// therefore lists every triangle that holds it, so the seed location tests only that list
// with exact orientation signs and keeps the lowest id (no walk, no tie-break search), and
// the integrator's walk falls back to the same list when it meets a boundary edge.
#include "tri_device.cuh"

#include <math.h>

#include <algorithm>
#include <vector>

namespace {

// inverse of E = [v1 - v0, v2 - v0] (columns) in FP64, rounded to FP32
__global__ void tri_map_kernel(const float2 *__restrict__ xy, const int4 *__restrict__ tris, long long nc,
                               float4 *__restrict__ tmap, float2 *__restrict__ tv0)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= nc) return;
    const int4 q = tris[t];
    const float2 p0 = xy[q.x], p1 = xy[q.y], p2 = xy[q.z];
    const double e00 = (double)p1.x - p0.x, e01 = (double)p2.x - p0.x;
    const double e10 = (double)p1.y - p0.y, e11 = (double)p2.y - p0.y;
    const double id = 1.0 / (e00 * e11 - e01 * e10);
    tmap[t] = make_float4((float)(e11 * id), (float)(-e01 * id), (float)(-e10 * id), (float)(e00 * id));
    tv0[t] = p0;
}

struct TriBins {
    float lo[2], inv[2];
    int n[2];
};

__device__ __forceinline__ void tri_bbox_bins(const TriBins &B, const float2 *xy, int4 q, int *b0, int *b1)
{
    const float2 a = xy[q.x], b = xy[q.y], c = xy[q.z];
    const float lo[2] = {fminf(a.x, fminf(b.x, c.x)), fminf(a.y, fminf(b.y, c.y))};
    const float hi[2] = {fmaxf(a.x, fmaxf(b.x, c.x)), fmaxf(a.y, fmaxf(b.y, c.y))};
    for (int d = 0; d < 2; ++d) {
        b0[d] = mesh_bin_axis(lo[d], B.lo[d], B.inv[d], B.n[d]);
        b1[d] = mesh_bin_axis(hi[d], B.lo[d], B.inv[d], B.n[d]);
    }
}

__global__ void tri_bin_count_kernel(const float2 *__restrict__ xy, const int4 *__restrict__ tris, long long nc,
                                     TriBins B, int *__restrict__ count)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= nc) return;
    int b0[2], b1[2];
    tri_bbox_bins(B, xy, tris[t], b0, b1);
    for (int y = b0[1]; y <= b1[1]; ++y)
        for (int x = b0[0]; x <= b1[0]; ++x) atomicAdd(count + x + B.n[0] * y, 1);
}

__global__ void tri_bin_fill_kernel(const float2 *__restrict__ xy, const int4 *__restrict__ tris, long long nc,
                                    TriBins B, const int *__restrict__ start, int *__restrict__ cursor,
                                    int *__restrict__ list)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= nc) return;
    int b0[2], b1[2];
    tri_bbox_bins(B, xy, tris[t], b0, b1);
    for (int y = b0[1]; y <= b1[1]; ++y)
        for (int x = b0[0]; x <= b1[0]; ++x) {
            const int b = x + B.n[0] * y;
            list[start[b] + atomicAdd(cursor + b, 1)] = (int)t;
        }
}

// each bin's list in increasing id (insertion sort: lists are short)
__global__ void tri_bin_sort_kernel(const int *__restrict__ start, long long nbins, int *__restrict__ list)
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

// exact signs of the barycentric coordinates of p in triangle c (either orientation)
__device__ bool tri_exact_contains(const TriDev &T, int c, const float *p)
{
    const int4 q = T.tris[c];
    const float2 A = T.xy[q.x], B = T.xy[q.y], C = T.xy[q.z];
    const float a[2] = {A.x, A.y}, b[2] = {B.x, B.y}, cc[2] = {C.x, C.y};
    const int D = orient2d_sign(a, b, cc);
    const int s0 = D * orient2d_sign(p, b, cc), s1 = D * orient2d_sign(a, p, cc), s2 = D * orient2d_sign(a, b, p);
    return s0 >= 0 && s1 >= 0 && s2 >= 0;
}

// lowest id among the closed triangles holding the seed, -1 if none
__global__ void tri_seed_locate_kernel(TriDev T, const float *__restrict__ seeds, long long N, int *__restrict__ cells)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float p[2] = {seeds[i], seeds[N + i]};
    int res = -1;
    if (isfinite(p[0]) && isfinite(p[1])) {
        const int b = mesh_bin_axis(p[0], T.blo[0], T.binv[0], T.bn[0]) +
                      T.bn[0] * mesh_bin_axis(p[1], T.blo[1], T.binv[1], T.bn[1]);
        for (int q = T.bstart[b]; q < T.bstart[b + 1]; ++q) {
            const int4 v = T.tris[T.blist[q]];
            const float2 A = T.xy[v.x], B = T.xy[v.y], C = T.xy[v.z];
            if (p[0] < fminf(A.x, fminf(B.x, C.x)) || p[0] > fmaxf(A.x, fmaxf(B.x, C.x)) ||
                p[1] < fminf(A.y, fminf(B.y, C.y)) || p[1] > fmaxf(A.y, fmaxf(B.y, C.y)))
                continue;  // the bounding box misses p: not a holder
            if (tri_exact_contains(T, T.blist[q], p)) {
                res = T.blist[q];  // ids increase along the list: the first holder is the lowest
                break;
            }
        }
    }
    cells[i] = res;
}

// a boundary edge (a, b) with the triangle's third vertex `in` on its interior side: the mesh is
// concave at a vertex of the edge when the neighbouring boundary edge's far vertex w lies strictly
// on the other side (exact signs)
__global__ void tri_convex_kernel(const float2 *__restrict__ xy, const int *__restrict__ chk, long long n,
                                  int *__restrict__ convex)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int *q = chk + 4 * i;
    float v[4][2];
    for (int k = 0; k < 4; ++k) {
        const float2 p = xy[q[k]];
        v[k][0] = p.x;
        v[k][1] = p.y;
    }
    const int s_in = orient2d_sign(v[0], v[1], v[2]), s_w = orient2d_sign(v[0], v[1], v[3]);
    if (s_in * s_w < 0) atomicExch(convex, 0);
}

// For every boundary vertex shared by exactly two boundary edges, two checks (edge, interior
// vertex, far vertex of the other edge) as 4 node ids each; false when some boundary vertex is
// not (then the mesh is not treated as convex).
bool tri_convexity_checks(const int *tris, const int *nbrs, long long nc, std::vector<int> &chk)
{
    struct V {
        int v;
        long long tj;  // boundary edge: triangle * 3 + j
        int w;         // the edge's other end
    };
    std::vector<V> e;
    for (long long t = 0; t < nc; ++t)
        for (int j = 0; j < 3; ++j) {
            if (nbrs[3 * t + j] >= 0) continue;
            const int a = tris[3 * t + (j + 1) % 3], b = tris[3 * t + (j + 2) % 3];
            e.push_back({a, 3 * t + j, b});
            e.push_back({b, 3 * t + j, a});
        }
    std::sort(e.begin(), e.end(), [](const V &x, const V &y) { return x.v != y.v ? x.v < y.v : x.tj < y.tj; });
    for (size_t i = 0; i < e.size();) {
        size_t k = i;
        while (k < e.size() && e[k].v == e[i].v) ++k;
        if (k - i != 2) return false;
        for (int s = 0; s < 2; ++s) {
            const long long t = e[i + s].tj / 3;
            const int j = (int)(e[i + s].tj % 3);
            chk.insert(chk.end(), {tris[3 * t + (j + 1) % 3], tris[3 * t + (j + 2) % 3], tris[3 * t + j],
                                   e[i + 1 - s].w});
        }
        i = k;
    }
    return true;
}

// triangle across the edge opposite vertex j, by matching sorted vertex pairs
void build_tri_neighbours(const int *tris, long long nc, std::vector<int> &nbrs)
{
    struct Edge {
        int a, b;
        long long tj;  // triangle * 3 + j
    };
    std::vector<Edge> e((size_t)nc * 3);
    for (long long t = 0; t < nc; ++t)
        for (int j = 0; j < 3; ++j) {
            int u = tris[3 * t + (j + 1) % 3], v = tris[3 * t + (j + 2) % 3];
            if (u > v) std::swap(u, v);
            e[(size_t)(3 * t + j)] = {u, v, 3 * t + j};
        }
    std::sort(e.begin(), e.end(), [](const Edge &x, const Edge &y) {
        if (x.a != y.a) return x.a < y.a;
        if (x.b != y.b) return x.b < y.b;
        return x.tj < y.tj;
    });
    nbrs.assign((size_t)nc * 3, -1);
    for (size_t i = 0; i + 1 < e.size(); ++i)
        if (e[i].a == e[i + 1].a && e[i].b == e[i + 1].b) {
            nbrs[(size_t)e[i].tj] = (int)(e[i + 1].tj / 3);
            nbrs[(size_t)e[i + 1].tj] = (int)(e[i].tj / 3);
            ++i;
        }
}

}  // namespace

cudaError_t tri_build_store(lcs_field *f, const float *xy_host, const int *tris_host, const int *nbrs_host,
                            cudaStream_t s)
{
    const long long nn = f->nodes, nc = f->ncells;
    std::vector<int> nb_built;
    if (!nbrs_host) {
        build_tri_neighbours(tris_host, nc, nb_built);
        nbrs_host = nb_built.data();
    }
    std::vector<int4> t4((size_t)nc), n4((size_t)nc);
    for (long long t = 0; t < nc; ++t) {
        t4[(size_t)t] = make_int4(tris_host[3 * t], tris_host[3 * t + 1], tris_host[3 * t + 2], 0);
        n4[(size_t)t] = make_int4(nbrs_host[3 * t], nbrs_host[3 * t + 1], nbrs_host[3 * t + 2], -1);
    }
    float lo[2] = {INFINITY, INFINITY}, hi[2] = {-INFINITY, -INFINITY};
    for (long long i = 0; i < nn; ++i)
        for (int d = 0; d < 2; ++d) {
            lo[d] = std::min(lo[d], xy_host[2 * i + d]);
            hi[d] = std::max(hi[d], xy_host[2 * i + d]);
        }
    TriBins B;
    const double area = std::max(1e-30, (double)(hi[0] - lo[0]) * (hi[1] - lo[1]));
    const double cell = sqrt(area / std::max(1.0, (double)nc / 2.0));  // about two triangles per bin
    for (int d = 0; d < 2; ++d) {
        const double ext = std::max((double)(hi[d] - lo[d]), 1e-30);
        B.n[d] = (int)std::min(8192.0, std::max(1.0, ceil(ext / cell)));
        B.lo[d] = lo[d];
        B.inv[d] = (float)(B.n[d] / ext);
        f->bin_n[d] = B.n[d];
        f->bin_lo[d] = B.lo[d];
        f->bin_inv[d] = B.inv[d];
    }
    f->bin_n[2] = 1;
    const long long nbins = (long long)B.n[0] * B.n[1];
    f->nbins = nbins;
    int *count = nullptr, *cursor = nullptr;
    cudaError_t e = cudaMalloc(&f->d_xy, sizeof(float2) * nn);
    if (e == cudaSuccess) e = cudaMalloc(&f->d_tets, sizeof(int4) * nc);
    if (e == cudaSuccess) e = cudaMalloc(&f->d_nbrs, sizeof(int4) * nc);
    if (e == cudaSuccess) e = cudaMalloc(&f->d_trimap, sizeof(float4) * nc);
    if (e == cudaSuccess) e = cudaMalloc(&f->d_triv0, sizeof(float2) * nc);
    if (e == cudaSuccess) e = cudaMalloc(&f->d_bstart, sizeof(int) * (nbins + 1));
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&count, sizeof(int) * nbins, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&cursor, sizeof(int) * nbins, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f->d_xy, xy_host, sizeof(float2) * nn, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f->d_tets, t4.data(), sizeof(int4) * nc, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f->d_nbrs, n4.data(), sizeof(int4) * nc, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, sizeof(int) * nbins, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cursor, 0, sizeof(int) * nbins, s);
    const int bt = 256;
    const unsigned gc = (unsigned)((nc + bt - 1) / bt);
    if (e == cudaSuccess) {
        tri_map_kernel<<<gc, bt, 0, s>>>(f->d_xy, f->d_tets, nc, f->d_trimap, f->d_triv0);
        tri_bin_count_kernel<<<gc, bt, 0, s>>>(f->d_xy, f->d_tets, nc, B, count);
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
        tri_bin_fill_kernel<<<gc, bt, 0, s>>>(f->d_xy, f->d_tets, nc, B, f->d_bstart, cursor, f->d_blist);
        tri_bin_sort_kernel<<<(unsigned)((nbins + bt - 1) / bt), bt, 0, s>>>(f->d_bstart, nbins, f->d_blist);
        e = cudaGetLastError();
    }
    // convex (connected, every boundary vertex convex): then a walk that meets the boundary is outside
    std::vector<int> chk;
    int convex = mesh_connected(nbrs_host, nc, 3) && tri_convexity_checks(tris_host, nbrs_host, nc, chk) ? 1 : 0;
    int *dchk = nullptr, *dflag = nullptr;
    const long long nchk = (long long)chk.size() / 4;
    if (e == cudaSuccess && convex && nchk > 0) {
        e = cudaMallocAsync((void **)&dchk, sizeof(int) * chk.size(), s);
        if (e == cudaSuccess) e = cudaMallocAsync((void **)&dflag, sizeof(int), s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dchk, chk.data(), sizeof(int) * chk.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dflag, &convex, sizeof(int), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) {
            tri_convex_kernel<<<(unsigned)((nchk + bt - 1) / bt), bt, 0, s>>>(f->d_xy, dchk, nchk, dflag);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(&convex, dflag, sizeof(int), cudaMemcpyDeviceToHost, s);
    }
    if (count) cudaFreeAsync(count, s);
    if (cursor) cudaFreeAsync(cursor, s);
    if (dchk) cudaFreeAsync(dchk, s);
    if (dflag) cudaFreeAsync(dflag, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host values above go out of scope
    f->convex = e == cudaSuccess ? convex : 0;
    return e;
}

TriDev tri_dev(const lcs_field *f, int walk_limit)
{
    TriDev T;
    T.xy = f->d_xy;
    T.tris = f->d_tets;
    T.nbrs = f->d_nbrs;
    T.tmap = f->d_trimap;
    T.tv0 = f->d_triv0;
    T.bstart = f->d_bstart;
    T.blist = f->d_blist;
    for (int d = 0; d < 2; ++d) {
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

cudaError_t tri_locate_seeds(const lcs_field *f, const float *seeds, long long N, int *cells, cudaStream_t s)
{
    if (N == 0) return cudaSuccess;
    const TriDev T = tri_dev(f, 0);
    const int bt = 128;
    tri_seed_locate_kernel<<<(unsigned)((N + bt - 1) / bt), bt, 0, s>>>(T, seeds, N, cells);
    return cudaGetLastError();
}
