// autotune.cu -- lcs_autotune: choose launch options of lcs_advect by timing.
//
// Candidates (kernel variant, threads per block, tracers per thread, steps per
// re-bundling episode) are timed with CUDA events on the caller's real inputs; the
// fastest is written back into the options and remembered in a plain-text cache,
// one line per call shape:  <signature> \t variant block_threads tracers_per_thread
// episode_steps milliseconds.
#include "lcs_internal.cuh"

#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

namespace {

struct Cand {
    int variant, bt, tpt, E;
};

std::string signature(int device, const lcs_field *f, const lcs_seeds *s, const lcs_advect_opts *o)
{
    cudaDeviceProp prop;
    memset(&prop, 0, sizeof prop);
    cudaGetDeviceProperties(&prop, device);
    int njobs = o->njobs > 1 ? o->njobs : 1;
    double adt = fabs(o->dt);
    long long steps = 0, smax = 0;
    for (int j = 0; j < njobs; ++j) {
        double T = o->njobs > 1 ? o->job_T[j] : o->T;
        long long n = adt > 0 ? (long long)floor(fabs(T) / adt + 0.5) : 0;
        steps += n;
        smax = n > smax ? n : smax;
    }
    char buf[512];
    snprintf(buf, sizeof buf, "%s|sm%d%d|dim%d|n%d,%d,%d|nf%d|st%d|per%d%d%d|N%lld|jobs%d|steps%lld|max%lld|m%d|snap%d",
             prop.name, prop.major, prop.minor, f->dim, f->n[0], f->n[1], f->n[2], f->nframes, f->storage,
             f->periodic[0], f->periodic[1], f->periodic[2], s->N, njobs, steps, smax, o->method,
             o->nsnap > 0 ? o->nsnap : 0);
    std::string sig = buf;
    for (auto &c : sig)
        if (c == ' ' || c == '\t' || c == '\n') c = '_';
    return sig;
}

bool cache_lookup(const char *path, const std::string &sig, Cand &c)
{
    if (!path) return false;
    FILE *fp = fopen(path, "r");
    if (!fp) return false;
    char line[1024];
    bool found = false;
    while (fgets(line, sizeof line, fp)) {
        char *tab = strchr(line, '\t');
        if (!tab) continue;
        *tab = 0;
        if (sig != line) continue;
        Cand t;
        double ms;
        if (sscanf(tab + 1, "%d %d %d %d %lf", &t.variant, &t.bt, &t.tpt, &t.E, &ms) == 5) {
            c = t;
            found = true;  // the last matching line wins
        }
    }
    fclose(fp);
    return found;
}

void cache_store(const char *path, const std::string &sig, const Cand &c, double ms)
{
    if (!path) return;
    FILE *fp = fopen(path, "a");
    if (!fp) return;
    fprintf(fp, "%s\t%d %d %d %d %.4f\n", sig.c_str(), c.variant, c.bt, c.tpt, c.E, ms);
    fclose(fp);
}

void apply(lcs_advect_opts *o, const Cand &c)
{
    o->variant = c.variant;
    o->block_threads = c.bt;
    o->tracers_per_thread = c.tpt;
    o->episode_steps = c.E;
}

}  // namespace

extern "C" lcs_status lcs_autotune(lcs_ctx *ctx, const lcs_field *f, const lcs_seeds *s, lcs_advect_opts *o,
                                   const char *cache_path)
{
    if (!ctx) return LCS_EINVAL;
    if (!f || !s || !o) {
        ctx->err = "lcs_autotune: null argument";
        return LCS_EINVAL;
    }
    if (o->method != LCS_RK4 || f->kind != LCS_RECTILINEAR) {
        ctx->err = "lcs_autotune: tunes RK4 on rectilinear fields";
        return LCS_EUNSUPPORTED;
    }
    const std::string sig = signature(ctx->device, f, s, o);
    Cand best{0, 0, 0, 0};
    if (cache_lookup(cache_path, sig, best)) {
        apply(o, best);
        return LCS_OK;
    }
    const int njobs = o->njobs > 1 ? o->njobs : 1;
    std::vector<Cand> cands;
    if (f->dim == 2) {
        const bool ring = 3 * f->frame_stride <= ctx->smem_optin;
        for (int bt : {128, 256})
            cands.push_back({1, bt, 1, 0});
        if (f->kind == LCS_RECTILINEAR)
            for (int bt : {128, 256})
                cands.push_back({5, bt, 1, 0});
        if (ring)
            for (int v : {2, 4}) {
                if (v == 4 && njobs < 2) continue;
                for (int bt : {128, 256, 512})
                    for (int tpt : {1, 2})
                        cands.push_back({v, bt, tpt, 0});
            }
    } else {
        cands.push_back({1, 256, 1, 0});
        if (s->N >= 32 * 1024)
            for (int E : {8, 16, 32, 48})
                for (int bt : {128, 256})
                    cands.push_back({3, bt, 1, E});
    }
    lcs_flowmap *fm = nullptr;
    const int nsnap = o->nsnap > 0 && o->nsnap <= LCS_MAX_SNAP ? o->nsnap : 0;
    lcs_status st = lcs_flowmap_create(ctx, s, njobs * (1 + nsnap), &fm);
    if (st != LCS_OK) return st;
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        lcs_free_flowmap(fm);
        if (a) cudaEventDestroy(a);
        ctx->err = "lcs_autotune: event creation failed";
        return LCS_ECUDA;
    }
    double best_ms = 1e300;
    for (const Cand &c : cands) {
        lcs_advect_opts t = *o;
        t.use_graph = 0;
        apply(&t, c);
        st = lcs_advect(ctx, f, s, &t, fm);  // warm-up (and scratch growth)
        if (st != LCS_OK) break;
        cudaEventRecord(a, ctx->stream);
        st = lcs_advect(ctx, f, s, &t, fm);
        cudaEventRecord(b, ctx->stream);
        if (st != LCS_OK) break;
        if (cudaEventSynchronize(b) != cudaSuccess) {
            st = LCS_ECUDA;
            ctx->err = "lcs_autotune: timing failed";
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a, b);
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    lcs_free_flowmap(fm);
    if (st != LCS_OK) return st;
    apply(o, best);
    cache_store(cache_path, sig, best, best_ms);
    return LCS_OK;
}
