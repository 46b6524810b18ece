// dp45_args.cuh -- parameters of the adaptive Dormand-Prince 5(4) launch (advect_tet.cu).
#pragma once

#include "lcs_internal.cuh"

struct Dp45Args {
    const float *seeds;        // [3][N]
    const int *cells0;         // [N] start cells (tets) or null
    long long N;
    const double *job_t0, *job_T;  // [njobs] (device)
    float h0, rtol, atol;
    long long max_steps;
    int rect_left;             // apply the rectilinear LEFT test after accepted steps
    const double *times;       // [nf] frame times (device, FP64)
    int nf, tp;
    float period;
    float *out_xyz;            // [njobs][3][N]
    unsigned char *out_status; // [njobs][N]
    float *out_texit;          // [njobs][N]
    int *out_steps;            // [njobs][N] accepted steps, or null
    unsigned *errword;
};

cudaError_t launch_dp45(lcs_ctx *ctx, const lcs_field *f, const Dp45Args &A, int njobs, int block_threads,
                        int walk_limit, cudaStream_t s);
