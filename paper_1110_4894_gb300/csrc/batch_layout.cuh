// batch_layout.cuh -- device tables of the batched trace (one entry per cone
// plus the launch arguments of the persistent kernel).
#pragma once
#include "rt3d_internal.cuh"

namespace rt3d {

struct BatchCone {
    DevField f;
    RayState rs;           // view into the batch's ray arrays (stride = padded ray count)
    TraceParams tp;
    const double *theta;   // this cone's bundle angles
    double *dlam;          // this cone's step table
    float2 *partials;      // S * 4 * n_rays split partials
    unsigned long long *cnt;  // [0], [1] rays in flight after even / odd steps; [2] active ray-stages
    double *rout;          // optional per-ray final states (compact)
    double *prism;         // mean-subtracted cones: kPrismRec doubles per bundle, else null
    double chi_s;          // written by the schedule kernel
    double z_s, chi_l, s_asinh, mfac;
    int64_t per_split, ray_base, b_base;
    int S, flags, total_steps, kind;
    int grid;              // 1: the field is a grid (g), read by grid items; S = 1
    GridDev g;
};

struct BatchArgs {
    BatchCone *cones;
    int n_cones;
    const int4 *items;     // (cone, ray block, split, kind); split -1: the prism records of a
                           // block of NT bundles; kind 1: grid evaluation of a ray block
    int64_t n_items;
    const int *rb2cone;    // cone of each padded ray block
    int64_t T;             // padded ray count
    int RB;                // rays per block
    int g_end;             // global stages to run
    unsigned *bar;         // [0] barrier count, [1] generation, [2] error word, [4], [5] work queues
    int *err;              // watchdog / error word
    unsigned long long limit_ns;
    double *bout;
};

inline BatchArgs make_batch_args(void *cones, int n_cones, const int4 *items, int64_t n_items, const int *rb2cone,
                                 int64_t T, int RB, int g_end, unsigned *bar, int *err, double watchdog_s,
                                 double *bout)
{
    BatchArgs A;
    A.cones = (BatchCone *)cones;
    A.n_cones = n_cones;
    A.items = items;
    A.n_items = n_items;
    A.rb2cone = rb2cone;
    A.T = T;
    A.RB = RB;
    A.g_end = g_end;
    A.bar = bar;
    A.err = err;
    A.limit_ns = (unsigned long long)(watchdog_s * 1e9);
    A.bout = bout;
    return A;
}

// MODE: 4 or 8 = bundle-centric pair sum for rings of that size, 0 = packed
cudaError_t batch_resident_blocks(int NT, int MODE, int *out);
// one bounded wait on a word nothing changes (the watchdog self-test)
cudaError_t launch_watchdog_probe(unsigned *d_word, int *d_err, double limit_s, cudaStream_t st);
cudaError_t batch_launch(const BatchArgs &B, int NT, int MODE, int grid, int max_sched_steps, int64_t n_b_total,
                         cudaStream_t st);

}  // namespace rt3d
