// force.cuh -- pair-sum kernels: phi and grad phi of a Plummer-softened
// particle set at every ray's stage position (Eqs. psi, derivs with
// phi = a psi, Eq. phicotophys), as partial sums over particle splits.
//
// Layout and precision
// * Particles are int4 (grid position qx, qy, qz in units of delta = 2^-e Mpc,
//   mass mu_G m 2^ms as FP32 bits).  A block stages a tile of TILE particles
//   in shared memory, applying the replica transform (exact integer
//   arithmetic) and re-centring on an anchor: the grid point nearest the
//   block's first ray.  The integer offset from the anchor converts to FP32
//   exactly up to 2^24 grid units and is then scaled by delta (a power of
//   two, also exact) so that the arithmetic runs in Mpc, where 1/d^3 stays
//   inside the FP32 range; each ray's offset is rounded once from FP64.
// * Every ray of a thread reuses each staged particle (register blocking R);
//   all threads of the block read the same shared word (broadcast).
// * Sums are accumulated in FP32 over chunks of CHUNK particles and merged
//   into a (hi, lo) pair by an error-free TwoSum per chunk.
// * Block (x = ray block, y = particle split) writes (hi, lo) per output to
//   partials[split][output][ray]; the integrator stage adds them in FP64.
#pragma once
#include <limits.h>

#include "rt3d_internal.cuh"

namespace rt3d {

constexpr int kTile = 256;
constexpr int kTile64 = 128;
constexpr int kChunk = 64;

struct ForceArgs {
    DevField f;
    const double *px, *py, *pz;  // point positions (SoA, FP64, world frame)
    const int *rep;              // replica per group of points (may be null: 0)
    int group;                   // points per group (rays per bundle)
    int64_t n;                   // points
    int64_t per_split;           // particles per split (multiple of kTile)
    void *out;                   // partials
    const unsigned long long *gate;  // non-null: skip when *gate == 0
};

__device__ __forceinline__ float rsqrt_mufu(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// error-free transformation: hi + lo absorbs x exactly up to the final add to lo
__device__ __forceinline__ void two_sum_into(float &hi, float &lo, float x)
{
    const float s = hi + x;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (x - bb);
    hi = s;
    lo += err;
}

template <int R, int NT>
__device__ __forceinline__ void block_replica_range(const ForceArgs &A, int64_t base, int myrep[R], int &rmin,
                                                    int &rmax)
{
    __shared__ int s_rmin, s_rmax;
    if (threadIdx.x == 0) {
        s_rmin = INT_MAX;
        s_rmax = INT_MIN;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int64_t i = base + (int64_t)k * NT + threadIdx.x;
        myrep[k] = -1;
        if (i < A.n) {
            myrep[k] = A.rep ? A.rep[i / A.group] : 0;
            atomicMin(&s_rmin, myrep[k]);
            atomicMax(&s_rmax, myrep[k]);
        }
    }
    __syncthreads();
    rmin = s_rmin;
    rmax = s_rmax;
}

template <int R, int NT, bool REPL, bool PEPS>
__global__ void __launch_bounds__(NT) k_force_mixed(ForceArgs A)
{
    if (A.gate && *A.gate == 0ull) return;
    __shared__ float4 s_p[kTile];
    __shared__ float s_e[PEPS ? kTile : 1];
    const DevField &f = A.f;
    const int tid = threadIdx.x;
    const int64_t base = (int64_t)blockIdx.x * (NT * R);
    const int split = blockIdx.y;
    int myrep[R], rmin, rmax;
    block_replica_range<R, NT>(A, base, myrep, rmin, rmax);

    float hi[R][4], lo[R][4];
#pragma unroll
    for (int k = 0; k < R; ++k)
#pragma unroll
        for (int o = 0; o < 4; ++o) hi[k][o] = lo[k][o] = 0.0f;

    const int64_t p0 = (int64_t)split * A.per_split;
    const int64_t p1 = min(f.n, p0 + A.per_split);
    const float dlt = (float)f.delta;
    for (int j = rmin; j <= rmax; ++j) {
        double o[3];
        frame_origin(f, j, o);
        const long long ax = __double2ll_rn((A.px[base] - o[0]) * f.inv_delta);
        const long long ay = __double2ll_rn((A.py[base] - o[1]) * f.inv_delta);
        const long long az = __double2ll_rn((A.pz[base] - o[2]) * f.inv_delta);
        float rx[R], ry[R], rz[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int64_t i = base + (int64_t)k * NT + tid;
            if (i < A.n && myrep[k] == j) {
                rx[k] = (float)(((A.px[i] - o[0]) * f.inv_delta - (double)ax) * f.delta);
                ry[k] = (float)(((A.py[i] - o[1]) * f.inv_delta - (double)ay) * f.delta);
                rz[k] = (float)(((A.pz[i] - o[2]) * f.inv_delta - (double)az) * f.delta);
            } else {  // far sentinel: every contribution is exactly zero
                rx[k] = ry[k] = rz[k] = 1e30f;
            }
        }
        for (int64_t t0 = p0; t0 < p1; t0 += kTile) {
            __syncthreads();
            for (int q = tid; q < kTile; q += NT) {
                const int64_t pi = t0 + q;
                float4 v = make_float4(1e18f, 1e18f, 1e18f, 0.0f);
                float e2 = 0.0f;
                if (pi < p1) {
                    const int4 pr = f.part[pi];
                    long long qq[3] = {pr.x, pr.y, pr.z};
                    if (REPL) replica_q(f, j, pr.x, pr.y, pr.z, qq);
                    v = make_float4((float)(qq[0] - ax) * dlt, (float)(qq[1] - ay) * dlt,
                                    (float)(qq[2] - az) * dlt, __int_as_float(pr.w));
                    if (PEPS) e2 = f.eps2[pi];
                }
                s_p[q] = v;
                if (PEPS) s_e[q] = e2;
            }
            __syncthreads();
            for (int c0 = 0; c0 < kTile; c0 += kChunk) {
                float ca[R][4];
#pragma unroll
                for (int k = 0; k < R; ++k)
#pragma unroll
                    for (int o2 = 0; o2 < 4; ++o2) ca[k][o2] = 0.0f;
#pragma unroll 8
                for (int jj = c0; jj < c0 + kChunk; ++jj) {
                    const float4 p = s_p[jj];
                    const float e2 = PEPS ? s_e[jj] : f.eps2u;
#pragma unroll
                    for (int k = 0; k < R; ++k) {
                        const float dx = p.x - rx[k], dy = p.y - ry[k], dz = p.z - rz[k];
                        const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, e2)));
                        const float inv = rsqrt_mufu(r2);
                        const float mi = p.w * inv;
                        const float mi3 = mi * (inv * inv);
                        ca[k][0] += mi;
                        ca[k][1] = fmaf(dx, mi3, ca[k][1]);
                        ca[k][2] = fmaf(dy, mi3, ca[k][2]);
                        ca[k][3] = fmaf(dz, mi3, ca[k][3]);
                    }
                }
#pragma unroll
                for (int k = 0; k < R; ++k)
#pragma unroll
                    for (int o2 = 0; o2 < 4; ++o2) two_sum_into(hi[k][o2], lo[k][o2], ca[k][o2]);
            }
        }
    }
    float2 *out = (float2 *)A.out;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int64_t i = base + (int64_t)k * NT + tid;
        if (i < A.n)
#pragma unroll
            for (int o2 = 0; o2 < 4; ++o2) out[((int64_t)split * 4 + o2) * A.n + i] = make_float2(hi[k][o2], lo[k][o2]);
    }
}

// FP64 twin (the all-FP64 path): same staging, FP64 arithmetic, plain sums.
template <int R, int NT, bool REPL, bool PEPS>
__global__ void __launch_bounds__(NT) k_force_fp64(ForceArgs A)
{
    if (A.gate && *A.gate == 0ull) return;
    __shared__ double4 s_p[kTile64];
    __shared__ double s_e[PEPS ? kTile64 : 1];
    const DevField &f = A.f;
    const int tid = threadIdx.x;
    const int64_t base = (int64_t)blockIdx.x * (NT * R);
    const int split = blockIdx.y;
    int myrep[R], rmin, rmax;
    block_replica_range<R, NT>(A, base, myrep, rmin, rmax);
    double acc[R][4];
#pragma unroll
    for (int k = 0; k < R; ++k)
#pragma unroll
        for (int o = 0; o < 4; ++o) acc[k][o] = 0.0;
    const int64_t p0 = (int64_t)split * A.per_split;
    const int64_t p1 = min(f.n, p0 + A.per_split);
    for (int j = rmin; j <= rmax; ++j) {
        double o[3];
        frame_origin(f, j, o);
        const long long ax = __double2ll_rn((A.px[base] - o[0]) * f.inv_delta);
        const long long ay = __double2ll_rn((A.py[base] - o[1]) * f.inv_delta);
        const long long az = __double2ll_rn((A.pz[base] - o[2]) * f.inv_delta);
        double rx[R], ry[R], rz[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int64_t i = base + (int64_t)k * NT + tid;
            if (i < A.n && myrep[k] == j) {
                rx[k] = ((A.px[i] - o[0]) * f.inv_delta - (double)ax) * f.delta;
                ry[k] = ((A.py[i] - o[1]) * f.inv_delta - (double)ay) * f.delta;
                rz[k] = ((A.pz[i] - o[2]) * f.inv_delta - (double)az) * f.delta;
            } else {
                rx[k] = ry[k] = rz[k] = 1e150;
            }
        }
        for (int64_t t0 = p0; t0 < p1; t0 += kTile64) {
            __syncthreads();
            for (int q = tid; q < kTile64; q += NT) {
                const int64_t pi = t0 + q;
                double4 v = make_double4(1e100, 1e100, 1e100, 0.0);
                double e2 = 0.0;
                if (pi < p1) {
                    const int4 pr = f.part[pi];
                    long long qq[3] = {pr.x, pr.y, pr.z};
                    if (REPL) replica_q(f, j, pr.x, pr.y, pr.z, qq);
                    v = make_double4((double)(qq[0] - ax) * f.delta, (double)(qq[1] - ay) * f.delta,
                                     (double)(qq[2] - az) * f.delta, f.m64[pi]);
                    if (PEPS) e2 = f.eps2_64[pi];
                }
                s_p[q] = v;
                if (PEPS) s_e[q] = e2;
            }
            __syncthreads();
#pragma unroll 4
            for (int jj = 0; jj < kTile64; ++jj) {
                const double4 p = s_p[jj];
                const double e2 = PEPS ? s_e[jj] : f.eps2u64;
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    const double dx = p.x - rx[k], dy = p.y - ry[k], dz = p.z - rz[k];
                    const double r2 = dx * dx + dy * dy + dz * dz + e2;
                    const double inv = rsqrt(r2);
                    const double mi = p.w * inv;
                    const double mi3 = mi * inv * inv;
                    acc[k][0] += mi;
                    acc[k][1] += dx * mi3;
                    acc[k][2] += dy * mi3;
                    acc[k][3] += dz * mi3;
                }
            }
        }
    }
    double *out = (double *)A.out;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int64_t i = base + (int64_t)k * NT + tid;
        if (i < A.n)
#pragma unroll
            for (int o2 = 0; o2 < 4; ++o2) out[((int64_t)split * 4 + o2) * A.n + i] = acc[k][o2];
    }
}

}  // namespace rt3d
