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
//   partials[split][output][ray]; the integrator stage adds them as FP32
//   double-float numbers and converts once to FP64.
#pragma once
#include <cooperative_groups.h>
#include <limits.h>

#include "rt3d_internal.cuh"

namespace rt3d {

namespace cg = cooperative_groups;

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

// grid coordinate of a block's anchor: the offset of x from the frame origin
// o, rounded to the grid; 0 (the frame origin itself) when x is not finite or
// lies beyond 2^62 grid units, so that one bad point cannot spoil the offsets
// of the other points of its block (a NaN fails the comparison)
__device__ __forceinline__ long long anchor_q(double x, double o, double inv_delta)
{
    const double q = (x - o) * inv_delta;
    return fabs(q) < 4.0e18 ? __double2ll_rn(q) : 0ll;
}

// replica index r of a point, or -1 (the point takes part in no replica's
// pass and its sums stay zero) when r is outside [0, n_rep)
__device__ __forceinline__ int checked_replica(int r, int n_rep) { return (r >= 0 && r < n_rep) ? r : -1; }

// Replica range [rmin, rmax] of the block's points (rmin > rmax when no point
// has a valid replica).  Indices outside [0, n_rep) are left out.
template <int R, int NT>
__device__ __forceinline__ void block_replica_range(const ForceArgs &A, int n_rep, int64_t base, int myrep[R],
                                                    int &rmin, int &rmax)
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
            myrep[k] = checked_replica(A.rep ? A.rep[i / A.group] : 0, n_rep);
            if (myrep[k] >= 0) {
                atomicMin(&s_rmin, myrep[k]);
                atomicMax(&s_rmax, myrep[k]);
            }
        }
    }
    __syncthreads();
    rmin = s_rmin;
    rmax = s_rmax;
}

// true in every thread of the block when some thread holds a point of replica
// j (a block barrier: every thread of the block must call it)
template <int R>
__device__ __forceinline__ bool block_uses_replica(const int myrep[R], int j)
{
    int mine = 0;
#pragma unroll
    for (int k = 0; k < R; ++k) mine |= myrep[k] == j;
    return __syncthreads_or(mine) != 0;
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
    block_replica_range<R, NT>(A, f.n_rep, base, myrep, rmin, rmax);

    float hi[R][4], lo[R][4];
#pragma unroll
    for (int k = 0; k < R; ++k)
#pragma unroll
        for (int o = 0; o < 4; ++o) hi[k][o] = lo[k][o] = 0.0f;

    const int64_t p0 = (int64_t)split * A.per_split;
    const int64_t p1 = min(f.n, p0 + A.per_split);
    const float dlt = (float)f.delta;
    for (int j = rmin; j <= rmax; ++j) {
        if (!block_uses_replica<R>(myrep, j)) continue;  // no point of this block is in replica j
        double o[3];
        frame_origin(f, j, o);
        const long long ax = anchor_q(A.px[base], o[0], f.inv_delta);
        const long long ay = anchor_q(A.py[base], o[1], f.inv_delta);
        const long long az = anchor_q(A.pz[base], o[2], f.inv_delta);
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

// Packed variant: P pairs of rays per thread, every FP32 operation of the pair
// sum issued as a Blackwell f32x2 instruction (FADD2 / FMUL2 / FFMA2), which
// halves the instruction count of the hot loop.  The particle tile is staged
// duplicated, (x, x, y, y) and (z, z, m, m), so that each shared load yields
// aligned register pairs.  The potential (which enters the geodesic equation
// only at first order in phi) is summed plainly; the gradient is compensated
// per chunk as in the scalar kernel.  UMASS: all particles share one mass,
// which the integrator stage applies in FP64 (saves one multiply per pair).
__device__ __forceinline__ void two_sum2_into(float2 &hi, float2 &lo, float2 x)
{
    const float2 s = __fadd2_rn(hi, x);
    const float2 bb = __fadd2_rn(s, make_float2(-hi.x, -hi.y));
    const float2 t = __fadd2_rn(s, make_float2(-bb.x, -bb.y));
    const float2 e1 = __fadd2_rn(hi, make_float2(-t.x, -t.y));
    const float2 e2 = __fadd2_rn(x, make_float2(-bb.x, -bb.y));
    hi = s;
    lo = __fadd2_rn(lo, __fadd2_rn(e1, e2));
}

// Sum of one block's rays over particles [p0, p1) of field f: the body shared
// by the pair-sum launch and the batched persistent kernel.  Rays
// base + k*NT + tid (k < 2P, index < n) with replica rep[i / group]; output
// (hi, lo) pairs to out[(split*4 + o)*n + i] (phi: (sum, 0)).
template <int P, int NT, bool REPL, bool PEPS, bool UMASS>
__device__ __forceinline__ void packed_block_sum(const DevField &f, const double *__restrict__ px,
                                                 const double *__restrict__ py, const double *__restrict__ pz,
                                                 const int *__restrict__ rep, int group, int64_t n, int64_t base,
                                                 int64_t p0, int64_t p1, int split, float2 *__restrict__ out,
                                                 float4 *s_a, float4 *s_b, float2 *s_e)
{
    constexpr int R = 2 * P;
    const int tid = threadIdx.x;
    ForceArgs A;
    A.rep = rep;
    A.group = group;
    A.n = n;
    int myrep[R], rmin, rmax;
    block_replica_range<R, NT>(A, f.n_rep, base, myrep, rmin, rmax);

    float2 phi[P], hx[P], hy[P], hz[P], lx[P], ly[P], lz[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        phi[p] = hx[p] = hy[p] = hz[p] = lx[p] = ly[p] = lz[p] = make_float2(0.0f, 0.0f);
    }
    const float dlt = (float)f.delta;
    const float2 E2u = make_float2(f.eps2u, f.eps2u);
    for (int j = rmin; j <= rmax; ++j) {
        if (!block_uses_replica<R>(myrep, j)) continue;  // no point of this block is in replica j
        double o[3];
        frame_origin(f, j, o);
        const long long ax = anchor_q(px[base], o[0], f.inv_delta);
        const long long ay = anchor_q(py[base], o[1], f.inv_delta);
        const long long az = anchor_q(pz[base], o[2], f.inv_delta);
        // negated ray offsets: d = particle + (-ray)
        float2 nx[P], ny[P], nz[P];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            float v[2][3];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = 2 * p + h;
                const int64_t i = base + (int64_t)k * NT + tid;
                if (i < n && myrep[k] == j) {
                    v[h][0] = -(float)(((px[i] - o[0]) * f.inv_delta - (double)ax) * f.delta);
                    v[h][1] = -(float)(((py[i] - o[1]) * f.inv_delta - (double)ay) * f.delta);
                    v[h][2] = -(float)(((pz[i] - o[2]) * f.inv_delta - (double)az) * f.delta);
                } else {  // far sentinel: every contribution is exactly zero
                    v[h][0] = v[h][1] = v[h][2] = -1e30f;
                }
            }
            nx[p] = make_float2(v[0][0], v[1][0]);
            ny[p] = make_float2(v[0][1], v[1][1]);
            nz[p] = make_float2(v[0][2], v[1][2]);
        }
        for (int64_t t0 = p0; t0 < p1; t0 += kTile) {
            __syncthreads();
            for (int q = tid; q < kTile; q += NT) {
                const int64_t pi = t0 + q;
                float x = 1e18f, y = 1e18f, z = 1e18f, m = 0.0f, e2 = 0.0f;
                if (pi < p1) {
                    const int4 pr = f.part[pi];
                    long long qq[3] = {pr.x, pr.y, pr.z};
                    if (REPL) replica_q(f, j, pr.x, pr.y, pr.z, qq);
                    x = (float)(qq[0] - ax) * dlt;
                    y = (float)(qq[1] - ay) * dlt;
                    z = (float)(qq[2] - az) * dlt;
                    m = __int_as_float(pr.w);
                    if (PEPS) e2 = f.eps2[pi];
                }
                s_a[q] = make_float4(x, x, y, y);
                s_b[q] = make_float4(z, z, m, m);
                if (PEPS) s_e[q] = make_float2(e2, e2);
            }
            __syncthreads();
            for (int c0 = 0; c0 < kTile; c0 += kChunk) {
                float2 cx[P], cy[P], cz[P];
#pragma unroll
                for (int p = 0; p < P; ++p) cx[p] = cy[p] = cz[p] = make_float2(0.0f, 0.0f);
#pragma unroll 4
                for (int jj = c0; jj < c0 + kChunk; ++jj) {
                    const float4 a = s_a[jj];
                    const float4 b = s_b[jj];
                    const float2 PX = make_float2(a.x, a.y), PY = make_float2(a.z, a.w);
                    const float2 PZ = make_float2(b.x, b.y), M2 = make_float2(b.z, b.w);
                    const float2 E2 = PEPS ? s_e[jj] : E2u;
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        const float2 dx = __fadd2_rn(PX, nx[p]);
                        const float2 dy = __fadd2_rn(PY, ny[p]);
                        const float2 dz = __fadd2_rn(PZ, nz[p]);
                        float2 r2 = __ffma2_rn(dz, dz, E2);
                        r2 = __ffma2_rn(dy, dy, r2);
                        r2 = __ffma2_rn(dx, dx, r2);
                        const float2 inv = make_float2(rsqrt_mufu(r2.x), rsqrt_mufu(r2.y));
                        const float2 i2 = __fmul2_rn(inv, inv);
                        float2 mi3;
                        if (UMASS) {
                            phi[p] = __fadd2_rn(phi[p], inv);
                            mi3 = __fmul2_rn(inv, i2);
                        } else {
                            const float2 mi = __fmul2_rn(M2, inv);
                            phi[p] = __fadd2_rn(phi[p], mi);
                            mi3 = __fmul2_rn(mi, i2);
                        }
                        cx[p] = __ffma2_rn(dx, mi3, cx[p]);
                        cy[p] = __ffma2_rn(dy, mi3, cy[p]);
                        cz[p] = __ffma2_rn(dz, mi3, cz[p]);
                    }
                }
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    two_sum2_into(hx[p], lx[p], cx[p]);
                    two_sum2_into(hy[p], ly[p], cy[p]);
                    two_sum2_into(hz[p], lz[p], cz[p]);
                }
            }
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t i = base + (int64_t)(2 * p + h) * NT + tid;
            if (i >= n) continue;
            const float ph = h ? phi[p].y : phi[p].x;
            out[((int64_t)split * 4 + 0) * n + i] = make_float2(ph, 0.0f);
            out[((int64_t)split * 4 + 1) * n + i] = h ? make_float2(hx[p].y, lx[p].y) : make_float2(hx[p].x, lx[p].x);
            out[((int64_t)split * 4 + 2) * n + i] = h ? make_float2(hy[p].y, ly[p].y) : make_float2(hy[p].x, ly[p].x);
            out[((int64_t)split * 4 + 3) * n + i] = h ? make_float2(hz[p].y, lz[p].y) : make_float2(hz[p].x, lz[p].x);
        }
    }
}

template <int P, int NT, bool REPL, bool PEPS, bool UMASS>
__global__ void __launch_bounds__(NT) k_force_packed(ForceArgs A)
{
    if (A.gate && *A.gate == 0ull) return;
    __shared__ float4 s_a[kTile];            // (x, x, y, y)
    __shared__ float4 s_b[kTile];            // (z, z, m, m)
    __shared__ float2 s_e[PEPS ? kTile : 1]; // (eps2, eps2)
    const int64_t base = (int64_t)blockIdx.x * (NT * 2 * P);
    const int split = blockIdx.y;
    const int64_t p0 = (int64_t)split * A.per_split;
    const int64_t p1 = min(A.f.n, p0 + A.per_split);
    packed_block_sum<P, NT, REPL, PEPS, UMASS>(A.f, A.px, A.py, A.pz, A.rep, A.group, A.n, base, p0, p1, split,
                                               (float2 *)A.out, s_a, s_b, s_e);
}

// Potential sum of a ring ray to first order about its bundle's central ray:
// with S0 = sum m / r and S = sum m d / r^3 (d = particle - ray), phi = -S0
// and grad phi = -S (times the mass scale), so phi(r_k) = phi(r_c) + (r_k -
// r_c) . grad phi(r_c) gives S0_k = S0_c - e_k . S_c for e_k = r_c - r_k.  The
// potential enters the geodesic equation only in terms of order phi times
// a-dot (App. A), where the neglected second-order term, e_k^T H e_k / 2 of
// the particles nearest the ray, acts over a path of the order of their
// distance: its effect on a ray's direction is below 1e-14 rad for the
// softened fields here, against bundle differential deflections of 1e-8 rad
// and more.  The gradient sums themselves stay exact per ray.
__device__ __forceinline__ float ring_phi(float s0_c, const float e[3], float gx, float gy, float gz)
{
    return s0_c - fmaf(e[0], gx, fmaf(e[1], gy, e[2] * gz));
}

// Bundle-centric variant: one thread per bundle (central ray + NRING rays).
// Each satellite's offset from a particle is formed from the central ray's,
//   d_k = (p - r_c) + (r_c - r_k),
// with r_c - r_k taken in FP64 and rounded once.  The large, rounded
// quantities (the particle's and the central ray's offsets from the block
// anchor) are then common to every ray of the bundle and cancel from the
// bundle's differential deflection, which sets the magnification: its
// position error is ulp(|d|), not ulp(|anchor distance|).  The central ray
// runs in scalar FP32, the satellites in f32x2 pairs.  Particles are staged
// once, (x, y, z, m), plus eps^2 when it varies per particle.
template <int NT, int NRING, bool REPL, bool PEPS, bool UMASS>
__device__ __forceinline__ void bundle_block_sum(const DevField &f, const double *__restrict__ px,
                                                 const double *__restrict__ py, const double *__restrict__ pz,
                                                 const int *__restrict__ rep, int64_t n_b, int64_t n_rays,
                                                 int64_t b0, int64_t p0, int64_t p1, int split,
                                                 float2 *__restrict__ out, float4 *s_p, float *s_e)
{
    constexpr int NR = NRING + 1, PP = NRING / 2;
    const int tid = threadIdx.x;
    const int64_t b = b0 + tid;
    const bool valid = b < n_b;
    const int64_t ic = b * NR;  // central ray
    __shared__ int s_rmin, s_rmax;
    if (tid == 0) {
        s_rmin = INT_MAX;
        s_rmax = INT_MIN;
    }
    __syncthreads();
    const int myrep = valid ? checked_replica(rep ? rep[b] : 0, f.n_rep) : -1;
    if (myrep >= 0) {
        atomicMin(&s_rmin, myrep);
        atomicMax(&s_rmax, myrep);
    }
    __syncthreads();
    const int rmin = s_rmin, rmax = s_rmax;

    // satellite offsets r_c - r_k (FP64 difference, one rounding)
    float2 ex[PP], ey[PP], ez[PP];
#pragma unroll
    for (int p = 0; p < PP; ++p) {
        float v[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
        if (valid) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t ik = ic + 1 + 2 * p + h;
                v[h][0] = (float)(px[ic] - px[ik]);
                v[h][1] = (float)(py[ic] - py[ik]);
                v[h][2] = (float)(pz[ic] - pz[ik]);
            }
        }
        ex[p] = make_float2(v[0][0], v[1][0]);
        ey[p] = make_float2(v[0][1], v[1][1]);
        ez[p] = make_float2(v[0][2], v[1][2]);
    }
    float c_phi = 0.f, c_hx = 0.f, c_hy = 0.f, c_hz = 0.f, c_lx = 0.f, c_ly = 0.f, c_lz = 0.f;
    float2 hx[PP], hy[PP], hz[PP], lx[PP], ly[PP], lz[PP];
#pragma unroll
    for (int p = 0; p < PP; ++p) hx[p] = hy[p] = hz[p] = lx[p] = ly[p] = lz[p] = make_float2(0.f, 0.f);
    const float dlt = (float)f.delta;
    const int64_t ia = b0 * NR;  // anchor: the block's first central ray
    for (int j = rmin; j <= rmax; ++j) {
        if (!__syncthreads_or(myrep == j)) continue;  // no point of this block is in replica j
        double o[3];
        frame_origin(f, j, o);
        const long long ax = anchor_q(px[ia], o[0], f.inv_delta);
        const long long ay = anchor_q(py[ia], o[1], f.inv_delta);
        const long long az = anchor_q(pz[ia], o[2], f.inv_delta);
        float nx = -1e30f, ny = -1e30f, nz = -1e30f;  // far sentinel
        if (valid && myrep == j) {
            nx = -(float)(((px[ic] - o[0]) * f.inv_delta - (double)ax) * f.delta);
            ny = -(float)(((py[ic] - o[1]) * f.inv_delta - (double)ay) * f.delta);
            nz = -(float)(((pz[ic] - o[2]) * f.inv_delta - (double)az) * f.delta);
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
                    v = make_float4((float)(qq[0] - ax) * dlt, (float)(qq[1] - ay) * dlt, (float)(qq[2] - az) * dlt,
                                    __int_as_float(pr.w));
                    if (PEPS) e2 = f.eps2[pi];
                }
                s_p[q] = v;
                if (PEPS) s_e[q] = e2;
            }
            __syncthreads();
            for (int c0 = 0; c0 < kTile; c0 += kChunk) {
                float ccx = 0.f, ccy = 0.f, ccz = 0.f;
                float2 cx[PP], cy[PP], cz[PP];
#pragma unroll
                for (int p = 0; p < PP; ++p) cx[p] = cy[p] = cz[p] = make_float2(0.f, 0.f);
#pragma unroll 2
                for (int jj = c0; jj < c0 + kChunk; ++jj) {
                    const float4 a = s_p[jj];
                    const float e2 = PEPS ? s_e[jj] : f.eps2u;
                    // central ray (scalar)
                    const float dx = a.x + nx, dy = a.y + ny, dz = a.z + nz;
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, e2)));
                    const float inv = rsqrt_mufu(r2);
                    const float i2 = inv * inv;
                    float mi3;
                    if (UMASS) {
                        c_phi += inv;
                        mi3 = inv * i2;
                    } else {
                        const float mi = a.w * inv;
                        c_phi += mi;
                        mi3 = mi * i2;
                    }
                    ccx = fmaf(dx, mi3, ccx);
                    ccy = fmaf(dy, mi3, ccy);
                    ccz = fmaf(dz, mi3, ccz);
                    // satellites in pairs: d_k = d_c + (r_c - r_k)
                    const float2 DX = make_float2(dx, dx), DY = make_float2(dy, dy), DZ = make_float2(dz, dz);
                    const float2 E2 = make_float2(e2, e2);
#pragma unroll
                    for (int p = 0; p < PP; ++p) {
                        const float2 qx = __fadd2_rn(DX, ex[p]);
                        const float2 qy = __fadd2_rn(DY, ey[p]);
                        const float2 qz = __fadd2_rn(DZ, ez[p]);
                        float2 s2 = __ffma2_rn(qz, qz, E2);
                        s2 = __ffma2_rn(qy, qy, s2);
                        s2 = __ffma2_rn(qx, qx, s2);
                        const float2 w = make_float2(rsqrt_mufu(s2.x), rsqrt_mufu(s2.y));
                        const float2 w2 = __fmul2_rn(w, w);
                        const float2 m3 = UMASS ? __fmul2_rn(w, w2) : __fmul2_rn(__fmul2_rn(make_float2(a.w, a.w), w), w2);
                        cx[p] = __ffma2_rn(qx, m3, cx[p]);
                        cy[p] = __ffma2_rn(qy, m3, cy[p]);
                        cz[p] = __ffma2_rn(qz, m3, cz[p]);
                    }
                }
                two_sum_into(c_hx, c_lx, ccx);
                two_sum_into(c_hy, c_ly, ccy);
                two_sum_into(c_hz, c_lz, ccz);
#pragma unroll
                for (int p = 0; p < PP; ++p) {
                    two_sum2_into(hx[p], lx[p], cx[p]);
                    two_sum2_into(hy[p], ly[p], cy[p]);
                    two_sum2_into(hz[p], lz[p], cz[p]);
                }
            }
        }
    }
    if (!valid) return;
    const int64_t sn = (int64_t)split * 4;
    out[(sn + 0) * n_rays + ic] = make_float2(c_phi, 0.f);
    out[(sn + 1) * n_rays + ic] = make_float2(c_hx, c_lx);
    out[(sn + 2) * n_rays + ic] = make_float2(c_hy, c_ly);
    out[(sn + 3) * n_rays + ic] = make_float2(c_hz, c_lz);
    // ring potentials to first order about the central ray (ring_phi)
    const float gcx = c_hx + c_lx, gcy = c_hy + c_ly, gcz = c_hz + c_lz;
#pragma unroll
    for (int p = 0; p < PP; ++p)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t i = ic + 1 + 2 * p + h;
            const float e[3] = {h ? ex[p].y : ex[p].x, h ? ey[p].y : ey[p].x, h ? ez[p].y : ez[p].x};
            out[(sn + 0) * n_rays + i] = make_float2(ring_phi(c_phi, e, gcx, gcy, gcz), 0.f);
            out[(sn + 1) * n_rays + i] = h ? make_float2(hx[p].y, lx[p].y) : make_float2(hx[p].x, lx[p].x);
            out[(sn + 2) * n_rays + i] = h ? make_float2(hy[p].y, ly[p].y) : make_float2(hy[p].x, ly[p].x);
            out[(sn + 3) * n_rays + i] = h ? make_float2(hz[p].y, lz[p].y) : make_float2(hz[p].x, lz[p].x);
        }
}

// Two bundles per thread, fully packed: bundles A = b0 + tid and B = b0 + NT
// + tid form f32x2 pairs ray by ray, (A_c, B_c) for the central rays and
// (A_k, B_k) for each ring position, so every FP32 operation of the pair sum
// is an f32x2 instruction and no operand needs duplicating.  The satellite
// pairs are formed from the central pair as in bundle_block_sum.  The
// compensated (hi, lo) gradient sums live in shared memory (merged once per
// chunk) to keep the register count low; the potential is summed plainly.
constexpr int kChunk2 = 256;  // one merge per staged tile (measured 2.7 % faster than 128)

template <int NT, int NRING, bool REPL, bool PEPS, bool UMASS>
__device__ __forceinline__ void bundle2_block_sum(const DevField &f, const double *__restrict__ px,
                                                  const double *__restrict__ py, const double *__restrict__ pz,
                                                  const int *__restrict__ rep, int64_t n_b, int64_t n_rays,
                                                  int64_t b0, int64_t p0, int64_t p1, int split,
                                                  float2 *__restrict__ out, float4 *s_a, float4 *s_b, float2 *s_e,
                                                  float2 *s_hl)
{
    constexpr int NR = NRING + 1;
    const int tid = threadIdx.x;
    int64_t bb[2] = {b0 + tid, b0 + NT + tid};
    bool valid[2] = {bb[0] < n_b, bb[1] < n_b};
    __shared__ int s_rmin, s_rmax;
    if (tid == 0) {
        s_rmin = INT_MAX;
        s_rmax = INT_MIN;
    }
    __syncthreads();
    int myrep[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        myrep[h] = valid[h] ? checked_replica(rep ? rep[bb[h]] : 0, f.n_rep) : -1;
        if (myrep[h] >= 0) {
            atomicMin(&s_rmin, myrep[h]);
            atomicMax(&s_rmax, myrep[h]);
        }
    }
    __syncthreads();
    const int rmin = s_rmin, rmax = s_rmax;
    // ring offsets r_c - r_k of both bundles, paired (A, B)
    float2 ex[NRING], ey[NRING], ez[NRING];
#pragma unroll
    for (int k = 0; k < NRING; ++k) {
        float v[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
        for (int h = 0; h < 2; ++h)
            if (valid[h]) {
                const int64_t ic = bb[h] * NR, ik = ic + 1 + k;
                v[h][0] = (float)(px[ic] - px[ik]);
                v[h][1] = (float)(py[ic] - py[ik]);
                v[h][2] = (float)(pz[ic] - pz[ik]);
            }
        ex[k] = make_float2(v[0][0], v[1][0]);
        ey[k] = make_float2(v[0][1], v[1][1]);
        ez[k] = make_float2(v[0][2], v[1][2]);
    }
    // (hi, lo) of group g (0 central, 1.. ring) and output o in shared memory
    float2 *s_hi = s_hl, *s_lo = s_hl + NR * 3 * NT;
#pragma unroll
    for (int q = 0; q < NR * 3; ++q) s_hi[q * NT + tid] = s_lo[q * NT + tid] = make_float2(0.f, 0.f);
    float2 phi = make_float2(0.f, 0.f);  // central rays; the ring's follow in the epilogue
    const float dlt = (float)f.delta;
    const float2 E2u = make_float2(f.eps2u, f.eps2u);
    const int64_t ia = b0 * NR;  // anchor: the block's first central ray
    for (int j = rmin; j <= rmax; ++j) {
        if (!block_uses_replica<2>(myrep, j)) continue;  // no point of this block is in replica j
        double o[3];
        frame_origin(f, j, o);
        const long long ax = anchor_q(px[ia], o[0], f.inv_delta);
        const long long ay = anchor_q(py[ia], o[1], f.inv_delta);
        const long long az = anchor_q(pz[ia], o[2], f.inv_delta);
        float nc[2][3];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            nc[h][0] = nc[h][1] = nc[h][2] = -1e30f;  // far sentinel
            if (valid[h] && myrep[h] == j) {
                const int64_t ic = bb[h] * NR;
                nc[h][0] = -(float)(((px[ic] - o[0]) * f.inv_delta - (double)ax) * f.delta);
                nc[h][1] = -(float)(((py[ic] - o[1]) * f.inv_delta - (double)ay) * f.delta);
                nc[h][2] = -(float)(((pz[ic] - o[2]) * f.inv_delta - (double)az) * f.delta);
            }
        }
        const float2 NX = make_float2(nc[0][0], nc[1][0]), NY = make_float2(nc[0][1], nc[1][1]),
                     NZ = make_float2(nc[0][2], nc[1][2]);
        for (int64_t t0 = p0; t0 < p1; t0 += kTile) {
            __syncthreads();
            for (int q = tid; q < kTile; q += NT) {
                const int64_t pi = t0 + q;
                float x = 1e18f, y = 1e18f, z = 1e18f, m = 0.0f, e2 = 0.0f;
                if (pi < p1) {
                    const int4 pr = f.part[pi];
                    long long qq[3] = {pr.x, pr.y, pr.z};
                    if (REPL) replica_q(f, j, pr.x, pr.y, pr.z, qq);
                    x = (float)(qq[0] - ax) * dlt;
                    y = (float)(qq[1] - ay) * dlt;
                    z = (float)(qq[2] - az) * dlt;
                    m = __int_as_float(pr.w);
                    if (PEPS) e2 = f.eps2[pi];
                }
                s_a[q] = make_float4(x, x, y, y);
                s_b[q] = make_float4(z, z, m, m);
                if (PEPS) s_e[q] = make_float2(e2, e2);
            }
            __syncthreads();
            for (int c0 = 0; c0 < kTile; c0 += kChunk2) {
                float2 cx[NR], cy[NR], cz[NR];
#pragma unroll
                for (int g = 0; g < NR; ++g) cx[g] = cy[g] = cz[g] = make_float2(0.f, 0.f);
#pragma unroll 1
                for (int jj = c0; jj < c0 + kChunk2; ++jj) {
                    const float4 a = s_a[jj];
                    const float4 b = s_b[jj];
                    const float2 E2 = PEPS ? s_e[jj] : E2u;
                    const float2 M2 = make_float2(b.z, b.w);
                    // central pair: d_c = p - r_c for bundles A and B
                    const float2 DX = __fadd2_rn(make_float2(a.x, a.y), NX);
                    const float2 DY = __fadd2_rn(make_float2(a.z, a.w), NY);
                    const float2 DZ = __fadd2_rn(make_float2(b.x, b.y), NZ);
#pragma unroll
                    for (int g = 0; g < NR; ++g) {
                        const float2 qx = g == 0 ? DX : __fadd2_rn(DX, ex[g - 1]);
                        const float2 qy = g == 0 ? DY : __fadd2_rn(DY, ey[g - 1]);
                        const float2 qz = g == 0 ? DZ : __fadd2_rn(DZ, ez[g - 1]);
                        float2 s2 = __ffma2_rn(qz, qz, E2);
                        s2 = __ffma2_rn(qy, qy, s2);
                        s2 = __ffma2_rn(qx, qx, s2);
                        const float2 w = make_float2(rsqrt_mufu(s2.x), rsqrt_mufu(s2.y));
                        const float2 w2 = __fmul2_rn(w, w);
                        float2 m3;
                        if (UMASS) {
                            if (g == 0) phi = __fadd2_rn(phi, w);
                            m3 = __fmul2_rn(w, w2);
                        } else {
                            const float2 mw = __fmul2_rn(M2, w);
                            if (g == 0) phi = __fadd2_rn(phi, mw);
                            m3 = __fmul2_rn(mw, w2);
                        }
                        cx[g] = __ffma2_rn(qx, m3, cx[g]);
                        cy[g] = __ffma2_rn(qy, m3, cy[g]);
                        cz[g] = __ffma2_rn(qz, m3, cz[g]);
                    }
                }
#pragma unroll
                for (int g = 0; g < NR; ++g) {
                    const float2 cc[3] = {cx[g], cy[g], cz[g]};
#pragma unroll
                    for (int oo = 0; oo < 3; ++oo) {
                        const int q = (g * 3 + oo) * NT + tid;
                        float2 hi = s_hi[q], lo = s_lo[q];
                        two_sum2_into(hi, lo, cc[oo]);
                        s_hi[q] = hi;
                        s_lo[q] = lo;
                    }
                }
            }
        }
    }
    const int64_t sn = (int64_t)split * 4;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (!valid[h]) continue;
        const int64_t ic = bb[h] * NR;
        const float pc = h ? phi.y : phi.x;
        float gc[3];
#pragma unroll
        for (int oo = 0; oo < 3; ++oo) {
            const float2 hi = s_hi[oo * NT + tid], lo = s_lo[oo * NT + tid];
            gc[oo] = h ? hi.y + lo.y : hi.x + lo.x;
        }
#pragma unroll
        for (int g = 0; g < NR; ++g) {
            const int64_t i = ic + g;
            float pg = pc;
            if (g > 0) {  // ring potentials to first order about the central ray (ring_phi)
                const float e[3] = {h ? ex[g - 1].y : ex[g - 1].x, h ? ey[g - 1].y : ey[g - 1].x,
                                    h ? ez[g - 1].y : ez[g - 1].x};
                pg = ring_phi(pc, e, gc[0], gc[1], gc[2]);
            }
            out[(sn + 0) * n_rays + i] = make_float2(pg, 0.f);
#pragma unroll
            for (int oo = 0; oo < 3; ++oo) {
                const int q = (g * 3 + oo) * NT + tid;
                const float2 hi = s_hi[q], lo = s_lo[q];
                out[(sn + 1 + oo) * n_rays + i] = h ? make_float2(hi.y, lo.y) : make_float2(hi.x, lo.x);
            }
        }
    }
}

// bounded for 512 resident threads per SM (128 registers, no spills)
template <int NT, int NRING, bool REPL, bool PEPS, bool UMASS>
__global__ void __launch_bounds__(NT, 512 / NT) k_force_bundle2(ForceArgs A)
{
    if (A.gate && *A.gate == 0ull) return;
    __shared__ float4 s_a[kTile];
    __shared__ float4 s_b[kTile];
    __shared__ float2 s_e[PEPS ? kTile : 1];
    __shared__ float2 s_hl[2 * (NRING + 1) * 3 * NT];
    const int64_t n_b = A.n / (NRING + 1);
    const int64_t b0 = (int64_t)blockIdx.x * 2 * NT;
    const int split = blockIdx.y;
    const int64_t p0 = (int64_t)split * A.per_split;
    const int64_t p1 = min(A.f.n, p0 + A.per_split);
    bundle2_block_sum<NT, NRING, REPL, PEPS, UMASS>(A.f, A.px, A.py, A.pz, A.rep, n_b, A.n, b0, p0, p1, split,
                                                    (float2 *)A.out, s_a, s_b, s_e, s_hl);
}

// Two bundles per thread with the ring separations expanded about the
// central ray.  With d_c = p - r_c and e_k = r_c - r_k the ring ray's
// separation is d_k = d_c + e_k, so
//   |d_k|^2 + eps^2 = (|d_c|^2 + eps^2) + (2 e_k . d_c + |e_k|^2)
//   sum m d_k / r_k^3 = sum m d_c / r_k^3 + e_k sum m / r_k^3.
// The central ray's softened squared distance is shared by the ring, each
// ring ray adds a three-FMA correction (its own rounding is one add), and the
// ring gradient splits into a sum along d_c plus e_k times a positive scalar
// sum S_k, combined once per block.  Per particle and pair of bundles this is
// 52 f32x2 operations for 10 interactions (the unexpanded kernel: 56).
// (Taking 1/r^2 from MUFU rcp instead of rsqrt^2 saves 5 more but was
// measured 26 % slower: the MUFU pipe then limits.)
// AHEAD: read the next particle's records one iteration ahead, so that the
// shared-memory latency overlaps the current particle's arithmetic (s_a and
// s_b then hold kTile + 1 records).  It pays in the single-trace kernel;
// the persistent batched kernel runs faster without it.
template <int NT, int NRING, bool REPL, bool PEPS, bool UMASS, int CL, bool AHEAD = true>
__device__ __forceinline__ void bundle2x_block_sum(const DevField &f, const double *__restrict__ px,
                                                   const double *__restrict__ py, const double *__restrict__ pz,
                                                   const int *__restrict__ rep, int64_t n_b, int64_t n_rays,
                                                   int64_t b0, int64_t p0, int64_t p1, int split,
                                                   float2 *__restrict__ out, float4 *s_a, float4 *s_b, float *s_e,
                                                   float2 *s_hl)
{
    constexpr int NR = NRING + 1;
    constexpr int NQ = NR * 3 + NRING;  // compensated sums per bundle: G (3 per ray) and S (ring)
    const int tid = threadIdx.x;
    int64_t bb[2] = {b0 + tid, b0 + NT + tid};
    bool valid[2] = {bb[0] < n_b, bb[1] < n_b};
    __shared__ int s_rmin, s_rmax;
    if (tid == 0) {
        s_rmin = INT_MAX;
        s_rmax = INT_MIN;
    }
    __syncthreads();
    int myrep[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        myrep[h] = valid[h] ? checked_replica(rep ? rep[bb[h]] : 0, f.n_rep) : -1;
        if (myrep[h] >= 0) {
            atomicMin(&s_rmin, myrep[h]);
            atomicMax(&s_rmax, myrep[h]);
        }
    }
    __syncthreads();
    const int rmin = s_rmin, rmax = s_rmax;
    // 2 e_k (exact doubling of the once-rounded FP64 offset) and |e_k|^2, paired (A, B)
    float2 fx[NRING], fy[NRING], fz[NRING], ee[NRING];
#pragma unroll
    for (int k = 0; k < NRING; ++k) {
        float v[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
        for (int h = 0; h < 2; ++h)
            if (valid[h]) {
                const int64_t ic = bb[h] * NR, ik = ic + 1 + k;
                v[h][0] = (float)(px[ic] - px[ik]);
                v[h][1] = (float)(py[ic] - py[ik]);
                v[h][2] = (float)(pz[ic] - pz[ik]);
            }
        fx[k] = make_float2(2.f * v[0][0], 2.f * v[1][0]);
        fy[k] = make_float2(2.f * v[0][1], 2.f * v[1][1]);
        fz[k] = make_float2(2.f * v[0][2], 2.f * v[1][2]);
        ee[k] = make_float2(fmaf(v[0][0], v[0][0], fmaf(v[0][1], v[0][1], v[0][2] * v[0][2])),
                            fmaf(v[1][0], v[1][0], fmaf(v[1][1], v[1][1], v[1][2] * v[1][2])));
    }
    // (hi, lo) per bundle pair: q = 3 g + o for G of ray g, 3 NR + k for S_k
    float2 *s_hi = s_hl, *s_lo = s_hl + NQ * NT;
#pragma unroll
    for (int q = 0; q < NQ; ++q) s_hi[q * NT + tid] = s_lo[q * NT + tid] = make_float2(0.f, 0.f);
    float2 phi = make_float2(0.f, 0.f);  // central rays; the ring's follow in the epilogue
    const float dlt = (float)f.delta;
    const float2 E2u = make_float2(f.eps2u, f.eps2u);
    const int64_t ia = b0 * NR;  // anchor: the block's first central ray
    for (int j = rmin; j <= rmax; ++j) {
        if (!block_uses_replica<2>(myrep, j)) continue;  // no point of this block is in replica j
        double o[3];
        frame_origin(f, j, o);
        const long long ax = anchor_q(px[ia], o[0], f.inv_delta);
        const long long ay = anchor_q(py[ia], o[1], f.inv_delta);
        const long long az = anchor_q(pz[ia], o[2], f.inv_delta);
        float nc[2][3];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            nc[h][0] = nc[h][1] = nc[h][2] = -1e30f;  // far sentinel
            if (valid[h] && myrep[h] == j) {
                const int64_t ic = bb[h] * NR;
                nc[h][0] = -(float)(((px[ic] - o[0]) * f.inv_delta - (double)ax) * f.delta);
                nc[h][1] = -(float)(((py[ic] - o[1]) * f.inv_delta - (double)ay) * f.delta);
                nc[h][2] = -(float)(((pz[ic] - o[2]) * f.inv_delta - (double)az) * f.delta);
            }
        }
        const float2 NX = make_float2(nc[0][0], nc[1][0]), NY = make_float2(nc[0][1], nc[1][1]),
                     NZ = make_float2(nc[0][2], nc[1][2]);
        for (int64_t t0 = p0; t0 < p1; t0 += kTile) {
            __syncthreads();
            for (int q = tid; q < kTile; q += NT) {
                const int64_t pi = t0 + q;
                float x = 1e18f, y = 1e18f, z = 1e18f, m = 0.0f, e2 = 0.0f;
                if (pi < p1) {
                    const int4 pr = f.part[pi];
                    long long qq[3] = {pr.x, pr.y, pr.z};
                    if (REPL) replica_q(f, j, pr.x, pr.y, pr.z, qq);
                    x = (float)(qq[0] - ax) * dlt;
                    y = (float)(qq[1] - ay) * dlt;
                    z = (float)(qq[2] - az) * dlt;
                    m = __int_as_float(pr.w);
                    if (PEPS) e2 = f.eps2[pi];
                }
                s_a[q] = make_float4(x, x, y, y);
                s_b[q] = make_float4(z, z, m, m);
                if (PEPS) s_e[q] = e2;
            }
            __syncthreads();
            for (int c0 = 0; c0 < kTile; c0 += kChunk2) {
                float2 cx[NR], cy[NR], cz[NR], cs[NRING];
#pragma unroll
                for (int g = 0; g < NR; ++g) cx[g] = cy[g] = cz[g] = make_float2(0.f, 0.f);
#pragma unroll
                for (int k = 0; k < NRING; ++k) cs[k] = make_float2(0.f, 0.f);
                float4 a_nx, b_nx;  // read-ahead registers (AHEAD)
                if constexpr (AHEAD) {
                    a_nx = s_a[c0];
                    b_nx = s_b[c0];
                }
#pragma unroll 1
                for (int jj = c0; jj < c0 + kChunk2; ++jj) {
                    float4 a, b;
                    if constexpr (AHEAD) {
                        a = a_nx;
                        b = b_nx;
                        a_nx = s_a[jj + 1];
                        b_nx = s_b[jj + 1];
                    } else {
                        a = s_a[jj];
                        b = s_b[jj];
                    }
                    const float2 E2 = PEPS ? make_float2(s_e[jj], s_e[jj]) : E2u;
                    const float2 M2 = make_float2(b.z, b.w);
                    const float2 DX = __fadd2_rn(make_float2(a.x, a.y), NX);
                    const float2 DY = __fadd2_rn(make_float2(a.z, a.w), NY);
                    const float2 DZ = __fadd2_rn(make_float2(b.x, b.y), NZ);
                    float2 R2 = __ffma2_rn(DZ, DZ, E2);
                    R2 = __ffma2_rn(DY, DY, R2);
                    R2 = __ffma2_rn(DX, DX, R2);
#pragma unroll
                    for (int g = 0; g < NR; ++g) {
                        float2 s2 = R2;
                        if (g > 0) {
                            float2 t = __ffma2_rn(fz[g - 1], DZ, ee[g - 1]);
                            t = __ffma2_rn(fy[g - 1], DY, t);
                            t = __ffma2_rn(fx[g - 1], DX, t);
                            s2 = __fadd2_rn(R2, t);
                        }
                        const float2 w = make_float2(rsqrt_mufu(s2.x), rsqrt_mufu(s2.y));
                        const float2 u = __fmul2_rn(w, w);
                        float2 m3;
                        if (UMASS) {
                            if (g == 0) phi = __fadd2_rn(phi, w);
                            m3 = __fmul2_rn(w, u);
                        } else {
                            const float2 mw = __fmul2_rn(M2, w);
                            if (g == 0) phi = __fadd2_rn(phi, mw);
                            m3 = __fmul2_rn(mw, u);
                        }
                        if (g > 0) cs[g - 1] = __fadd2_rn(cs[g - 1], m3);
                        cx[g] = __ffma2_rn(DX, m3, cx[g]);
                        cy[g] = __ffma2_rn(DY, m3, cy[g]);
                        cz[g] = __ffma2_rn(DZ, m3, cz[g]);
                    }
                }
#pragma unroll
                for (int g = 0; g < NR; ++g) {
                    const float2 cc[3] = {cx[g], cy[g], cz[g]};
#pragma unroll
                    for (int oo = 0; oo < 3; ++oo) {
                        const int q = (g * 3 + oo) * NT + tid;
                        float2 hi = s_hi[q], lo = s_lo[q];
                        two_sum2_into(hi, lo, cc[oo]);
                        s_hi[q] = hi;
                        s_lo[q] = lo;
                    }
                }
#pragma unroll
                for (int k = 0; k < NRING; ++k) {
                    const int q = (NR * 3 + k) * NT + tid;
                    float2 hi = s_hi[q], lo = s_lo[q];
                    two_sum2_into(hi, lo, cs[k]);
                    s_hi[q] = hi;
                    s_lo[q] = lo;
                }
            }
        }
    }
    // gradient of ring ray k: G_k + e_k S_k, as an FP32 (hi, lo) pair (the
    // product's rounding error recovered by an FMA, the sum by TwoSum).
    // Outputs per thread: slot g (< NR) holds (phi_A, phi_B) of ray g, slot
    // NR + (h NR + g) 3 + o - 1 the (hi, lo) of gradient component o of ray g
    // of bundle h.
    constexpr int NSLOT = NR + 2 * NR * 3;
    float2 res[NSLOT];
    res[0] = phi;
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int g = 0; g < NR; ++g) {
            float shi = 0.f, slo = 0.f;
            if (g > 0) {
                const float2 a = s_hi[(NR * 3 + g - 1) * NT + tid], c = s_lo[(NR * 3 + g - 1) * NT + tid];
                shi = h ? a.y : a.x;
                slo = h ? c.y : c.x;
            }
#pragma unroll
            for (int oo = 0; oo < 3; ++oo) {
                const int q = (g * 3 + oo) * NT + tid;
                const float2 a = s_hi[q], c = s_lo[q];
                float hi = h ? a.y : a.x, lo = h ? c.y : c.x;
                if (g > 0) {
                    const float2 f2 = oo == 0 ? fx[g - 1] : (oo == 1 ? fy[g - 1] : fz[g - 1]);
                    const float e = 0.5f * (h ? f2.y : f2.x);
                    const float p = e * shi;
                    const float pe = fmaf(e, shi, -p);
                    const float sm = hi + p;
                    const float bv = sm - hi;
                    const float err = (hi - (sm - bv)) + (p - bv);
                    lo = lo + (err + fmaf(e, slo, pe));
                    hi = sm;
                }
                res[NR + (h * NR + g) * 3 + oo] = make_float2(hi, lo);
            }
        }
    // ring potentials to first order about the central ray (ring_phi), from
    // the central gradient; e_k = r_c - r_k is half the stored 2 e_k
#pragma unroll
    for (int g = 1; g < NR; ++g) {
        float v[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float2 *gc = res + NR + (h * NR) * 3;
            const float e[3] = {0.5f * (h ? fx[g - 1].y : fx[g - 1].x), 0.5f * (h ? fy[g - 1].y : fy[g - 1].x),
                                0.5f * (h ? fz[g - 1].y : fz[g - 1].x)};
            v[h] = ring_phi(h ? phi.y : phi.x, e, gc[0].x + gc[0].y, gc[1].x + gc[1].y, gc[2].x + gc[2].y);
        }
        res[g] = make_float2(v[0], v[1]);
    }
    if (CL == 1) {
        const int64_t sn = (int64_t)split * 4;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (!valid[h]) continue;
            const int64_t ic = bb[h] * NR;
#pragma unroll
            for (int g = 0; g < NR; ++g) {
                out[(sn + 0) * n_rays + ic + g] = make_float2(h ? res[g].y : res[g].x, 0.f);
#pragma unroll
                for (int oo = 0; oo < 3; ++oo) out[(sn + 1 + oo) * n_rays + ic + g] = res[NR + (h * NR + g) * 3 + oo];
            }
        }
        return;
    }
    // cluster of CL blocks (consecutive splits of the same bundle block): the
    // partials are added in distributed shared memory, in rank order, and one
    // partial per cluster is written (split / CL)
    static_assert(NSLOT <= 2 * (NR * 3 + NRING), "outputs must fit the (hi, lo) buffer");
    __syncthreads();  // every thread has read its (hi, lo) sums
#pragma unroll
    for (int q = 0; q < NSLOT; ++q) s_hl[q * NT + tid] = res[q];
    cg::cluster_group cluster = cg::this_cluster();
    cluster.sync();
    const int rank = (int)cluster.block_rank();
    constexpr int TPR = NT / CL;  // threads' outputs each rank reduces
    const int64_t sn = (int64_t)(split / CL) * 4;
    for (int it = tid; it < NSLOT * TPR; it += NT) {
        const int q = it / TPR, t = rank * TPR + it % TPR;
        float hx = 0.f, lx = 0.f, hy = 0.f, ly = 0.f;
#pragma unroll
        for (int r = 0; r < CL; ++r) {
            const float2 v = cluster.map_shared_rank(s_hl, r)[q * NT + t];
            if (q < NR) {  // potential of bundles A and B: plain sums
                hx += v.x;
                hy += v.y;
            } else {  // (hi, lo) gradient: TwoSum on the high parts
                const float sm = hx + v.x;
                const float bv = sm - hx;
                lx += ((hx - (sm - bv)) + (v.x - bv)) + v.y;
                hx = sm;
            }
        }
        if (q < NR) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t bh = b0 + h * NT + t;
                if (bh < n_b) out[sn * n_rays + bh * NR + q] = make_float2(h ? hy : hx, 0.f);
            }
        } else {
            const int k = q - NR, h = k / (NR * 3), g = (k / 3) % NR, oo = k % 3;
            const int64_t bh = b0 + h * NT + t;
            if (bh < n_b) out[(sn + 1 + oo) * n_rays + bh * NR + g] = make_float2(hx, lx);
        }
        (void)ly;
    }
    cluster.sync();  // no block leaves while the others read its shared memory
}

// TPSM: resident threads per SM the register allocation is bounded for;
// AHEAD: the particle loop's read-ahead (bundle2x_block_sum)
template <int NT, int NRING, bool REPL, bool PEPS, bool UMASS, int TPSM, int CL, bool AHEAD = true>
__global__ void __launch_bounds__(NT, TPSM / NT) k_force_bundle2x(ForceArgs A)
{
    if (A.gate && *A.gate == 0ull) return;
    __shared__ float4 s_a[kTile + 1];  // + 1: the particle loop reads one record ahead
    __shared__ float4 s_b[kTile + 1];
    __shared__ float s_e[PEPS ? kTile : 1];
    __shared__ float2 s_hl[2 * ((NRING + 1) * 3 + NRING) * NT];
    const int64_t n_b = A.n / (NRING + 1);
    const int64_t b0 = (int64_t)blockIdx.x * 2 * NT;
    const int split = blockIdx.y;
    const int64_t p0 = (int64_t)split * A.per_split;
    const int64_t p1 = min(A.f.n, p0 + A.per_split);
    bundle2x_block_sum<NT, NRING, REPL, PEPS, UMASS, CL, AHEAD>(A.f, A.px, A.py, A.pz, A.rep, n_b, A.n, b0, p0, p1,
                                                            split, (float2 *)A.out, s_a, s_b, s_e, s_hl);
}

// ForceArgs for the bundle kernel: n = rays, group = rays per bundle; rep is
// the per-bundle replica array.
template <int NT, int NRING, bool REPL, bool PEPS, bool UMASS>
__global__ void __launch_bounds__(NT) k_force_bundle(ForceArgs A)
{
    if (A.gate && *A.gate == 0ull) return;
    __shared__ float4 s_p[kTile];
    __shared__ float s_e[PEPS ? kTile : 1];
    const int64_t n_b = A.n / (NRING + 1);
    const int64_t b0 = (int64_t)blockIdx.x * NT;
    const int split = blockIdx.y;
    const int64_t p0 = (int64_t)split * A.per_split;
    const int64_t p1 = min(A.f.n, p0 + A.per_split);
    bundle_block_sum<NT, NRING, REPL, PEPS, UMASS>(A.f, A.px, A.py, A.pz, A.rep, n_b, A.n, b0, p0, p1, split,
                                                   (float2 *)A.out, s_p, s_e);
}

// FP64 twin (the all-FP64 path): same staging, FP64 arithmetic, plain sums.
template <int R, int NT, bool REPL, bool PEPS>
__global__ void __launch_bounds__(NT) k_force_fp64(ForceArgs A)
{
    if (A.gate && *A.gate == 0ull) return;
    __shared__ double4_16a s_p[kTile64];
    __shared__ double s_e[PEPS ? kTile64 : 1];
    const DevField &f = A.f;
    const int tid = threadIdx.x;
    const int64_t base = (int64_t)blockIdx.x * (NT * R);
    const int split = blockIdx.y;
    int myrep[R], rmin, rmax;
    block_replica_range<R, NT>(A, f.n_rep, base, myrep, rmin, rmax);
    double acc[R][4];
#pragma unroll
    for (int k = 0; k < R; ++k)
#pragma unroll
        for (int o = 0; o < 4; ++o) acc[k][o] = 0.0;
    const int64_t p0 = (int64_t)split * A.per_split;
    const int64_t p1 = min(f.n, p0 + A.per_split);
    for (int j = rmin; j <= rmax; ++j) {
        if (!block_uses_replica<R>(myrep, j)) continue;  // no point of this block is in replica j
        double o[3];
        frame_origin(f, j, o);
        const long long ax = anchor_q(A.px[base], o[0], f.inv_delta);
        const long long ay = anchor_q(A.py[base], o[1], f.inv_delta);
        const long long az = anchor_q(A.pz[base], o[2], f.inv_delta);
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
                double4_16a v = make_double4_16a(1e100, 1e100, 1e100, 0.0);
                double e2 = 0.0;
                if (pi < p1) {
                    const int4 pr = f.part[pi];
                    long long qq[3] = {pr.x, pr.y, pr.z};
                    if (REPL) replica_q(f, j, pr.x, pr.y, pr.z, qq);
                    v = make_double4_16a((double)(qq[0] - ax) * f.delta, (double)(qq[1] - ay) * f.delta,
                                         (double)(qq[2] - az) * f.delta, f.m64[pi]);
                    if (PEPS) e2 = f.eps2_64[pi];
                }
                s_p[q] = v;
                if (PEPS) s_e[q] = e2;
            }
            __syncthreads();
#pragma unroll 4
            for (int jj = 0; jj < kTile64; ++jj) {
                const double4_16a p = s_p[jj];
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
