// born.cu -- the Born approximation (Sec. 6): convergence and shear of each
// line of sight from the Hessian of psi = phi / a along the unperturbed ray
// x(chi) = (theta_x chi, theta_y chi, chi):
//   kappa  = int W (d11 + d22) psi dchi,   gamma1 = int W (d11 - d22) psi dchi,
//   gamma2 = 2 int W d12 psi dchi,          W = chi (chi_s - chi) / chi_s,
// over the trace's node table by the trapezoid rule in the node variable.
// The Hessian pair sum runs in FP32 with chunked TwoSum accumulation (the
// same anchoring as the field kernels); node weights, the mean-density prism
// and the accumulation over nodes are FP64.
#include <algorithm>

#include "force.cuh"
#include "trace_device.cuh"

namespace rt3d {

// node positions and weights: w_k = trapezoid weight x d chi / d u x W / a
__global__ void k_born_nodes(Cosmo c, double z_s, int kind, int n, double chi_l, double s, double *__restrict__ x,
                             double *__restrict__ w)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > n) return;
    const double chi_s = comoving_distance(c, z_s);
    const double xk = sched_node(kind, n, k, chi_s, chi_l, s);
    double du, jac;
    if (kind == RT3D_SCHED_UNIFORM) {
        du = chi_s / n;
        jac = 1.0;
    } else {
        du = (asinh((chi_s - chi_l) / s) - asinh(-chi_l / s)) / n;
        jac = sqrt(s * s + (xk - chi_l) * (xk - chi_l));
    }
    const double W = xk * (chi_s - xk) / chi_s;
    x[k] = xk;
    w[k] = ((k == 0 || k == n) ? 0.5 : 1.0) * du * jac * W * (1.0 + redshift_at(c, xk));
}

// points of nodes [k0, k0 + K) for every bundle, node-major (neighbouring
// bundles of one node are neighbours in space, as the rays of a stage are)
__global__ void k_born_points(DevField f, int64_t n_b, const double *__restrict__ theta, const double *__restrict__ x,
                              int k0, int K, double *__restrict__ pts, int *__restrict__ rep)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t m = (int64_t)K * n_b;
    if (q >= m) return;
    const int64_t b = q % n_b;
    const double xk = x[k0 + q / n_b];
    pts[q] = theta[2 * b] * xk;
    pts[m + q] = theta[2 * b + 1] * xk;
    pts[2 * m + q] = xk;
    rep[q] = replica_of(f, xk);
}

// Hessian pair sum: for every point, sums over particles [p0, p1) of
//   A = m (2 / r^3 - 3 (dx^2 + dy^2) / r^5),  B = m (dy^2 - dx^2) / r^5,
//   C = m dx dy / r^5          (d = point - particle, r^2 = |d|^2 + eps^2)
// so that (d11 + d22) phi = A, (d11 - d22) phi = 3 B, d12 phi = -3 C (times
// mu_G / 2^ms); (hi, lo) partials at out[(split * 3 + o) * n + i].
template <int R, int NT, bool REPL, bool PEPS>
__global__ void __launch_bounds__(NT) k_hess(ForceArgs A)
{
    __shared__ float4 s_p[kTile];
    __shared__ float s_e[PEPS ? kTile : 1];
    const DevField &f = A.f;
    const int tid = threadIdx.x;
    const int64_t base = (int64_t)blockIdx.x * (NT * R);
    const int split = blockIdx.y;
    int myrep[R], rmin, rmax;
    block_replica_range<R, NT>(A, f.n_rep, base, myrep, rmin, rmax);
    float hi[R][3], lo[R][3];
#pragma unroll
    for (int k = 0; k < R; ++k)
#pragma unroll
        for (int o = 0; o < 3; ++o) hi[k][o] = lo[k][o] = 0.0f;
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
            } else {  // far sentinel: every contribution is exactly zero (squares stay finite)
                rx[k] = ry[k] = rz[k] = 5e18f;
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
                    v = make_float4((float)(qq[0] - ax) * dlt, (float)(qq[1] - ay) * dlt, (float)(qq[2] - az) * dlt,
                                    __int_as_float(pr.w));
                    if (PEPS) e2 = f.eps2[pi];
                }
                s_p[q] = v;
                if (PEPS) s_e[q] = e2;
            }
            __syncthreads();
            for (int c0 = 0; c0 < kTile; c0 += kChunk) {
                float ca[R][3];
#pragma unroll
                for (int k = 0; k < R; ++k) ca[k][0] = ca[k][1] = ca[k][2] = 0.0f;
#pragma unroll 4
                for (int jj = c0; jj < c0 + kChunk; ++jj) {
                    const float4 p = s_p[jj];
                    const float e2 = PEPS ? s_e[jj] : f.eps2u;
#pragma unroll
                    for (int k = 0; k < R; ++k) {
                        const float dx = rx[k] - p.x, dy = ry[k] - p.y, dz = rz[k] - p.z;
                        const float dxx = dx * dx, dyy = dy * dy;
                        const float r2 = fmaf(dz, dz, dxx + dyy) + e2;
                        const float inv = rsqrt_mufu(r2);
                        const float i2 = inv * inv;
                        const float m3 = p.w * inv * i2, m5 = m3 * i2;
                        ca[k][0] += fmaf(-3.0f * (dxx + dyy), m5, 2.0f * m3);
                        ca[k][1] = fmaf(dyy - dxx, m5, ca[k][1]);
                        ca[k][2] = fmaf(dx * dy, m5, ca[k][2]);
                    }
                }
#pragma unroll
                for (int k = 0; k < R; ++k)
#pragma unroll
                    for (int o2 = 0; o2 < 3; ++o2) two_sum_into(hi[k][o2], lo[k][o2], ca[k][o2]);
            }
        }
    }
    float2 *out = (float2 *)A.out;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int64_t i = base + (int64_t)k * NT + tid;
        if (i < A.n)
#pragma unroll
            for (int o2 = 0; o2 < 3; ++o2) out[((int64_t)split * 3 + o2) * A.n + i] = make_float2(hi[k][o2], lo[k][o2]);
    }
}

// per bundle: add the chunk's nodes (FP64, node order) to out[b] = (kappa, gamma1, gamma2)
__global__ void k_born_accum(DevField f, int64_t n_b, int S, const float2 *__restrict__ partials,
                             const double *__restrict__ pts, const int *__restrict__ rep, const double *__restrict__ w,
                             int k0, int K, double *__restrict__ out)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_b) return;
    const int64_t m = (int64_t)K * n_b;
    double acc[3] = {out[3 * b], out[3 * b + 1], out[3 * b + 2]};
    for (int kk = 0; kk < K; ++kk) {
        const int64_t q = (int64_t)kk * n_b + b;
        double v[3];
#pragma unroll
        for (int o = 0; o < 3; ++o) {
            float h = 0.0f, l = 0.0f;
            for (int s = 0; s < S; ++s) {
                const float2 p = partials[((int64_t)s * 3 + o) * m + q];
                const float t = h + p.x;
                const float bb = t - h;
                l += ((h - (t - bb)) + (p.x - bb)) + p.y;
                h = t;
            }
            v[o] = ((double)h + (double)l) * f.mscale_inv;
        }
        double lap = v[0], dif = 3.0 * v[1], mix = -3.0 * v[2];
        if (f.replicated && f.mean_subtract) {  // minus the replica's uniform mean density
            const double p[3] = {pts[q], pts[m + q], pts[2 * m + q]};
            const int r = rep[q];
            const double lo[3] = {-0.5 * f.L, -0.5 * f.L, (double)r * f.L};
            const double hi[3] = {0.5 * f.L, 0.5 * f.L, (double)(r + 1) * f.L};
            double I[4], H[6];
            prism_field_hess<double>(lo, hi, p, I, H);
            lap += f.rho_term * (H[0] + H[3]);
            dif += f.rho_term * (H[0] - H[3]);
            mix += f.rho_term * H[1];
        }
        const double wk = w[k0 + kk];
        acc[0] += wk * lap;
        acc[1] += wk * dif;
        acc[2] += wk * 2.0 * mix;
    }
    out[3 * b] = acc[0];
    out[3 * b + 1] = acc[1];
    out[3 * b + 2] = acc[2];
}

static cudaError_t launch_hess(const ForceArgs &A, int splits, cudaStream_t st)
{
    constexpr int R = 4, NT = 128;
    const dim3 grid((unsigned)((A.n + R * NT - 1) / (R * NT)), (unsigned)splits);
    const bool repl = A.f.replicated != 0, peps = A.f.eps2 != nullptr;
    if (repl && peps) k_hess<R, NT, true, true><<<grid, NT, 0, st>>>(A);
    else if (repl) k_hess<R, NT, true, false><<<grid, NT, 0, st>>>(A);
    else if (peps) k_hess<R, NT, false, true><<<grid, NT, 0, st>>>(A);
    else k_hess<R, NT, false, false><<<grid, NT, 0, st>>>(A);
    return cudaGetLastError();
}

// Scratch layout (doubles unless noted): x[n+1], w[n+1], pts[3 K n_b],
// rep (int)[K n_b], partials (float2)[splits 3 K n_b]; sizes from born_scratch.
size_t born_scratch_bytes(int64_t n_b, int n_steps, int K, int splits)
{
    const size_t m = (size_t)K * (size_t)n_b;
    return sizeof(double) * (2 * (size_t)(n_steps + 1) + 3 * m) + sizeof(int) * m + sizeof(float2) * 3 * m * splits +
           256;
}

cudaError_t born_run(const Cosmo &c, const DevField &f, int64_t n_particles, double z_s, int64_t n_b,
                     const double *d_theta, int kind, int n_steps, double chi_l, double s, int K, int splits,
                     void *scratch, double *d_out, cudaStream_t st)
{
    const int n = n_steps;
    const size_t m = (size_t)K * (size_t)n_b;
    double *x = (double *)scratch, *w = x + (n + 1), *pts = w + (n + 1);
    int *rep = (int *)(pts + 3 * m);
    float2 *part = (float2 *)(((uintptr_t)(rep + m) + 255) & ~(uintptr_t)255);
    cudaError_t e;
    k_born_nodes<<<(n + 1 + 127) / 128, 128, 0, st>>>(c, z_s, kind, n, chi_l, s, x, w);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(d_out, 0, sizeof(double) * 3 * n_b, st)) != cudaSuccess) return e;
    const int64_t tiles = std::max<int64_t>(1, (n_particles + kTile - 1) / kTile);
    const int64_t tps = (tiles + splits - 1) / splits;
    const int S = (int)((tiles + tps - 1) / tps);
    for (int k0 = 0; k0 <= n; k0 += K) {
        const int Kc = std::min(K, n + 1 - k0);
        const int64_t mc = (int64_t)Kc * n_b;
        k_born_points<<<(unsigned)((mc + 255) / 256), 256, 0, st>>>(f, n_b, d_theta, x, k0, Kc, pts, rep);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        ForceArgs A;
        A.f = f;
        A.px = pts;
        A.py = pts + mc;
        A.pz = pts + 2 * mc;
        A.rep = rep;
        A.group = 1;
        A.n = mc;
        A.per_split = tps * kTile;
        A.out = part;
        A.gate = nullptr;
        // the point arrays of a chunk are contiguous at stride mc (not m)
        if (n_particles > 0) {
            if ((e = launch_hess(A, S, st)) != cudaSuccess) return e;
        } else {
            if ((e = cudaMemsetAsync(part, 0, sizeof(float2) * 3 * mc, st)) != cudaSuccess) return e;
        }
        k_born_accum<<<(unsigned)((n_b + 127) / 128), 128, 0, st>>>(f, n_b, n_particles > 0 ? S : 1, part, pts, rep,
                                                                   w, k0, Kc, d_out);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace rt3d
