// grid.cu -- the paper's grid force path (Sec. 3.3 and App. B).
//
// Build, once per mass distribution:
//   1. cloud-in-cell assignment of the particle masses to n^3 nodes, summed in
//      64-bit fixed point with integer atomics (order-independent, so the
//      node masses are bit-reproducible);
//   2. optional subtraction of the mean node mass (Sec. 3.3 removes the mean
//      density);
//   3. phi and grad phi on the nodes: the zero-padded (2n)^3 FFT convolution
//      of the node masses with the Plummer kernels (Eqs. psi, derivs with
//      phi = a psi), by cuFFT (double precision, real-to-complex);
//   4. the natural-spline second derivatives of every node line along x3
//      (App. B: computed once).
// Per RK4 stage, App. B's interpolation at every ray: along x3 from the
// global line splines, then natural splines through the 2 n_int nodes around
// the ray along x1 and along x2.  A natural spline through unit-spaced values
// is linear in them, so the x1 and x2 splines are applied as weight vectors
// (computed once per point) to the four fields at once.  One thread per point;
// the node table keeps, per node, the four field values and their x3-spline
// second derivatives side by side (64 bytes), so the two nodes a point reads on
// each x3 line are one contiguous 128-byte span.
#include <cufft.h>

#include <algorithm>
#include <new>
#include <thread>
#include <vector>

#include "grid_device.cuh"
#include "rt3d_internal.cuh"

namespace rt3d {

constexpr int kMaxGridN = 1024;

// ---------------------------------------------------------------------------
// build kernels
// ---------------------------------------------------------------------------
__global__ void k_cic(int64_t np, const double *__restrict__ pos, const double *__restrict__ mass, double lo0,
                      double lo1, double lo2, double inv_h, int n, double qscale,
                      unsigned long long *__restrict__ node_q)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const double u[3] = {(pos[3 * p] - lo0) * inv_h, (pos[3 * p + 1] - lo1) * inv_h, (pos[3 * p + 2] - lo2) * inv_h};
    int64_t i0[3];
    double f[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double fl = floor(u[d]);
        i0[d] = (int64_t)fl;
        f[d] = u[d] - fl;
    }
    const double m = mass[p] * qscale;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int64_t a = i0[0] + (c & 1), b = i0[1] + ((c >> 1) & 1), z = i0[2] + ((c >> 2) & 1);
        if (a < 0 || a >= n || b < 0 || b >= n || z < 0 || z >= n) continue;
        const double w = ((c & 1) ? f[0] : 1.0 - f[0]) * (((c >> 1) & 1) ? f[1] : 1.0 - f[1]) *
                         (((c >> 2) & 1) ? f[2] : 1.0 - f[2]);
        const unsigned long long q = (unsigned long long)__double2ll_rn(m * w);
        atomicAdd(&node_q[(a * n + b) * n + z], q);
    }
}

__global__ void k_sum_q(int64_t m, const unsigned long long *__restrict__ q, unsigned long long *__restrict__ total)
{
    __shared__ unsigned long long s[256];
    unsigned long long acc = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        acc += q[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(total, s[0]);
}

// padded (P = 2n)^3 real array: node masses (minus the mean) in the first n^3 corner
__global__ void k_fill_mass(int n, const unsigned long long *__restrict__ q, const unsigned long long *__restrict__ total,
                            double qinv, int mean_subtract, double *__restrict__ buf)
{
    const int P = 2 * n;
    const int64_t m = (int64_t)P * P * P;
    const double mean = mean_subtract ? (double)*total * qinv / ((double)n * n * n) : 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int k3 = (int)(i % P), k2 = (int)((i / P) % P), k1 = (int)(i / ((int64_t)P * P));
        double v = 0.0;
        if (k1 < n && k2 < n && k3 < n) v = (double)q[((int64_t)k1 * n + k2) * n + k3] * qinv - mean;
        buf[i] = v;
    }
}

// kernel f on the padded grid, indexed by node displacement
// (k < n: +k, k > n: k - 2n, k = n: unused, zero)
__global__ void k_fill_kernel(int n, int f, double h, double eps2, double *__restrict__ buf)
{
    const int P = 2 * n;
    const int64_t m = (int64_t)P * P * P;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int k[3] = {(int)(i / ((int64_t)P * P)), (int)((i / P) % P), (int)(i % P)};
        double d[3];
        bool ok = true;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ok = ok && k[c] != n;
            d[c] = (double)(k[c] < n ? k[c] : k[c] - P) * h;
        }
        const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + eps2;
        double v = 0.0;
        if (ok && r2 > 0.0) {
            const double inv = 1.0 / sqrt(r2);
            v = f == 0 ? -kMuG * inv : kMuG * d[f - 1] * inv * inv * inv;
        }
        buf[i] = v;
    }
}

// out = a b scale (out may be b)
__global__ void k_cmul(int64_t m, const cufftDoubleComplex *__restrict__ a, const cufftDoubleComplex *b,
                       cufftDoubleComplex *out, double scale)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const cufftDoubleComplex x = a[i], y = b[i];
        out[i] = make_cuDoubleComplex((x.x * y.x - x.y * y.y) * scale, (x.x * y.y + x.y * y.x) * scale);
    }
}

__global__ void k_extract(int n, const double *__restrict__ buf, double *__restrict__ out)
{
    const int P = 2 * n;
    const int64_t m = (int64_t)n * n * n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k3 = i % n, k2 = (i / n) % n, k1 = i / ((int64_t)n * n);
        out[i] = buf[(k1 * P + k2) * P + k3];
    }
}

// natural cubic spline along each x3 line (unit spacing):
// y2[i-1] + 4 y2[i] + y2[i+1] = 6 (y[i+1] - 2 y[i] + y[i-1]), y2 = 0 at the ends.
// The elimination factors depend on n only and are shared by all lines.
__global__ void k_spline_lines(int n, int64_t lines, const double *__restrict__ val, double *__restrict__ y2)
{
    __shared__ double s_den[kMaxGridN];
    if (threadIdx.x == 0) {
        double cp = 0.0;
        for (int i = 1; i <= n - 2; ++i) {
            s_den[i] = 4.0 - cp;
            cp = 1.0 / s_den[i];
        }
    }
    __syncthreads();
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= lines) return;
    const double *y = val + l * n;
    double *z = y2 + l * n;
    z[0] = 0.0;
    z[n - 1] = 0.0;
    if (n < 3) return;
    double dp = 0.0;
    for (int i = 1; i <= n - 2; ++i) {
        dp = (6.0 * (y[i + 1] - 2.0 * y[i] + y[i - 1]) - dp) / s_den[i];
        z[i] = dp;
    }
    for (int i = n - 3; i >= 1; --i) z[i] = z[i] - z[i + 1] / s_den[i];
}

// node table: per node the four values, then the four x3-spline second
// derivatives (kGridRec doubles); tab32 holds the same numbers rounded to FP32
// (either may be null)
__global__ void k_interleave(int64_t n3, const double *__restrict__ val, const double *__restrict__ y2,
                             double *__restrict__ tab, float *__restrict__ tab32)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
        const double r[kGridRec] = {val[i], val[n3 + i], val[2 * n3 + i], val[3 * n3 + i],
                                    y2[i],  y2[n3 + i],  y2[2 * n3 + i],  y2[3 * n3 + i]};
        if (tab) {
            double2 *t = reinterpret_cast<double2 *>(tab + kGridRec * i);
            t[0] = make_double2(r[0], r[1]);
            t[1] = make_double2(r[2], r[3]);
            t[2] = make_double2(r[4], r[5]);
            t[3] = make_double2(r[6], r[7]);
        }
        if (tab32) {
            float4 *t32 = reinterpret_cast<float4 *>(tab32 + kGridRec * i);
            t32[0] = make_float4((float)r[0], (float)r[1], (float)r[2], (float)r[3]);
            t32[1] = make_float4((float)r[4], (float)r[5], (float)r[6], (float)r[7]);
        }
    }
}

// ---------------------------------------------------------------------------
// App. B evaluation
// ---------------------------------------------------------------------------
// Weights c of the natural cubic spline through W unit-spaced values y,
// evaluated at u in [0, W-1]: S(u) = sum_j c[j] y[j].  The second derivatives
// z of the spline through the unit vector e_j solve the same tridiagonal
// system as any data (z[i-1] + 4 z[i] + z[i+1] = 6 (e[i+1] - 2 e[i] + e[i-1]),
// z = 0 at the ends); they are constants of W.
template <int W>
__device__ __forceinline__ void spline_weights(double u, double (&c)[W])
{
    int k = (int)floor(u);
    k = k > W - 2 ? W - 2 : k;
    k = k < 0 ? 0 : k;
    const double A = (double)(k + 1) - u, B = u - (double)k;
    const double cA = (A * A * A - A) / 6.0, cB = (B * B * B - B) / 6.0;
#pragma unroll
    for (int j = 0; j < W; ++j) {
        double z[W];
        z[0] = 0.0;
        z[W - 1] = 0.0;
        if (W >= 3) {
            double den[W], dp = 0.0, cp = 0.0;
#pragma unroll
            for (int i = 1; i <= W - 2; ++i) {
                const double e = (i + 1 == j ? 1.0 : 0.0) - 2.0 * (i == j ? 1.0 : 0.0) + (i - 1 == j ? 1.0 : 0.0);
                den[i] = 4.0 - cp;
                cp = 1.0 / den[i];
                dp = (6.0 * e - dp) / den[i];
                z[i] = dp;
            }
#pragma unroll
            for (int i = W - 3; i >= 1; --i) z[i] = z[i] - z[i + 1] / den[i];
        }
        double zk = z[0], zk1 = z[1];
#pragma unroll
        for (int i = 1; i < W - 1; ++i)
            if (k == i) {
                zk = z[i];
                zk1 = z[i + 1];
            }
        c[j] = (j == k ? A : 0.0) + (j == k + 1 ? B : 0.0) + (cA * zk + cB * zk1);
    }
}

// group: points per bundle; a cube-tiled box takes the cube holding the x3
// of the group's first point (the bundle's central ray), as the direct sum
// takes its replica
template <int NI>
__global__ void __launch_bounds__(128) k_grid_eval(GridDev g, const double *__restrict__ px,
                                                   const double *__restrict__ py, const double *__restrict__ pz,
                                                   int64_t n_pts, int mode, void *__restrict__ out,
                                                   const unsigned long long *__restrict__ gate, int group)
{
    constexpr int W = 2 * NI;
    if (gate && *gate == 0ull) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pts) return;
    const int n = g.n;
    const double r[3] = {px[i], py[i], pz[i]};
    double lo[3] = {g.lo[0], g.lo[1], g.lo[2]};
    const double *tab = g.tab;
    if (g.cubes > 0) {
        const double x3 = pz[(i / group) * group];
        double q = floor(x3 / g.L);
        const int j = q < 0.0 ? 0 : (q > (double)(g.n_rep - 1) ? g.n_rep - 1 : (int)q);
        double cq = floor((x3 - (double)j * g.L) / g.W);
        const int c = cq < 0.0 ? 0 : (cq > (double)(g.cubes - 1) ? g.cubes - 1 : (int)cq);
        lo[0] = -0.5 * g.W;
        lo[1] = -0.5 * g.W;
        lo[2] = (double)j * g.L + (double)c * g.W;
        tab += ((int64_t)j * g.cubes + c) * kGridRec * (int64_t)n * n * n;
    }
    double u[3];
    int s[3];
    bool inside = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        u[d] = (r[d] - lo[d]) / g.h;
        inside = inside && (u[d] >= -g.margin && u[d] <= (double)(n - 1) + g.margin);
        int sd = inside ? (int)floor(u[d]) - NI + 1 : 0;
        sd = sd > n - W ? n - W : sd;
        s[d] = sd < 0 ? 0 : sd;
    }
    double F[4] = {0.0, 0.0, 0.0, 0.0};
    if (inside) {
        int k3 = (int)floor(u[2]);
        k3 = k3 > n - 2 ? n - 2 : k3;
        k3 = k3 < 0 ? 0 : k3;
        const double A = (double)(k3 + 1) - u[2], B = u[2] - (double)k3;
        const double cA = (A * A * A - A) / 6.0, cB = (B * B * B - B) / 6.0;
        double c1[W], c2[W];
        spline_weights<W>(u[0] - (double)s[0], c1);
        spline_weights<W>(u[1] - (double)s[1], c2);
#pragma unroll
        for (int b = 0; b < W; ++b) {
            double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
            for (int a = 0; a < W; ++a) {
                // along x3 on node line (s1 + a, s2 + b): the global spline
                // from nodes k3 and k3 + 1 (values, then second derivatives)
                const int64_t node = ((int64_t)(s[0] + a) * n + (s[1] + b)) * n + k3;
                const double2 *p = reinterpret_cast<const double2 *>(tab + kGridRec * node);
                const double2 v01 = __ldg(p), v23 = __ldg(p + 1), y01 = __ldg(p + 2), y23 = __ldg(p + 3);
                const double2 w01 = __ldg(p + 4), w23 = __ldg(p + 5), z01 = __ldg(p + 6), z23 = __ldg(p + 7);
                const double t0 = A * v01.x + B * w01.x + (cA * y01.x + cB * z01.x);
                const double t1 = A * v01.y + B * w01.y + (cA * y01.y + cB * z01.y);
                const double t2 = A * v23.x + B * w23.x + (cA * y23.x + cB * z23.x);
                const double t3 = A * v23.y + B * w23.y + (cA * y23.y + cB * z23.y);
                // along x1
                acc[0] += c1[a] * t0;
                acc[1] += c1[a] * t1;
                acc[2] += c1[a] * t2;
                acc[3] += c1[a] * t3;
            }
            // along x2
#pragma unroll
            for (int f = 0; f < 4; ++f) F[f] += c2[b] * acc[f];
        }
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        if (mode == 2) {
            ((double *)out)[4 * i + f] = F[f];
        } else if (mode == 1) {
            ((double *)out)[(int64_t)f * n_pts + i] = -F[f];
        } else {
            const float hi = (float)(-F[f]);
            const float lo2 = (float)(-F[f] - (double)hi);
            ((float2 *)out)[(int64_t)f * n_pts + i] = make_float2(hi, lo2);
        }
    }
}

// The mixed path's evaluation (grid_device.cuh): output modes 0 (hi = -F,
// lo = 0) and 2.
template <int NI>
__global__ void __launch_bounds__(128) k_grid_eval32(GridDev g, const double *__restrict__ px,
                                                     const double *__restrict__ py, const double *__restrict__ pz,
                                                     int64_t n_pts, int mode, void *__restrict__ out,
                                                     const unsigned long long *__restrict__ gate, int group)
{
    if (gate && *gate == 0ull) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pts) return;
    float F[4];
    grid_eval32_point<NI>(g, px, py, pz, i, group, F);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        if (mode == 2)
            ((double *)out)[4 * i + f] = (double)F[f];
        else
            ((float2 *)out)[(int64_t)f * n_pts + i] = make_float2(-F[f], 0.0f);
    }
}

cudaError_t launch_grid_eval(const GridDev &g, const double *px, const double *py, const double *pz, int64_t n,
                             int mode, void *out, const unsigned long long *gate, cudaStream_t st, int group)
{
    if (n <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((n + 127) / 128);
    // the FP32 table serves the mixed path (mode 0) and, where it is the only
    // table, point evaluation (mode 2)
    if (g.tab32 && (mode == 0 || !g.tab)) {
        if (mode == 1) return cudaErrorInvalidValue;
        switch (g.n_int) {
        case 1: k_grid_eval32<1><<<grid, 128, 0, st>>>(g, px, py, pz, n, mode, out, gate, group); break;
        case 2: k_grid_eval32<2><<<grid, 128, 0, st>>>(g, px, py, pz, n, mode, out, gate, group); break;
        case 3: k_grid_eval32<3><<<grid, 128, 0, st>>>(g, px, py, pz, n, mode, out, gate, group); break;
        case 4: k_grid_eval32<4><<<grid, 128, 0, st>>>(g, px, py, pz, n, mode, out, gate, group); break;
        default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    if (!g.tab) return cudaErrorInvalidValue;
    switch (g.n_int) {
    case 1: k_grid_eval<1><<<grid, 128, 0, st>>>(g, px, py, pz, n, mode, out, gate, group); break;
    case 2: k_grid_eval<2><<<grid, 128, 0, st>>>(g, px, py, pz, n, mode, out, gate, group); break;
    case 3: k_grid_eval<3><<<grid, 128, 0, st>>>(g, px, py, pz, n, mode, out, gate, group); break;
    case 4: k_grid_eval<4><<<grid, 128, 0, st>>>(g, px, py, pz, n, mode, out, gate, group); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// build orchestration
// ---------------------------------------------------------------------------
void grid_free(GridDev &g)
{
    cudaFree(g.tab);
    cudaFree(g.tab32);
    g.tab = nullptr;
    g.tab32 = nullptr;
}

static unsigned blocks_for(int64_t m)
{
    const int64_t b = (m + 255) / 256, cap = (int64_t)device_sm_count() * 64;
    return (unsigned)(b < cap ? (b > 0 ? b : 1) : cap);
}

namespace {
// Device state for building grids of one shape (n nodes per side, spacing h,
// softening eps): FFT buffers and plans, node-mass and value temporaries, and
// (when cache_kernels) the four kernel spectra, which depend on the shape
// only and so serve every cube of a replicated box.  Freed on every exit.
struct Builder {
    int n = 0;
    double h = 0.0, eps2 = 0.0;
    bool cache = false, have_k = false;
    double *pos = nullptr, *mass = nullptr, *buf = nullptr, *val = nullptr, *y2 = nullptr;
    int64_t cap = 0;
    unsigned long long *q = nullptr, *total = nullptr;
    cufftDoubleComplex *fm = nullptr, *fk = nullptr, *kspec = nullptr;
    cufftHandle r2c = 0, c2r = 0;
    bool have_r2c = false, have_c2r = false;
    std::string *err = nullptr;
    ~Builder()
    {
        cudaFree(pos);
        cudaFree(mass);
        cudaFree(buf);
        cudaFree(val);
        cudaFree(y2);
        cudaFree(q);
        cudaFree(total);
        cudaFree(fm);
        cudaFree(fk);
        cudaFree(kspec);
        if (have_r2c) cufftDestroy(r2c);
        if (have_c2r) cufftDestroy(c2r);
    }
    int cuda_fail(cudaError_t e, const char *what)
    {
        *err = std::string(what) + ": " + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? RT3D_ENOMEM : RT3D_ECUDA;
    }
    int fft_fail(cufftResult r, const char *what)
    {
        *err = std::string(what) + ": cuFFT error " + std::to_string((int)r);
        return r == CUFFT_ALLOC_FAILED ? RT3D_ENOMEM : RT3D_ECUDA;
    }
    int64_t P3() const { return 8 * (int64_t)n * n * n; }
    int64_t Pc() const { return 4 * (int64_t)n * n * (n + 1); }
    int64_t n3() const { return (int64_t)n * n * n; }
};
}  // namespace

#define GCK(x, what)                                        \
    do {                                                    \
        cudaError_t e_ = (x);                               \
        if (e_ != cudaSuccess) return B.cuda_fail(e_, what); \
    } while (0)
#define FCK(x, what)                                        \
    do {                                                    \
        cufftResult r_ = (x);                               \
        if (r_ != CUFFT_SUCCESS) return B.fft_fail(r_, what); \
    } while (0)

static int builder_init(Builder &B, int n, double h, double soft, bool cache_kernels, cudaStream_t st,
                        std::string &err)
{
    B.n = n;
    B.h = h;
    B.eps2 = soft * soft;
    B.err = &err;
    const int P = 2 * n;
    // the four kernel spectra stay resident only where they are small
    B.cache = cache_kernels && 4 * B.Pc() * (int64_t)sizeof(cufftDoubleComplex) <= ((int64_t)8 << 30);
    GCK(cudaMalloc(&B.q, sizeof(unsigned long long) * (size_t)B.n3()), "grid node buffer");
    GCK(cudaMalloc(&B.total, sizeof(unsigned long long)), "grid total");
    GCK(cudaMalloc(&B.buf, sizeof(double) * (size_t)B.P3()), "grid FFT buffer");
    GCK(cudaMalloc(&B.fm, sizeof(cufftDoubleComplex) * (size_t)B.Pc()), "grid FFT buffer");
    GCK(cudaMalloc(&B.fk, sizeof(cufftDoubleComplex) * (size_t)B.Pc()), "grid FFT buffer");
    GCK(cudaMalloc(&B.val, sizeof(double) * 4 * (size_t)B.n3()), "grid values");
    GCK(cudaMalloc(&B.y2, sizeof(double) * 4 * (size_t)B.n3()), "grid spline table");
    if (B.cache) GCK(cudaMalloc(&B.kspec, sizeof(cufftDoubleComplex) * 4 * (size_t)B.Pc()), "grid kernel spectra");
    FCK(cufftPlan3d(&B.r2c, P, P, P, CUFFT_D2Z), "cufftPlan3d D2Z");
    B.have_r2c = true;
    FCK(cufftPlan3d(&B.c2r, P, P, P, CUFFT_Z2D), "cufftPlan3d Z2D");
    B.have_c2r = true;
    FCK(cufftSetStream(B.r2c, st), "cufftSetStream");
    FCK(cufftSetStream(B.c2r, st), "cufftSetStream");
    return RT3D_OK;
}

// one grid: the particles' CIC node masses on the nodes lo + h i, optionally
// minus their mean, convolved with the four Plummer kernels; the node table
// (kGridRec n^3 doubles) goes to dest, its FP32 copy to dest32
static int builder_run(Builder &B, int64_t np, const double *pos, const double *mass, const double lo[3],
                       int mean_subtract, double *dest, float *dest32, cudaStream_t st)
{
    const int n = B.n;
    const int64_t n3 = B.n3(), P3 = B.P3(), Pc = B.Pc();
    // fixed-point scale: the node sums stay below 2^62 for any assignment
    double msum = 0.0;
    for (int64_t i = 0; i < np; ++i) msum += mass[i];
    const int e = msum > 0.0 ? 61 - (int)ceil(log2(msum)) : 0;
    const double qscale = ldexp(1.0, e), qinv = ldexp(1.0, -e);
    GCK(cudaMemsetAsync(B.q, 0, sizeof(unsigned long long) * (size_t)n3, st), "memset");
    GCK(cudaMemsetAsync(B.total, 0, sizeof(unsigned long long), st), "memset");
    if (np > 0) {
        if (np > B.cap) {
            GCK(cudaStreamSynchronize(st), "grid build");
            cudaFree(B.pos);
            cudaFree(B.mass);
            B.pos = B.mass = nullptr;
            B.cap = 0;
            GCK(cudaMalloc(&B.pos, sizeof(double) * 3 * (size_t)np), "particle upload");
            GCK(cudaMalloc(&B.mass, sizeof(double) * (size_t)np), "particle upload");
            B.cap = np;
        }
        GCK(cudaMemcpyAsync(B.pos, pos, sizeof(double) * 3 * (size_t)np, cudaMemcpyHostToDevice, st), "upload");
        GCK(cudaMemcpyAsync(B.mass, mass, sizeof(double) * (size_t)np, cudaMemcpyHostToDevice, st), "upload");
        k_cic<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(np, B.pos, B.mass, lo[0], lo[1], lo[2], 1.0 / B.h, n,
                                                             qscale, B.q);
        GCK(cudaGetLastError(), "k_cic");
    }
    k_sum_q<<<blocks_for(n3), 256, 0, st>>>(n3, B.q, B.total);
    GCK(cudaGetLastError(), "k_sum_q");
    k_fill_mass<<<blocks_for(P3), 256, 0, st>>>(n, B.q, B.total, qinv, mean_subtract, B.buf);
    GCK(cudaGetLastError(), "k_fill_mass");
    FCK(cufftExecD2Z(B.r2c, B.buf, B.fm), "cufftExecD2Z");
    for (int f = 0; f < 4; ++f) {
        cufftDoubleComplex *ks = B.cache ? B.kspec + f * Pc : B.fk;
        if (!B.cache || !B.have_k) {
            k_fill_kernel<<<blocks_for(P3), 256, 0, st>>>(n, f, B.h, B.eps2, B.buf);
            GCK(cudaGetLastError(), "k_fill_kernel");
            FCK(cufftExecD2Z(B.r2c, B.buf, ks), "cufftExecD2Z");
        }
        k_cmul<<<blocks_for(Pc), 256, 0, st>>>(Pc, B.fm, ks, B.fk, 1.0 / (double)P3);
        GCK(cudaGetLastError(), "k_cmul");
        FCK(cufftExecZ2D(B.c2r, B.fk, B.buf), "cufftExecZ2D");
        k_extract<<<blocks_for(n3), 256, 0, st>>>(n, B.buf, B.val + f * n3);
        GCK(cudaGetLastError(), "k_extract");
    }
    B.have_k = B.cache;
    const int64_t lines = 4 * (int64_t)n * n;
    k_spline_lines<<<(unsigned)((lines + 127) / 128), 128, 0, st>>>(n, lines, B.val, B.y2);
    GCK(cudaGetLastError(), "k_spline_lines");
    k_interleave<<<blocks_for(n3), 256, 0, st>>>(n3, B.val, B.y2, dest, dest32);
    GCK(cudaGetLastError(), "k_interleave");
    return RT3D_OK;
}

int grid_build(GridDev &g, int64_t np, const double *pos, const double *mass, double soft, int mean_subtract,
               bool fp64, cudaStream_t st, std::string &err)
{
    Builder B;
    int rc = builder_init(B, g.n, g.h, soft, false, st, err);
    if (rc != RT3D_OK) return rc;
    if (fp64)
        GCK(cudaMalloc(&g.tab, sizeof(double) * kGridRec * (size_t)B.n3()), "grid node table");
    else
        GCK(cudaMalloc(&g.tab32, sizeof(float) * kGridRec * (size_t)B.n3()), "grid node table");
    rc = builder_run(B, np, pos, mass, g.lo, mean_subtract, g.tab, g.tab32, st);
    if (rc != RT3D_OK) return rc;
    GCK(cudaStreamSynchronize(st), "grid build");
    return RT3D_OK;
}

int grid_build_box(GridDev &g, int64_t np, const double *pos, const double *mass, double soft,
                   const int32_t *rot, const double *shift, int mean_subtract, bool fp64, cudaStream_t st,
                   std::string &err)
{
    const int R = g.n_rep, C = g.cubes;
    const double L = g.L, W = g.W, c = 0.5 * L;
    // every replica's prism particles, cube by cube (host threads over replicas)
    std::vector<std::vector<double>> cp((size_t)R * C), cm((size_t)R * C);
    auto select = [&](int j) {
        const int32_t *Rm = rot + 9 * j;
        const double *sh = shift + 3 * j;
        for (int64_t i = 0; i < np; ++i) {
            const double *p = pos + 3 * i;
            double w[3];
            for (int r = 0; r < 3; ++r) {
                double v = 0.0;
                for (int k = 0; k < 3; ++k) v += (double)Rm[3 * r + k] * (p[k] - c);
                v = v + c + sh[r];
                while (v >= L) v -= L;
                while (v < 0.0) v += L;
                w[r] = v;
            }
            w[0] -= c;
            w[1] -= c;
            w[2] += (double)j * L;
            if (!(w[0] >= -0.5 * W && w[0] < 0.5 * W && w[1] >= -0.5 * W && w[1] < 0.5 * W)) continue;
            for (int q = 0; q < C; ++q) {
                const double z0 = (double)j * L + (double)q * W;
                if (w[2] >= z0 && w[2] < z0 + W) {
                    std::vector<double> &P = cp[(size_t)j * C + q];
                    P.insert(P.end(), w, w + 3);
                    cm[(size_t)j * C + q].push_back(mass[i]);
                    break;
                }
            }
        }
    };
    {
        const int nt = std::max(1, std::min(R, (int)std::thread::hardware_concurrency()));
        std::vector<std::thread> th;
        std::vector<char> oom((size_t)nt, 0);
        for (int t = 0; t < nt; ++t)
            th.emplace_back([&, t] {
                try {
                    for (int j = t; j < R; j += nt) select(j);
                } catch (const std::bad_alloc &) {
                    oom[(size_t)t] = 1;
                }
            });
        for (auto &x : th) x.join();
        for (char o : oom)
            if (o) {
                err = "host memory for the prism particles";
                return RT3D_ENOMEM;
            }
    }
    Builder B;
    int rc = builder_init(B, g.n, g.h, soft, true, st, err);
    if (rc != RT3D_OK) return rc;
    const size_t stride = kGridRec * (size_t)B.n3();
    if (fp64)
        GCK(cudaMalloc(&g.tab, sizeof(double) * stride * (size_t)R * C), "grid node tables");
    else
        GCK(cudaMalloc(&g.tab32, sizeof(float) * stride * (size_t)R * C), "grid node tables");
    for (int j = 0; j < R; ++j)
        for (int q = 0; q < C; ++q) {
            const size_t cell = (size_t)j * C + q;
            const double lo[3] = {-0.5 * W, -0.5 * W, (double)j * L + (double)q * W};
            rc = builder_run(B, (int64_t)cm[cell].size(), cp[cell].data(), cm[cell].data(), lo, mean_subtract,
                             g.tab ? g.tab + cell * stride : nullptr, g.tab32 ? g.tab32 + cell * stride : nullptr,
                             st);
            if (rc != RT3D_OK) return rc;
            // the host lists of this cube must outlive its asynchronous upload
            GCK(cudaStreamSynchronize(st), "grid build");
        }
    return RT3D_OK;
}
#undef GCK
#undef FCK

}  // namespace rt3d
