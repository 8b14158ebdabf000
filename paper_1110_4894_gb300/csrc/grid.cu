// grid.cu -- the paper's grid force path (Sec. 3.3 and App. B).
//
// Build, once per mass distribution:
//   1. cloud-in-cell assignment of the particle masses to n^3 nodes, summed in
//      64-bit fixed point with integer atomics (order-independent, so the
//      node masses are bit-reproducible);
//   2. optional subtraction of the mean node mass ("the mean matter density
//      is then subtracted off");
//   3. phi and grad phi on the nodes: the zero-padded (2n)^3 FFT convolution
//      of the node masses with the Plummer kernels (Eqs. psi, derivs with
//      phi = a psi), by cuFFT (double precision, real-to-complex);
//   4. the natural-spline second derivatives of every node line along x3
//      (App. B: computed once).
// Per RK4 stage, App. B's interpolation at every ray: along x3 from the
// global line splines, then natural splines through the 2 n_int nodes around
// the ray along x1 and along x2.  One thread per (point, field); the four
// fields of a point are blockIdx.y = 0..3.
#include <cufft.h>

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

__global__ void k_cmul(int64_t m, const cufftDoubleComplex *__restrict__ a, cufftDoubleComplex *__restrict__ b,
                       double scale)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const cufftDoubleComplex x = a[i], y = b[i];
        b[i] = make_cuDoubleComplex((x.x * y.x - x.y * y.y) * scale, (x.x * y.y + x.y * y.x) * scale);
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

// ---------------------------------------------------------------------------
// App. B evaluation
// ---------------------------------------------------------------------------
__device__ __forceinline__ double splint_at(const double *y, const double *y2, int m, double u)
{
    int k = (int)floor(u);
    k = k > m - 2 ? m - 2 : k;
    k = k < 0 ? 0 : k;
    const double A = (double)(k + 1) - u, B = u - (double)k;
    return A * y[k] + B * y[k + 1] + ((A * A * A - A) * y2[k] + (B * B * B - B) * y2[k + 1]) / 6.0;
}

// natural spline through W unit-spaced values, evaluated at u in [0, W-1]
template <int W>
__device__ __forceinline__ double local_spline(const double (&t)[W], double u)
{
    double z[W];
    z[0] = 0.0;
    z[W - 1] = 0.0;
    if (W >= 3) {
        double den[W], dp = 0.0, cp = 0.0;
#pragma unroll
        for (int i = 1; i <= W - 2; ++i) {
            den[i] = 4.0 - cp;
            cp = 1.0 / den[i];
            dp = (6.0 * (t[i + 1] - 2.0 * t[i] + t[i - 1]) - dp) / den[i];
            z[i] = dp;
        }
#pragma unroll
        for (int i = W - 3; i >= 1; --i) z[i] = z[i] - z[i + 1] / den[i];
    }
    int k = (int)floor(u);
    k = k > W - 2 ? W - 2 : k;
    k = k < 0 ? 0 : k;
    const double A = (double)(k + 1) - u, B = u - (double)k;
    double yk = t[0], yk1 = t[1], zk = z[0], zk1 = z[1];
#pragma unroll
    for (int i = 1; i < W - 1; ++i)
        if (k == i) {
            yk = t[i];
            yk1 = t[i + 1];
            zk = z[i];
            zk1 = z[i + 1];
        }
    return A * yk + B * yk1 + ((A * A * A - A) * zk + (B * B * B - B) * zk1) / 6.0;
}

// group: points per bundle; a cube-tiled box takes the cube holding the x3
// of the group's first point (the bundle's central ray), as the direct sum
// takes its replica
template <int NI>
__global__ void k_grid_eval(GridDev g, const double *__restrict__ px, const double *__restrict__ py,
                            const double *__restrict__ pz, int64_t n_pts, int mode, void *__restrict__ out,
                            const unsigned long long *__restrict__ gate, int group)
{
    constexpr int W = 2 * NI;
    if (gate && *gate == 0ull) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int f = blockIdx.y;
    if (i >= n_pts) return;
    const int n = g.n;
    const double r[3] = {px[i], py[i], pz[i]};
    double lo[3] = {g.lo[0], g.lo[1], g.lo[2]};
    const double *val = g.val, *y2t = g.y2;
    if (g.cubes > 0) {
        const double x3 = pz[(i / group) * group];
        double q = floor(x3 / g.L);
        const int j = q < 0.0 ? 0 : (q > (double)(g.n_rep - 1) ? g.n_rep - 1 : (int)q);
        double cq = floor((x3 - (double)j * g.L) / g.W);
        const int c = cq < 0.0 ? 0 : (cq > (double)(g.cubes - 1) ? g.cubes - 1 : (int)cq);
        lo[0] = -0.5 * g.W;
        lo[1] = -0.5 * g.W;
        lo[2] = (double)j * g.L + (double)c * g.W;
        const int64_t cell = (int64_t)j * g.cubes + c, stride = 4 * (int64_t)n * n * n;
        val += cell * stride;
        y2t += cell * stride;
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
    double F = 0.0;
    if (inside) {
        const int64_t n3 = (int64_t)n * n * n;
        const double *v = val + f * n3, *y2 = y2t + f * n3;
        int k3 = (int)floor(u[2]);
        k3 = k3 > n - 2 ? n - 2 : k3;
        k3 = k3 < 0 ? 0 : k3;
        const double A = (double)(k3 + 1) - u[2], B = u[2] - (double)k3;
        const double cA = (A * A * A - A) / 6.0, cB = (B * B * B - B) / 6.0;
        double w2[W];
#pragma unroll
        for (int b = 0; b < W; ++b) {
            double t[W];
#pragma unroll
            for (int a = 0; a < W; ++a) {
                // step 1: along x3 on node line (s1 + a, s2 + b), global spline
                const int64_t line = ((int64_t)(s[0] + a) * n + (s[1] + b)) * n + k3;
                t[a] = A * v[line] + B * v[line + 1] + (cA * y2[line] + cB * y2[line + 1]);
            }
            // steps 2-3: along x1
            w2[b] = local_spline<W>(t, u[0] - (double)s[0]);
        }
        // steps 4-5: along x2
        F = local_spline<W>(w2, u[1] - (double)s[1]);
    }
    if (mode == 2) {
        ((double *)out)[4 * i + f] = F;
    } else if (mode == 1) {
        ((double *)out)[(int64_t)f * n_pts + i] = -F;
    } else {
        const float hi = (float)(-F);
        const float lo = (float)(-F - (double)hi);
        ((float2 *)out)[(int64_t)f * n_pts + i] = make_float2(hi, lo);
    }
}

cudaError_t launch_grid_eval(const GridDev &g, const double *px, const double *py, const double *pz, int64_t n,
                             int mode, void *out, const unsigned long long *gate, cudaStream_t st, int group)
{
    if (n <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((n + 127) / 128), 4);
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
    cudaFree(g.val);
    cudaFree(g.y2);
    g.val = g.y2 = nullptr;
}

static unsigned blocks_for(int64_t m)
{
    const int64_t b = (m + 255) / 256;
    return (unsigned)(b < 152 * 64 ? (b > 0 ? b : 1) : 152 * 64);
}

namespace {
struct Tmp {  // temporary device buffers of a build, freed on every exit
    double *pos = nullptr, *mass = nullptr, *buf = nullptr;
    unsigned long long *q = nullptr, *total = nullptr;
    cufftDoubleComplex *fm = nullptr, *fk = nullptr;
    cufftHandle r2c = 0, c2r = 0;
    bool have_r2c = false, have_c2r = false;
    ~Tmp()
    {
        cudaFree(pos);
        cudaFree(mass);
        cudaFree(buf);
        cudaFree(q);
        cudaFree(total);
        cudaFree(fm);
        cudaFree(fk);
        if (have_r2c) cufftDestroy(r2c);
        if (have_c2r) cufftDestroy(c2r);
    }
};
}  // namespace

int grid_build(GridDev &g, int64_t np, const double *pos, const double *mass, double soft, int mean_subtract,
               cudaStream_t st, std::string &err)
{
    const int n = g.n, P = 2 * n;
    const int64_t n3 = (int64_t)n * n * n, P3 = (int64_t)P * P * P, Pc = (int64_t)P * P * (P / 2 + 1);
    Tmp t;
    auto cuda_fail = [&](cudaError_t e, const char *what) {
        err = std::string(what) + ": " + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? RT3D_ENOMEM : RT3D_ECUDA;
    };
#define GCK(x, what)                                       \
    do {                                                   \
        cudaError_t e_ = (x);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)
#define FCK(x, what)                                                      \
    do {                                                                  \
        cufftResult r_ = (x);                                             \
        if (r_ != CUFFT_SUCCESS) {                                        \
            err = std::string(what) + ": cuFFT error " + std::to_string((int)r_); \
            return r_ == CUFFT_ALLOC_FAILED ? RT3D_ENOMEM : RT3D_ECUDA;   \
        }                                                                 \
    } while (0)
    // fixed-point scale: the node sums stay below 2^62 for any assignment
    double msum = 0.0;
    for (int64_t i = 0; i < np; ++i) msum += mass[i];
    const int e = msum > 0.0 ? 61 - (int)ceil(log2(msum)) : 0;
    const double qscale = ldexp(1.0, e), qinv = ldexp(1.0, -e);
    GCK(cudaMalloc(&t.q, sizeof(unsigned long long) * (size_t)n3), "grid node buffer");
    GCK(cudaMalloc(&t.total, sizeof(unsigned long long)), "grid total");
    GCK(cudaMemsetAsync(t.q, 0, sizeof(unsigned long long) * (size_t)n3, st), "memset");
    GCK(cudaMemsetAsync(t.total, 0, sizeof(unsigned long long), st), "memset");
    if (np > 0) {
        GCK(cudaMalloc(&t.pos, sizeof(double) * 3 * (size_t)np), "particle upload");
        GCK(cudaMalloc(&t.mass, sizeof(double) * (size_t)np), "particle upload");
        GCK(cudaMemcpyAsync(t.pos, pos, sizeof(double) * 3 * (size_t)np, cudaMemcpyHostToDevice, st), "upload");
        GCK(cudaMemcpyAsync(t.mass, mass, sizeof(double) * (size_t)np, cudaMemcpyHostToDevice, st), "upload");
        k_cic<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(np, t.pos, t.mass, g.lo[0], g.lo[1], g.lo[2], 1.0 / g.h, n,
                                                             qscale, t.q);
        GCK(cudaGetLastError(), "k_cic");
    }
    k_sum_q<<<blocks_for(n3), 256, 0, st>>>(n3, t.q, t.total);
    GCK(cudaGetLastError(), "k_sum_q");
    GCK(cudaMalloc(&t.buf, sizeof(double) * (size_t)P3), "grid FFT buffer");
    GCK(cudaMalloc(&t.fm, sizeof(cufftDoubleComplex) * (size_t)Pc), "grid FFT buffer");
    GCK(cudaMalloc(&t.fk, sizeof(cufftDoubleComplex) * (size_t)Pc), "grid FFT buffer");
    GCK(cudaMalloc(&g.val, sizeof(double) * 4 * (size_t)n3), "grid values");
    GCK(cudaMalloc(&g.y2, sizeof(double) * 4 * (size_t)n3), "grid spline table");
    FCK(cufftPlan3d(&t.r2c, P, P, P, CUFFT_D2Z), "cufftPlan3d D2Z");
    t.have_r2c = true;
    FCK(cufftPlan3d(&t.c2r, P, P, P, CUFFT_Z2D), "cufftPlan3d Z2D");
    t.have_c2r = true;
    FCK(cufftSetStream(t.r2c, st), "cufftSetStream");
    FCK(cufftSetStream(t.c2r, st), "cufftSetStream");
    k_fill_mass<<<blocks_for(P3), 256, 0, st>>>(n, t.q, t.total, qinv, mean_subtract, t.buf);
    GCK(cudaGetLastError(), "k_fill_mass");
    FCK(cufftExecD2Z(t.r2c, t.buf, t.fm), "cufftExecD2Z");
    for (int f = 0; f < 4; ++f) {
        k_fill_kernel<<<blocks_for(P3), 256, 0, st>>>(n, f, g.h, soft * soft, t.buf);
        GCK(cudaGetLastError(), "k_fill_kernel");
        FCK(cufftExecD2Z(t.r2c, t.buf, t.fk), "cufftExecD2Z");
        k_cmul<<<blocks_for(Pc), 256, 0, st>>>(Pc, t.fm, t.fk, 1.0 / (double)P3);
        GCK(cudaGetLastError(), "k_cmul");
        FCK(cufftExecZ2D(t.c2r, t.fk, t.buf), "cufftExecZ2D");
        k_extract<<<blocks_for(n3), 256, 0, st>>>(n, t.buf, g.val + f * n3);
        GCK(cudaGetLastError(), "k_extract");
    }
    const int64_t lines = 4 * (int64_t)n * n;
    k_spline_lines<<<(unsigned)((lines + 127) / 128), 128, 0, st>>>(n, lines, g.val, g.y2);
    GCK(cudaGetLastError(), "k_spline_lines");
    GCK(cudaStreamSynchronize(st), "grid build");
#undef GCK
#undef FCK
    return RT3D_OK;
}

}  // namespace rt3d
