// kernels.cu -- FP64 kernels of the trace: step schedule (cosmology
// precompute), bundle initialiser, RK4 integrator stage, bundle reducer,
// muPDF histogram and particle staging.
#include "trace_device.cuh"

namespace rt3d {

// ---------------------------------------------------------------------------
// background cosmology on the device (Sec. 3.5, Eq. raytracedistance)
// ---------------------------------------------------------------------------
// One block computes chi_s; every thread then fills dlam[k] = int a^2 dchi over
// [x_k, x_{k+1}] (the affine step of the unperturbed ray with dx3/dl = 1 at the
// observer), by composite Boole's rule with 4 panels.
// a(t) and h da/dt at t = j h (the closed forms of Eq. scalefac2)
__global__ void k_atab(Cosmo c, int n, double h, double *__restrict__ tab)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double a = cosmo_a_exact(c, (double)j * h);
    tab[2 * j] = a;
    tab[2 * j + 1] = h * cosmo_adot(c, a);
}

cudaError_t launch_atab(const Cosmo &c, int n, double h, double *d_tab, cudaStream_t st)
{
    k_atab<<<(n + 255) / 256, 256, 0, st>>>(c, n, h, d_tab);
    return cudaGetLastError();
}

__global__ void k_schedule(Cosmo c, double z_s, int kind, int n, double chi_l, double s, double *dlam,
                           double *misc)
{
    __shared__ double s_chi;
    if (threadIdx.x == 0) {
        s_chi = comoving_distance(c, z_s);
        if (blockIdx.x == 0) misc[0] = s_chi;
    }
    __syncthreads();
    const double chi_s = s_chi;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        dlam[k] = schedule_step(c, kind, n, k, chi_s, chi_l, s);
}

cudaError_t launch_schedule(const Cosmo &c, double z_s, int kind, int n, double chi_l, double s, double *d_dlam,
                            double *d_misc, cudaStream_t st)
{
    int blocks = (n + 127) / 128;
    if (blocks > 1024) blocks = 1024;
    k_schedule<<<blocks, 128, 0, st>>>(c, z_s, kind, n, chi_l, s, d_dlam, d_misc);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// bundle initialiser (Sec. 3.1, ray bundle; initial state of Sec. 3.4)
// ---------------------------------------------------------------------------
__global__ void k_init(TraceParams tp, DevField f, const double *__restrict__ theta, RayState rs,
                       unsigned long long *cnt)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        cnt[0] = cnt[1] = cnt[2] = 0ull;
    }
    if (i >= rs.n_rays) return;
    init_ray(tp, f, theta, rs, i);
}

cudaError_t launch_init(const TraceParams &tp, const DevField &f, const double *d_theta, RayState rs,
                        unsigned long long *d_counters, cudaStream_t st)
{
    const int64_t blocks = (rs.n_rays + 255) / 256;
    k_init<<<(unsigned)(blocks > 0 ? blocks : 1), 256, 0, st>>>(tp, f, d_theta, rs, d_counters);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// integrator stage (Eq. geodesiceqn with the App. A symbols, classical RK4,
// termination on x3 with linear interpolation: Sec. 3.4)
// ---------------------------------------------------------------------------
// A block of 256 threads serves 64 rays: first every thread reduces one
// output of one ray's split partials (mixed precision: four threads per ray,
// which keeps four times more loads in flight), then one thread per ray runs
// the FP64 stage update with whole warps active.
constexpr int kStageRays = 64;
// from this many rays on (four blocks of 256 per SM), one ray per thread
// still gives every SM several blocks
static int64_t stage_wide_rays() { return (int64_t)device_sm_count() * 4 * 256; }

int device_sm_count()
{
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    if (dev >= 0 && dev < 64 && cache[dev] > 0) return cache[dev];
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return 152;
    if (dev >= 0 && dev < 64) cache[dev] = sms;
    return sms;
}

// the bundles' prism records of this stage (mean-subtracted boxes), read by
// every ray of the bundle in k_stage
__global__ void k_prism(TraceParams tp, DevField f, RayState rs, int step, int stage, const unsigned long long *cnt,
                        double *__restrict__ prism)
{
    if (step >= tp.n_steps && cnt[(step - 1) & 1] == 0ull) return;  // every ray is across
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= rs.n_b) return;
    bundle_prism(f, rs, step * 4 + stage, b, prism);
}

cudaError_t launch_prism(const TraceParams &tp, const DevField &f, RayState rs, int step, int stage,
                         const unsigned long long *d_counters, double *d_prism, cudaStream_t st)
{
    const int64_t blocks = (rs.n_b + 127) / 128;
    k_prism<<<(unsigned)(blocks > 0 ? blocks : 1), 128, 0, st>>>(tp, f, rs, step, stage, d_counters, d_prism);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_stage(TraceParams tp, DevField f, RayState rs, int S, int fp64,
                                              double mfac, const void *__restrict__ partials,
                                              const double *__restrict__ dlam,
                                              const double *__restrict__ misc, int step, int stage,
                                              unsigned long long *cnt, const double *__restrict__ prism)
{
    if (stage == 0 && blockIdx.x == 0 && threadIdx.x == 0) cnt[step & 1] = 0ull;
    if (step >= tp.n_steps && cnt[(step - 1) & 1] == 0ull) return;  // every ray is across
    __shared__ double s_acc[kStageRays][4];
    __shared__ unsigned s_active;
    if (threadIdx.x == 0) s_active = 0;
    const int64_t r0 = (int64_t)blockIdx.x * kStageRays;
    if (!fp64) {
        const int local = threadIdx.x >> 2, o = threadIdx.x & 3;
        const int64_t i = r0 + local;
        if (i < rs.n_rays) s_acc[local][o] = reduce_partials_mixed((const float2 *)partials, S, rs.n_rays, i, o);
    }
    __syncthreads();
    if (threadIdx.x < kStageRays) {
        const int64_t i = r0 + threadIdx.x;
        if (i < rs.n_rays && stage_ray(tp, f, rs, S, fp64 != 0, mfac, partials, dlam, misc[0], step, stage, cnt, i,
                                       fp64 ? nullptr : s_acc[threadIdx.x], prism))
            atomicAdd(&s_active, 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_active) atomicAdd(&cnt[2], (unsigned long long)s_active);
}

// One ray per thread, its four outputs reduced by the same thread: for few
// splits (the grid path) or enough rays to fill the GPU, where the FP64
// stage, not the reduction, needs the threads.
__global__ void __launch_bounds__(256) k_stage_wide(TraceParams tp, DevField f, RayState rs, int S, int fp64,
                                                   double mfac, const void *__restrict__ partials,
                                                   const double *__restrict__ dlam,
                                                   const double *__restrict__ misc, int step, int stage,
                                                   unsigned long long *cnt, const double *__restrict__ prism)
{
    if (stage == 0 && blockIdx.x == 0 && threadIdx.x == 0) cnt[step & 1] = 0ull;
    if (step >= tp.n_steps && cnt[(step - 1) & 1] == 0ull) return;  // every ray is across
    __shared__ unsigned s_active;
    if (threadIdx.x == 0) s_active = 0;
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < rs.n_rays) {
        double acc[4];
        if (!fp64) {
#pragma unroll
            for (int o = 0; o < 4; ++o) acc[o] = reduce_partials_mixed((const float2 *)partials, S, rs.n_rays, i, o);
        }
        if (stage_ray(tp, f, rs, S, fp64 != 0, mfac, partials, dlam, misc[0], step, stage, cnt, i,
                      fp64 ? nullptr : acc, prism))
            atomicAdd(&s_active, 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_active) atomicAdd(&cnt[2], (unsigned long long)s_active);
}

cudaError_t launch_stage(const TraceParams &tp, const DevField &f, RayState rs, const ForceShape &sh, bool fp64,
                         const void *d_partials, const double *d_dlam, const double *d_misc, int step, int stage,
                         unsigned long long *d_counters, cudaStream_t st, const double *d_prism)
{
    const int S = partial_splits(sh);
    const double mfac = partial_mass_factor(f, sh);
    if (S <= 8 || rs.n_rays >= stage_wide_rays()) {
        const int64_t blocks = (rs.n_rays + 255) / 256;
        k_stage_wide<<<(unsigned)blocks, 256, 0, st>>>(tp, f, rs, S, fp64 ? 1 : 0, mfac, d_partials, d_dlam, d_misc,
                                                       step, stage, d_counters, d_prism);
    } else {
        const int64_t blocks = (rs.n_rays + kStageRays - 1) / kStageRays;
        k_stage<<<(unsigned)blocks, 256, 0, st>>>(tp, f, rs, S, fp64 ? 1 : 0, mfac, d_partials, d_dlam, d_misc, step,
                                                 stage, d_counters, d_prism);
    }
    return cudaGetLastError();
}

// field at arbitrary points (rt3d_potential): reduce partials + mean subtraction
__global__ void k_field_points(DevField f, int S, int fp64, double mfac, const void *__restrict__ partials,
                               const double *__restrict__ pts, const int *__restrict__ rep, int64_t n,
                               double *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double p[3] = {pts[i], pts[n + i], pts[2 * n + i]};
    const int r = rep ? rep[i] : 0;
    double F[4];
    if (r < 0 || r >= f.n_rep || !isfinite(p[0]) || !isfinite(p[1]) || !isfinite(p[2])) {
        // a replica index outside [0, n_rep) or a non-finite point: the pair
        // sum skipped it, and its result is NaN rather than a silent value
#pragma unroll
        for (int o = 0; o < 4; ++o) out[4 * i + o] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    gather_field(f, S, fp64 != 0, partials, n, i, r, p, mfac, F);
#pragma unroll
    for (int o = 0; o < 4; ++o) out[4 * i + o] = F[o];
}

cudaError_t launch_stage_field(const DevField &f, const ForceShape &sh, bool fp64, const void *d_partials,
                               const double *d_pts, const int *d_rep, int64_t n, double *d_out, cudaStream_t st)
{
    const int64_t blocks = (n + 255) / 256;
    k_field_points<<<(unsigned)(blocks > 0 ? blocks : 1), 256, 0, st>>>(
        f, partial_splits(sh), fp64 ? 1 : 0, partial_mass_factor(f, sh), d_partials, d_pts, d_rep, n, d_out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// bundle reducer: least-squares lens-map Jacobian of the polygon offsets
// (Sec. 3.1; Eqs. lensmap, magnification), in FP64
// ---------------------------------------------------------------------------
__global__ void k_reduce(TraceParams tp, const double *__restrict__ theta, RayState rs,
                         const double *__restrict__ misc, double *__restrict__ bout, double *__restrict__ rout)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= rs.n_b) return;
    reduce_bundle(tp, theta, rs, misc[0], b, bout + 6 * b, rout);
}

cudaError_t launch_reduce(const TraceParams &tp, const double *d_theta, RayState rs, const double *d_misc,
                          double *d_bout, double *d_rout, cudaStream_t st)
{
    const int64_t blocks = (rs.n_b + 127) / 128;
    k_reduce<<<(unsigned)(blocks > 0 ? blocks : 1), 128, 0, st>>>(tp, d_theta, rs, d_misc, d_bout, d_rout);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// muPDF (Sec. 5.3, Eq. weighthisto): integer counts and fixed-point weights
// by atomics (order-independent, so bit-reproducible), moments by one block
// in a fixed order.
// ---------------------------------------------------------------------------
// value binned and weight base of entry i: v = |mu| (muPDF) or, with a shear
// pair, v = |gamma| = sqrt(g1^2 + g2^2) (shear PDF, Sec. 5.4, products and sum
// rounded separately as in the FP64 definition); the weight is 1/|mu| in both
struct HistIn {
    const double *mu;
    int stride;
    const int *fl;
    const double *fld;
    const double *g1, *g2;  // shear PDF; null for the muPDF
};

__device__ __forceinline__ bool hist_take(const HistIn &h, int64_t i, double &m, double &v)
{
    m = h.mu[i * h.stride];
    int f = h.fl ? h.fl[i] : (h.fld ? (int)h.fld[i * h.stride] : 0);
    if ((f & (RT3D_F_NOCROSS | RT3D_F_NONFINITE)) || !isfinite(m) || m == 0.0) return false;
    if (h.g1) {
        const double a = h.g1[i], b = h.g2[i];
        v = sqrt(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)));
        if (!isfinite(v)) return false;
    } else {
        v = fabs(m);
    }
    return true;
}

__global__ void k_hist_bins(int64_t n, HistIn h, int bins, double lmin, double dl, unsigned long long *counts,
                            unsigned long long *wfix, unsigned long long *scal)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double m, v;
    if (!hist_take(h, i, m, v)) {
        atomicAdd(&scal[4], 1ull);
        return;
    }
    atomicAdd(&scal[0], 1ull);
    if (m < 0.0) atomicAdd(&scal[3], 1ull);
    m = fabs(m);
    const double bb = floor((log10(v) - lmin) / dl);
    if (bb < 0.0) {
        atomicAdd(&scal[1], 1ull);
    } else if (bb >= (double)bins) {
        atomicAdd(&scal[2], 1ull);
    } else {
        const int k = (int)bb;
        atomicAdd(&counts[k], 1ull);
        atomicAdd(&wfix[k], (unsigned long long)__double2ll_rn(ldexp(1.0 / m, 32)));
    }
}

__global__ void __launch_bounds__(1024) k_hist_moments(int64_t n, HistIn h,
                                                       const unsigned long long *__restrict__ scal, double *out8)
{
    __shared__ double sw[1024], s1[1024];
    double w = 0.0, a1 = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        double m, v;
        if (!hist_take(h, i, m, v)) continue;
        const double iw = 1.0 / fabs(m);
        w += iw;
        a1 += iw * v;
    }
    sw[threadIdx.x] = w;
    s1[threadIdx.x] = a1;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) {
            sw[threadIdx.x] += sw[threadIdx.x + k];
            s1[threadIdx.x] += s1[threadIdx.x + k];
        }
        __syncthreads();
    }
    const double W = sw[0], mean = W > 0.0 ? s1[0] / W : 0.0;
    __syncthreads();
    double a2 = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        double m, v;
        if (!hist_take(h, i, m, v)) continue;
        const double d = v - mean;
        a2 += d * d / fabs(m);
    }
    sw[threadIdx.x] = a2;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) sw[threadIdx.x] += sw[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int q = 0; q < 5; ++q) out8[q] = (double)scal[q];  // used, under, over, negative, excluded
        out8[5] = W;
        out8[6] = mean;
        out8[7] = W > 0.0 ? sqrt(sw[0] / W) : 0.0;
    }
}

cudaError_t launch_histogram(int64_t n, const double *d_mu, int mu_stride, const int *d_flags, const double *d_flagsd,
                             int bins, double mu_min, double mu_max, unsigned long long *d_counts,
                             unsigned long long *d_wfix, unsigned long long *d_scal, double *d_out8,
                             cudaStream_t st, const double *d_g1, const double *d_g2)
{
    const double lmin = log10(mu_min);
    const double dl = (log10(mu_max) - lmin) / (double)bins;
    HistIn h{d_mu, mu_stride, d_flags, d_flagsd, d_g1, d_g2};
    cudaError_t e;
    if ((e = cudaMemsetAsync(d_counts, 0, sizeof(unsigned long long) * bins, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(d_wfix, 0, sizeof(unsigned long long) * bins, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(d_scal, 0, sizeof(unsigned long long) * 5, st)) != cudaSuccess) return e;
    if (n > 0) {
        const int64_t blocks = (n + 255) / 256;
        k_hist_bins<<<(unsigned)blocks, 256, 0, st>>>(n, h, bins, lmin, dl, d_counts, d_wfix, d_scal);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_hist_moments<<<1, 1024, 0, st>>>(n, h, d_scal, d_out8);
    return cudaGetLastError();
}

}  // namespace rt3d
