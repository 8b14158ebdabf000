// rt3d_internal.cuh -- shared definitions of the sm_103a ray-bundle library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rt3d.h"

namespace rt3d {

// ---------------------------------------------------------------------------
// physical constants (IAU nominal G Msun, SI c, Mpc)
// ---------------------------------------------------------------------------
constexpr double kGMsun = 1.32712440018e20;          // m^3 s^-2
constexpr double kC = 299792458.0;                   // m s^-1
constexpr double kMpc = 3.0856775814913673e22;       // m
constexpr double kMuG = kGMsun / (kC * kC) / kMpc;   // G Msun / c^2 in Mpc
constexpr double kCkms = 299792.458;                 // c in km s^-1

struct Cosmo {
    double om, ol, h;
    double H0;  // H0 / c in 1/Mpc
    double t0;  // lookback time of the big bang (Mpc)
    double k;   // 1.5 sqrt(OL) H0
    double r;   // OM / OL
    // a(t) and atab_h da/dt at t = j atab_h, j < atab_n (interleaved), or
    // null: the closed form is then evaluated at every call
    const double *atab = nullptr;
    int atab_n = 0;
    double atab_h = 0.0, atab_ih = 0.0;  // node spacing and its inverse
};

// Eq. scalefac2: a(t) for t the lookback time, closed form.
__device__ __forceinline__ double cosmo_a_exact(const Cosmo &c, double t)
{
    double s = sinh(c.k * (c.t0 - t));
    return cbrt(c.r * s * s);
}

// a(t) by cubic Hermite interpolation of the table (a and da/dt at the
// nodes): the remainder h^4 max|d^4a/dt^4| / 384 is below 1e-13 of a up to
// z = 5 for the 4096-node table, against the closed form's FP64 rounding of a
// few 1e-16; outside the table, the closed form.  It replaces an FP64 sinh
// and cbrt per ray and stage on a GPU whose FP64 rate is 1/64 of FP32.
__device__ __forceinline__ double cosmo_a(const Cosmo &c, double t)
{
    if (c.atab) {
        const double u = t * c.atab_ih;
        if (u >= 0.0 && u < (double)(c.atab_n - 1)) {
            const int j = (int)u;
            const double s = u - (double)j;
            const double a0 = c.atab[2 * j], d0 = c.atab[2 * j + 1];
            const double a1 = c.atab[2 * j + 2], d1 = c.atab[2 * j + 3];
            // the cubic through (a0, d0) at s = 0 and (a1, d1) at s = 1, in powers of s
            const double D = a1 - a0;
            const double c2 = 3.0 * D - 2.0 * d0 - d1, c3 = d0 + d1 - 2.0 * D;
            return a0 + s * (d0 + s * (c2 + s * c3));
        }
    }
    return cosmo_a_exact(c, t);
}

// d a / d t (lookback): -a H(a) for the same flat Lemaitre model.
__device__ __forceinline__ double cosmo_adot(const Cosmo &c, double a)
{
    return -a * c.H0 * sqrt(c.om / (a * a * a) + c.ol);
}

// the same with ia = 1 / a already at hand
__device__ __forceinline__ double cosmo_adot_ia(const Cosmo &c, double a, double ia)
{
    return -a * c.H0 * sqrt(c.om * (ia * ia * ia) + c.ol);
}

// ---------------------------------------------------------------------------
// field of a uniform rectangular prism (mean subtraction, Sec. 3.3):
// I = int dV / |r - r'| and dI/dr, from the closed-form antiderivative.
// ---------------------------------------------------------------------------
// log(u + rho) with rho = |(u, v, w)|, q = v^2 + w^2; stable for u < 0.
template <typename T>
__device__ __forceinline__ T prism_log(T u, T rho, T q)
{
    if (u >= T(0)) return log(u + rho);
    if (q == T(0)) return T(0);  // only ever multiplied by a zero coefficient
    return log(q / (rho - u));
}

template <typename T>
__device__ __forceinline__ void prism_corner(T x, T y, T z, T &F, T &Hx, T &Hy, T &Hz)
{
    T xx = x * x, yy = y * y, zz = z * z;
    T rho = sqrt(xx + yy + zz);
    T lx = prism_log(x, rho, yy + zz), ly = prism_log(y, rho, xx + zz), lz = prism_log(z, rho, xx + yy);
    T tx = (x != T(0)) ? atan(y * z / (x * rho)) : T(0);
    T ty = (y != T(0)) ? atan(z * x / (y * rho)) : T(0);
    T tz = (z != T(0)) ? atan(x * y / (z * rho)) : T(0);
    F = x * y * lz + y * z * lx + z * x * ly - T(0.5) * (xx * tx + yy * ty + zz * tz);
    Hx = y * lz + z * ly - x * tx;
    Hy = z * lx + x * lz - y * ty;
    Hz = x * ly + y * lx - z * tz;
}

// out = (I, dI/dx1, dI/dx2, dI/dx3) for the prism [lo, hi] at point p.
template <typename T>
__device__ __forceinline__ void prism_field(const T lo[3], const T hi[3], const T p[3], T out[4])
{
    T I = 0, gx = 0, gy = 0, gz = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const T x = ((c & 1) ? hi[0] : lo[0]) - p[0];
        const T y = ((c & 2) ? hi[1] : lo[1]) - p[1];
        const T z = ((c & 4) ? hi[2] : lo[2]) - p[2];
        T F, Hx, Hy, Hz;
        prism_corner(x, y, z, F, Hx, Hy, Hz);
        // inclusion-exclusion over the corners: (-1)^(number of lower limits)
        const T sg = ((3 - __popc(c)) & 1) ? T(-1) : T(1);
        I += sg * F;
        gx -= sg * Hx;
        gy -= sg * Hy;
        gz -= sg * Hz;
    }
    out[0] = I;
    out[1] = gx;
    out[2] = gy;
    out[3] = gz;
}

// As prism_field, plus the Hessian d2I/dp_i dp_j (h = xx, xy, xz, yy, yz,
// zz) from the same logarithms and arctangents: for the corner function,
// d2F/dx2 = -atan(yz / (x rho)) and d2F/dx dy = log(z + rho) (cyclically).
template <typename T>
__device__ __forceinline__ void prism_field_hess(const T lo[3], const T hi[3], const T p[3], T out[4], T h[6])
{
    T I = 0, gx = 0, gy = 0, gz = 0, hxx = 0, hxy = 0, hxz = 0, hyy = 0, hyz = 0, hzz = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const T x = ((c & 1) ? hi[0] : lo[0]) - p[0];
        const T y = ((c & 2) ? hi[1] : lo[1]) - p[1];
        const T z = ((c & 4) ? hi[2] : lo[2]) - p[2];
        const T xx = x * x, yy = y * y, zz = z * z;
        const T rho = sqrt(xx + yy + zz);
        const T lx = prism_log(x, rho, yy + zz), ly = prism_log(y, rho, xx + zz), lz = prism_log(z, rho, xx + yy);
        const T tx = (x != T(0)) ? atan(y * z / (x * rho)) : T(0);
        const T ty = (y != T(0)) ? atan(z * x / (y * rho)) : T(0);
        const T tz = (z != T(0)) ? atan(x * y / (z * rho)) : T(0);
        const T sg = ((3 - __popc(c)) & 1) ? T(-1) : T(1);
        I += sg * (x * y * lz + y * z * lx + z * x * ly - T(0.5) * (xx * tx + yy * ty + zz * tz));
        gx -= sg * (y * lz + z * ly - x * tx);
        gy -= sg * (z * lx + x * lz - y * ty);
        gz -= sg * (x * ly + y * lx - z * tz);
        hxx -= sg * tx;
        hyy -= sg * ty;
        hzz -= sg * tz;
        hxy += sg * lz;
        hyz += sg * lx;
        hxz += sg * ly;
    }
    out[0] = I;
    out[1] = gx;
    out[2] = gy;
    out[3] = gz;
    h[0] = hxx;
    h[1] = hxy;
    h[2] = hxz;
    h[3] = hyy;
    h[4] = hyz;
    h[5] = hzz;
}

// ---------------------------------------------------------------------------
// device-side particle field
// ---------------------------------------------------------------------------
struct DevField {
    const int4 *part;      // (qx, qy, qz, m32 bits): integer grid position, scaled mass (FP32)
    const float *eps2;     // per-particle eps^2 (Mpc^2), or nullptr
    const double *m64;     // scaled masses (FP64 path)
    const double *eps2_64; // per-particle eps^2 (FP64 path) or nullptr
    const int *rot;        // n_rep * 9
    const int *shift;      // n_rep * 3, grid units
    int64_t n;
    float eps2u;           // uniform eps^2 (Mpc^2)
    double eps2u64;
    int replicated, mean_subtract, n_rep;
    int Lq;                // box length in grid units (replicated)
    double delta, inv_delta;  // grid spacing 2^-e (Mpc) and its inverse
    double O[3];           // world position of grid origin (isolated fields)
    double L;              // box length (Mpc)
    double mscale_inv;     // 1 / 2^ms (masses are stored as mu_G m 2^ms)
    double rho_term;       // mu_G * mean density (mean subtraction), Mpc^-2
    int uniform_mass;      // every particle has the same mass
    double m_uniform;      // that mass, scaled as stored (mu_G m 2^ms)
};

// world position of the grid origin of replica j (replicated) or the field origin
__device__ __forceinline__ void frame_origin(const DevField &f, int j, double o[3])
{
    if (f.replicated) {
        o[0] = -0.5 * f.L;
        o[1] = -0.5 * f.L;
        o[2] = (double)j * f.L;
    } else {
        o[0] = f.O[0];
        o[1] = f.O[1];
        o[2] = f.O[2];
    }
}

// replica transform of a box-frame grid position (exact integer arithmetic):
// q' = wrap(R (q - c) + c + s), c = Lq/2
__device__ __forceinline__ void replica_q(const DevField &f, int j, int qx, int qy, int qz, long long out[3])
{
    const long long c = f.Lq / 2;
    const long long d[3] = {qx - c, qy - c, qz - c};
    const int *R = f.rot + 9 * j;
    const int *S = f.shift + 3 * j;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        long long v = (long long)R[3 * r] * d[0] + (long long)R[3 * r + 1] * d[1] + (long long)R[3 * r + 2] * d[2];
        v += c + S[r];
        if (v >= f.Lq) v -= f.Lq;
        if (v >= f.Lq) v -= f.Lq;
        if (v < 0) v += f.Lq;
        out[r] = v;
    }
}

__device__ __forceinline__ int replica_of(const DevField &f, double x3)
{
    if (!f.replicated) return 0;
    double q = floor(x3 / f.L);
    if (q < 0.0) return 0;
    if (q > (double)(f.n_rep - 1)) return f.n_rep - 1;
    return (int)q;
}

// ---------------------------------------------------------------------------
// ray state (SoA, FP64): index [component * n_rays + ray]
// ---------------------------------------------------------------------------
struct RayState {
    double *y;     // 8 x nr  current state
    double *ys;    // 8 x nr  stage state (positions read by the pair sum)
    double *ks;    // 8 x nr  RK4 accumulator
    double *fin;   // 8 x nr  state interpolated to x3 = chi_s
    int *done;     // nr
    int *steps;    // nr
    int *rep;      // 2 x n_bundles: replica of each bundle for even / odd stages
    int64_t n_rays, n_b;
    int nr;        // rays per bundle (1 + n_ring)
    int64_t stride;  // component stride of y, ys, ks, fin (n_rays for a single trace)
};

struct TraceParams {
    Cosmo cosmo;
    double chi_s;
    int n_ring;
    double theta_r, phase;
    int christoffel;
    int n_steps, max_extra;
};

// force launch shape
struct ForceShape {
    int R;        // rays per thread
    int NT;       // threads per block
    int splits;   // particle splits (blocks along y)
    int variant;  // 0 packed FP32x2, 1 scalar FP32, 2 FP64, 3-5 bundle-centric, 6 grid path
    int umass;    // packed kernel without per-particle masses (uniform-mass field)
    int cl = 1;   // thread-block cluster size along the splits: the cluster adds its
                  // CTAs' partials in distributed shared memory, one partial per cluster
};
// split partials a shape leaves for the integrator stage
inline int partial_splits(const ForceShape &sh) { return sh.splits / sh.cl; }

// device scratch of a trace (grow-only, owned by the context)
struct Scratch {
    void *partials = nullptr;      // splits * 4 * n_rays (float2 or double)
    size_t partials_bytes = 0;
    double *dlam = nullptr;        // n_steps
    size_t dlam_n = 0;
    double *misc = nullptr;        // [0] chi_s, [1..] spare
    unsigned long long *counters = nullptr; // [0] active-after slot 0, [1] slot 1, [2] active ray-stages
    double *state = nullptr;       // 32 * n_rays
    size_t state_rays = 0;
    int *ints = nullptr;           // 2 * n_rays + n_b
    size_t ints_n = 0;
    double *theta = nullptr;       // n_b * 2
    size_t theta_n = 0;
    double *bout = nullptr;        // n_b * 6
    size_t bout_n = 0;
    double *rout = nullptr;        // n_rays * 8
    size_t rout_n = 0;
    double *prism = nullptr;       // n_b * 13 bundle prism records
    size_t prism_n = 0;
    char *planes = nullptr;        // lens-plane table of the multi-plane system
    size_t planes_bytes = 0;
};

// streaming multiprocessors of the current device (queried once per device;
// 152 on GB300), for grid sizes counted in waves of resident blocks
int device_sm_count();

// kernels (launch wrappers; return cudaError_t of the launch)
// fill the a(t) table of c (n nodes, spacing h) at d_tab
cudaError_t launch_atab(const Cosmo &c, int n, double h, double *d_tab, cudaStream_t st);
cudaError_t launch_schedule(const Cosmo &c, double z_s, int kind, int n, double chi_l, double s,
                            double *d_dlam, double *d_misc, cudaStream_t st);
cudaError_t launch_init(const TraceParams &tp, const DevField &f, const double *d_theta, RayState rs,
                        unsigned long long *d_counters, cudaStream_t st);
cudaError_t launch_force(const DevField &f, const RayState &rs, const ForceShape &sh, bool fp64,
                         void *d_partials, const unsigned long long *d_active, int gate, cudaStream_t st);
cudaError_t launch_stage(const TraceParams &tp, const DevField &f, RayState rs, const ForceShape &sh,
                         bool fp64, const void *d_partials, const double *d_dlam, const double *d_misc,
                         int step, int stage, unsigned long long *d_counters, cudaStream_t st,
                         const double *d_prism = nullptr);
// per-bundle prism records (value, gradient, Hessian at the central ray) of a
// mean-subtracted replicated field, for launch_stage: kPrismRec doubles each
constexpr int kPrismRec = 13;
cudaError_t launch_prism(const TraceParams &tp, const DevField &f, RayState rs, int step, int stage,
                         const unsigned long long *d_counters, double *d_prism, cudaStream_t st);
// factor the integrator stage applies to the pair-sum partials of shape sh
inline double partial_mass_factor(const DevField &f, const ForceShape &sh)
{
    return sh.umass ? f.m_uniform : 1.0;
}
cudaError_t launch_reduce(const TraceParams &tp, const double *d_theta, RayState rs, const double *d_misc,
                          double *d_bout, double *d_rout, cudaStream_t st);
cudaError_t launch_histogram(int64_t n, const double *d_mu, int mu_stride, const int *d_flags,
                             const double *d_flagsd, int bins, double mu_min, double mu_max,
                             unsigned long long *d_counts, unsigned long long *d_wfix,
                             unsigned long long *d_scal, double *d_out8, cudaStream_t st,
                             const double *d_g1 = nullptr, const double *d_g2 = nullptr);
cudaError_t launch_potential(const DevField &f, bool fp64, const double *d_pts, const int *d_rep,
                             int64_t n, const ForceShape &sh, void *d_partials, double *d_out,
                             cudaStream_t st);
cudaError_t launch_stage_field(const DevField &f, const ForceShape &sh, bool fp64, const void *d_partials,
                               const double *d_pts, const int *d_rep, int64_t n, double *d_out,
                               cudaStream_t st);

// gridded field (Sec. 3.3 grid path, App. B): node values and x3 spline
// second derivatives, 4 n^3 doubles each, [f][i1][i2][i3] with i3 fastest
// doubles per grid node in the node table: phi, dphi/dx1, dphi/dx2, dphi/dx3,
// then their natural-spline second derivatives along x3 (App. B)
constexpr int kGridRec = 8;
struct GridDev {
    int n = 0, n_int = 0;
    double lo[3] = {0.0, 0.0, 0.0};
    double h = 0.0;
    // one of the two: [i1][i2][i3][kGridRec], i3 fastest, in FP64 (FP64
    // contexts) or rounded to FP32 (mixed contexts)
    double *tab = nullptr;
    float *tab32 = nullptr;
    // cube-tiled replicated box (cubes > 0): n_rep * cubes node tables stored
    // one after the other (stride kGridRec n^3), replica-major; cube c of
    // replica j has lo = (-W/2, -W/2, j L + c W) and spacing W / (n - 1)
    int cubes = 0, n_rep = 1;
    double L = 0.0, W = 0.0;
    // points up to margin node spacings outside the node range take the end
    // intervals' cubics (box cubes: 1, for the rays of a bundle near a cube
    // face); farther out the field is zero
    double margin = 0.0;
};
// build g.tab (fp64) or g.tab32 (allocated here) from host particles; returns
// an rt3d status and sets err on failure
int grid_build(GridDev &g, int64_t np, const double *pos, const double *mass, double soft, int mean_subtract,
               bool fp64, cudaStream_t st, std::string &err);
// build the n_rep * cubes node tables of a cube-tiled replicated box (g.n,
// n_rep, cubes, L, W, h set by the caller; g.tab allocated here) from the
// box's host particles, each replica placed by rot[9 j] and shift[3 j]
int grid_build_box(GridDev &g, int64_t np, const double *pos, const double *mass, double soft,
                   const int32_t *rot, const double *shift, int mean_subtract, bool fp64, cudaStream_t st,
                   std::string &err);
void grid_free(GridDev &g);
// App. B evaluation at n points (SoA px, py, pz) from the grid's table.  mode
// 0 (mixed path, FP32 table): -F as (hi, 0) pairs in the pair-sum partial
// layout (one split); 1 (FP64 table): -F as FP64 partials; 2: F at
// out[4 i + f] as FP64 numbers
cudaError_t launch_grid_eval(const GridDev &g, const double *px, const double *py, const double *pz, int64_t n,
                             int mode, void *out, const unsigned long long *gate, cudaStream_t st,
                             int group = 1);

// Born approximation (born.cu): scratch size and the run over node chunks of
// K nodes with the Hessian pair sum split `splits` ways; d_out = n_b x 3
size_t born_scratch_bytes(int64_t n_b, int n_steps, int K, int splits);
cudaError_t born_run(const Cosmo &c, const DevField &f, int64_t n_particles, double z_s, int64_t n_b,
                     const double *d_theta, int kind, int n_steps, double chi_l, double s, int K, int splits,
                     void *scratch, double *d_out, cudaStream_t st);

int force_max_splits(const ForceShape &sh, int64_t n_particles);
size_t partials_bytes(const ForceShape &sh, int64_t n_rays, bool fp64);

// multiple lens-plane comparison system (multiplane.cu)
size_t mp_plane_bytes();
size_t mp_partials_bytes(int n_ring, int64_t n_b, int splits, bool fp64);
cudaError_t mp_run(const Cosmo &c, const DevField &f, double z_s, int slices, double x3_lo, double x3_hi,
                   const TraceParams &tp, const double *d_theta, RayState rs, void *d_planes, int n_pl, void *partials,
                   int splits, bool fp64, bool umass, double *misc, unsigned long long *count, double *d_bout,
                   double *d_rout, cudaStream_t st);

}  // namespace rt3d
