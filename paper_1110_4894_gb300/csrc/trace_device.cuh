// trace_device.cuh -- device functions of one trace shared by the per-stage
// kernels and the batched persistent kernel: background cosmology and the
// step table, bundle initialiser, field gather with mean subtraction, the
// geodesic right-hand side, one RK4 stage of one ray, and the bundle reducer.
#pragma once
#include <math_constants.h>

#include "rt3d_internal.cuh"

namespace rt3d {

// ---------------------------------------------------------------------------
// background cosmology on the device (Sec. 3.5, Eq. raytracedistance)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double hubble_E(const Cosmo &c, double z)
{
    double u = 1.0 + z;
    return sqrt(c.om * u * u * u + c.ol);
}

// chi(z) = (1/H0) int_0^z dz'/E(z') by composite Boole's rule (5-point
// Newton-Cotes, error O(h^7)), panels no wider than 0.02 in z.
static __device__ double comoving_distance(const Cosmo &c, double z)
{
    if (z <= 0.0) return 0.0;
    int panels = (int)ceil(z / 0.02);
    if (panels < 1) panels = 1;
    const double w = z / panels, h = 0.25 * w;
    double acc = 0.0;
    for (int p = 0; p < panels; ++p) {
        const double z0 = p * w;
        const double f0 = 1.0 / hubble_E(c, z0), f1 = 1.0 / hubble_E(c, z0 + h),
                     f2 = 1.0 / hubble_E(c, z0 + 2 * h), f3 = 1.0 / hubble_E(c, z0 + 3 * h),
                     f4 = 1.0 / hubble_E(c, z0 + w);
        acc += (7.0 * (f0 + f4) + 32.0 * (f1 + f3) + 12.0 * f2) * (2.0 * h / 45.0);
    }
    return acc / c.H0;
}

// redshift at comoving distance chi (Newton on chi(z), d chi/dz = 1/(H0 E))
static __device__ double redshift_at(const Cosmo &c, double chi)
{
    if (chi <= 0.0) return 0.0;
    double z = chi * c.H0;
    for (int it = 0; it < 40; ++it) {
        const double dz = (comoving_distance(c, z) - chi) * c.H0 * hubble_E(c, z);
        z -= dz;
        if (fabs(dz) <= 2e-16 * (1.0 + z)) break;
    }
    return z;
}

__device__ __forceinline__ double a2_at(const Cosmo &c, double chi)
{
    const double a = 1.0 / (1.0 + redshift_at(c, chi));
    return a * a;
}

__device__ __forceinline__ double sched_node(int kind, int n, int k, double chi_s, double chi_l, double s)
{
    if (k == 0) return 0.0;
    if (k == n) return chi_s;
    if (kind == RT3D_SCHED_UNIFORM) return chi_s * (double)k / (double)n;
    const double u0 = asinh((0.0 - chi_l) / s), u1 = asinh((chi_s - chi_l) / s);
    return chi_l + s * sinh(u0 + (u1 - u0) * (double)k / (double)n);
}


// affine step k of the unperturbed ray: int a^2 dchi over [x_k, x_{k+1}] by
// composite Boole's rule with 4 panels
__device__ __forceinline__ double schedule_step(const Cosmo &c, int kind, int n, int k, double chi_s, double chi_l,
                                                double s)
{
    const double x0 = sched_node(kind, n, k, chi_s, chi_l, s), x1 = sched_node(kind, n, k + 1, chi_s, chi_l, s);
    const double w = (x1 - x0) * 0.25, h = 0.25 * w;
    double acc = 0.0;
    double fl = a2_at(c, x0);
    for (int p = 0; p < 4; ++p) {
        const double xa = x0 + p * w;
        const double f1 = a2_at(c, xa + h), f2 = a2_at(c, xa + 2 * h), f3 = a2_at(c, xa + 3 * h);
        const double f4 = a2_at(c, p == 3 ? x1 : xa + w);
        acc += (7.0 * (fl + f4) + 32.0 * (f1 + f3) + 12.0 * f2) * (2.0 * h / 45.0);
        fl = f4;
    }
    return acc;
}

// ---------------------------------------------------------------------------
// bundle initialiser (Sec. 3.1, ray bundle; initial state of Sec. 3.4)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ray_theta(const TraceParams &tp, const double *theta, int64_t b, int k,
                                          double &tx, double &ty)
{
    tx = theta[2 * b];
    ty = theta[2 * b + 1];
    if (k > 0) {
        const double ang = tp.phase + 2.0 * CUDART_PI * (double)(k - 1) / (double)tp.n_ring;
        double sn, cs;
        sincos(ang, &sn, &cs);
        tx += tp.theta_r * cs;
        ty += tp.theta_r * sn;
    }
}


// bundle initialiser for ray i (Sec. 3.1; initial state of Sec. 3.4)
__device__ __forceinline__ void init_ray(const TraceParams &tp, const DevField &f, const double *__restrict__ theta,
                                         const RayState &rs, int64_t i)
{
    const int64_t b = i / rs.nr;
    const int k = (int)(i % rs.nr);
    double tx, ty;
    ray_theta(tp, theta, b, k, tx, ty);
    // observer: t = 0 (lookback), x = 0, direction (theta_x, theta_y, 1) with
    // dx3/dl = 1; dt/dl is set from the null condition at the first stage
    const double v[8] = {0.0, 0.0, 0.0, 0.0, sqrt(tx * tx + ty * ty + 1.0), tx, ty, 1.0};
    const int64_t n = rs.stride;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        rs.y[q * n + i] = v[q];
        rs.ys[q * n + i] = v[q];
        rs.ks[q * n + i] = 0.0;
        rs.fin[q * n + i] = 0.0;
    }
    rs.done[i] = 0;
    rs.steps[i] = -1;
    if (k == 0) rs.rep[b] = replica_of(f, 0.0);  // stage parity 0
}

// ---------------------------------------------------------------------------
// integrator stage (Eq. geodesiceqn with the App. A symbols, classical RK4,
// termination on x3 with linear interpolation: Sec. 3.4)
// ---------------------------------------------------------------------------
// phi and grad phi from the reduced pair sums, plus the mean subtraction.
// The sums hold sum m'' / |d| and sum m'' d / |d|^3 (Mpc) with d = particle -
// point and m'' = mu_G m 2^ms (or the same sums without m'' for a uniform-mass
// field, mfac = m''): phi = -S0 mfac / 2^ms, grad phi = -S mfac / 2^ms.
// Bundle prism record (kPrismRec doubles per bundle): the central ray's stage
// position, and the replica prism's I, grad I and Hessian there.
// A ray whose offset e from its bundle's central ray is below 1/kPrismNear of
// the central ray's distance to every face of the prism takes I and grad I
// from the second-order Taylor expansion about the central ray; the
// remainder is O(|e|^3 / d) in I and O(|e|^2 / d) in grad I, d the face
// distance (the prism's third derivatives fall off as 1/d inside), i.e. a
// relative 1/(2 kPrismNear) of the tidal term H e.  Other rays use the
// closed form.
constexpr double kPrismNear = 1000.0;

__device__ __forceinline__ void prism_of_ray(const DevField &f, int rep, const double p[3],
                                             const double *__restrict__ rec, double I[4])
{
    const double lo[3] = {-0.5 * f.L, -0.5 * f.L, (double)rep * f.L};
    const double hi[3] = {0.5 * f.L, 0.5 * f.L, (double)(rep + 1) * f.L};
    if (rec) {
        const double e[3] = {p[0] - rec[0], p[1] - rec[1], p[2] - rec[2]};
        const double en = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
        double d = rec[0] - lo[0];
        d = fmin(d, hi[0] - rec[0]);
        d = fmin(d, rec[1] - lo[1]);
        d = fmin(d, hi[1] - rec[1]);
        d = fmin(d, rec[2] - lo[2]);
        d = fmin(d, hi[2] - rec[2]);
        if (d > kPrismNear * en) {
            const double *g = rec + 3, *h = rec + 7;  // g = (I, grad I)
            const double he[3] = {h[0] * e[0] + h[1] * e[1] + h[2] * e[2], h[1] * e[0] + h[3] * e[1] + h[4] * e[2],
                                  h[2] * e[0] + h[4] * e[1] + h[5] * e[2]};
            I[0] = g[0] + (g[1] * e[0] + g[2] * e[1] + g[3] * e[2]) +
                   0.5 * (e[0] * he[0] + e[1] * he[1] + e[2] * he[2]);
            I[1] = g[1] + he[0];
            I[2] = g[2] + he[1];
            I[3] = g[3] + he[2];
            return;
        }
    }
    prism_field<double>(lo, hi, p, I);
}

// rec: the bundle's prism record, or null (closed form at p)
__device__ __forceinline__ void field_from_sums(const DevField &f, const double acc[4], int rep, const double p[3],
                                                double mfac, double F[4], const double *rec = nullptr)
{
    const double sp = f.mscale_inv * mfac, sg = sp;
    F[0] = -acc[0] * sp;
    F[1] = -acc[1] * sg;
    F[2] = -acc[2] * sg;
    F[3] = -acc[3] * sg;
    if (f.replicated && f.mean_subtract) {
        // remove the field of the replica's uniform mean density (Sec. 3.3)
        double I[4];
        prism_of_ray(f, rep, p, rec, I);
        F[0] += f.rho_term * I[0];
        F[1] += f.rho_term * I[1];
        F[2] += f.rho_term * I[2];
        F[3] += f.rho_term * I[3];
    }
}

// the prism record of bundle b at its central ray's stage position
__device__ __forceinline__ void bundle_prism(const DevField &f, const RayState &rs, int g, int64_t b,
                                             double *__restrict__ rec)
{
    const int64_t ic = b * rs.nr, st = rs.stride;
    const int rep = rs.rep[(g & 1) * rs.n_b + b];
    const double p[3] = {rs.ys[st + ic], rs.ys[2 * st + ic], rs.ys[3 * st + ic]};
    const double lo[3] = {-0.5 * f.L, -0.5 * f.L, (double)rep * f.L};
    const double hi[3] = {0.5 * f.L, 0.5 * f.L, (double)(rep + 1) * f.L};
    double I[4], h[6];
    prism_field_hess<double>(lo, hi, p, I, h);
    double *r = rec + kPrismRec * b;
    r[0] = p[0];
    r[1] = p[1];
    r[2] = p[2];
#pragma unroll
    for (int q = 0; q < 4; ++q) r[3 + q] = I[q];
#pragma unroll
    for (int q = 0; q < 6; ++q) r[7 + q] = h[q];
}

// One output of one ray's split partials, as a double-float sum in FP32
// (TwoSum on the high parts, low parts carried), converted once to FP64.
__device__ __forceinline__ double reduce_partials_mixed(const float2 *__restrict__ pm, int S, int64_t n, int64_t i,
                                                        int o)
{
    float hi = 0.0f, lo = 0.0f;
    for (int s = 0; s < S; ++s) {
        const float2 v = pm[((int64_t)s * 4 + o) * n + i];
        const float t = hi + v.x;
        const float bb = t - hi;
        const float err = (hi - (t - bb)) + (v.x - bb);
        hi = t;
        lo += err + v.y;
    }
    return (double)hi + (double)lo;
}

// Reduce the pair-sum partials of one ray and add the mean subtraction:
// F = (phi, dphi/dx1, dphi/dx2, dphi/dx3) at the ray's stage position.
__device__ __forceinline__ void gather_field(const DevField &f, int S, bool fp64, const void *partials, int64_t n,
                                             int64_t i, int rep, const double p[3], double mfac, double F[4],
                                             const double *rec = nullptr)
{
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (fp64) {
        const double *pd = (const double *)partials;
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int o = 0; o < 4; ++o) acc[o] += pd[((int64_t)s * 4 + o) * n + i];
    } else {
        // the (hi, lo) FP32 pairs are added as double-float numbers (TwoSum on
        // hi, lo carried separately): ~48-bit sums on the FP32 pipe, converted
        // to FP64 once, instead of 2S conversions and adds on the FP64 pipe
        const float2 *pm = (const float2 *)partials;
        float hi[4] = {0.0f, 0.0f, 0.0f, 0.0f}, lo[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const float2 v = pm[((int64_t)s * 4 + o) * n + i];
                const float t = hi[o] + v.x;
                const float bb = t - hi[o];
                const float err = (hi[o] - (t - bb)) + (v.x - bb);
                hi[o] = t;
                lo[o] += err + v.y;
            }
#pragma unroll
        for (int o = 0; o < 4; ++o) acc[o] = (double)hi[o] + (double)lo[o];
    }
    field_from_sums(f, acc, rep, p, mfac, F, rec);
}

// d y / d lambda for y = (t, x1, x2, x3, dt/dl, dx1/dl, dx2/dl, dx3/dl):
// d^2 x^a / dl^2 = -Gamma^a_bc u^b u^c with App. A's first-order symbols
//   Gamma^t_tt = -a' phi / a^2,  Gamma^t_ti = phi_i / a,  Gamma^t_ii = a' (a + phi)
//   Gamma^i_tt = phi_i / a^3,    Gamma^i_ti = a' (a + phi) / a^2,
//   Gamma^i_jk = (-phi_k d_ij - phi_j d_ik + phi_i d_jk) / a
// (christoffel = DERIVED replaces Gamma^t_ii by a' (a - 3 phi)).
__device__ __forceinline__ void geodesic_rhs(const double y[8], const double F[4], double a, double ia, double ad,
                                             int christoffel, double k[8])
{
    const double T = y[4], vx = y[5], vy = y[6], vz = y[7];
    const double phi = F[0], gx = F[1], gy = F[2], gz = F[3];
    const double gv = gx * vx + gy * vy + gz * vz;
    const double v2 = vx * vx + vy * vy + vz * vz;
    const double gtii = christoffel == RT3D_CHRISTOFFEL_DERIVED ? ad * (a - 3.0 * phi) : ad * (a + phi);
    const double gitj = ad * (a + phi) * ia * ia;
    k[0] = T;
    k[1] = vx;
    k[2] = vy;
    k[3] = vz;
    k[4] = ad * phi * ia * ia * T * T - 2.0 * ia * gv * T - gtii * v2;
    const double tt = T * T * ia * ia * ia;
    const double drag = 2.0 * gitj * T;
    k[5] = -gx * tt - drag * vx - ia * (gx * v2 - 2.0 * vx * gv);
    k[6] = -gy * tt - drag * vy - ia * (gy * v2 - 2.0 * vy * gv);
    k[7] = -gz * tt - drag * vz - ia * (gz * v2 - 2.0 * vz * gv);
}

// One ray's RK4 stage: gather phi and grad phi, set dt/dl from the null
// condition at the observer, evaluate the geodesic right-hand side, update the
// stage state or (stage 3) combine, terminate and interpolate.  rs is a view:
// ray i of this trace lives at index i with component stride rs.stride, and
// its partials at ((s * 4 + o) * rs.n_rays + i).  Returns whether the ray was
// still in flight (counts towards interactions).
__device__ __forceinline__ bool stage_ray(const TraceParams &tp, const DevField &f, const RayState &rs, int S,
                                          bool fp64, double mfac, const void *__restrict__ partials,
                                          const double *__restrict__ dlam, double chi_s, int step, int stage,
                                          unsigned long long *cnt, int64_t i, const double *pre = nullptr,
                                          const double *prism = nullptr)
{
    const int64_t st = rs.stride;
    const int64_t b = i / rs.nr;
    const int g = step * 4 + stage;  // global stage index: replica buffers alternate on its parity
    const int rep = rs.rep[(g & 1) * rs.n_b + b];
    double ys[8], y[8], k[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        ys[q] = rs.ys[q * st + i];
        y[q] = rs.y[q * st + i];
    }
    double F[4];
    const double *rec = prism ? prism + kPrismRec * b : nullptr;
    if (pre) field_from_sums(f, pre, rep, ys + 1, mfac, F, rec);
    else gather_field(f, S, fp64, partials, rs.n_rays, i, rep, ys + 1, mfac, F, rec);
    const double a = cosmo_a(tp.cosmo, ys[0]);
    const double ia = 1.0 / a;
    const double ad = cosmo_adot_ia(tp.cosmo, a, ia);
    if (step == 0 && stage == 0) {
        // null condition of Eq. expandingmetric with psi = phi / a
        const double vn = sqrt(ys[5] * ys[5] + ys[6] * ys[6] + ys[7] * ys[7]);
        const double T = a * vn * sqrt((1.0 - 2.0 * F[0] / a) / (1.0 + 2.0 * F[0] / a));
        ys[4] = T;
        y[4] = T;
        rs.y[4 * st + i] = T;
    }
    geodesic_rhs(ys, F, a, ia, ad, tp.christoffel, k);
    const double dl = dlam[step < tp.n_steps ? step : tp.n_steps - 1];
    const int done = rs.done[i];
    double nx[8];
    if (stage < 3) {
        const double c = stage == 2 ? dl : 0.5 * dl;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const double acc = stage == 0 ? k[q] : rs.ks[q * st + i] + 2.0 * k[q];
            rs.ks[q * st + i] = acc;
            nx[q] = y[q] + c * k[q];
            rs.ys[q * st + i] = nx[q];
        }
    } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) nx[q] = y[q] + dl * (1.0 / 6.0) * (rs.ks[q * st + i] + k[q]);
        if (!done && nx[3] >= chi_s) {
            const double s = (chi_s - y[3]) / (nx[3] - y[3]);
#pragma unroll
            for (int q = 0; q < 8; ++q) rs.fin[q * st + i] = y[q] + s * (nx[q] - y[q]);
            rs.done[i] = 1;
            rs.steps[i] = step + 1;
        } else if (!done) {
            atomicAdd(&cnt[step & 1], 1ull);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            rs.y[q * st + i] = nx[q];
            rs.ys[q * st + i] = nx[q];
        }
    }
    if (i % rs.nr == 0) rs.rep[((g + 1) & 1) * rs.n_b + b] = replica_of(f, nx[3]);
    return !done;
}

// One bundle's lens-map Jacobian from its rays' states at x3 = chi_s; writes
// (mu, kappa, gamma1, gamma2, omega, flags) to o[0..5] and, when rout is
// given, each ray's final state to rout[(b * nr + k) * 8 + q].
__device__ __forceinline__ void reduce_bundle(const TraceParams &tp, const double *__restrict__ theta,
                                              const RayState &rs, double chi_s, int64_t b, double *__restrict__ o,
                                              double *__restrict__ rout)
{
    const int64_t n = rs.stride;
    int flags = 0;
    double x0 = 0, y0 = 0, tx0 = 0, ty0 = 0;
    double M00 = 0, M01 = 0, M10 = 0, M11 = 0, N00 = 0, N01 = 0, N10 = 0, N11 = 0;
    for (int k = 0; k < rs.nr; ++k) {
        const int64_t i = b * rs.nr + k;
        const int done = rs.done[i];
        const double *src = done ? rs.fin : rs.y;
        if (!done) flags |= RT3D_F_NOCROSS;
        double st[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            st[q] = src[q * n + i];
            if (!isfinite(st[q])) flags |= RT3D_F_NONFINITE;
        }
        if (rout)
#pragma unroll
            for (int q = 0; q < 8; ++q) rout[i * 8 + q] = st[q];
        double tx, ty;
        ray_theta(tp, theta, b, k, tx, ty);
        if (k == 0) {
            x0 = st[1];
            y0 = st[2];
            tx0 = tx;
            ty0 = ty;
        } else {
            const double dbx = (st[1] - x0) / chi_s, dby = (st[2] - y0) / chi_s;
            const double dtx = tx - tx0, dty = ty - ty0;
            M00 += dbx * dtx;
            M01 += dbx * dty;
            M10 += dby * dtx;
            M11 += dby * dty;
            N00 += dtx * dtx;
            N01 += dtx * dty;
            N10 += dty * dtx;
            N11 += dty * dty;
        }
    }
    const double dn = N00 * N11 - N01 * N10;
    const double i00 = N11 / dn, i01 = -N01 / dn, i10 = -N10 / dn, i11 = N00 / dn;
    const double A00 = M00 * i00 + M01 * i10, A01 = M00 * i01 + M01 * i11;
    const double A10 = M10 * i00 + M11 * i10, A11 = M10 * i01 + M11 * i11;
    const double det = A00 * A11 - A01 * A10;
    const double mu = 1.0 / det;
    if (!isfinite(mu)) flags |= RT3D_F_NONFINITE;
    if (mu < 0.0) flags |= RT3D_F_NEGPARITY;
    o[0] = mu;
    o[1] = 1.0 - 0.5 * (A00 + A11);
    o[2] = 0.5 * (A11 - A00);
    o[3] = -0.5 * (A01 + A10);
    o[4] = 0.5 * (A01 - A10);
    o[5] = (double)flags;
}

}  // namespace rt3d
